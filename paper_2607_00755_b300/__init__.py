"""Thin Python binding of libkx (the B300 collision-operator library).

Argument marshalling only: every step of the computation runs in the CUDA
kernels of ``libkx.so`` behind the C ABI of ``include/kx.h``.  torch is used
for device memory and streams.  Loading fails loudly if the library has not
been built (``python -m paper_2607_00755_b300.build``); there is no CPU path.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libkx.so")

OK, PENDING = 0, 1
EINVAL, ENOMEM, EADMIT, ENEG, ENONFINITE = -1, -2, -3, -4, -5
ESINGULAR, ENOCONV, ETIMEOUT, ECUDA, ENOTSUP = -6, -7, -8, -9, -10
MEASURE_ENERGY, MEASURE_LITERAL = 0, 1
FP64, FP32, SPLIT_TF32 = 0, 1, 2

EXPORTS = (
    "kx_create", "kx_destroy", "kx_set_stream", "kx_strerror", "kx_last_error",
    "kx_build_kernel", "kx_kernel_retain", "kx_kernel_release", "kx_kernel_get_info",
    "kx_kernel_grid", "kx_kernel_row", "kx_collision", "kx_collision_host", "kx_step",
    "kx_solve", "kx_solve_host", "kx_mb_fit", "kx_launch_count", "kx_time_contraction",
    "kx_time_contractions", "kx_time_collision",
    "kx_collision_noalloc", "kx_server_start", "kx_submit", "kx_poll", "kx_server_get_stats",
    "kx_server_stop", "kx_math_check", "kx_profile_attempts", "kx_measure_peaks", "kx_measure_mma_rate", "kx_server_reset_latency", "kx_check_status", "kx_check_probe", "kx_set_split_tuning", "kx_set_gain_operand", "kx_get_split_tuning", "kx_wait_check", "kx_set_stream_variant", "kx_get_stream_variant",
    "kx_source_higgs_decay", "kx_source_condensate", "kx_solve_expanding", "kx_solve_grouped",
)


class GridDesc(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("q", ctypes.c_void_p), ("a", ctypes.c_double),
                ("mass", ctypes.c_double), ("n_mu", ctypes.c_int), ("measure", ctypes.c_int),
                ("stats", ctypes.c_int), ("precision", ctypes.c_int), ("loss_terms", ctypes.c_int)]


class Source(ctypes.Structure):
    _fields_ = [("n_src", ctypes.c_int), ("shape", ctypes.c_void_p), ("rate", ctypes.c_void_p),
                ("tau", ctypes.c_void_p), ("t_on", ctypes.c_void_p)]


class SolveParams(ctypes.Structure):
    _fields_ = [("t0", ctypes.c_double), ("t_end", ctypes.c_double), ("h0", ctypes.c_double),
                ("rtol", ctypes.c_double), ("atol", ctypes.c_double), ("h_min", ctypes.c_double),
                ("h_max", ctypes.c_double), ("l1_tol", ctypes.c_double),
                ("max_attempts", ctypes.c_int), ("fixed_step", ctypes.c_int),
                ("check_every", ctypes.c_int), ("project", ctypes.c_int), ("chains", ctypes.c_int)]


class Diag(ctypes.Structure):
    _fields_ = [(k, ctypes.c_double) for k in ("eps_N_raw", "eps_E_raw", "eps_N_proj",
                                               "eps_E_proj", "R_N", "R_E", "alpha", "beta",
                                               "f_max")] + \
               [("singular", ctypes.c_int), ("status", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Result(ctypes.Structure):
    _fields_ = [(k, ctypes.c_double) for k in ("t", "h", "l1_to_mb", "T_mb", "ln_z_mb",
                                               "latency_s")] + \
               [(k, ctypes.c_longlong) for k in ("steps", "rejects", "evals")] + \
               [("status", ctypes.c_int), ("converged", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class ExpansionResult(ctypes.Structure):
    _fields_ = [("r", Result), ("u_switch", ctypes.c_double), ("gamma_over_H", ctypes.c_double),
                ("rk4_steps", ctypes.c_longlong), ("checks", ctypes.c_longlong)]

    def as_dict(self):
        d = self.r.as_dict()
        d.update(u=self.r.t, u_switch=self.u_switch, gamma_over_H=self.gamma_over_H,
                 rk4_steps=self.rk4_steps, checks=self.checks)
        return d


class KernelInfo(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("n_mu", ctypes.c_int), ("measure", ctypes.c_int),
                ("precision", ctypes.c_int), ("unique_elements", ctypes.c_longlong),
                ("nonzero_elements", ctypes.c_longlong), ("tensor_bytes", ctypes.c_longlong),
                ("build_ms", ctypes.c_double), ("stream_bytes", ctypes.c_longlong)]


class Expansion(ctypes.Structure):
    _fields_ = [("n_h", ctypes.c_int), ("u", ctypes.c_void_p), ("ln_H", ctypes.c_void_p),
                ("u0", ctypes.c_double), ("u_end", ctypes.c_double), ("du_rk4", ctypes.c_double),
                ("check_every", ctypes.c_int), ("eps_switch", ctypes.c_double)]


class ServerConfig(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_longlong), ("slots_per_group", ctypes.c_int),
                ("attempts_per_tick", ctypes.c_int), ("precision", ctypes.c_int),
                ("n_mu", ctypes.c_int), ("measure", ctypes.c_int), ("par", SolveParams),
                ("grid_div", ctypes.c_int), ("loss_terms", ctypes.c_int)]


class ServerStats(ctypes.Structure):
    _fields_ = [(k, ctypes.c_longlong) for k in ("submitted", "completed", "failed", "queued",
                                                 "active", "kernels_built", "kernel_cache_hits",
                                                 "evictions")] + \
               [(k, ctypes.c_double) for k in ("p50_latency_s", "p99_latency_s", "mean_latency_s",
                                               "p50_wait_s")] + \
               [(k, ctypes.c_longlong) for k in ("evals", "converged", "ticks_shared", "ticks_whole")] + \
               [(k, ctypes.c_double) for k in ("p99_wait_s", "p50_service_s", "p99_service_s")] + \
               [("stream_bytes", ctypes.c_longlong)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None
_libs = {}
LIB_CHECK_PATH = os.path.join(_HERE, "libkx_check.so")


def load_checked_library():
    """Load libkx_check.so, the bounds-checked build (kx_check_status)."""
    return _open_library(LIB_CHECK_PATH)


def load_library(path: str = LIB_PATH):
    """Load libkx.so (raises if it is missing: the product has no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    _lib = _open_library(path)
    return _lib


def _open_library(path: str):
    if path in _libs:
        return _libs[path]
    if not os.path.exists(path):
        raise RuntimeError(f"{os.path.basename(path)} not built at {path}; "
                           "run python -m paper_2607_00755_b300.build")
    lib = ctypes.CDLL(path)
    i, vp, d = ctypes.c_int, ctypes.c_void_p, ctypes.c_double
    sig = {
        "kx_create": (i, [vp, i, vp]),
        "kx_destroy": (None, [vp]),
        "kx_set_stream": (i, [vp, vp]),
        "kx_strerror": (ctypes.c_char_p, [i]),
        "kx_last_error": (ctypes.c_char_p, [vp]),
        "kx_build_kernel": (i, [vp, ctypes.POINTER(GridDesc), vp]),
        "kx_kernel_retain": (None, [vp]),
        "kx_kernel_release": (None, [vp]),
        "kx_kernel_get_info": (i, [vp, ctypes.POINTER(KernelInfo)]),
        "kx_kernel_grid": (i, [vp, vp, vp, vp, vp, vp]),
        "kx_kernel_row": (i, [vp, i, vp, vp, vp]),
        "kx_collision": (i, [vp, vp, i, vp, vp, vp, i, vp]),
        "kx_collision_host": (i, [vp, vp, i, vp, vp, vp, i, vp]),
        "kx_step": (i, [vp, vp, i, vp, vp, i, ctypes.POINTER(SolveParams), vp, vp, vp, vp]),
        "kx_solve": (i, [vp, vp, i, vp, vp, i, ctypes.POINTER(SolveParams), vp, vp]),
        "kx_solve_host": (i, [vp, vp, i, vp, vp, i, ctypes.POINTER(SolveParams), vp, vp]),
        "kx_mb_fit": (i, [vp, vp, i, vp, vp]),
        "kx_math_check": (i, [vp, i, i, vp, vp]),
        "kx_profile_attempts": (i, [vp, vp, i, vp, vp, i, vp, vp, i, vp]),
        "kx_measure_peaks": (i, [vp, vp, vp]),
        "kx_measure_mma_rate": (i, [vp, i, i, vp, vp]),
        "kx_server_reset_latency": (i, [vp]),
        "kx_check_status": (i, [vp, i, vp, vp, vp, vp]),
        "kx_check_probe": (i, [vp, i, i, vp]),
        "kx_set_split_tuning": (i, [i]),
        "kx_get_split_tuning": (i, [vp, i, vp, vp, vp, vp, vp, vp]),
        "kx_set_gain_operand": (i, [i]),
        "kx_wait_check": (i, [vp, ctypes.c_longlong, vp]),
        "kx_set_stream_variant": (i, [vp, i, i, i]),
        "kx_get_stream_variant": (i, [vp, i, i, vp, vp]),
        "kx_source_higgs_decay": (i, [i, vp, d, d, d, d, d, d, vp, vp]),
        "kx_source_condensate": (i, [i, vp, d, d, d, d, d, vp, vp]),
        "kx_solve_grouped": (i, [vp, i, vp, vp, vp, ctypes.POINTER(SolveParams), vp, vp]),
        "kx_solve_expanding": (i, [vp, ctypes.POINTER(GridDesc), d, vp, ctypes.POINTER(Expansion),
                                   ctypes.POINTER(SolveParams), vp, ctypes.POINTER(ExpansionResult)]),
        "kx_launch_count": (ctypes.c_longlong, [vp]),
        "kx_time_contraction": (i, [vp, vp, i, vp, i, ctypes.c_longlong, vp]),
        "kx_time_contractions": (i, [vp, i, vp, i, vp, i, i, vp]),
        "kx_time_collision": (i, [vp, vp, i, vp, vp, vp, i, i, vp]),
        "kx_collision_noalloc": (i, [vp, vp, i, vp, vp, vp, i]),
        "kx_server_start": (i, [vp, ctypes.POINTER(ServerConfig), vp]),
        "kx_submit": (i, [vp, ctypes.POINTER(GridDesc), d, vp, d, d, d, vp, vp]),
        "kx_poll": (i, [vp, ctypes.c_uint64, d, vp, vp]),
        "kx_server_get_stats": (i, [vp, ctypes.POINTER(ServerStats)]),
        "kx_server_stop": (None, [vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _libs[path] = lib
    return lib


class KxError(RuntimeError):
    def __init__(self, code, msg=""):
        self.code = code
        super().__init__(f"kx error {code}: {msg}")


def _np(a, dtype=np.float64):
    return np.ascontiguousarray(a, dtype=dtype)


def _ptr(a):
    return ctypes.c_void_p(a.ctypes.data)


def _dptr(t):
    """Device pointer of a contiguous CUDA float64 torch tensor."""
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64
            and t.is_contiguous()):
        raise TypeError("expected a contiguous CUDA float64 tensor")
    return ctypes.c_void_p(t.data_ptr())


class Context:
    """kx_ctx bound to a CUDA device and a torch stream."""

    def __init__(self, device: int = 0, stream=None, lib=None):
        import torch
        self.lib = lib if lib is not None else load_library()
        self.device = device
        if stream is None:
            stream = torch.cuda.current_stream(device)
        self.stream = stream
        h = ctypes.c_void_p()
        rc = self.lib.kx_create(ctypes.byref(h), device, ctypes.c_void_p(stream.cuda_stream))
        if rc:
            raise KxError(rc, "kx_create")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self.lib.kx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def error(self, rc, what):
        msg = self.lib.kx_last_error(self.h) or b""
        return KxError(rc, f"{what}: {self.lib.kx_strerror(rc).decode()} {msg.decode()}")

    # -------------------------------------------------------------- kernels
    def build_kernel(self, q, mass=1.0, a=1.0, n_mu=18, measure=MEASURE_ENERGY,
                     precision=FP64, stats=0, loss_terms=0):
        q = _np(q)
        desc = GridDesc(q.size, q.ctypes.data, a, mass, n_mu, measure, stats, precision, loss_terms)
        h = ctypes.c_void_p()
        rc = self.lib.kx_build_kernel(self.h, ctypes.byref(desc), ctypes.byref(h))
        if rc:
            raise self.error(rc, "kx_build_kernel")
        return Kernel(self, h, q.size)

    # ------------------------------------------------------------ collision
    def collision(self, kernel, f, sigma=1.0, project=True, out=None, diag=False):
        """C[f] for f of shape [B, n] (CUDA float64); returns (C, diag list|None)."""
        import torch
        f2 = f if f.dim() == 2 else f.view(1, -1)
        B = f2.shape[0]
        sig = _np(np.broadcast_to(np.asarray(sigma, dtype=np.float64), (B,)))
        C = out if out is not None else torch.empty_like(f2)
        dg = (Diag * B)() if diag else None
        rc = self.lib.kx_collision(self.h, kernel.h, B, _ptr(sig), _dptr(f2), _dptr(C),
                                   int(project), dg)
        if rc and not (rc == ENONFINITE and diag):
            raise self.error(rc, "kx_collision")
        return C.view_as(f), ([x.as_dict() for x in dg] if diag else None)

    def collision_host(self, kernel, f, sigma=1.0, project=True, diag=False):
        f2 = _np(np.atleast_2d(f))
        B = f2.shape[0]
        sig = _np(np.broadcast_to(np.asarray(sigma, dtype=np.float64), (B,)))
        C = np.empty_like(f2)
        dg = (Diag * B)() if diag else None
        rc = self.lib.kx_collision_host(self.h, kernel.h, B, _ptr(sig), _ptr(f2), _ptr(C),
                                        int(project), dg)
        if rc and not (rc == ENONFINITE and diag):
            raise self.error(rc, "kx_collision_host")
        return C.reshape(np.shape(f)), ([x.as_dict() for x in dg] if diag else None)

    # ---------------------------------------------------------- integration
    @staticmethod
    def _sources(sources, B, n):
        """sources: None, one dict (shared) or a list of B dicts."""
        if sources is None:
            return None, 0, []
        lst = [sources] if isinstance(sources, dict) else list(sources)
        keep = []
        arr = (Source * len(lst))()
        for s, src in enumerate(lst):
            shape = _np(np.atleast_2d(src["shape"]))
            rate, tau, t_on = (_np(src[k]) for k in ("rate", "tau", "t_on"))
            keep += [shape, rate, tau, t_on]
            arr[s] = Source(shape.shape[0], shape.ctypes.data, rate.ctypes.data,
                            tau.ctypes.data, t_on.ctypes.data)
        return arr, len(lst), keep

    @staticmethod
    def params(**kw):
        p = dict(t0=0.0, t_end=1.0, h0=1e-3, rtol=1e-6, atol=1e-12, h_min=0.0, h_max=0.0,
                 l1_tol=0.0, max_attempts=1_000_000, fixed_step=0, check_every=10, project=1,
                 chains=0)
        p.update(kw)
        return SolveParams(**{k: p[k] for k, _ in SolveParams._fields_})

    def solve(self, kernel, f, sigma, sources=None, **params):
        """Integrate f ([B, n] CUDA float64, in place).  Returns list of result dicts."""
        f2 = f if f.dim() == 2 else f.view(1, -1)
        B = f2.shape[0]
        sig = _np(np.broadcast_to(np.asarray(sigma, dtype=np.float64), (B,)))
        src, ns, keep = self._sources(sources, B, kernel.n)
        par = self.params(**params)
        res = (Result * B)()
        rc = self.lib.kx_solve(self.h, kernel.h, B, _ptr(sig), src, ns, ctypes.byref(par),
                               _dptr(f2), res)
        del keep
        if rc in (EINVAL, ENOMEM, ECUDA, ETIMEOUT, ENOTSUP):
            raise self.error(rc, "kx_solve")
        return [r.as_dict() for r in res]

    def set_split_tuning(self, enabled):
        """Switch the split path's launch-choice timing on or off (off forgets the choices)."""
        self.lib.kx_set_split_tuning(int(bool(enabled)))

    def split_tuning(self, kernel, batch):
        """The split path's launch choices for kernel and batch (kx_get_split_tuning)."""
        v = [ctypes.c_int(0) for _ in range(6)]
        rc = self.lib.kx_get_split_tuning(kernel.h, int(batch), *[ctypes.byref(x) for x in v])
        if rc:
            raise self.error(rc, "kx_get_split_tuning")
        return {"gain_S": v[0].value, "gain_fs": v[1].value, "loss_S": v[2].value, "loss_ipl": v[3].value,
                "tuned": v[4].value, "gain_atm": v[5].value}

    def set_gain_operand(self, where):
        """Where the split path's gain GEMM keeps its generated A operand
        (kx_set_gain_operand): "any", "shared" or "tensor"."""
        rc = self.lib.kx_set_gain_operand({"any": 0, "shared": 1, "tensor": 2}[where])
        if rc:
            raise self.error(rc, "kx_set_gain_operand")

    def check_status(self, reset=False):
        """Bounds-check record (kx_check_status): checked build?, failures,
        first failing site and index."""
        c, nf, site, idx = ctypes.c_int(0), ctypes.c_longlong(0), ctypes.c_int(0), ctypes.c_longlong(0)
        rc = self.lib.kx_check_status(self.h, int(bool(reset)), ctypes.byref(c), ctypes.byref(nf),
                                      ctypes.byref(site), ctypes.byref(idx))
        if rc:
            raise self.error(rc, "kx_check_status")
        return {"checked": bool(c.value), "failures": nf.value, "first_site": site.value,
                "first_index": idx.value}

    def check_probe(self, index, limit):
        """Result of passing index through the bounds check with the given limit."""
        r = ctypes.c_int(0)
        rc = self.lib.kx_check_probe(self.h, int(index), int(limit), ctypes.byref(r))
        if rc:
            raise self.error(rc, "kx_check_probe")
        return r.value

    def measure_mma_rate(self, kind, n):
        """(FLOP per clock per SM, cycles per MMA) of tcgen05.mma M=128, N=n: kind 0
        TF32 (K = 8), kind 1 BF16 (K = 16)."""
        a, b = ctypes.c_double(0.0), ctypes.c_double(0.0)
        rc = self.lib.kx_measure_mma_rate(self.h, int(kind), int(n), ctypes.byref(a), ctypes.byref(b))
        if rc:
            raise self.error(rc, "kx_measure_mma_rate")
        return a.value, b.value

    def measure_peaks(self):
        """(FP64 flop/s, ex2/s) of the device from the library's throughput kernels."""
        a, b = ctypes.c_double(0.0), ctypes.c_double(0.0)
        rc = self.lib.kx_measure_peaks(self.h, ctypes.byref(a), ctypes.byref(b))
        if rc:
            raise self.error(rc, "kx_measure_peaks")
        return a.value, b.value

    def profile_attempts(self, kernel, f, sigma, sources=None, attempts=200, **params):
        """Average device microseconds of the four kernels of a Heun attempt
        (contraction 1, stage 1, contraction 2, stage 2), launched in plain
        stream order with CUDA events between them; f (CUDA float64 [B, n]) is
        advanced by the attempts."""
        f2 = f if f.dim() == 2 else f.view(1, -1)
        B = f2.shape[0]
        sig = _np(np.broadcast_to(np.asarray(sigma, dtype=np.float64), (B,)))
        src, ns, keep = self._sources(sources, B, kernel.n)
        par = self.params(**params)
        us = (ctypes.c_double * 4)()
        rc = self.lib.kx_profile_attempts(self.h, kernel.h, B, _ptr(sig), src, ns, ctypes.byref(par),
                                          _dptr(f2), int(attempts), us)
        del keep
        if rc:
            raise self.error(rc, "kx_profile_attempts")
        return {"contraction_1_us": us[0], "stage_1_us": us[1], "contraction_2_us": us[2],
                "stage_2_us": us[3]}

    def solve_host(self, kernel, f, sigma, sources=None, **params):
        """Host-buffer variant: f numpy [B, n] copied in and out inside the call."""
        f2 = _np(np.atleast_2d(f)).copy()
        B = f2.shape[0]
        sig = _np(np.broadcast_to(np.asarray(sigma, dtype=np.float64), (B,)))
        src, ns, keep = self._sources(sources, B, kernel.n)
        par = self.params(**params)
        res = (Result * B)()
        rc = self.lib.kx_solve_host(self.h, kernel.h, B, _ptr(sig), src, ns, ctypes.byref(par),
                                    _ptr(f2), res)
        del keep
        if rc in (EINVAL, ENOMEM, ECUDA, ETIMEOUT, ENOTSUP):
            raise self.error(rc, "kx_solve_host")
        return f2, [r.as_dict() for r in res]

    def step(self, kernel, f, sigma, t, h, sources=None, **params):
        """One Heun attempt per instance; t, h numpy [B] updated in place."""
        f2 = f if f.dim() == 2 else f.view(1, -1)
        B = f2.shape[0]
        sig = _np(np.broadcast_to(np.asarray(sigma, dtype=np.float64), (B,)))
        src, ns, keep = self._sources(sources, B, kernel.n)
        par = self.params(**params)
        res = (Result * B)()
        rc = self.lib.kx_step(self.h, kernel.h, B, _ptr(sig), src, ns, ctypes.byref(par),
                              _ptr(t), _ptr(h), _dptr(f2), res)
        del keep
        if rc in (EINVAL, ENOMEM, ECUDA, ETIMEOUT, ENOTSUP):
            raise self.error(rc, "kx_step")
        return [r.as_dict() for r in res]

    def solve_grouped(self, kernels, fs, sigmas, **params):
        """Uneven batch (kx_solve_grouped): kernels[g] with the CUDA float64
        tensor fs[g] [B_g, n_g] (in place) and sigmas[g] [B_g]; returns one list
        of result dicts per group."""
        G = len(kernels)
        Bs = [f.shape[0] for f in fs]
        sig = [_np(np.broadcast_to(np.asarray(s_, dtype=np.float64), (b,))) for s_, b in zip(sigmas, Bs)]
        karr = (ctypes.c_void_p * G)(*[k.h for k in kernels])
        barr = (ctypes.c_int * G)(*Bs)
        sarr = (ctypes.c_void_p * G)(*[x.ctypes.data for x in sig])
        farr = (ctypes.c_void_p * G)(*[f.data_ptr() for f in fs])
        res = [(Result * b)() for b in Bs]
        rarr = (ctypes.c_void_p * G)(*[ctypes.addressof(r) for r in res])
        par = self.params(**params)
        rc = self.lib.kx_solve_grouped(self.h, G, karr, barr, sarr, ctypes.byref(par), farr, rarr)
        if rc in (EINVAL, ENOMEM, ECUDA, ETIMEOUT, ENOTSUP):
            raise self.error(rc, "kx_solve_grouped")
        return [[x.as_dict() for x in r] for r in res]

    def solve_expanding(self, q, f, sigma, hu, ln_H, u0, u_end, du_rk4=0.05, check_every=1,
                        eps_switch=1e-2, sources=None, precision=FP64, mass=1.0, n_mu=18,
                        measure=MEASURE_ENERGY, **params):
        """One distribution in an expanding universe (kx_solve_expanding): f is
        a CUDA float64 tensor [n] on the comoving grid q, updated in place."""
        q = _np(q)
        hu_a, hl_a = _np(np.atleast_1d(hu)), _np(np.atleast_1d(ln_H))
        desc = GridDesc(q.size, q.ctypes.data, 1.0, mass, n_mu, measure, 0, precision, 0)
        ex = Expansion(hl_a.size, hu_a.ctypes.data, hl_a.ctypes.data, float(u0), float(u_end),
                       float(du_rk4), int(check_every), float(eps_switch))
        src, ns, keep = self._sources(sources, 1, q.size)
        par = self.params(**params)
        res = ExpansionResult()
        rc = self.lib.kx_solve_expanding(self.h, ctypes.byref(desc), float(sigma), src, ctypes.byref(ex),
                                         ctypes.byref(par), _dptr(f), ctypes.byref(res))
        del keep
        if rc in (EINVAL, ENOMEM, ECUDA, ETIMEOUT, ENOTSUP):
            raise self.error(rc, "kx_solve_expanding")
        return res.as_dict()

    def launch_count(self) -> int:
        return int(self.lib.kx_launch_count(self.h))

    def time_contraction(self, kernel, f, iters=20, flush_bytes=0):
        """Mean device time (ms) of one contraction launch for f [B, n]."""
        f2 = f if f.dim() == 2 else f.view(1, -1)
        ms = ctypes.c_double()
        rc = self.lib.kx_time_contraction(self.h, kernel.h, f2.shape[0], _dptr(f2), int(iters),
                                          int(flush_bytes), ctypes.byref(ms))
        if rc:
            raise self.error(rc, "kx_time_contraction")
        return ms.value

    def time_collision(self, kernel, f, sigma=1.0, project=True, iters=20):
        """Device time (ms) of one full evaluation of C[f] for f [B, n] (graph
        replay); returns (ms, C)."""
        import torch
        f2 = f if f.dim() == 2 else f.view(1, -1)
        B = f2.shape[0]
        sig = _np(np.broadcast_to(np.asarray(sigma, dtype=np.float64), (B,)))
        C = torch.empty_like(f2)
        ms = ctypes.c_double()
        rc = self.lib.kx_time_collision(self.h, kernel.h, B, _ptr(sig), _dptr(f2), _dptr(C),
                                        int(project), int(iters), ctypes.byref(ms))
        if rc:
            raise self.error(rc, "kx_time_collision")
        return ms.value, C.view_as(f)

    def time_contractions(self, kernels, f, iters=10, pdl=False):
        """Mean device time (ms) per launch of the kernels' contractions issued
        back to back (rotating tables), for f [B, n]; pdl: programmatic
        dependent launch, as inside the solve's graphs."""
        f2 = f if f.dim() == 2 else f.view(1, -1)
        arr = (ctypes.c_void_p * len(kernels))(*[k.h for k in kernels])
        ms = ctypes.c_double()
        rc = self.lib.kx_time_contractions(self.h, len(kernels), arr, f2.shape[0], _dptr(f2),
                                           int(iters), int(bool(pdl)), ctypes.byref(ms))
        if rc:
            raise self.error(rc, "kx_time_contractions")
        return ms.value

    def mb_fit(self, kernel, f):
        f2 = f if f.dim() == 2 else f.view(1, -1)
        out = np.empty((f2.shape[0], 3))
        rc = self.lib.kx_mb_fit(self.h, kernel.h, f2.shape[0], _dptr(f2), _ptr(out))
        if rc:
            raise self.error(rc, "kx_mb_fit")
        return out

    def set_stream_variant(self, n, batch, variant):
        """Pin (0 .. 4) or forget (-1) the streaming variant for (n, batch)."""
        rc = self.lib.kx_set_stream_variant(self.h, int(n), int(batch), int(variant))
        if rc:
            raise self.error(rc, "kx_set_stream_variant")

    def stream_variant(self, n, batch):
        """(variant, tuned) of the FP32 streaming contraction for (n, batch)."""
        var, tun = ctypes.c_int(-1), ctypes.c_int(0)
        rc = self.lib.kx_get_stream_variant(self.h, int(n), int(batch), ctypes.byref(var),
                                            ctypes.byref(tun))
        if rc:
            raise self.error(rc, "kx_get_stream_variant")
        return var.value, bool(tun.value)

    def math_check(self, which, x):
        """(library value, CUDA value) of x (a CUDA float64 tensor) for the
        helper `which` (0 log2, 1 exp, 2 double-float log2, 3 double -> float,
        4 float -> double of the float nearest x); returns a [n, 2] tensor."""
        import torch
        out = torch.empty((x.numel(), 2), dtype=torch.float64, device=x.device)
        rc = self.lib.kx_math_check(self.h, int(which), x.numel(), _dptr(x), _dptr(out))
        if rc:
            raise self.error(rc, "kx_math_check")
        torch.cuda.synchronize()
        return out

    def wait_check(self, cycles):
        """1 if a bounded device wait of `cycles` SM cycles on an mbarrier that
        nothing arrives on gave up (kx_wait_check)."""
        out = ctypes.c_int(-1)
        rc = self.lib.kx_wait_check(self.h, int(cycles), ctypes.byref(out))
        if rc:
            raise self.error(rc, "kx_wait_check")
        return out.value


def source_higgs_decay(q, mass, m_h, T, coupling, g_chi=1.0, a=1.0):
    """Higgs-decay source row (eq. C_higgs_decay): (shape [n], rate)."""
    lib = load_library()
    q = _np(q)
    shape = np.empty(q.size)
    rate = ctypes.c_double()
    rc = lib.kx_source_higgs_decay(q.size, _ptr(q), float(a), float(mass), float(m_h), float(T),
                                   float(coupling), float(g_chi), _ptr(shape), ctypes.byref(rate))
    if rc:
        raise KxError(rc, "kx_source_higgs_decay")
    return shape, rate.value


def source_condensate(q, mass, m_phi, gamma_n, g_chi=1.0, a=1.0):
    """Condensate-decay source row (eq. C_condensate_decay): (shape [n], rate)."""
    lib = load_library()
    q = _np(q)
    shape = np.empty(q.size)
    rate = ctypes.c_double()
    rc = lib.kx_source_condensate(q.size, _ptr(q), float(a), float(mass), float(m_phi), float(g_chi),
                                  float(gamma_n), _ptr(shape), ctypes.byref(rate))
    if rc:
        raise KxError(rc, "kx_source_condensate")
    return shape, rate.value


class Server:
    """Continuous-batching solve server (kx_server): submit solves, poll results."""

    def __init__(self, ctx: Context, budget_bytes=8 << 30, slots_per_group=16,
                 attempts_per_tick=8, precision=FP32, n_mu=18, measure=MEASURE_ENERGY,
                 grid_div=0, loss_terms=0, **params):
        self.ctx, self.lib = ctx, ctx.lib
        cfg = ServerConfig(int(budget_bytes), int(slots_per_group), int(attempts_per_tick),
                           int(precision), int(n_mu), int(measure), Context.params(**params),
                           int(grid_div), int(loss_terms))
        h = ctypes.c_void_p()
        rc = self.lib.kx_server_start(ctx.h, ctypes.byref(cfg), ctypes.byref(h))
        if rc:
            raise ctx.error(rc, "kx_server_start")
        self.h = h

    def submit(self, q, f0, sigma, sources=None, t0=0.0, t_end=1.0, h0=1e-3, mass=1.0, a=1.0):
        """Queue one solve; returns a ticket (int).  Raises KxError (e.g. KX_EADMIT)."""
        q, f0 = _np(q), _np(f0)
        desc = GridDesc(q.size, q.ctypes.data, a, mass, 0, 0, 0, 0, 0)
        src, ns, keep = Context._sources(sources, 1, q.size)
        t = ctypes.c_uint64()
        rc = self.lib.kx_submit(self.h, ctypes.byref(desc), float(sigma), src, float(t0),
                                float(t_end), float(h0), _ptr(f0), ctypes.byref(t))
        del keep
        if rc:
            raise KxError(rc, self.lib.kx_strerror(rc).decode())
        return t.value

    def poll(self, ticket, n, timeout=0.0):
        """(status, f, result dict): status OK when done, PENDING otherwise."""
        f = np.empty(n)
        res = Result()
        rc = self.lib.kx_poll(self.h, ctypes.c_uint64(ticket), float(timeout), _ptr(f),
                              ctypes.byref(res))
        return rc, f, res.as_dict()

    def stats(self):
        st = ServerStats()
        self.lib.kx_server_get_stats(self.h, ctypes.byref(st))
        return st.as_dict()

    def reset_latency(self):
        """New sample for the latency quantiles (requests completed from now on)."""
        rc = self.lib.kx_server_reset_latency(self.h)
        if rc:
            raise KxError(rc, "kx_server_reset_latency")

    def stop(self):
        if getattr(self, "h", None):
            self.lib.kx_server_stop(self.h)
            self.h = None

    def __del__(self):
        try:
            self.stop()
        except Exception:
            pass


class Kernel:
    """Reference-counted kernel-tensor handle (kx_kernel)."""

    def __init__(self, ctx: Context, h, n: int):
        self.ctx, self.h, self.n = ctx, h, n

    def info(self):
        inf = KernelInfo()
        self.ctx.lib.kx_kernel_get_info(self.h, ctypes.byref(inf))
        return {k: getattr(inf, k) for k, _ in KernelInfo._fields_}

    def grid(self):
        out = {k: np.empty(self.n) for k in ("p", "E", "dp", "dE", "h")}
        self.ctx.lib.kx_kernel_grid(self.h, *(_ptr(out[k]) for k in ("p", "E", "dp", "dE", "h")))
        return out

    def row(self, i: int):
        P = self.n * (self.n + 1) // 2
        W, jl, om = np.empty(P), np.empty(P, dtype=np.int32), np.empty(P)
        rc = self.ctx.lib.kx_kernel_row(self.h, i, _ptr(W), _ptr(jl), _ptr(om))
        if rc:
            raise self.ctx.error(rc, "kx_kernel_row")
        return W, jl, om

    def release(self):
        if self.h:
            self.ctx.lib.kx_kernel_release(self.h)
            self.h = None

    def __del__(self):
        try:
            self.release()
        except Exception:
            pass
