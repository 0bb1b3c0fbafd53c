// kx_serve.cu -- continuous-batching solve server (kx_server_*, kx_submit, kx_poll).
//
// A worker thread owns the GPU work.  Requests are grouped by kernel tensor
// (grid and mass); each group has a fixed number of device-resident slots, its
// own stream and one captured CUDA graph of `attempts_per_tick` Heun attempts
// over all its slots (free and finished slots are skipped on the device by
// their `done` flag).  Between graph launches the worker copies finished slots
// out, frees them and admits queued requests into free slots, so requests join
// and leave at step boundaries while the others keep integrating.  Kernel
// tensors stay cached (LRU) while the HBM budget allows.
#include <math.h>
#include <string.h>
#include <stdlib.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "kx_internal.cuh"

// groups with work above which their FP32 contractions share the GPU
#define KX_SHARE_MIN_GROUPS 8

namespace {

double kx_now() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

size_t kx_al(size_t x) { return (x + 255) & ~(size_t)255; }

struct Request {
    kx_ticket id = 0;
    int n = 0;
    std::vector<double> q;
    double a = 1, mass = 1, sigma = 1, t0 = 0, t_end = 0, h0 = 0;
    int n_src = 0;
    std::vector<double> shape, rate, tau, t_on;
    std::vector<double> f0, f_out;
    kx_result res;
    int status = KX_PENDING;
    double t_submit = 0, t_admit = 0, t_done = 0;
    std::string key;
};

struct Group {
    std::string key;
    kx_kernel *k = nullptr;
    int cap = 0, n = 0;
    void *mem = nullptr;
    size_t mem_bytes = 0;
    kx_batch_views v;
    kx_step_views sv;
    double *mb = nullptr;
    int *fin = nullptr;      // [cap] slots to fit on completion
    double *shapes = nullptr;
    kx_src_dev *src = nullptr;
    std::vector<std::shared_ptr<Request>> slot;
    cudaStream_t stream = nullptr;
    cudaGraph_t graph = nullptr;      // attempts with the shared contraction grid (1/grid_div)
    cudaGraphExec_t exec = nullptr;
    cudaGraph_t graph1 = nullptr;     // the same attempts with the whole GPU (grid_div > 1 only)
    cudaGraphExec_t exec1 = nullptr;
    kx_inst_state *h_st = nullptr;   // pinned [cap]
    cudaEvent_t ev = nullptr;
    bool in_flight = false;
    bool need_prep = false;
    int active = 0;
    double last_used = 0;
    size_t footprint() const { return mem_bytes + (size_t)(k ? k->bytes : 0); }
};

}  // namespace

struct kx_server {
    kx_ctx *ctx = nullptr;    // the caller's context (device)
    kx_ctx *wctx = nullptr;   // the worker's own context for kernel builds
    kx_server_config cfg;
    std::thread worker;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    bool stop = false;
    std::deque<std::shared_ptr<Request>> queue;
    std::unordered_map<kx_ticket, std::shared_ptr<Request>> reqs;
    std::vector<std::unique_ptr<Group>> groups;
    size_t used = 0;
    kx_ticket next_id = 1;
    kx_server_stats stats;
    std::vector<double> lat, wait, service;   // submit->done, submit->admit, admit->done
};

// ------------------------------------------------------------------ helpers
static std::string kx_key(const Request &r) {
    std::string k((const char *)r.q.data(), sizeof(double) * r.q.size());
    k.append((const char *)&r.a, sizeof(double));
    k.append((const char *)&r.mass, sizeof(double));
    return k;
}

// Device bytes of a group (kernel tables after the build + slot state), from
// the grid size alone, for admission before anything is built.
static size_t kx_group_estimate(const kx_server_config &cfg, int n) {
    kx_kernel d;
    d.n = n;
    d.precision = cfg.precision;
    d.P = (long long)n * (n + 1) / 2;
    long long V = 0;
    for (int a = 0; a < n; ++a) V += (n - a + 3) / 4;
    d.V = (int)V;
    d.cheb_K = cfg.precision == KX_SPLIT_TF32 ? cfg.loss_terms : 0;
    kx_split_geometry(&d);
    size_t tables;
    // FP32: upper bounds (every vector kept, rows padded to whole units, one
    // unit per task)
    const long long unit = n <= 160 ? 64 : 128, upr = (V + unit - 1) / unit;
    d.tslots = (int)(n * ((upr + 2) & ~1LL));
    if (cfg.precision == KX_FP32)
        tables = (size_t)n * upr * unit * (16 + 16 + 4) + (size_t)(n + 1) * 4 + (size_t)n * 8 +
                 (size_t)n * upr * 16;
    else if (cfg.precision == KX_FP64) tables = (size_t)n * d.P * 18 + 4 * d.P;
    else {   // split: gain (and Chebyshev) operand tiles, loss elements (with padding), segments, row tables
        const size_t segs = (size_t)n * (d.P / 64 + n + 1);   // at most P/64 + n per row
        tables = (size_t)((d.nis + 255) / 256) * std::min(4, d.nsubI) * (d.KBG + d.KBL) * 1024 * 8 +
                 ((size_t)n * d.P + 3 * segs) * 8 +
                 segs * 8 + (size_t)(34 * n + 1) * 4;
    }
    const int cap = cfg.slots_per_group;
    size_t mem = kx_al(kx_views_bytes(&d, cap)) + 3 * kx_al(sizeof(double) * cap * n) +
                 kx_al(sizeof(kx_inst_state) * cap) + kx_al(sizeof(kx_src_dev) * cap) +
                 kx_al(sizeof(double) * cap * KX_MAX_SRC * n) + kx_al(sizeof(double) * 3 * cap) +
                 kx_al(sizeof(int) * cap);
    return tables + mem + 5 * n * 8;
}

static void kx_free_group(Group *g) {
    if (!g) return;
    if (g->stream) cudaStreamSynchronize(g->stream);
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->graph) cudaGraphDestroy(g->graph);
    if (g->exec1) cudaGraphExecDestroy(g->exec1);
    if (g->graph1) cudaGraphDestroy(g->graph1);
    if (g->ev) cudaEventDestroy(g->ev);
    if (g->h_st) cudaFreeHost(g->h_st);
    if (g->mem) cudaFree(g->mem);
    if (g->stream) cudaStreamDestroy(g->stream);
    if (g->k) kx_kernel_release(g->k);
}

// One Heun attempt over all slots; after the first attempt of a captured tick
// every launch may start early (programmatic dependent launch, each kernel
// waits for its predecessor before reading its outputs).
static cudaError_t kx_group_attempt(Group *g, cudaStream_t s, bool first) {
    cudaError_t e;
    if ((e = kx_launch_contract(g->k, g->cap, g->sv.f, g->v, g->sv.st, 1, s, !first)) != cudaSuccess) return e;
    if ((e = kx_launch_stage(g->k, g->cap, g->v, g->sv, 1, s, true)) != cudaSuccess) return e;
    if ((e = kx_launch_contract(g->k, g->cap, g->sv.fp, g->v, g->sv.st, 2, s, true)) != cudaSuccess) return e;
    return kx_launch_stage(g->k, g->cap, g->v, g->sv, 2, s, true);
}

// Build (or fail) the group of request r.  Called on the worker thread.
static int kx_make_group(kx_server *srv, const Request &r, Group **out) {
    *out = nullptr;
    kx_grid_desc d;
    d.n = r.n;
    d.q = r.q.data();
    d.a = r.a;
    d.mass = r.mass;
    d.n_mu = srv->cfg.n_mu;
    d.measure = srv->cfg.measure;
    d.stats = 0;
    d.precision = srv->cfg.precision;
    d.loss_terms = srv->cfg.loss_terms;
    kx_kernel *k = nullptr;
    int rc = kx_build_kernel(srv->wctx, &d, &k);
    if (rc) return rc;
    std::unique_ptr<Group> g(new Group());
    g->key = r.key;
    g->k = k;
    g->cap = srv->cfg.slots_per_group;
    g->n = r.n;
    const int cap = g->cap, n = r.n;
    const size_t o_views = 0;
    size_t o = kx_al(kx_views_bytes(k, cap));
    const size_t o_f = o; o += kx_al(sizeof(double) * cap * n);
    const size_t o_k1 = o; o += kx_al(sizeof(double) * cap * n);
    const size_t o_fp = o; o += kx_al(sizeof(double) * cap * n);
    const size_t o_st = o; o += kx_al(sizeof(kx_inst_state) * cap);
    const size_t o_src = o; o += kx_al(sizeof(kx_src_dev) * cap);
    const size_t o_sh = o; o += kx_al(sizeof(double) * cap * KX_MAX_SRC * n);
    const size_t o_mb = o; o += kx_al(sizeof(double) * 3 * cap);
    const size_t o_fin = o; o += kx_al(sizeof(int) * cap);
    g->mem_bytes = o;
    if (cudaMalloc(&g->mem, o) != cudaSuccess) {
        cudaGetLastError();
        kx_free_group(g.get());
        return KX_ENOMEM;
    }
    char *base = (char *)g->mem;
    kx_carve_views(k, cap, base + o_views, &g->v);
    kx_step_views &sv = g->sv;
    sv.f = (double *)(base + o_f);
    sv.k1 = (double *)(base + o_k1);
    sv.fp = (double *)(base + o_fp);
    sv.st = (kx_inst_state *)(base + o_st);
    g->src = (kx_src_dev *)(base + o_src);
    g->shapes = (double *)(base + o_sh);
    sv.src = g->src;
    sv.shapes = g->shapes;
    g->mb = (double *)(base + o_mb);
    g->fin = (int *)(base + o_fin);
    const kx_solve_params &p = srv->cfg.par;
    sv.rtol = p.rtol;
    sv.atol = p.atol;
    sv.h_min = p.h_min;
    sv.h_max = p.h_max > 0 ? p.h_max : INFINITY;
    sv.l1_tol = p.l1_tol;
    sv.max_attempts = p.max_attempts;
    sv.fixed = p.fixed_step;
    sv.check_every = p.check_every;
    sv.project = p.project;
    sv.hscale = 1.0;
    cudaError_t e = cudaStreamCreateWithFlags(&g->stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&g->ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMallocHost((void **)&g->h_st, sizeof(kx_inst_state) * cap);
    std::vector<kx_inst_state> st(cap);
    for (auto &x : st) {
        memset(&x, 0, sizeof(x));
        x.done = 1;
    }
    std::vector<kx_src_dev> sd(cap);
    for (auto &x : sd) {
        memset(&x, 0, sizeof(x));
        x.t_off = -INFINITY;
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(g->mem, 0, o, g->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(sv.st, st.data(), sizeof(kx_inst_state) * cap, cudaMemcpyHostToDevice, g->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(g->src, sd.data(), sizeof(kx_src_dev) * cap, cudaMemcpyHostToDevice, g->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
    // pick the streaming variant for this size and slot count before capture
    // (timed on the group's zeroed tables: same work as real inputs)
    // (tuned for each grid share the group's graphs launch with)
    for (int pass = 0; pass < (srv->cfg.grid_div > 1 ? 2 : 1) && e == cudaSuccess; ++pass) {
        g->v.grid_div = pass == 0 ? srv->cfg.grid_div : 1;
        if (kx_tune_contraction(k, cap, g->sv.f, g->v, nullptr, g->stream, nullptr)) e = cudaErrorUnknown;
    }
    // captured graph of attempts_per_tick Heun attempts over all slots: one with
    // the shared contraction grid and, if that is a fraction, one with the
    // whole GPU (the worker picks by the number of groups with work)
    cudaStream_t cap_s = nullptr;
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&cap_s, cudaStreamNonBlocking);
    for (int pass = 0; pass < (srv->cfg.grid_div > 1 ? 2 : 1) && e == cudaSuccess; ++pass) {
        g->v.grid_div = pass == 0 ? srv->cfg.grid_div : 1;
        cudaGraph_t *gr = pass == 0 ? &g->graph : &g->graph1;
        e = cudaStreamBeginCapture(cap_s, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            for (int a = 0; a < srv->cfg.attempts_per_tick && e == cudaSuccess; ++a)
                e = kx_group_attempt(g.get(), cap_s, a == 0);
            cudaError_t e2 = cudaStreamEndCapture(cap_s, gr);
            if (e == cudaSuccess) e = e2;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(pass == 0 ? &g->exec : &g->exec1, *gr, 0);
    }
    g->v.grid_div = 1;
    if (cap_s) cudaStreamDestroy(cap_s);
    if (e != cudaSuccess) {
        kx_free_group(g.get());
        return kx_set_error(srv->wctx, KX_ECUDA, std::string("server group: ") + cudaGetErrorString(e));
    }
    g->slot.assign(cap, nullptr);
    g->last_used = kx_now();
    *out = g.release();
    return KX_OK;
}

// Write request r into free slot s of g (the group is not in flight).
static cudaError_t kx_admit(Group *g, int s, const std::shared_ptr<Request> &r) {
    const int n = g->n;
    kx_inst_state st;
    memset(&st, 0, sizeof(st));
    st.t = r->t0;
    st.h = r->h0;
    st.t_end = r->t_end;
    st.l1 = INFINITY;
    st.done = !(r->t0 < r->t_end);
    kx_src_dev sd;
    memset(&sd, 0, sizeof(sd));
    sd.t_off = -INFINITY;
    sd.n_src = r->n_src;
    sd.shape_off = (long long)s * KX_MAX_SRC * n;
    std::vector<double> shp((size_t)KX_MAX_SRC * n, 0.0);
    for (int k = 0; k < r->n_src; ++k) {
        double norm = 0.0;
        for (int j = 0; j < n; ++j) norm += g->k->h[j] * r->shape[(size_t)k * n + j];
        for (int j = 0; j < n; ++j) shp[(size_t)k * n + j] = r->shape[(size_t)k * n + j] / norm;
        sd.rate[k] = r->rate[k];
        sd.tau[k] = r->tau[k];
        sd.t_on[k] = r->t_on[k];
        sd.t_off = std::max(sd.t_off, r->t_on[k] + r->tau[k] * log(1e12));
    }
    const double M2 = 64.0 * 3.14159265358979323846 * g->k->mass * g->k->mass * r->sigma;
    cudaError_t e = cudaMemcpyAsync(g->sv.f + (size_t)s * n, r->f0.data(), sizeof(double) * n,
                                    cudaMemcpyHostToDevice, g->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(g->sv.st + s, &st, sizeof(st), cudaMemcpyHostToDevice, g->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(g->src + s, &sd, sizeof(sd), cudaMemcpyHostToDevice, g->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(g->shapes + (size_t)s * KX_MAX_SRC * n, shp.data(), sizeof(double) * shp.size(),
                            cudaMemcpyHostToDevice, g->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(g->v.M2 + s, &M2, sizeof(double), cudaMemcpyHostToDevice, g->stream);
    // the pageable copies above are staged before return; keep the host data alive anyway
    if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
    g->slot[s] = r;
    g->active++;
    g->need_prep = true;
    return e;
}

// Copy finished slots out (the group's graph has completed).
static void kx_complete(kx_server *srv, Group *g) {
    std::vector<int> fin;
    for (int s = 0; s < g->cap; ++s)
        if (g->slot[s] && g->h_st[s].done) fin.push_back(s);
    if (fin.empty()) return;
    const int n = g->n;
    std::vector<double> f((size_t)g->cap * n), mb((size_t)3 * g->cap);
    // fit only the finished slots (from their last in-solve fit's temperature)
    cudaError_t e = cudaMemcpyAsync(g->fin, fin.data(), sizeof(int) * fin.size(), cudaMemcpyHostToDevice,
                                    g->stream);
    if (e == cudaSuccess)
        e = kx_launch_mbfit(g->k, (int)fin.size(), g->sv.f, g->mb, g->stream, g->sv.st, g->fin);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(f.data(), g->sv.f, sizeof(double) * f.size(), cudaMemcpyDeviceToHost, g->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(mb.data(), g->mb, sizeof(double) * mb.size(), cudaMemcpyDeviceToHost, g->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
    const double t = kx_now();
    std::lock_guard<std::mutex> lock(srv->mu);
    for (int s : fin) {
        std::shared_ptr<Request> r = g->slot[s];
        const kx_inst_state &st = g->h_st[s];
        r->f_out.assign(f.begin() + (size_t)s * n, f.begin() + (size_t)(s + 1) * n);
        kx_result &o = r->res;
        o.t = st.t;
        o.h = st.h;
        o.T_mb = mb[3 * s];
        o.ln_z_mb = mb[3 * s + 1];
        o.l1_to_mb = mb[3 * s + 2];
        o.steps = st.steps;
        o.rejects = st.rejects;
        o.evals = st.evals;
        o.status = e == cudaSuccess ? st.status : KX_ECUDA;
        o.converged = st.converged;
        r->t_done = t;
        o.latency_s = r->t_done - r->t_submit;
        r->status = o.status;
        srv->stats.completed += o.status == KX_OK;
        srv->stats.converged += o.status == KX_OK && o.converged;
        srv->stats.failed += o.status != KX_OK;
        srv->service.push_back(r->t_done - r->t_admit);
        srv->stats.active--;
        srv->stats.evals += st.evals;
        srv->stats.stream_bytes += st.evals * g->k->stream_bytes;
        srv->lat.push_back(o.latency_s);
        g->slot[s] = nullptr;
        g->active--;
    }
    g->last_used = t;
    srv->cv_done.notify_all();
}

static bool kx_evict_for(kx_server *srv, size_t need) {
    while (srv->used + need > (size_t)srv->cfg.hbm_budget_bytes) {
        int victim = -1;
        for (int i = 0; i < (int)srv->groups.size(); ++i) {
            Group *g = srv->groups[i].get();
            if (g->active == 0 && !g->in_flight &&
                (victim < 0 || g->last_used < srv->groups[victim]->last_used))
                victim = i;
        }
        if (victim < 0) return false;
        srv->used -= srv->groups[victim]->footprint();
        kx_free_group(srv->groups[victim].get());
        delete srv->groups[victim].release();
        srv->groups.erase(srv->groups.begin() + victim);
        std::lock_guard<std::mutex> lock(srv->mu);
        srv->stats.evictions++;
    }
    return true;
}

static void kx_fail(kx_server *srv, const std::shared_ptr<Request> &r, int code) {
    std::lock_guard<std::mutex> lock(srv->mu);
    r->status = code;
    r->res.status = code;
    r->t_done = kx_now();
    srv->stats.failed++;
    srv->cv_done.notify_all();
}

static void kx_worker(kx_server *srv) {
    kx_nvtx range_("kx_server_worker");
    cudaSetDevice(srv->ctx->device);
    const double wall_limit = 3600.0;
    double t_stop = 0.0;
    for (;;) {
        bool progressed = false;
        // 1. graphs that finished: copy out finished requests
        for (auto &gp : srv->groups) {
            Group *g = gp.get();
            if (!g->in_flight) continue;
            cudaError_t q = cudaEventQuery(g->ev);
            if (q == cudaErrorNotReady) continue;
            g->in_flight = false;
            if (q != cudaSuccess) {
                for (int s = 0; s < g->cap; ++s) g->h_st[s].done = 1, g->h_st[s].status = KX_ECUDA;
            }
            kx_complete(srv, g);
            progressed = true;
        }
        // 2. admissions in arrival order
        std::vector<std::shared_ptr<Request>> pending;
        {
            std::lock_guard<std::mutex> lock(srv->mu);
            pending.assign(srv->queue.begin(), srv->queue.end());
        }
        std::vector<std::shared_ptr<Request>> admitted;
        for (auto &r : pending) {
            Group *g = nullptr;
            bool fresh = false;
            for (auto &gp : srv->groups)
                if (gp->key == r->key) g = gp.get();
            if (!g) {
                fresh = true;
                const size_t need = kx_group_estimate(srv->cfg, r->n);
                if (need > (size_t)srv->cfg.hbm_budget_bytes) {
                    kx_fail(srv, r, KX_EADMIT);
                    admitted.push_back(r);
                    continue;
                }
                if (!kx_evict_for(srv, need)) continue;   // wait for memory
                int rc = kx_make_group(srv, *r, &g);
                if (rc) {
                    kx_fail(srv, r, rc);
                    admitted.push_back(r);
                    continue;
                }
                srv->groups.emplace_back(g);
                srv->used += g->footprint();
                std::lock_guard<std::mutex> lock(srv->mu);
                srv->stats.kernels_built++;
            }
            if (g->in_flight) continue;
            int s = -1;
            for (int i = 0; i < g->cap; ++i)
                if (!g->slot[i]) {
                    s = i;
                    break;
                }
            if (s < 0) continue;
            if (kx_admit(g, s, r) != cudaSuccess) {
                kx_fail(srv, r, KX_ECUDA);
            } else {
                std::lock_guard<std::mutex> lock(srv->mu);
                r->t_admit = kx_now();
                srv->wait.push_back(r->t_admit - r->t_submit);
                srv->stats.active++;
                if (!fresh) srv->stats.kernel_cache_hits++;
            }
            admitted.push_back(r);
            progressed = true;
        }
        if (!admitted.empty()) {
            std::lock_guard<std::mutex> lock(srv->mu);
            for (auto &r : admitted) {
                auto it = std::find(srv->queue.begin(), srv->queue.end(), r);
                if (it != srv->queue.end()) srv->queue.erase(it);
            }
            srv->stats.queued = (long long)srv->queue.size();
        }
        // 3. launch a tick for every idle group with work; while more than 8
        // groups have work their contractions share the GPU (1/grid_div of it
        // each), else each takes the whole of it.  Measured on the Poisson
        // stream: 100 solves (85 grids at once) 5.9 solves/s against 3.8 with
        // the whole GPU throughout; its first 8 solves 2.3 against 1.3 with the
        // shared grid throughout.
        int busy = 0;
        for (auto &gp : srv->groups) busy += gp->active > 0;
        const bool shared = busy > KX_SHARE_MIN_GROUPS;
        for (auto &gp : srv->groups) {
            Group *g = gp.get();
            if (g->in_flight || g->active == 0) continue;
            cudaError_t e = cudaSuccess;
            if (g->need_prep) {
                e = kx_launch_prep(g->k, g->cap, g->sv.f, g->v, g->sv.st, g->stream);
                g->need_prep = false;
            }
            const bool on_share = shared || !g->exec1;
            if (e == cudaSuccess) e = cudaGraphLaunch(on_share ? g->exec : g->exec1, g->stream);
            if (e == cudaSuccess) {
                std::lock_guard<std::mutex> lock(srv->mu);
                if (on_share && srv->cfg.grid_div > 1) srv->stats.ticks_shared++;
                else srv->stats.ticks_whole++;
            }
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(g->h_st, g->sv.st, sizeof(kx_inst_state) * g->cap,
                                    cudaMemcpyDeviceToHost, g->stream);
            if (e == cudaSuccess) e = cudaEventRecord(g->ev, g->stream);
            g->in_flight = e == cudaSuccess;
            if (e != cudaSuccess) {
                for (int s = 0; s < g->cap; ++s) g->h_st[s].done = 1, g->h_st[s].status = KX_ECUDA;
                kx_complete(srv, g);
            }
            progressed = true;
        }
        // 4. exit or wait
        bool any_flight = false, any_active = false;
        for (auto &gp : srv->groups) {
            any_flight |= gp->in_flight;
            any_active |= gp->active > 0;
        }
        std::unique_lock<std::mutex> lock(srv->mu);
        if (srv->stop) {
            if (t_stop == 0.0) t_stop = kx_now();
            if ((srv->queue.empty() && !any_flight && !any_active) || kx_now() - t_stop > wall_limit)
                break;
        }
        if (!progressed) {
            if (any_flight) {
                lock.unlock();
                std::this_thread::sleep_for(std::chrono::microseconds(20));
            } else {
                srv->cv_work.wait_for(lock, std::chrono::milliseconds(2));
            }
        }
    }
    for (auto &gp : srv->groups) kx_free_group(gp.get());
    srv->groups.clear();
}

// ---------------------------------------------------------------------- ABI
extern "C" int kx_server_start(kx_ctx *ctx, const kx_server_config *cfg, kx_server **out) {
    if (!ctx || !cfg || !out) return KX_EINVAL;
    *out = nullptr;
    if (cfg->hbm_budget_bytes <= 0 || cfg->slots_per_group < 1 || cfg->slots_per_group > 256 ||
        cfg->attempts_per_tick < 1 || cfg->attempts_per_tick > 64 || cfg->n_mu < 1 ||
        cfg->n_mu > KX_MAX_NMU ||
        (cfg->precision != KX_FP32 && cfg->precision != KX_FP64 && cfg->precision != KX_SPLIT_TF32) ||
        !(cfg->par.rtol >= 0) || !(cfg->par.atol >= 0) || cfg->par.max_attempts < 1 ||
        cfg->grid_div < 0 || cfg->grid_div > 16 ||
        (cfg->loss_terms != 0 && (cfg->precision != KX_SPLIT_TF32 ||
                                  (cfg->loss_terms != 8 && cfg->loss_terms != 16 && cfg->loss_terms != 32))))
        return kx_set_error(ctx, KX_EINVAL, "bad server configuration");
    kx_server *srv = new (std::nothrow) kx_server();
    if (!srv) return KX_ENOMEM;
    srv->ctx = ctx;
    srv->cfg = *cfg;
    // a half grid per group measured best with many groups at once (a third and
    // a quarter were slower)
    if (srv->cfg.grid_div == 0) srv->cfg.grid_div = 2;
    if (srv->cfg.precision != KX_FP32) srv->cfg.grid_div = 1;   // only the FP32 streaming kernels use it
    memset(&srv->stats, 0, sizeof(srv->stats));
    int rc = kx_create(&srv->wctx, ctx->device, nullptr);
    if (rc) {
        delete srv;
        return rc;
    }
    srv->worker = std::thread(kx_worker, srv);
    *out = srv;
    return KX_OK;
}

extern "C" int kx_submit(kx_server *srv, const kx_grid_desc *grid, double sigma, const kx_source *src,
                         double t0, double t_end, double h0, const double *f0, kx_ticket *ticket) {
    if (!srv || !grid || !f0 || !ticket || !grid->q) return KX_EINVAL;
    const int n = grid->n;
    if (n < 4 || n > KX_MAX_N || !(grid->mass > 0) || !(grid->a > 0) || !(sigma > 0) ||
        !isfinite(sigma) || !(h0 > 0) || !(t_end >= t0))
        return KX_EINVAL;
    for (int i = 0; i < n; ++i) {
        if (!(grid->q[i] > 0) || (i && !(grid->q[i] > grid->q[i - 1]))) return KX_EINVAL;
        if (!isfinite(f0[i])) return KX_EINVAL;
    }
    auto r = std::make_shared<Request>();
    r->n = n;
    r->q.assign(grid->q, grid->q + n);
    r->a = grid->a;
    r->mass = grid->mass;
    r->sigma = sigma;
    r->t0 = t0;
    r->t_end = t_end;
    r->h0 = h0;
    r->f0.assign(f0, f0 + n);
    if (src && src->n_src > 0) {
        if (src->n_src > KX_MAX_SRC || !src->shape || !src->rate || !src->tau || !src->t_on)
            return KX_EINVAL;
        r->n_src = src->n_src;
        r->shape.assign(src->shape, src->shape + (size_t)src->n_src * n);
        r->rate.assign(src->rate, src->rate + src->n_src);
        r->tau.assign(src->tau, src->tau + src->n_src);
        r->t_on.assign(src->t_on, src->t_on + src->n_src);
        for (int k = 0; k < src->n_src; ++k) {
            double norm = 0.0;
            for (int j = 0; j < n; ++j) {
                if (!(r->shape[(size_t)k * n + j] >= 0)) return KX_EINVAL;
                norm += r->shape[(size_t)k * n + j];
            }
            if (!(norm > 0) || !(r->tau[k] > 0)) return KX_EINVAL;
        }
    }
    r->key = kx_key(*r);
    if (kx_fault("admit") || kx_group_estimate(srv->cfg, n) > (size_t)srv->cfg.hbm_budget_bytes)
        return KX_EADMIT;
    r->t_submit = kx_now();
    {
        std::lock_guard<std::mutex> lock(srv->mu);
        if (srv->stop) return KX_EINVAL;
        r->id = srv->next_id++;
        srv->reqs[r->id] = r;
        srv->queue.push_back(r);
        srv->stats.submitted++;
        srv->stats.queued = (long long)srv->queue.size();
    }
    srv->cv_work.notify_one();
    *ticket = r->id;
    return KX_OK;
}

extern "C" int kx_poll(kx_server *srv, kx_ticket ticket, double timeout_s, double *f_out,
                       kx_result *res) {
    if (!srv || !(timeout_s >= 0)) return KX_EINVAL;
    std::unique_lock<std::mutex> lock(srv->mu);
    auto it = srv->reqs.find(ticket);
    if (it == srv->reqs.end()) return KX_EINVAL;
    std::shared_ptr<Request> r = it->second;
    const auto deadline = std::chrono::steady_clock::now() + std::chrono::duration<double>(timeout_s);
    while (r->status == KX_PENDING) {
        if (srv->cv_done.wait_until(lock, deadline) == std::cv_status::timeout) break;
    }
    if (r->status == KX_PENDING) return KX_PENDING;
    if (res) *res = r->res;
    if (f_out && !r->f_out.empty()) memcpy(f_out, r->f_out.data(), sizeof(double) * r->n);
    const int st = r->status;
    srv->reqs.erase(it);
    return st;
}

static double kx_quantile(std::vector<double> v, double q) {
    if (v.empty()) return 0.0;
    std::sort(v.begin(), v.end());
    const double pos = q * (v.size() - 1);
    const size_t i = (size_t)pos;
    const double fr = pos - i;
    return i + 1 < v.size() ? v[i] * (1 - fr) + v[i + 1] * fr : v[i];
}

extern "C" int kx_server_get_stats(kx_server *srv, kx_server_stats *out) {
    if (!srv || !out) return KX_EINVAL;
    std::lock_guard<std::mutex> lock(srv->mu);
    *out = srv->stats;
    out->p50_latency_s = kx_quantile(srv->lat, 0.5);
    out->p99_latency_s = kx_quantile(srv->lat, 0.99);
    double m = 0.0;
    for (double x : srv->lat) m += x;
    out->mean_latency_s = srv->lat.empty() ? 0.0 : m / srv->lat.size();
    out->p50_wait_s = kx_quantile(srv->wait, 0.5);
    out->p99_wait_s = kx_quantile(srv->wait, 0.99);
    out->p50_service_s = kx_quantile(srv->service, 0.5);
    out->p99_service_s = kx_quantile(srv->service, 0.99);
    return KX_OK;
}

extern "C" int kx_server_reset_latency(kx_server *srv) {
    if (!srv) return KX_EINVAL;
    std::lock_guard<std::mutex> lock(srv->mu);
    srv->lat.clear();
    srv->wait.clear();
    srv->service.clear();
    return KX_OK;
}

extern "C" void kx_server_stop(kx_server *srv) {
    if (!srv) return;
    {
        std::lock_guard<std::mutex> lock(srv->mu);
        srv->stop = true;
    }
    srv->cv_work.notify_all();
    if (srv->worker.joinable()) srv->worker.join();
    kx_destroy(srv->wctx);
    delete srv;
}
