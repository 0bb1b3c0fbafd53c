"""The paper's two freeze-in source terms (Sec. 2, eqs. C_higgs_decay and
C_condensate_decay): the oracle's formulas pinned to closed forms, and the
library's host helpers against the oracle (no GPU needed)."""
import numpy as np
import pytest
from scipy.special import k1

import kx_inputs as ki
import oracle

M, MH, COUPLING, G = 1.0, 5.0, 0.3, 2.0


def trapezoid_number(q, C):
    g = oracle.grid(q)
    return np.sum(g["h"] * C)


@pytest.mark.parametrize("T", [0.5, 2.0, 10.0])
def test_higgs_source_number_rate_closed_form(T):
    """Integrated over momentum space the Higgs source injects
    c^2/(8 pi g) * k * T * K1(m_h / T) (k = sqrt(m_h^2 - 4 m^2)): the parent
    energies that feed a daughter energy E span [E_h^-, E_h^+], so swapping the
    order of integration leaves int dE_h p_h e^(-E_h/T) (k / m_h)
    = k T K1(m_h/T).  A dropped or mis-signed term in E_h^(+/-) breaks this."""
    q = ki.log_grid(6000, 1e-5, 60.0 * T + 60.0)
    C = oracle.higgs_decay_source(q, M, MH, T, COUPLING, G)
    k = np.sqrt(MH ** 2 - 4 * M ** 2)
    exact = COUPLING ** 2 / (8 * np.pi * G) * k * T * k1(MH / T)
    assert abs(trapezoid_number(q, C) / exact - 1) < 2e-5


def test_higgs_source_edges():
    """Support and limits: non-negative everywhere; at threshold m_h -> 2 m the
    source vanishes linearly in k = sqrt(m_h^2 - 4 m^2) (the bracket is
    exp(-E_h^-/T)(1 - exp(-m_h p k / (m^2 T))), E_h^- -> m_h^2 E / (2 m^2));
    at large p the daughter is suppressed like exp(-E_h^-/T)."""
    q = ki.log_grid(400, 1e-3, 50.0)
    C = oracle.higgs_decay_source(q, M, MH, 1.0, COUPLING, G)
    assert np.all(C >= 0) and np.all(np.isfinite(C))
    assert C[-1] < 1e-12 * np.max(C)
    eps = (1e-6, 4e-6)   # m_h = 2 m (1 + eps): k = 2 m sqrt(2 eps + eps^2)
    Cs = [oracle.higgs_decay_source(q[:40], M, 2 * M * (1 + e), 1.0, COUPLING, G) for e in eps]
    ks = [2 * M * np.sqrt(2 * e + e * e) for e in eps]
    np.testing.assert_allclose(Cs[1] / Cs[0], ks[1] / ks[0], rtol=2e-3)


def test_condensate_cell_and_rate():
    q = ki.log_grid(64, 1e-3, 10.0)
    for m_phi in (2.2, 3.0, 7.5):
        p0 = 0.5 * np.sqrt(m_phi ** 2 - 4 * M ** 2)
        i = oracle.condensate_source_cell(q, M, m_phi)
        assert i is not None
        lo = q[0] if i == 0 else 0.5 * (q[i - 1] + q[i])
        hi = q[-1] if i == q.size - 1 else 0.5 * (q[i] + q[i + 1])
        assert lo <= p0 <= hi
    assert oracle.condensate_source_cell(q, M, 40.0) is None


@pytest.fixture(scope="module")
def kx():
    import paper_2607_00755_b300 as kx
    from paper_2607_00755_b300 import build
    build.build()
    return kx


@pytest.mark.parametrize("T,a", [(0.7, 1.0), (3.0, 0.5)])
def test_library_higgs_source_matches_oracle(kx, T, a):
    q = ki.log_grid(96, 1e-3, 30.0)
    shape, rate = kx.source_higgs_decay(q, M, MH, T, COUPLING, G, a=a)
    ref = oracle.higgs_decay_source(q, M, MH, T, COUPLING, G, a=a)
    big = ref > 1e-200
    np.testing.assert_allclose(shape[big], ref[big], rtol=1e-10)
    g = oracle.grid(q, a=a, mass=M)
    assert abs(rate / np.sum(g["h"] * ref) - 1) < 1e-12


def test_library_condensate_source_matches_oracle(kx):
    q = ki.log_grid(80, 1e-3, 10.0)
    shape, rate = kx.source_condensate(q, M, 3.0, 0.25, G)
    i = oracle.condensate_source_cell(q, M, 3.0)
    assert np.count_nonzero(shape) == 1 and shape[i] == 1.0
    assert rate == pytest.approx(2 * np.pi ** 2 / G * 0.25, rel=1e-15)
    with pytest.raises(kx.KxError):
        kx.source_condensate(q, M, 40.0, 0.25, G)
    with pytest.raises(kx.KxError):
        kx.source_higgs_decay(q, M, 1.5, 1.0, COUPLING, G)   # m_h < 2 m
