"""The LHY interpolation tables of the CUDA path against the oracle's
Gauss-Legendre sums, on the host (no GPU): the library builds the tables for a
parameter set exactly as its engines do and evaluates them in FP64
(egpe_lhy_table_eval), for the FP64 and the FP32 engine.  mu_LHY must equal
the oracle's quadrature to ~1e-14 (FP64 tables) or ~5e-9 (FP32 tables) of
its magnitude at every density ratio (including minor fractions down to
1e-12), the energy density follows from Euler's identity, and the second
derivatives equal central differences of the oracle's mu_LHY."""
import numpy as np
import pytest

import oracle as O
from paper_2510_24543_gb300 import build as B
from paper_2510_24543_gb300 import egpe as E
from paper_2510_24543_gb300 import inputs as I

from . import _common as _cm


@pytest.fixture(scope="module")
def lib():
    B.build()
    return E.load()


def _cases():
    out = {k: I.PRESETS[k] for k in ("c1", "c2", "c3", "c5")}
    scan = I.scan_workloads()
    lo = min(scan, key=lambda w: w.g[0][1] - w.gdd[0][0])   # small g12, large g_dd: nodes left exact
    hi = max(scan, key=lambda w: w.g[0][1] - w.gdd[0][0])
    out["scan_lo"], out["scan_hi"] = lo, hi
    out["mixed"] = _cm.mixed_workload((8, 8, 8))
    rng = np.random.default_rng(11)
    for k in range(4):
        g11, g22 = rng.uniform(50, 500, 2)
        g12 = rng.uniform(-200, 400)
        d = rng.uniform(0, 600, 3)
        out[f"random{k}"] = I.Workload(f"r{k}", (8, 8, 8), (1, 1, 1), (1, 1, 1), ((g11, g12), (g12, g22)),
                                       ((d[0], d[2]), (d[2], d[1])), 60.0, 0, "kinetic", 32)
    return out


def _points(seed=5, m=400):
    rng = np.random.default_rng(seed)
    n = rng.uniform(0.001, 0.3, m)
    t = rng.uniform(0, 1, m)
    t[:40] = 10.0 ** rng.uniform(-12, -2, 40)       # component 2 dominant
    t[40:80] = 1 - 10.0 ** rng.uniform(-12, -2, 40)  # component 1 dominant
    t[80] = 0.0
    t[81] = 1.0
    t[82] = 0.5
    return n * t, n * (1 - t)


# table error bound per engine: the FP64 tables are checked to 2e-15 of each
# function's largest magnitude, the FP32 ones (degree 7) to 1e-9
_TOL = {E.EGPE_FP64: 2e-14, E.EGPE_FP32: 5e-9}


@pytest.mark.parametrize("prec", [E.EGPE_FP64, E.EGPE_FP32], ids=["fp64", "fp32"])
@pytest.mark.parametrize("name", list(_cases().keys()))
def test_tables_reproduce_the_quadrature(lib, name, prec):
    w = _cases()[name]
    prm = O.Params(w.g, w.gdd, w.kappa, w.eta_s, w.lhy_nodes, w.trap)
    n1, n2 = _points()
    mu, hs, (ni, nexact) = E.egpe_lhy_table_eval(E.params_from_workload(w), n1, n2, prec)
    tol = _TOL[prec]
    assert ni in (0, 32, 64) and 0 <= nexact <= w.lhy_nodes
    if name in ("c1", "c2", "c3", "c5", "mixed"):
        assert ni > 0 and nexact <= 1  # the workloads run almost entirely from the tables
    F, m1, m2 = O.lhy_density_and_mu(prm, n1, n2)
    n = n1 + n2
    for i, m in enumerate((m1, m2)):
        scale = np.max(np.abs(m) / n ** 1.5)
        assert np.max(np.abs(mu[:, i] - m) / n ** 1.5) < tol * scale, i
    Fe = 0.4 * (n1 * mu[:, 0] + n2 * mu[:, 1])
    assert np.max(np.abs(Fe - F) / n ** 2.5) < tol * np.max(np.abs(F) / n ** 2.5)
    # second derivatives against central differences of the oracle's mu (away
    # from the edges n_i = 0, where the one-sided behaviour spoils the stencil)
    sel = (n1 > 1e-3 * n) & (n2 > 1e-3 * n)
    a1, a2 = n1[sel], n2[sel]
    h = 1e-6 * (a1 + a2)
    d11 = (O.lhy_density_and_mu(prm, a1 + h, a2)[1] - O.lhy_density_and_mu(prm, a1 - h, a2)[1]) / (2 * h)
    d12 = (O.lhy_density_and_mu(prm, a1, a2 + h)[1] - O.lhy_density_and_mu(prm, a1, a2 - h)[1]) / (2 * h)
    d22 = (O.lhy_density_and_mu(prm, a1, a2 + h)[2] - O.lhy_density_and_mu(prm, a1, a2 - h)[2]) / (2 * h)
    na = np.sqrt(a1 + a2)
    for col, fd in ((0, d11), (1, d12), (2, d22)):
        scale = np.max(np.abs(fd) / na)
        assert np.max(np.abs(hs[sel, col] - fd) / na) < 1e-6 * scale, col


@pytest.mark.parametrize("prec", [E.EGPE_FP64, E.EGPE_FP32], ids=["fp64", "fp32"])
def test_tables_vanish_without_lhy(lib, prec):
    w = I.PRESETS["c1"]
    p = E.params_from_workload(w)
    p.lhy_kappa = 0.0
    mu, hs, _ = E.egpe_lhy_table_eval(p, *_points(), prec)
    assert np.all(mu == 0) and np.all(hs == 0)


def test_table_eval_rejects_other_precisions(lib):
    p = E.params_from_workload(I.PRESETS["c1"])
    with pytest.raises(E.EgpeError):
        E.egpe_lhy_table_eval(p, *_points(), E.EGPE_MIXED)
