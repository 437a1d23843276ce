"""Batched solves of several instances (the parameter scan's uneven grids):
every instance reaches the ground state a solve of that instance alone
reaches, the first iterations of instance 0 follow the oracle in lockstep, and
the mixed-precision batched scan agrees with the oracle's evaluation of each
returned state."""
import numpy as np
import pytest

import oracle as O
from paper_2510_24543_gb300 import inputs as I

from ._common import gauge_fix, oracle_case, rel

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def E():
    from paper_2510_24543_gb300 import build as B
    B.build()
    from paper_2510_24543_gb300 import egpe
    egpe.load()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return egpe


def _scan_subset(sizes_per_grid=2, nodes=32):
    """A few instances of each grid size of the parameter scan (the scan's
    own 32-node LHY rule)."""
    scan = I.scan_workloads()
    out = []
    for g in range(4):
        for k in range(sizes_per_grid):
            w = scan[16 * g + k]
            out.append(I.Workload(w.name, w.n, w.L, w.trap, w.g, w.gdd, w.lhy_c, w.seed, w.precond, nodes))
    return out


def _solve(E, ws, prec, batch, tol=1e-9, trace_cap=0, max_iter=3000, **kw):
    h = E.egpe_create([E.make_grid(w.n, w.L) for w in ws], [E.params_from_workload(w) for w in ws], prec)
    try:
        o = E.egpe_default_solve_opts()
        o.precond = E.PRECOND["kinetic"]
        o.tol_res = tol
        o.max_iter = max_iter
        o.batch = batch
        for k, v in kw.items():
            setattr(o, k, v)
        dt = torch.complex64 if prec == E.EGPE_FP32 else torch.complex128
        xs = [torch.from_numpy(I.gaussian_start(w)).to("cuda").to(dt) for w in ws]
        st, reps, tr = E.egpe_ncg_solve(h, xs, o, len(ws), trace_cap=trace_cap)
        return st, reps, tr, [x.cpu().numpy().astype(np.complex128) for x in xs]
    finally:
        E.egpe_destroy(h)


@pytest.mark.parametrize("batch", [1, 2])
def test_batched_equals_one_by_one(E, batch):
    """Eight instances on 48^3, 64^3, 80^3 and 96^3: batched solves (the grid
    shapes' launches in sequence, batch 1, or as concurrent graph branches,
    batch 2) and one-by-one solves reach the same energies and states (they
    differ only in how the per-block partial sums are grouped)."""
    ws = _scan_subset()
    st_b, rb, _, psi_b = _solve(E, ws, E.EGPE_FP64, batch)
    st_s, rs, _, psi_s = _solve(E, ws, E.EGPE_FP64, 0)
    assert st_b == 0 and st_s == 0
    for i in range(len(ws)):
        assert rb[i]["status"] == 0 and rs[i]["status"] == 0
        assert rb[i]["res"] < 1e-9
        assert rel(rb[i]["E"], rs[i]["E"]) < 1e-12, i
        assert abs(rb[i]["iters"] - rs[i]["iters"]) <= max(3, rs[i]["iters"] // 10), i
        assert np.max(np.abs(gauge_fix(psi_b[i]) - gauge_fix(psi_s[i]))) < 1e-7, i


def test_batched_lockstep_with_oracle(E):
    """Instance 0 of a batch (48^3) follows the oracle iteration by iteration
    while the other instances run in the same launches."""
    ws = _scan_subset(1)
    w = ws[0]
    g, prm = oracle_case(w)
    otr = []
    O.ncg_solve(g, prm, I.gaussian_start(w), O.SolveOpts(precond="kinetic", tol_res=1e-8, max_iter=6), trace=otr)
    st, reps, tr, _ = _solve(E, ws, E.EGPE_FP64, 2, max_iter=6, trace_cap=64)
    acc = [t for t in tr if t["flags"] & 1]
    oacc = [t for t in otr if t["accepted"]]
    assert len(acc) == len(oacc) == 6
    for a, b in zip(acc, oacc):
        assert rel(a["E"], b["E"]) < 1e-11
        assert rel(a["E_trial"], b["E_new"]) < 1e-11
        assert rel(a["res"], b["res"]) < 1e-8
    assert all(r["iters"] == 6 for r in reps)


def test_batched_mixed_scan_against_oracle(E):
    """Mixed precision (FP32 phase to 1e-4, FP64 polish to 1e-9) over the
    subset: converged, and the oracle's evaluation of two returned states
    (48^3 and 96^3) gives the reported energy and a residual below 1e-8."""
    ws = _scan_subset()
    st, reps, _, psis = _solve(E, ws, E.EGPE_MIXED, 2, tol_fp32_switch=1e-4)
    assert st == 0
    for r in reps:
        assert r["status"] == 0 and r["iters_fp32"] > 0 and r["res"] < 1e-9
    for i in (0, len(ws) - 1):
        g, prm = oracle_case(ws[i])
        ev = O.evaluate(g, prm, psis[i])
        assert rel(reps[i]["E"], ev.E) < 1e-12
        r = np.stack([ev.Hpsi[c] - ev.mu[c] * psis[i][c] for c in range(2)])
        assert np.sqrt(sum(O.inner(g, r[c], r[c]).real for c in range(2))) < 1e-8
