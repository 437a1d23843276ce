"""GPU parity on the workload sizes beyond 32^3: the 64^3 droplet couplings in
lockstep with the oracle and solved to the same ground state, the
256x256x128 energy/gradient element by element, and the 128x128x64 and 128^3
mixed-precision solves (FP32 phase + FP64 polish) whose results the oracle
evaluates independently."""
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


def _handle(E, w, prec):
    return E.egpe_create([E.make_grid(w.n, w.L)], [E.params_from_workload(w)], prec)


def test_c2_droplet_lockstep(E):
    """64^3 droplet couplings, kinetic+diagonal preconditioner: the first
    iterations agree with the oracle step by step."""
    w = I.PRESETS["c2"]
    psi0 = I.gaussian_start(w)
    g, prm = oracle_case(w)
    otr = []
    O.ncg_solve(g, prm, psi0, O.SolveOpts(precond="kinetic+diagonal", tol_res=1e-8, max_iter=6), trace=otr)
    h = _handle(E, w, E.EGPE_FP64)
    try:
        o = E.egpe_default_solve_opts()
        o.precond = E.PRECOND["kinetic+diagonal"]
        o.max_iter = 6
        x = torch.from_numpy(psi0).to("cuda")
        st, reps, tr = E.egpe_ncg_solve(h, [x], o, 1, trace_cap=64)
    finally:
        E.egpe_destroy(h)
    acc = [t for t in tr if t["flags"] & 1]
    oacc = [t for t in otr if t["accepted"]]
    assert len(acc) == len(oacc) == 6
    for a, b in zip(acc, oacc):
        assert rel(a["E"], b["E"]) < 1e-11
        assert rel(a["E_trial"], b["E_new"]) < 1e-11
        assert rel(a["res"], b["res"]) < 1e-8
        assert rel(a["alpha"], b["alpha"]) < 1e-7
        assert abs(a["beta"] - b["beta"]) < 1e-7 * max(1.0, abs(b["beta"]))


def test_c2_droplet_ground_state_matches_oracle(E):
    """64^3 droplet workload solved to ||r|| < 1e-11 by the GPU (FP64, P_Delta o
    P_V) and by the oracle from the same seeded start: the same ground state,
    relative energy within 1e-11 and max|psi| within 1e-9 after fixing the
    global phase of each component (the whole-solver comparison of Sec. VI with
    the residual stopping rule)."""
    w = I.PRESETS["c2"]
    psi0 = I.gaussian_start(w)
    g, prm = oracle_case(w)
    opsi, orep = O.ncg_solve(g, prm, psi0, O.SolveOpts(precond="kinetic+diagonal", tol_res=1e-11, max_iter=500))
    assert orep["status"] == "converged"
    h = _handle(E, w, E.EGPE_FP64)
    try:
        o = E.egpe_default_solve_opts()
        o.precond = E.PRECOND["kinetic+diagonal"]
        o.tol_res = 1e-11
        o.max_iter = 500
        x = torch.from_numpy(psi0).to("cuda")
        st, reps, _ = E.egpe_ncg_solve(h, [x], o, 1)
        psi = x.cpu().numpy()
    finally:
        E.egpe_destroy(h)
    assert st == 0 and reps[0]["status"] == 0
    assert rel(reps[0]["E"], orep["E"]) < 1e-11
    for i in range(2):
        assert rel(reps[0]["mu"][i], orep["mu"][i]) < 1e-9
    assert np.max(np.abs(gauge_fix(psi) - gauge_fix(opsi))) < 1e-9


def test_c3p_headline_mixed_solve_against_oracle(E):
    """The headline 128^3 workload through the headline path: FP32 fields to
    ||r|| < 1e-4, then the FP64 polish to ||r|| < 1e-10.  The oracle evaluates
    the returned state: its energy and chemical potentials equal the reported
    ones to 1e-11 and its own residual is below 1e-9; the FP64-only solve from
    the same start reaches the same energy."""
    w = I.PRESETS["c3p"]
    psi0 = I.gaussian_start(w)
    g, prm = oracle_case(w)
    out = {}
    for prec in (E.EGPE_MIXED, E.EGPE_FP64):
        h = _handle(E, w, prec)
        try:
            o = E.egpe_default_solve_opts()
            o.precond = E.PRECOND["kinetic+diagonal"]
            o.tol_res = 1e-10
            o.tol_fp32_switch = 1e-4
            o.max_iter = 2000
            x = torch.from_numpy(psi0).to("cuda")
            st, reps, _ = E.egpe_ncg_solve(h, [x], o, 1)
            out[prec] = (st, reps[0], x.cpu().numpy())
        finally:
            E.egpe_destroy(h)
    st_m, rep_m, psi_m = out[E.EGPE_MIXED]
    st_d, rep_d, _ = out[E.EGPE_FP64]
    assert st_m == 0 and st_d == 0
    assert 0 < rep_m["iters_fp32"] < rep_m["iters"]
    ev = O.evaluate(g, prm, psi_m)
    assert rel(rep_m["E"], ev.E) < 1e-11
    for i in range(2):
        assert rel(rep_m["mu"][i], ev.mu[i]) < 1e-11
        assert abs(O.inner(g, psi_m[i], psi_m[i]).real - 1.0) < 1e-12
    r = np.stack([ev.Hpsi[i] - ev.mu[i] * psi_m[i] for i in range(2)])
    assert np.sqrt(sum(O.inner(g, r[i], r[i]).real for i in range(2))) < 1e-9
    assert rel(rep_m["E"], rep_d["E"]) < 1e-11


def test_c5_energy_grad_full_size(E):
    """256x256x128 (8.4M points): every gradient element and every energy term."""
    w = I.PRESETS["c5"]
    psi = I.gaussian_start(w)
    g, prm = oracle_case(w)
    ev = O.evaluate(g, prm, psi)
    h = _handle(E, w, E.EGPE_FP64)
    try:
        x = torch.from_numpy(psi).to("cuda")
        grad = torch.empty_like(x)
        t = E.egpe_energy_terms_eval(h, 0, x, grad)
        G = grad.cpu().numpy()
    finally:
        E.egpe_destroy(h)
    assert rel(t["E"], ev.E) < 1e-12
    for k in ("kin1", "kin2", "trap", "contact", "dipolar", "lhy"):
        assert abs(t[k] - ev.terms[k]) < 1e-11 * max(abs(ev.terms[k]), 1e-3 * abs(ev.E)), k
    assert np.max(np.abs(G - ev.Hpsi)) < 1e-11 * np.max(np.abs(ev.Hpsi))


def test_c3_mixed_solve_energy_against_oracle(E):
    """128x128x64 mixed precision: FP32 phase to 1e-4, FP64 polish to 1e-9.  The
    oracle evaluates the returned state: same energy, small residual, unit norms;
    and the FP64-only solve reaches the same energy."""
    w = I.PRESETS["c3"]
    psi0 = I.gaussian_start(w)
    g, prm = oracle_case(w)
    out = {}
    for prec in (E.EGPE_MIXED, E.EGPE_FP64):
        h = _handle(E, w, prec)
        try:
            o = E.egpe_default_solve_opts()
            o.precond = E.PRECOND["kinetic+diagonal"]
            o.tol_res = 1e-9
            o.tol_fp32_switch = 1e-4
            x = torch.from_numpy(psi0).to("cuda")
            st, reps, _ = E.egpe_ncg_solve(h, [x], o, 1)
            out[prec] = (reps[0], x.cpu().numpy())
        finally:
            E.egpe_destroy(h)
    rep_m, psi_m = out[E.EGPE_MIXED]
    rep_d, psi_d = out[E.EGPE_FP64]
    assert rep_m["status"] == 0 and rep_d["status"] == 0
    assert rep_m["iters_fp32"] > 0
    ev = O.evaluate(g, prm, psi_m)
    assert rel(rep_m["E"], ev.E) < 1e-12
    r = np.stack([ev.Hpsi[i] - ev.mu[i] * psi_m[i] for i in range(2)])
    res = np.sqrt(sum(O.inner(g, r[i], r[i]).real for i in range(2)))
    assert res < 1e-8
    for i in range(2):
        assert abs(O.inner(g, psi_m[i], psi_m[i]).real - 1.0) < 1e-12
    # both precisions land on the same minimum (unique up to the residual tolerance)
    assert rel(rep_m["E"], rep_d["E"]) < 1e-11


def test_c5_param_grad_full_size(E):
    """256x256x128: the parameter derivatives of the energy (the autograd
    extension on the largest workload) against the oracle at the seeded start."""
    w = I.PRESETS["c5"]
    psi = I.gaussian_start(w)
    g, prm = oracle_case(w)
    ref = O.param_grad(g, prm, psi)
    h = _handle(E, w, E.EGPE_FP64)
    try:
        d = E.egpe_param_grad(h, 0, torch.from_numpy(psi).to("cuda"))
    finally:
        E.egpe_destroy(h)
    for k, v in ref.items():
        assert abs(d[k] - v) < 1e-11 * max(abs(v), 1e-6), (k, d[k], v)
