"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle on
identical seeded inputs, one row of the hot path at a time and then the whole
solver.  Tolerances (FP64 path): energies 1e-12 relative, fields 1e-11 of their
largest magnitude, final ground state 1e-11 relative energy and 1e-9 max|psi|
difference after a gauge fix.  FP32 fields are held to 2e-5 relative."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2510_24543_gb300 import inputs as I

from ._common import gauge_fix, mixed_workload, oracle_case, rel, workload

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


class Handle:
    def __init__(self, E, w, prec=0):
        self.E = E
        self.w = w
        self.h = E.egpe_create([E.make_grid(w.n, w.L)], [E.params_from_workload(w)], prec)
        self.cdtype = torch.complex64 if prec == 1 else torch.complex128

    def dev(self, a):
        return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=self.cdtype)

    def empty(self, nf=2):
        return torch.empty((nf,) + tuple(reversed(self.w.n)), dtype=self.cdtype, device="cuda")

    def close(self):
        self.E.egpe_destroy(self.h)
        self.h = None


def host(t):
    return t.detach().cpu().numpy().astype(np.complex128)


# ----------------------------------------------------------------- a1/a3: FFT
@pytest.mark.parametrize("n", [(16, 16, 16), (32, 16, 64), (64, 32, 16), (128, 64, 32), (256, 16, 32)])
@pytest.mark.parametrize("prec", [0, 1])
def test_fft_matches_numpy(E, n, prec):
    w = mixed_workload(n)
    H = Handle(E, w, prec)
    try:
        x = I.random_fields((3, n[2], n[1], n[0]), 40 + n[0])
        xd = H.dev(x)
        out = H.empty(3)
        E.egpe_fft(H.h, 0, xd, out, 3, inverse=False)
        ref = np.fft.fftn(x, axes=(1, 2, 3))
        tol = 1e-13 if prec == 0 else 3e-6
        assert np.max(np.abs(host(out) - ref)) < tol * np.max(np.abs(ref))
        back = H.empty(3)
        E.egpe_fft(H.h, 0, out, back, 3, inverse=True)
        refi = np.fft.ifftn(host(out), axes=(1, 2, 3)) * np.prod(n)
        assert np.max(np.abs(host(back) - refi)) < tol * np.max(np.abs(refi))
    finally:
        H.close()


# ----------------------------------------------------------------- a1-a6: energy and gradient
def _check_energy(H, w, psi, tolE=1e-12, tolG=1e-11):
    E = H.E
    g, prm = oracle_case(w)
    ev = O.evaluate(g, prm, psi)
    grad = H.empty()
    t = E.egpe_energy_terms_eval(H.h, 0, H.dev(psi), grad)
    for k in ("kin1", "kin2", "trap", "contact", "dipolar", "lhy"):
        scale = max(abs(ev.terms[k]), 1e-3 * abs(ev.E))
        assert abs(t[k] - ev.terms[k]) < tolE * scale * 10, (k, t[k], ev.terms[k])
    assert rel(t["E"], ev.E) < tolE, (t["E"], ev.E)
    for i in range(2):
        assert rel(t["mu"][i], ev.mu[i]) < tolE * 10
    G = host(grad)
    assert np.max(np.abs(G - ev.Hpsi)) < tolG * max(1.0, np.max(np.abs(ev.Hpsi)))
    return t, ev


def test_energy_grad_c1_start(E):
    w = I.PRESETS["c1"]
    H = Handle(E, w)
    try:
        _check_energy(H, w, I.gaussian_start(w))
    finally:
        H.close()


@pytest.mark.parametrize("n", [(32, 64, 16), (16, 32, 64), (64, 16, 32)])
def test_energy_grad_complex_anisotropic(E, n):
    w = mixed_workload(n)
    H = Handle(E, w)
    try:
        _check_energy(H, w, I.random_state(n, w.L, 17, width=(1.2, 1.5, 0.9)))
    finally:
        H.close()


def test_energy_grad_fp32_fields(E):
    w = I.PRESETS["c1"]
    H = Handle(E, w, prec=1)
    try:
        psi = I.gaussian_start(w)
        g, prm = oracle_case(w)
        ev = O.evaluate(g, prm, psi)
        grad = H.empty()
        t = E.egpe_energy_terms_eval(H.h, 0, H.dev(psi), grad)
        assert rel(t["E"], ev.E) < 2e-5
        assert np.max(np.abs(host(grad) - ev.Hpsi)) < 2e-5 * np.max(np.abs(ev.Hpsi))
    finally:
        H.close()


def test_energy_grad_full_size_headline_grid(E):
    """128^3 on the headline box: the full-size evaluation element by element."""
    w = I.PRESETS["c3p"]
    H = Handle(E, w)
    try:
        _check_energy(H, w, I.gaussian_start(w), tolE=1e-12, tolG=1e-11)
    finally:
        H.close()


# ----------------------------------------------------------------- a11: line-search coefficients
@pytest.mark.parametrize("case", ["c1", "mixed"])
def test_line_coeffs(E, case):
    if case == "c1":
        w = I.PRESETS["c1"]
        psi = I.gaussian_start(w)
    else:
        w = mixed_workload((32, 16, 64))
        psi = I.random_state(w.n, w.L, 21, width=(1.2, 1.5, 0.9))
    g, prm = oracle_case(w)
    p = O.project(g, psi, I.raw_direction(w.n, w.L, 22))
    H = Handle(E, w)
    try:
        c = E.egpe_line_coeffs(H.h, 0, H.dev(psi), H.dev(p))
        ref = O.line_coeffs(g, prm, psi, p)
        assert rel(c[0], ref[0]) < 1e-12
        assert abs(c[1] - ref[1]) < 1e-11 * max(1.0, abs(ref[1]))
        assert abs(c[2] - ref[2]) < 1e-11 * max(1.0, abs(ref[2]))
    finally:
        H.close()


# ----------------------------------------------------------------- a7/a8: preconditioners
@pytest.mark.parametrize("mode", ["none", "kinetic", "diagonal", "kinetic+diagonal", "blend"])
def test_precondition(E, mode):
    w = mixed_workload((32, 16, 64))
    psi = I.random_state(w.n, w.L, 31, width=(1.2, 1.5, 0.9))
    g, prm = oracle_case(w)
    ev = O.evaluate(g, prm, psi)
    r = np.stack([ev.Hpsi[i] - ev.mu[i] * psi[i] for i in range(2)])
    zref = O.precondition(g, prm, ev, psi, r, mode)
    H = Handle(E, w)
    try:
        z = H.empty()
        E.egpe_precondition(H.h, 0, E.PRECOND[mode], H.dev(psi), None, z)
        assert np.max(np.abs(host(z) - zref)) < 1e-11 * np.max(np.abs(zref))
        # given residual
        rr = I.random_fields(psi.shape, 32)
        z2 = H.empty()
        E.egpe_precondition(H.h, 0, E.PRECOND[mode], H.dev(psi), H.dev(rr), z2)
        zref2 = O.precondition(g, prm, ev, psi, rr, mode)
        assert np.max(np.abs(host(z2) - zref2)) < 1e-11 * np.max(np.abs(zref2))
    finally:
        H.close()


# ----------------------------------------------------------------- a12: retraction
def test_retract(E):
    w = mixed_workload((16, 32, 16))
    psi = I.random_state(w.n, w.L, 41)
    g, _ = oracle_case(w)
    p = O.project(g, psi, I.raw_direction(w.n, w.L, 42))
    H = Handle(E, w)
    try:
        out = H.empty()
        E.egpe_retract(H.h, 0, H.dev(psi), H.dev(p), (0.3, 1.2), out)
        ref = O.retract(g, psi, p, (0.3, 1.2))
        assert np.max(np.abs(host(out) - ref)) < 1e-13 * np.max(np.abs(ref))
    finally:
        H.close()


# ----------------------------------------------------------------- a9-a14: the whole solver
def _solve_gpu(E, w, psi0, precond, tol, prec=0, trace_cap=0, max_iter=2000, **kw):
    H = Handle(E, w, prec)
    try:
        o = E.egpe_default_solve_opts()
        o.precond = E.PRECOND[precond]
        o.tol_res = tol
        o.max_iter = max_iter
        for k, v in kw.items():
            setattr(o, k, v)
        x = H.dev(psi0) if prec != 2 else torch.from_numpy(psi0).to("cuda")
        st, reps, trace = E.egpe_ncg_solve(H.h, [x], o, 1, trace_cap=trace_cap)
        return st, reps[0], trace, host(x)
    finally:
        H.close()


@pytest.mark.parametrize("beta_rule", ["HS", "PR"])
def test_ncg_lockstep_first_iterations(E, beta_rule):
    """Per-iteration (E, ||r||, beta, alpha) of the first iterations against the oracle."""
    w = I.PRESETS["c1"]
    psi0 = I.gaussian_start(w)
    g, prm = oracle_case(w)
    otr = []
    O.ncg_solve(g, prm, psi0, O.SolveOpts(precond="kinetic", tol_res=1e-8, max_iter=12, beta_rule=beta_rule),
                trace=otr)
    st, rep, tr, _ = _solve_gpu(E, w, psi0, "kinetic", 1e-8, trace_cap=64, max_iter=12,
                                beta_rule=1 if beta_rule == "PR" else 0)
    acc = [t for t in tr if t["flags"] & 1]
    assert len(acc) >= 10
    oacc = [t for t in otr if t["accepted"]]
    for k in range(10):
        a, b = acc[k], oacc[k]
        assert a["n"] == b["n"]
        assert rel(a["E"], b["E"]) < 1e-11, k
        assert rel(a["res"], b["res"]) < 1e-8, k
        assert abs(a["beta"] - b["beta"]) < 1e-7 * max(1.0, abs(b["beta"])), k
        assert rel(a["alpha"], b["alpha"]) < 1e-7, k
        assert rel(a["E_trial"], b["E_new"]) < 1e-11, k


def test_ncg_lockstep_blended_preconditioner(E):
    """Weighted P_V / P_Delta combination (weight 0.3): iterations in lockstep."""
    w = I.PRESETS["c1"]
    psi0 = I.gaussian_start(w)
    g, prm = oracle_case(w)
    otr = []
    O.ncg_solve(g, prm, psi0, O.SolveOpts(precond="blend", blend=0.3, tol_res=1e-8, max_iter=8), trace=otr)
    st, rep, tr, _ = _solve_gpu(E, w, psi0, "blend", 1e-8, trace_cap=64, max_iter=8, pc_blend=0.3)
    acc = [t for t in tr if t["flags"] & 1]
    oacc = [t for t in otr if t["accepted"]]
    assert len(acc) == len(oacc) == 8
    for a, b in zip(acc, oacc):
        assert rel(a["E"], b["E"]) < 1e-11
        assert rel(a["res"], b["res"]) < 1e-8
        assert abs(a["beta"] - b["beta"]) < 1e-7 * max(1.0, abs(b["beta"]))
        assert rel(a["alpha"], b["alpha"]) < 1e-7


@pytest.mark.parametrize("precond", ["kinetic", "kinetic+diagonal"])
def test_ncg_ground_state_c1(E, precond):
    w = I.PRESETS["c1"]
    psi0 = I.gaussian_start(w)
    g, prm = oracle_case(w)
    psi_o, rep_o = O.ncg_solve(g, prm, psi0, O.SolveOpts(precond=precond, tol_res=1e-10))
    assert rep_o["status"] == "converged"
    st, rep, _, psi_g = _solve_gpu(E, w, psi0, precond, 1e-10)
    assert rep["status"] == 0, rep
    assert rep["res"] < 1e-10
    assert rel(rep["E"], rep_o["E"]) < 1e-11
    assert np.max(np.abs(gauge_fix(psi_g) - gauge_fix(psi_o))) < 1e-9
    for i in range(2):
        assert abs(O.inner(g, psi_g[i], psi_g[i]).real - 1.0) < 1e-12


def test_ncg_fp32_then_mixed_polish(E):
    """FP32 fields reach ~1e-4 residual; the mixed solve's FP64 polish then
    reaches the FP64 ground state."""
    w = I.PRESETS["c1"]
    psi0 = I.gaussian_start(w)
    g, prm = oracle_case(w)
    _, rep_o = O.ncg_solve(g, prm, psi0, O.SolveOpts(precond="kinetic+diagonal", tol_res=1e-10))
    st, rep, _, psi32 = _solve_gpu(E, w, psi0, "kinetic+diagonal", 1e-4, prec=1)
    assert rep["status"] == 0, rep
    assert rel(rep["E"], rep_o["E"]) < 1e-6
    st, rep, _, psi_m = _solve_gpu(E, w, psi0, "kinetic+diagonal", 1e-10, prec=2, tol_fp32_switch=1e-4)
    assert rep["status"] == 0, rep
    assert rep["iters_fp32"] > 0
    assert rel(rep["E"], rep_o["E"]) < 1e-11
