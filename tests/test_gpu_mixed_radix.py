"""GPU parity on the mixed-radix grid lengths 48, 80 and 96 (radix-3 and
radix-5 passes): transforms against numpy, every pipeline against the oracle on
uneven grids, and the first solver iterations on a 48^3 scan instance."""
import numpy as np
import pytest

import oracle as O
from paper_2510_24543_gb300 import inputs as I

from ._common import mixed_workload, oracle_case, rel

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
        self.prec = prec
        self.h = E.egpe_create([E.make_grid(w.n, w.L)], [E.params_from_workload(w)], prec)
        self.dt = torch.complex64 if prec == 1 else torch.complex128

    def dev(self, a):
        return torch.from_numpy(np.ascontiguousarray(a)).to("cuda").to(self.dt)

    def close(self):
        self.E.egpe_destroy(self.h)


def host(t):
    return t.detach().cpu().numpy().astype(np.complex128)


@pytest.mark.parametrize("n", [(48, 48, 48), (80, 96, 48), (96, 16, 80), (16, 80, 96), (48, 128, 80)])
@pytest.mark.parametrize("prec", [0, 1])
def test_fft_mixed_radix_matches_numpy(E, n, prec):
    w = mixed_workload(n)
    H = Handle(E, w, prec)
    try:
        x = I.random_fields((2, n[2], n[1], n[0]), 60 + n[0] + n[1])
        xd = H.dev(x)
        out = torch.empty_like(xd)
        E.egpe_fft(H.h, 0, xd, out, 2, inverse=False)
        ref = np.fft.fftn(x, axes=(1, 2, 3))
        tol = 1e-13 if prec == 0 else 3e-6
        assert np.max(np.abs(host(out) - ref)) < tol * np.max(np.abs(ref))
        back = torch.empty_like(xd)
        E.egpe_fft(H.h, 0, out, back, 2, inverse=True)
        refi = np.fft.ifftn(host(out), axes=(1, 2, 3)) * np.prod(n)
        assert np.max(np.abs(host(back) - refi)) < tol * np.max(np.abs(refi))
    finally:
        H.close()


@pytest.mark.parametrize("n", [(80, 96, 48), (48, 48, 96)])
def test_energy_grad_mixed_radix(E, n):
    w = mixed_workload(n)
    psi = I.random_state(n, w.L, 71, width=(1.2, 1.5, 0.9))
    g, prm = oracle_case(w)
    ev = O.evaluate(g, prm, psi)
    H = Handle(E, w)
    try:
        grad = torch.empty_like(H.dev(psi))
        t = E.egpe_energy_terms_eval(H.h, 0, H.dev(psi), grad)
        assert rel(t["E"], ev.E) < 1e-12
        for k in ("kin1", "kin2", "trap", "contact", "dipolar", "lhy"):
            assert abs(t[k] - ev.terms[k]) < 1e-11 * max(abs(ev.terms[k]), 1e-3 * abs(ev.E)), k
        assert np.max(np.abs(host(grad) - ev.Hpsi)) < 1e-11 * np.max(np.abs(ev.Hpsi))
    finally:
        H.close()


def test_line_coeffs_and_precondition_mixed_radix(E):
    n = (96, 48, 80)
    w = mixed_workload(n)
    psi = I.random_state(n, w.L, 81, width=(1.2, 1.5, 0.9))
    g, prm = oracle_case(w)
    ev = O.evaluate(g, prm, psi)
    p = O.project(g, psi, I.raw_direction(n, w.L, 82))
    H = Handle(E, w)
    try:
        c = E.egpe_line_coeffs(H.h, 0, H.dev(psi), H.dev(p))
        ref = O.line_coeffs(g, prm, psi, p, ev)
        assert rel(c[0], ref[0]) < 1e-12
        assert abs(c[1] - ref[1]) < 1e-11 * max(1.0, abs(ref[1]))
        assert abs(c[2] - ref[2]) < 1e-11 * max(1.0, abs(ref[2]))
        r = np.stack([ev.Hpsi[i] - ev.mu[i] * psi[i] for i in range(2)])
        for mode in ("kinetic", "kinetic+diagonal"):
            zref = O.precondition(g, prm, ev, psi, r, mode)
            z = torch.empty_like(H.dev(psi))
            E.egpe_precondition(H.h, 0, E.PRECOND[mode], H.dev(psi), None, z)
            assert np.max(np.abs(host(z) - zref)) < 1e-11 * np.max(np.abs(zref)), mode
    finally:
        H.close()


def test_ncg_lockstep_scan_instance_48(E):
    """First iterations of a 48^3 instance of the parameter scan, in lockstep."""
    w = I.scan_workloads()[3]
    assert w.n == (48, 48, 48)
    psi0 = I.gaussian_start(w)
    g, prm = oracle_case(w)
    otr = []
    O.ncg_solve(g, prm, psi0, O.SolveOpts(precond="kinetic", tol_res=1e-8, max_iter=6), trace=otr)
    H = Handle(E, w)
    try:
        o = E.egpe_default_solve_opts()
        o.precond = E.PRECOND["kinetic"]
        o.max_iter = 6
        st, reps, tr = E.egpe_ncg_solve(H.h, [H.dev(psi0)], o, 1, trace_cap=64)
    finally:
        H.close()
    acc = [t for t in tr if t["flags"] & 1]
    oacc = [t for t in otr if t["accepted"]]
    assert len(acc) == len(oacc) == 6
    for a, b in zip(acc, oacc):
        assert rel(a["E"], b["E"]) < 1e-11
        assert rel(a["E_trial"], b["E_new"]) < 1e-11
        assert rel(a["res"], b["res"]) < 1e-8
        assert rel(a["alpha"], b["alpha"]) < 1e-7


def test_ite_steps_mixed_radix(E):
    n = (48, 80, 48)
    w = mixed_workload(n)
    psi0 = I.gaussian_start(w)
    g, prm = oracle_case(w)
    psi_o, rep_o = O.ite_solve(g, prm, psi0, dtau=1e-3, tol_dE=0.0, max_steps=3)
    H = Handle(E, w)
    try:
        o = E.egpe_default_ite_opts()
        o.dtau = 1e-3
        o.tol_dE = 1e-300
        o.max_steps = 3
        x = H.dev(psi0)
        st, reps = E.egpe_ite_solve(H.h, [x], o)
        psi = host(x)
    finally:
        H.close()
    assert reps[0]["iters"] == 3
    assert rel(reps[0]["E"], rep_o["E"]) < 1e-12
    assert np.max(np.abs(psi - psi_o)) < 1e-12 * np.max(np.abs(psi_o))
