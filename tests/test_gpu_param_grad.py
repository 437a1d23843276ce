"""GPU parameter derivatives and the autograd binding: dE/d(g, g_dd, kappa,
eta_s, trap) against the oracle, parameter updates in place, the psi and
theta gradients of EnergyFn against central differences of GPU energies, and
the Hellmann-Feynman identity at converged ground states."""
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


def _theta(w):
    from paper_2510_24543_gb300 import autograd as AG
    return AG.params_vector(w.g, w.gdd, w.kappa, w.eta_s, w.trap)


def _check(d, ref, E_scale, tol):
    for k, v in ref.items():
        assert abs(d[k] - v) < tol * max(abs(v), 1e-3 * abs(E_scale)), (k, d[k], v)


@pytest.mark.parametrize("case", ["c1", "mixed"])
@pytest.mark.parametrize("prec", [0, 1])
def test_param_grad_matches_oracle(E, case, prec):
    if case == "c1":
        w = I.PRESETS["c1"]
        psi = I.gaussian_start(w)
    else:
        w = mixed_workload((48, 16, 32))
        psi = I.random_state(w.n, w.L, 91, width=(1.2, 1.5, 0.9))
    g, prm = oracle_case(w)
    ref = O.param_grad(g, prm, psi)
    Eref = O.evaluate(g, prm, psi).E
    h = E.egpe_create([E.make_grid(w.n, w.L)], [E.params_from_workload(w)], prec)
    try:
        dt = torch.complex64 if prec == E.EGPE_FP32 else torch.complex128
        d = E.egpe_param_grad(h, 0, torch.from_numpy(psi).to("cuda").to(dt))
    finally:
        E.egpe_destroy(h)
    _check(d, ref, Eref, 1e-11 if prec == E.EGPE_FP64 else 2e-5)


def test_set_params_in_place(E):
    w = mixed_workload((32, 16, 48))
    psi = I.random_state(w.n, w.L, 92)
    w2 = I.Workload("mixed2", w.n, w.L, (1.4, 0.8, 2.2), ((280.0, 90.0), (90.0, 240.0)),
                    ((150.0, 60.0), (60.0, 210.0)), 20.0, 3, "kinetic", w.lhy_nodes)
    g, prm2 = oracle_case(w2)
    h = E.egpe_create([E.make_grid(w.n, w.L)], [E.params_from_workload(w)], E.EGPE_MIXED)
    try:
        x = torch.from_numpy(psi).to("cuda")
        E.egpe_energy_grad(h, 0, x)  # evaluated once with the old parameters
        E.egpe_set_params(h, 0, E.params_from_workload(w2))
        Ev, _ = E.egpe_energy_grad(h, 0, x)
        d = E.egpe_param_grad(h, 0, x)
    finally:
        E.egpe_destroy(h)
    ev = O.evaluate(g, prm2, psi)
    assert rel(Ev, ev.E) < 1e-12
    _check(d, O.param_grad(g, prm2, psi), ev.E, 1e-11)


def test_autograd_psi_and_theta_against_differences(E):
    from paper_2510_24543_gb300 import autograd as AG
    w = mixed_workload((32, 16, 16))
    theta0 = _theta(w)
    model = AG.EnergyModel(w.n, w.L, theta0, nodes=w.lhy_nodes)
    try:
        psi = torch.from_numpy(I.random_state(w.n, w.L, 93)).to("cuda").requires_grad_(True)
        theta = theta0.clone().requires_grad_(True)
        model.energy(psi, theta).backward()
        delta = torch.from_numpy(I.random_fields(tuple(psi.shape), 94, scale=1e-2)).to("cuda")
        eps = 1e-3
        with torch.no_grad():
            Ep = model.energy(psi + eps * delta, theta0).item()
            Em = model.energy(psi - eps * delta, theta0).item()
        fd = (Ep - Em) / (2 * eps)
        lin = torch.sum(torch.conj(psi.grad) * delta).real.item()
        assert abs(fd - lin) < 1e-6 * max(abs(fd), 1e-6), (fd, lin)
        for k in (1, 4, 6, 7, 10):  # g12, gdd12, kappa, eta_s, trap_z
            hk = 1e-4 * abs(theta0[k].item())
            tp, tm = theta0.clone(), theta0.clone()
            tp[k] += hk
            tm[k] -= hk
            with torch.no_grad():
                fdk = (model.energy(psi, tp).item() - model.energy(psi, tm).item()) / (2 * hk)
            assert abs(fdk - theta.grad[k].item()) < 1e-6 * max(1.0, abs(fdk)), k
    finally:
        model.close()


def test_hellmann_feynman_at_ground_states(E):
    """dE0/dtheta from the ground-state energy's backward (the partial
    derivatives at psi*) against central differences of converged ground-state
    energies, on the 32^3 workload."""
    from paper_2510_24543_gb300 import autograd as AG
    w = I.PRESETS["c1"]
    theta0 = _theta(w)
    model = AG.EnergyModel(w.n, w.L, theta0, nodes=w.lhy_nodes)
    try:
        o = E.egpe_default_solve_opts()
        o.precond = E.PRECOND["kinetic+diagonal"]
        o.tol_res = 1e-11
        psi0 = torch.from_numpy(I.gaussian_start(w)).to("cuda")
        theta = theta0.clone().requires_grad_(True)
        model.ground_state_energy(psi0, theta, o).backward()
        for k in (1, 4, 6, 10):  # g12, gdd12, kappa, trap_z
            hk = 1e-4 * abs(theta0[k].item())
            tp, tm = theta0.clone(), theta0.clone()
            tp[k] += hk
            tm[k] -= hk
            with torch.no_grad():
                fd = (model.ground_state_energy(psi0, tp, o).item()
                      - model.ground_state_energy(psi0, tm, o).item()) / (2 * hk)
            assert abs(fd - theta.grad[k].item()) < 1e-6 * max(1.0, abs(fd)), (k, fd, theta.grad[k].item())
    finally:
        model.close()
