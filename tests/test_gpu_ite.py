"""GPU imaginary-time evolution (the baseline the paper compares NCG with,
Sec. VI.B) against the oracle's Strang-split ITE: states after a few steps
element by element, the step count to the |Delta E| stopping rule of Sec. VI.A,
and the ground state it reaches against the NCG solver's."""
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


def _ite(E, w, psi0, prec, dtau, tol_dE, max_steps, use_graph=1, poll=32):
    h = E.egpe_create([E.make_grid(w.n, w.L)], [E.params_from_workload(w)], prec)
    try:
        o = E.egpe_default_ite_opts()
        o.dtau = dtau
        o.tol_dE = tol_dE
        o.max_steps = max_steps
        o.use_graph = use_graph
        o.poll_every = poll
        dt = torch.complex64 if prec == E.EGPE_FP32 else torch.complex128
        x = torch.from_numpy(psi0).to("cuda").to(dt)
        st, reps = E.egpe_ite_solve(h, [x], o)
        return st, reps[0], x.cpu().numpy().astype(np.complex128)
    finally:
        E.egpe_destroy(h)


@pytest.mark.parametrize("case", ["c1", "mixed"])
@pytest.mark.parametrize("use_graph", [1, 0])
def test_ite_steps_match_oracle(E, case, use_graph):
    """Four Strang steps: every element of the state and the energy."""
    w = I.PRESETS["c1"] if case == "c1" else mixed_workload((32, 16, 64))
    psi0 = I.gaussian_start(w)
    g, prm = oracle_case(w)
    dtau = 1e-3
    psi_o, rep_o = O.ite_solve(g, prm, psi0, dtau=dtau, tol_dE=0.0, max_steps=4)
    st, rep, psi = _ite(E, w, psi0, E.EGPE_FP64, dtau, 1e-300, 4, use_graph=use_graph, poll=1)
    assert rep["status"] == 5  # not converged: the step limit ended it
    assert rep["iters"] == 4
    assert rep["ffts"] == 6 + 4 * 20
    assert rel(rep["E"], rep_o["E"]) < 1e-12
    for i in range(2):
        assert abs(rep["mu"][i] - rep_o["mu"][i]) < 1e-11 * abs(rep_o["mu"][i])
    assert np.max(np.abs(psi - psi_o)) < 1e-12 * np.max(np.abs(psi_o))


def test_ite_fp32_steps_match_oracle(E):
    """FP32 fields: the same four steps within single-precision round-off."""
    w = I.PRESETS["c1"]
    psi0 = I.gaussian_start(w)
    g, prm = oracle_case(w)
    psi_o, rep_o = O.ite_solve(g, prm, psi0, dtau=1e-3, tol_dE=0.0, max_steps=4)
    st, rep, psi = _ite(E, w, psi0, E.EGPE_FP32, 1e-3, 1e-300, 4)
    assert rep["iters"] == 4
    assert rel(rep["E"], rep_o["E"]) < 2e-6
    assert np.max(np.abs(psi - psi_o)) < 2e-5 * np.max(np.abs(psi_o))


def test_ite_stops_where_the_oracle_stops(E):
    """dtau = 0.01 to |E^{k+1} - E^k| < 1e-4: same step count, same state."""
    w = I.PRESETS["c1"]
    psi0 = I.gaussian_start(w)
    g, prm = oracle_case(w)
    psi_o, rep_o = O.ite_solve(g, prm, psi0, dtau=1e-2, tol_dE=1e-4, max_steps=1000)
    assert rep_o["status"] == "converged"
    st, rep, psi = _ite(E, w, psi0, E.EGPE_FP64, 1e-2, 1e-4, 1000)
    assert st == 0 and rep["status"] == 0
    assert rep["iters"] == rep_o["steps"]
    assert rel(rep["E"], rep_o["E"]) < 1e-11
    assert np.max(np.abs(psi - psi_o)) < 1e-10 * np.max(np.abs(psi_o))


def test_ite_and_ncg_reach_the_same_ground_state(E):
    """64^3 droplet couplings: ITE (dtau = 1e-3, |Delta E| < 1e-10) and NCG
    (||r|| < 1e-9) agree on the energy to 1e-6 relative (the paper's
    comparison criterion), and ITE never goes below the NCG minimum."""
    w = I.PRESETS["c2"]
    psi0 = I.gaussian_start(w)
    st, rep_i, psi_i = _ite(E, w, psi0, E.EGPE_FP64, 1e-3, 1e-10, 50000)
    assert rep_i["status"] == 0
    h = E.egpe_create([E.make_grid(w.n, w.L)], [E.params_from_workload(w)], E.EGPE_FP64)
    try:
        o = E.egpe_default_solve_opts()
        o.precond = E.PRECOND["kinetic+diagonal"]
        o.tol_res = 1e-9
        x = torch.from_numpy(psi0).to("cuda")
        st, reps, _ = E.egpe_ncg_solve(h, [x], o, 1)
        rep_c = reps[0]
    finally:
        E.egpe_destroy(h)
    assert rep_c["status"] == 0
    assert abs(rep_i["E"] - rep_c["E"]) < 1e-6 * abs(rep_c["E"])
    assert rep_i["E"] > rep_c["E"] - 1e-10 * abs(rep_c["E"])
    # the comparison the paper draws: NCG needs far fewer transforms
    assert rep_c["ffts"] < rep_i["ffts"]
