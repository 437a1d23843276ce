"""The boundary's error statuses, reached through the C ABI with failures made
on the host: a non-finite start (EGPE_ERR_NONFINITE), an acceptance rule that
no trial step can meet so the Armijo halvings run out (EGPE_ERR_STAGNATED, the
last paragraph of Sec. V), and a device wait budget of zero polls
(EGPE_ERR_TIMEOUT).  After each, the process and the GPU stay usable: a fresh
or restored handle solves normally.  The oracle takes the same decisions on
the same inputs."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2510_24543_gb300 import inputs as I

from ._common import oracle_case, workload

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


def _case():
    w = workload("c1", n=(16, 16, 16), nodes=16)
    return w, I.gaussian_start(w)


def _opts(E, **kw):
    o = E.egpe_default_solve_opts()
    o.precond = E.PRECOND["kinetic"]
    o.tol_res = 1e-8
    o.max_iter = 400
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def _solve(E, w, psi_np, prec, o):
    h = E.egpe_create([E.make_grid(w.n, w.L)], [E.params_from_workload(w)], prec)
    try:
        x = torch.from_numpy(psi_np).to("cuda").to(torch.complex64 if prec == 1 else torch.complex128)
        st, reps, tr = E.egpe_ncg_solve(h, [x], o, 1, trace_cap=8)
        rep = dict(reps[0])
        rep["trace"] = [{k: t[k] for k in ("n", "kind", "armijo", "flags", "E", "E_trial", "res", "beta", "alpha")}
                        for t in tr[:4]]
        return st, rep, x
    finally:
        E.egpe_destroy(h)


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_nonfinite_start(E, prec):
    w, psi = _case()
    bad = psi.copy()
    bad[0, 3, 4, 5] = np.nan
    st, rep, _ = _solve(E, w, bad, prec, _opts(E))
    assert st == 4 and rep["status"] == 4, rep
    g, prm = oracle_case(w)
    with np.errstate(invalid="ignore"):
        _, orep = O.ncg_solve(g, prm, bad, O.SolveOpts(precond="kinetic", tol_res=1e-8, max_iter=5))
    assert orep["status"] == "nonfinite"
    # the next solve on a fresh handle is unaffected (a tolerance above the
    # FP32 fields' round-off floor when there is an FP32 phase)
    st, rep, _ = _solve(E, w, psi, prec, _opts(E, tol_res=1e-6 if prec == 0 else 1e-4))
    assert st == 0 and rep["status"] == 0, rep


def test_stagnated_when_the_halvings_run_out(E):
    """accept_rtol = -0.9 asks every trial for a decrease of 90% of the
    energy, more than the ground state lies below the start, so no step along
    the geodesic is accepted: the first trial and armijo_max halvings are
    rejected and the solve ends STAGNATED after armijo_max + 1 trial
    evaluations, as in the oracle."""
    w, psi = _case()
    st, rep, _ = _solve(E, w, psi, 0, _opts(E, accept_rtol=-0.9, armijo_max=2))
    assert st == 6 and rep["status"] == 6, rep
    assert rep["attempts"] == 3 and rep["armijo_steps"] == 3 and rep["iters"] == 0
    g, prm = oracle_case(w)
    _, orep = O.ncg_solve(g, prm, psi, O.SolveOpts(precond="kinetic", tol_res=1e-8, accept_rtol=-0.9, armijo_max=2))
    assert orep["status"] == "stagnated" and orep["armijo_steps"] == 3 and orep["iters"] == 0


@pytest.mark.parametrize("prec", [0, 1])
def test_timeout_of_a_device_wait(E, prec):
    """With a wait budget of 0 polls every TMA tile wait of the column passes
    gives up at once; the pass lets its issued copies land (full budget), marks
    the run, and the solve and a standalone evaluation report
    EGPE_ERR_TIMEOUT.  Restoring the budget on the same handle, and a fresh
    handle, both solve normally."""
    w, psi = _case()
    grid, prm = E.make_grid(w.n, w.L), E.params_from_workload(w)
    h = E.egpe_create([grid], [prm], prec)
    cd = torch.complex64 if prec == 1 else torch.complex128
    try:
        E.egpe_set_wait_limit(h, 0)
        x = torch.from_numpy(psi).to("cuda").to(cd)
        st, reps, _ = E.egpe_ncg_solve(h, [x], _opts(E, tol_res=1e-4), 1)
        assert st == 7 and reps[0]["status"] == 7, reps[0]
        with pytest.raises(E.EgpeError) as ei:
            E.egpe_energy_grad(h, 0, x)
        assert ei.value.status == 7
        E.egpe_set_wait_limit(h, 1 << 20)
        x = torch.from_numpy(psi).to("cuda").to(cd)
        st, reps, _ = E.egpe_ncg_solve(h, [x], _opts(E, tol_res=1e-4), 1)
        assert st == 0 and reps[0]["status"] == 0
        E_restored = reps[0]["E"]
    finally:
        E.egpe_destroy(h)
    st, rep, _ = _solve(E, w, psi, prec, _opts(E, tol_res=1e-4))
    assert st == 0 and rep["status"] == 0, rep
    assert abs(rep["E"] - E_restored) <= 1e-12 * abs(E_restored)
