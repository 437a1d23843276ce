"""GPU: the launch-shape autotuner returns a shape for every kernel of an
attempt, never picks a shape slower than the untuned one it timed, and solves
after tuning reach the same result as untuned solves."""
import numpy as np
import pytest

from paper_2510_24543_gb300 import inputs as I

from ._common import rel

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


@pytest.mark.parametrize("prec", [0, 1])
def test_autotune_then_solve(E, prec):
    w = I.PRESETS["c2"]
    psi0 = I.gaussian_start(w)
    dt = torch.complex64 if prec == E.EGPE_FP32 else torch.complex128
    out = {}
    for tuned in (False, True):
        h = E.egpe_create([E.make_grid(w.n, w.L)], [E.params_from_workload(w)], prec)
        try:
            if tuned:
                res = E.egpe_autotune(h, 0, 0 if prec == E.EGPE_FP64 else 1, torch.from_numpy(psi0).to("cuda").to(dt),
                                      E.PRECOND["kinetic+diagonal"], reps=3)
                assert len(res) >= 8
                for r in res:
                    assert r["ms_best"] <= r["ms_default"] + 1e-9
                    assert (r["kind"] == 0 and r["choice"] >= 1) or (r["kind"] == 1 and r["choice"] in (0, 1))
            o = E.egpe_default_solve_opts()
            o.precond = E.PRECOND["kinetic+diagonal"]
            o.tol_res = 1e-9 if prec == E.EGPE_FP64 else 1e-4
            x = torch.from_numpy(psi0).to("cuda").to(dt)
            st, reps, _ = E.egpe_ncg_solve(h, [x], o, 1)
            out[tuned] = reps[0]
        finally:
            E.egpe_destroy(h)
    assert out[True]["status"] == 0 and out[False]["status"] == 0
    tol = 1e-12 if prec == E.EGPE_FP64 else 1e-6
    assert rel(out[True]["E"], out[False]["E"]) < tol
