"""GPU: the launch-shape autotuner returns a shape for every kernel of an
attempt (and one column tile width), never picks a shape slower than the
untuned one it timed, and solves after tuning reach the same result as untuned
solves; every column tile width gives the same gradient."""
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
                    assert ((r["kind"] == 0 and r["choice"] >= 1) or (r["kind"] == 1 and r["choice"] in (0, 1))
                            or (r["kind"] == 2 and r["choice"] in (64, 128, 256)))
                assert sum(r["kind"] == 2 for r in res) == 1
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


@pytest.mark.parametrize("prec", [0, 1])
def test_column_tile_widths_give_the_same_gradient(E, prec):
    """The tile width only regroups the columns of the y and z transforms: the
    gradient is bitwise the same at 64-, 128- and 256-byte tile rows, and the
    energy differs only by the grouping of its block partial sums."""
    w = I.PRESETS["c3p"]
    psi = torch.from_numpy(I.gaussian_start(w)).to("cuda")
    dt = torch.complex64 if prec == E.EGPE_FP32 else torch.complex128
    psi = psi.to(dt)
    res = {}
    for width in (128, 64, 256):
        h = E.egpe_create([E.make_grid(w.n, w.L)], [E.params_from_workload(w)], prec)
        try:
            E.egpe_set_tuning(h, 0, 0 if prec == E.EGPE_FP64 else 1, [{"key": "column tile row bytes", "choice": width}])
            g = torch.empty_like(psi)
            e, _ = E.egpe_energy_grad(h, 0, psi, g)
            res[width] = (e, g)
        finally:
            E.egpe_destroy(h)
    e0, g0 = res[128]
    tol = 1e-13 if prec == E.EGPE_FP64 else 1e-7
    for width in (64, 256):
        e, g = res[width]
        assert torch.equal(g, g0), width
        assert rel(e, e0) < tol, width
