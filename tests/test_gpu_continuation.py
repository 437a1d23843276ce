"""GPU continuation along a parameter path: every point reaches the ground
state a cold solve reaches, warm starts need fewer iterations in total, the
per-point states handed back are those ground states, and the oracle's
evaluation of the last one agrees."""
import numpy as np
import pytest

import oracle as O
from paper_2510_24543_gb300 import inputs as I

from ._common import oracle_case, rel

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


def _path(n=5):
    return [I.Workload(f"path{k}", (48, 48, 48), (10.0, 10.0, 10.0), (1.0, 1.0, 2.0),
                       ((400.0, g12), (g12, 400.0)), ((260.0, 260.0), (260.0, 260.0)), 60.0, 2100, "kinetic+diagonal",
                       16)
            for k, g12 in enumerate(np.linspace(120.0, 220.0, n))]


def test_continuation_matches_cold_solves(E):
    ws = _path()
    grid = E.make_grid(ws[0].n, ws[0].L)
    o = E.egpe_default_solve_opts()
    o.precond = E.PRECOND["kinetic+diagonal"]
    o.tol_res = 1e-9
    psi0 = torch.from_numpy(I.gaussian_start(ws[0])).to("cuda")
    cold = []
    h = E.egpe_create([grid], [E.params_from_workload(ws[0])], E.EGPE_FP64)
    try:
        for w in ws:
            E.egpe_set_params(h, 0, E.params_from_workload(w))
            x = psi0.clone()
            st, reps, _ = E.egpe_ncg_solve(h, [x], o, 1)
            cold.append(reps[0])
        E.egpe_set_params(h, 0, E.params_from_workload(ws[0]))
        x = psi0.clone()
        outs = [torch.empty_like(psi0) for _ in ws]
        st, warm = E.egpe_ncg_continuation(h, 0, [E.params_from_workload(w) for w in ws], x, o, psi_out=outs)
        assert st == 0
        for k, w in enumerate(ws):
            assert cold[k]["status"] == 0 and warm[k]["status"] == 0
            assert rel(warm[k]["E"], cold[k]["E"]) < 1e-10, k
            E.egpe_set_params(h, 0, E.params_from_workload(w))
            Ek, _ = E.egpe_energy_grad(h, 0, outs[k])
            assert rel(Ek, warm[k]["E"]) < 1e-13, k
        assert torch.equal(outs[-1], x)
        assert sum(r["iters"] for r in warm[1:]) < sum(r["iters"] for r in cold[1:])
    finally:
        E.egpe_destroy(h)
    g, prm = oracle_case(ws[-1])
    psi = outs[-1].cpu().numpy()
    ev = O.evaluate(g, prm, psi)
    assert rel(ev.E, warm[-1]["E"]) < 1e-12
    r = np.stack([ev.Hpsi[c] - ev.mu[c] * psi[c] for c in range(2)])
    assert np.sqrt(sum(O.inner(g, r[c], r[c]).real for c in range(2))) < 1e-8
