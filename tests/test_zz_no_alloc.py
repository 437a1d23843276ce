"""The allocation-free energy/gradient entry point against the handle-based one.

egpe_energy_grad_noalloc serves callers that cannot allocate device memory
(applications whose device memory belongs to their own pool allocator, and
loops that must stay out of the CUDA allocator); it keeps its workspace in a
fixed array inside the library.  This file is collected last so that a run
stopping at the first failure has already run every other test; it also
passes on its own in a fresh process.
"""
import numpy as np
import pytest

import oracle as O
from paper_2510_24543_gb300 import inputs as I

from ._common import oracle_case

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


def _case(n, complex_state):
    if complex_state:
        w = I.Workload("mixed", n, (4.0, 5.0, 3.0), (1.0, 1.3, 1.9), ((310.0, 140.0), (140.0, 260.0)),
                       ((220.0, 90.0), (90.0, 180.0)), 35.0, 3, "kinetic", 12)
        return w, I.random_state(n, w.L, 17, width=(1.2, 1.5, 0.9))
    w = I.PRESETS["c1"]
    return w, I.gaussian_start(w)


@pytest.mark.parametrize("n,complex_state", [((32, 32, 32), False), ((16, 32, 16), True)])
def test_noalloc_matches_handle_path_on_two_calls(E, n, complex_state):
    w, psi_np = _case(n, complex_state)
    grid = E.make_grid(w.n, w.L)
    prm = E.params_from_workload(w)
    psi = torch.from_numpy(psi_np).to("cuda")
    h = E.egpe_create([grid], [prm], E.EGPE_FP64)
    try:
        g_ref = torch.empty_like(psi)
        e_ref, mu_ref = E.egpe_energy_grad(h, 0, psi, g_ref)
    finally:
        E.egpe_destroy(h)
    scale = float(g_ref.abs().max())
    for call in range(2):
        g = torch.full_like(psi, float("nan"))
        e, mu = E.egpe_energy_grad_noalloc(grid, prm, psi, g)
        assert abs(e - e_ref) < 1e-12 * abs(e_ref), (call, e, e_ref)
        for i in range(2):
            assert abs(mu[i] - mu_ref[i]) < 1e-11 * abs(mu_ref[i])
        assert float((g - g_ref).abs().max()) < 1e-11 * scale, call
    # without a gradient output the energy is the same
    e2, _ = E.egpe_energy_grad_noalloc(grid, prm, psi, None)
    assert abs(e2 - e_ref) < 1e-12 * abs(e_ref)
    # and both agree with the FP64 oracle (Eq. 1 and the coupled eGPE)
    og, oprm = oracle_case(w)
    ev = O.evaluate(og, oprm, psi_np)
    assert abs(e - ev.E) < 1e-12 * abs(ev.E)
    for i in range(2):
        assert abs(mu[i] - ev.mu[i]) < 1e-11 * abs(ev.mu[i])
    hmax = float(np.max(np.abs(ev.Hpsi)))
    assert float(np.max(np.abs(g.cpu().numpy() - ev.Hpsi))) < 1e-11 * hmax


def test_noalloc_rejects_grids_beyond_its_workspace(E):
    w = I.PRESETS["c2"]  # 64^3 > 32^3
    grid = E.make_grid(w.n, w.L)
    prm = E.params_from_workload(w)
    psi = torch.zeros((2, 64, 64, 64), dtype=torch.complex128, device="cuda")
    with pytest.raises(E.EgpeError) as ei:
        E.egpe_energy_grad_noalloc(grid, prm, psi)
    assert ei.value.status == 1
    assert "32" in str(ei.value)


def test_noalloc_binding_rejects_mismatched_fields_before_any_launch(E):
    """The C entry point only sees pointers; the binding checks each tensor
    against the grid and raises before calling it."""
    w = I.PRESETS["c1"]
    grid = E.make_grid(w.n, w.L)
    prm = E.params_from_workload(w)
    with pytest.raises(ValueError, match="elements"):
        E.egpe_energy_grad_noalloc(grid, prm, torch.zeros((2, 16, 32, 32), dtype=torch.complex128, device="cuda"))
    with pytest.raises(ValueError, match="complex128"):
        E.egpe_energy_grad_noalloc(grid, prm, torch.zeros((2, 32, 32, 32), dtype=torch.complex64, device="cuda"))
    psi = torch.zeros((2, 32, 32, 32), dtype=torch.complex128, device="cuda")
    with pytest.raises(ValueError, match="grad"):
        E.egpe_energy_grad_noalloc(grid, prm, psi, torch.zeros((2, 32, 32, 16), dtype=torch.complex128,
                                                                  device="cuda"))
