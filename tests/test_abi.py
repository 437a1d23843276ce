"""Host-side checks of the C ABI (no GPU needed): the library builds for
sm_103a, loads, exports every function include/egpe.h declares, and rejects
invalid arguments before touching the device."""
import ctypes as ct
import os
import re

import pytest

from paper_2510_24543_gb300 import build as B
from paper_2510_24543_gb300 import egpe as E

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return E.load()


def declared_functions():
    with open(os.path.join(ROOT, "include", "egpe.h")) as f:
        src = f.read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(egpe_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("egpe_create", "egpe_energy_grad", "egpe_line_coeffs", "egpe_ncg_solve", "egpe_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_version_and_status_strings(lib):
    assert E.egpe_version() == 103
    for s in range(9):
        assert E.egpe_status_string(s)
    assert E.egpe_status_string(99) == "unknown status"


def test_default_options(lib):
    o = E.egpe_default_solve_opts()
    assert o.precond == 1 and o.restart_period == 20 and o.armijo_max == 30
    assert o.tol_res == 1e-8 and o.accept_rtol == 1e-13 and o.theta_max > 1.57


@pytest.mark.parametrize("n", [(12, 16, 16), (16, 16, 512), (8, 16, 16)])
def test_create_rejects_unsupported_grid_sizes(lib, n):
    g = E.make_grid(n, (1.0, 1.0, 1.0))
    p = E.make_params(((1, 0), (0, 1)), ((0, 0), (0, 0)), 0.0, 1.0, 4, (1, 1, 1))
    h = ct.c_void_p()
    st = lib.egpe_create(ct.byref(g), ct.byref(p), 1, 0, None, ct.byref(h))
    assert st == 1 and not h.value


def test_create_rejects_bad_parameters(lib):
    g = E.make_grid((16, 16, 16), (1.0, 1.0, 1.0))
    h = ct.c_void_p()
    bad = [
        E.make_params(((1, 2), (3, 1)), ((0, 0), (0, 0)), 0.0, 1.0, 4, (1, 1, 1)),   # asymmetric g
        E.make_params(((1, 0), (0, 1)), ((0, 1), (2, 0)), 0.0, 1.0, 4, (1, 1, 1)),   # asymmetric gdd
        E.make_params(((1, 0), (0, 1)), ((0, 0), (0, 0)), 0.0, 0.0, 4, (1, 1, 1)),   # eta_s = 0
        E.make_params(((1, 0), (0, 1)), ((0, 0), (0, 0)), 0.0, 1.0, 0, (1, 1, 1)),   # Q = 0
        E.make_params(((1, 0), (0, 1)), ((0, 0), (0, 0)), 0.0, 1.0, 65, (1, 1, 1)),  # Q too large
    ]
    for p in bad:
        assert lib.egpe_create(ct.byref(g), ct.byref(p), 1, 0, None, ct.byref(h)) == 1
    g2 = E.make_grid((16, 16, 16), (1.0, -1.0, 1.0))
    p = E.make_params(((1, 0), (0, 1)), ((0, 0), (0, 0)), 0.0, 1.0, 4, (1, 1, 1))
    assert lib.egpe_create(ct.byref(g2), ct.byref(p), 1, 0, None, ct.byref(h)) == 1
    assert lib.egpe_create(ct.byref(g), ct.byref(p), 0, 0, None, ct.byref(h)) == 1
    assert lib.egpe_create(ct.byref(g), ct.byref(p), 1, 7, None, ct.byref(h)) == 1


def test_null_handle_calls_are_rejected(lib):
    assert lib.egpe_energy_grad(None, 0, None, None, None, None) == 1
    assert lib.egpe_line_coeffs(None, 0, None, None, None) == 1
    assert lib.egpe_ncg_solve(None, None, None, None) == 1
    lib.egpe_destroy(None)


def test_binding_fails_loudly_without_the_library(tmp_path):
    import importlib
    mod = importlib.import_module("paper_2510_24543_gb300.egpe")
    saved = mod._lib
    try:
        mod._lib = None
        with pytest.raises(RuntimeError):
            mod.load(str(tmp_path / "missing.so"))
    finally:
        mod._lib = saved


def test_source_digest_ignores_the_machine_include_path(monkeypatch):
    """The digest that stamps builds and committed profiles names the sources
    and compiler options, not where the repository sits on a machine."""
    d0 = B._digest()
    monkeypatch.setattr(B, "FLAGS", [f if not f.startswith("-I") else "-I/elsewhere/include" for f in B.FLAGS])
    assert B._digest() == d0
    monkeypatch.setattr(B, "FLAGS", B.FLAGS + ["-DEXTRA"])
    assert B._digest() != d0


def test_wait_limit_rejects_bad_arguments(lib):
    assert lib.egpe_set_wait_limit(None, 5) == 1


def test_noalloc_binding_checks_fields_on_the_host(lib):
    """egpe_energy_grad_noalloc only receives pointers, so the binding checks
    the tensors against the grid before the call: device, dtype, contiguity
    and element count (a short buffer would be read out of bounds)."""
    torch = pytest.importorskip("torch")
    g = E.make_grid((16, 16, 16), (3.0, 3.0, 3.0))
    p = E.make_params(((1, 0), (0, 1)), ((0, 0), (0, 0)), 0.0, 1.0, 4, (1, 1, 1))
    with pytest.raises(ValueError, match="CUDA"):
        E.egpe_energy_grad_noalloc(g, p, torch.zeros((2, 16, 16, 16), dtype=torch.complex128))
    with pytest.raises(ValueError, match="torch CUDA tensor"):
        E.egpe_energy_grad_noalloc(g, p, 12345)


def test_binding_checks_handle_fields_on_the_host():
    """Tensor arguments of handle calls are checked against the handle's
    precision and grid before their pointers reach the library (host tensors
    stand in here for the psi_on_host case; device tensors get the same
    dtype and size checks)."""
    torch = pytest.importorskip("torch")
    h = 0xABC0
    E._HANDLES[h] = (E.EGPE_FP32, [(16, 16, 16), (32, 16, 16)])
    try:
        ok = torch.zeros((2, 16, 16, 16), dtype=torch.complex64)
        assert E._field(h, 0, ok, on_host=True) == ok.data_ptr()
        with pytest.raises(ValueError, match="complex64"):
            E._field(h, 0, ok.to(torch.complex128), on_host=True)
        with pytest.raises(ValueError, match="elements"):
            E._field(h, 1, ok, on_host=True)
        with pytest.raises(ValueError, match="CUDA"):
            E._field(h, 0, ok)
        with pytest.raises(ValueError, match="complex128"):
            E._field(h, 0, ok, on_host=True, engine=0)
        assert E._field(h, 0, 1234) == 1234  # raw pointers pass unchecked
    finally:
        E._HANDLES.pop(h, None)
