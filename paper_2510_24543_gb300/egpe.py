"""Thin ctypes binding of libegpe.so (include/egpe.h): argument marshalling only.

The functions keep the C names.  Field arguments are torch CUDA tensors of
shape (2, nz, ny, nx) (complex128 for FP64/MIXED handles, complex64 for FP32
handles) or raw device pointers; every step of the computation runs in the
library's CUDA kernels.  There is no fallback: if the library cannot be
loaded, every call raises.
"""
from __future__ import annotations

import ctypes as ct
import os
from typing import Optional, Sequence

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libegpe.so")

EGPE_OK = 0
STATUS = {0: "ok", 1: "invalid argument", 2: "CUDA error", 3: "out of device memory", 4: "non-finite value",
          5: "not converged", 6: "stagnated", 7: "timeout", 8: "unsupported"}
EGPE_FP64, EGPE_FP32, EGPE_MIXED = 0, 1, 2
PRECOND = {"none": 0, "kinetic": 1, "diagonal": 2, "kinetic+diagonal": 3, "blend": 4}
# order of egpe_param_grad's output (EGPE_P_*)
PARAM_NAMES = ("g11", "g12", "g22", "gdd11", "gdd12", "gdd22", "kappa", "eta_s", "trap_x", "trap_y", "trap_z")


class egpe_grid(ct.Structure):
    _fields_ = [("n", ct.c_int * 3), ("L", ct.c_double * 3)]


class egpe_params(ct.Structure):
    _fields_ = [("g", (ct.c_double * 2) * 2), ("gdd", (ct.c_double * 2) * 2), ("lhy_kappa", ct.c_double),
                ("lhy_eta_scale", ct.c_double), ("lhy_nodes", ct.c_int), ("trap", ct.c_double * 3)]


class egpe_energy_terms(ct.Structure):
    _fields_ = [("E", ct.c_double), ("kin", ct.c_double * 2), ("trap", ct.c_double), ("contact", ct.c_double),
                ("dipolar", ct.c_double), ("lhy", ct.c_double), ("mu", ct.c_double * 2),
                ("norm2", ct.c_double * 2), ("shift", ct.c_double * 2)]


class egpe_solve_opts(ct.Structure):
    _fields_ = [("precond", ct.c_int), ("beta_rule", ct.c_int), ("restart_period", ct.c_int),
                ("max_iter", ct.c_int), ("armijo_max", ct.c_int), ("poll_every", ct.c_int),
                ("use_graph", ct.c_int), ("psi_on_host", ct.c_int), ("tol_res", ct.c_double),
                ("tol_dE", ct.c_double), ("armijo_c1", ct.c_double), ("theta_max", ct.c_double),
                ("accept_rtol", ct.c_double), ("accept_rtol_fp32", ct.c_double), ("pv_floor", ct.c_double),
                ("tol_fp32_switch", ct.c_double), ("max_iter_fp32", ct.c_int), ("trace_cap", ct.c_int),
                ("trace", ct.c_void_p), ("batch", ct.c_int), ("stall_iters_fp32", ct.c_int),
                ("pc_blend", ct.c_double)]


class egpe_trace_entry(ct.Structure):
    _fields_ = [("n", ct.c_int), ("kind", ct.c_int), ("armijo", ct.c_int), ("flags", ct.c_int),
                ("E", ct.c_double), ("E_trial", ct.c_double), ("res", ct.c_double), ("beta", ct.c_double),
                ("alpha", ct.c_double), ("theta", ct.c_double * 2), ("Ep", ct.c_double), ("Epp", ct.c_double)]


class egpe_ite_opts(ct.Structure):
    _fields_ = [("dtau", ct.c_double), ("tol_dE", ct.c_double), ("max_steps", ct.c_int), ("poll_every", ct.c_int),
                ("use_graph", ct.c_int), ("psi_on_host", ct.c_int)]


class egpe_tuning(ct.Structure):
    _fields_ = [("key", ct.c_char * 160), ("name", ct.c_char * 48), ("L", ct.c_int), ("kind", ct.c_int),
                ("choice", ct.c_int), ("default_choice", ct.c_int), ("ms_best", ct.c_double),
                ("ms_default", ct.c_double)]


class egpe_report(ct.Structure):
    _fields_ = [("status", ct.c_int), ("iters", ct.c_int), ("iters_fp32", ct.c_int), ("attempts", ct.c_int),
                ("restarts", ct.c_int), ("armijo_steps", ct.c_int), ("trace_len", ct.c_int),
                ("graph_launches", ct.c_int), ("E", ct.c_double), ("mu", ct.c_double * 2), ("res", ct.c_double),
                ("seconds", ct.c_double), ("ffts", ct.c_longlong), ("kernels", ct.c_longlong)]


_lib = None

_SIGS = {
    "egpe_create": (ct.c_int, [ct.POINTER(egpe_grid), ct.POINTER(egpe_params), ct.c_int, ct.c_int, ct.c_void_p,
                               ct.POINTER(ct.c_void_p)]),
    "egpe_destroy": (None, [ct.c_void_p]),
    "egpe_energy_grad": (ct.c_int, [ct.c_void_p, ct.c_int, ct.c_void_p, ct.POINTER(ct.c_double),
                                    ct.POINTER(ct.c_double), ct.c_void_p]),
    "egpe_energy_terms_eval": (ct.c_int, [ct.c_void_p, ct.c_int, ct.c_void_p, ct.POINTER(egpe_energy_terms),
                                          ct.c_void_p]),
    "egpe_line_coeffs": (ct.c_int, [ct.c_void_p, ct.c_int, ct.c_void_p, ct.c_void_p, ct.POINTER(ct.c_double)]),
    "egpe_precondition": (ct.c_int, [ct.c_void_p, ct.c_int, ct.c_int, ct.c_void_p, ct.c_void_p, ct.c_void_p]),
    "egpe_retract": (ct.c_int, [ct.c_void_p, ct.c_int, ct.c_void_p, ct.c_void_p, ct.POINTER(ct.c_double),
                                ct.c_void_p]),
    "egpe_fft": (ct.c_int, [ct.c_void_p, ct.c_int, ct.c_void_p, ct.c_void_p, ct.c_int, ct.c_int]),
    "egpe_ncg_solve": (ct.c_int, [ct.c_void_p, ct.POINTER(ct.c_void_p), ct.POINTER(egpe_solve_opts),
                                  ct.POINTER(egpe_report)]),
    "egpe_profile_attempt": (ct.c_int, [ct.c_void_p, ct.c_int, ct.c_int, ct.c_void_p, ct.c_int, ct.c_int, ct.c_int,
                                        ct.c_char_p, ct.POINTER(ct.c_double), ct.POINTER(ct.c_double),
                                        ct.POINTER(ct.c_int)]),
    "egpe_solver_start": (ct.c_int, [ct.c_void_p, ct.c_int, ct.c_int, ct.c_void_p, ct.POINTER(egpe_solve_opts)]),
    "egpe_solver_step": (ct.c_int, [ct.c_void_p, ct.c_int, ct.c_int, ct.c_int]),
    "egpe_solver_read": (ct.c_int, [ct.c_void_p, ct.c_int, ct.c_int, ct.POINTER(egpe_report), ct.c_void_p]),
    "egpe_energy_grad_noalloc": (ct.c_int, [ct.POINTER(egpe_grid), ct.POINTER(egpe_params), ct.c_void_p,
                                            ct.POINTER(ct.c_double), ct.POINTER(ct.c_double), ct.c_void_p,
                                            ct.c_void_p]),
    "egpe_ite_solve": (ct.c_int, [ct.c_void_p, ct.POINTER(ct.c_void_p), ct.POINTER(egpe_ite_opts),
                                  ct.POINTER(egpe_report)]),
    "egpe_default_ite_opts": (None, [ct.POINTER(egpe_ite_opts)]),
    "egpe_param_grad": (ct.c_int, [ct.c_void_p, ct.c_int, ct.c_void_p, ct.POINTER(ct.c_double)]),
    "egpe_ncg_continuation": (ct.c_int, [ct.c_void_p, ct.c_int, ct.POINTER(egpe_params), ct.c_int, ct.c_void_p,
                                         ct.POINTER(ct.c_void_p), ct.POINTER(egpe_solve_opts),
                                         ct.POINTER(egpe_report)]),
    "egpe_set_params": (ct.c_int, [ct.c_void_p, ct.c_int, ct.POINTER(egpe_params)]),
    "egpe_autotune": (ct.c_int, [ct.c_void_p, ct.c_int, ct.c_int, ct.c_void_p, ct.c_int, ct.c_int,
                                 ct.POINTER(egpe_tuning), ct.c_int, ct.POINTER(ct.c_int)]),
    "egpe_set_tuning": (ct.c_int, [ct.c_void_p, ct.c_int, ct.c_int, ct.POINTER(egpe_tuning), ct.c_int]),
    "egpe_set_wait_limit": (ct.c_int, [ct.c_void_p, ct.c_longlong]),
    "egpe_lhy_table_eval": (ct.c_int, [ct.POINTER(egpe_params), ct.c_int, ct.c_int, ct.c_void_p, ct.c_void_p,
                                       ct.c_void_p, ct.c_void_p, ct.POINTER(ct.c_int)]),
    "egpe_default_solve_opts": (None, [ct.POINTER(egpe_solve_opts)]),
    "egpe_status_string": (ct.c_char_p, [ct.c_int]),
    "egpe_last_error": (ct.c_char_p, []),
    "egpe_version": (ct.c_int, []),
}


def load(path: Optional[str] = None):
    """Load libegpe.so (raises if it is missing: there is no fallback path)."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"libegpe.so not built ({p}); run paper_2510_24543_gb300.build.build()")
    lib = ct.CDLL(p)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class EgpeError(RuntimeError):
    def __init__(self, where: str, status: int):
        lib = load()
        msg = lib.egpe_last_error().decode(errors="replace")
        super().__init__(f"{where}: {STATUS.get(status, status)} ({msg})")
        self.status = status


def _check(where: str, status: int):
    if status != EGPE_OK:
        raise EgpeError(where, status)


def _ptr(x) -> int:
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("field tensors must be contiguous")
        return x.data_ptr()
    raise TypeError(type(x))


# Handles created through this binding: precision and grid sizes, so that
# tensor arguments can be checked before the library sees their pointers.
_HANDLES = {}


def _field(h: int, inst: int, t, name: str = "psi", nf: int = 2, engine: Optional[int] = None,
           on_host: bool = False):
    """Pointer of a field argument.  A tensor is checked against the handle:
    a CUDA tensor (a host tensor when on_host), contiguous, complex64 for the
    FP32 engine and complex128 otherwise, with nf*nx*ny*nz elements of
    instance inst's grid; ValueError otherwise.  Raw integer pointers are
    passed through unchecked."""
    if t is None or isinstance(t, int):
        return t
    info = _HANDLES.get(h)
    if info is not None and hasattr(t, "dtype"):
        prec, grids = info
        if not 0 <= inst < len(grids):
            raise ValueError(f"instance {inst} out of range")
        n = grids[inst]
        if engine is None:
            engine = 1 if prec == EGPE_FP32 else 0
        want_dtype = "torch.complex64" if engine == 1 else "torch.complex128"
        want = nf * n[0] * n[1] * n[2]
        if bool(t.is_cuda) == bool(on_host):
            raise ValueError(f"{name} must be a {'host' if on_host else 'CUDA'} tensor")
        if str(t.dtype) != want_dtype:
            raise ValueError(f"{name} must be {want_dtype[6:]} for this handle/engine, not {t.dtype}")
        if not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
        if t.numel() != want:
            raise ValueError(f"{name} has {t.numel()} elements; instance {inst} needs {want}")
    return _ptr(t)


def make_grid(n, L) -> egpe_grid:
    g = egpe_grid()
    for a in range(3):
        g.n[a] = int(n[a])
        g.L[a] = float(L[a])
    return g


def make_params(g, gdd, kappa, eta_s, nodes, trap) -> egpe_params:
    p = egpe_params()
    for i in range(2):
        for j in range(2):
            p.g[i][j] = float(g[i][j])
            p.gdd[i][j] = float(gdd[i][j])
    p.lhy_kappa = float(kappa)
    p.lhy_eta_scale = float(eta_s)
    p.lhy_nodes = int(nodes)
    for a in range(3):
        p.trap[a] = float(trap[a])
    return p


def egpe_create(grids: Sequence[egpe_grid], params: Sequence[egpe_params], prec: int = EGPE_FP64,
                stream: int = 0) -> int:
    lib = load()
    n = len(grids)
    G = (egpe_grid * n)(*grids)
    P = (egpe_params * n)(*params)
    h = ct.c_void_p()
    _check("egpe_create", lib.egpe_create(G, P, n, prec, ct.c_void_p(stream or None), ct.byref(h)))
    _HANDLES[h.value] = (prec, [tuple(g.n) for g in grids])
    return h.value


def egpe_destroy(h: int):
    if h:
        _HANDLES.pop(h, None)
        load().egpe_destroy(ct.c_void_p(h))


def egpe_energy_terms_eval(h: int, inst: int, psi, grad=None) -> dict:
    t = egpe_energy_terms()
    _check("egpe_energy_terms_eval",
           load().egpe_energy_terms_eval(ct.c_void_p(h), inst, ct.c_void_p(_field(h, inst, psi)), ct.byref(t),
                                         ct.c_void_p(_field(h, inst, grad, "grad"))))
    return dict(E=t.E, kin1=t.kin[0], kin2=t.kin[1], trap=t.trap, contact=t.contact, dipolar=t.dipolar,
                lhy=t.lhy, mu=(t.mu[0], t.mu[1]), norm2=(t.norm2[0], t.norm2[1]), shift=(t.shift[0], t.shift[1]))


def egpe_energy_grad(h: int, inst: int, psi, grad=None):
    E = ct.c_double()
    mu = (ct.c_double * 2)()
    _check("egpe_energy_grad", load().egpe_energy_grad(ct.c_void_p(h), inst, ct.c_void_p(_field(h, inst, psi)),
                                                       ct.byref(E), mu, ct.c_void_p(_field(h, inst, grad, "grad"))))
    return E.value, (mu[0], mu[1])


def _check_field(name: str, t, grid: egpe_grid, dtype_name: str):
    """Host-side check that a field tensor matches the grid it is used with:
    a CUDA tensor of the given complex dtype, contiguous, with 2*nx*ny*nz
    elements.  The C entry points receive bare pointers and cannot check this."""
    if not hasattr(t, "data_ptr") or not hasattr(t, "is_cuda"):
        raise ValueError(f"{name} must be a torch CUDA tensor, not {type(t).__name__}")
    want = 2 * grid.n[0] * grid.n[1] * grid.n[2]
    if not t.is_cuda:
        raise ValueError(f"{name} must live on a CUDA device")
    if str(t.dtype) != "torch." + dtype_name:
        raise ValueError(f"{name} must be {dtype_name}, not {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if t.numel() != want:
        raise ValueError(f"{name} has {t.numel()} elements; the grid needs 2*nx*ny*nz = {want}")


def egpe_energy_grad_noalloc(grid: egpe_grid, params: egpe_params, psi, grad=None, stream: int = 0):
    """Energy and gradient with the library's fixed workspace (no device
    allocation; at most 32 points per axis).  psi (and grad, if given) must be
    contiguous complex128 CUDA tensors of 2*nx*ny*nz elements: checked here,
    before the call, since the library only sees pointers.  Returns (E, (mu1, mu2))."""
    _check_field("psi", psi, grid, "complex128")
    if grad is not None:
        _check_field("grad", grad, grid, "complex128")
    E = ct.c_double()
    mu = (ct.c_double * 2)()
    _check("egpe_energy_grad_noalloc",
           load().egpe_energy_grad_noalloc(ct.byref(grid), ct.byref(params), ct.c_void_p(_ptr(psi)), ct.byref(E), mu,
                                           ct.c_void_p(_ptr(grad)), ct.c_void_p(stream or None)))
    return E.value, (mu[0], mu[1])


def egpe_line_coeffs(h: int, inst: int, psi, p):
    c = (ct.c_double * 3)()
    _check("egpe_line_coeffs", load().egpe_line_coeffs(ct.c_void_p(h), inst, ct.c_void_p(_field(h, inst, psi)),
                                                       ct.c_void_p(_field(h, inst, p, "p")), c))
    return c[0], c[1], c[2]


def egpe_precondition(h: int, inst: int, mode: int, psi, r, z):
    _check("egpe_precondition", load().egpe_precondition(ct.c_void_p(h), inst, int(mode),
                                                         ct.c_void_p(_field(h, inst, psi)),
                                                         ct.c_void_p(_field(h, inst, r, "r")),
                                                         ct.c_void_p(_field(h, inst, z, "z"))))


def egpe_retract(h: int, inst: int, psi, p, theta, out):
    th = (ct.c_double * 2)(float(theta[0]), float(theta[1]))
    _check("egpe_retract", load().egpe_retract(ct.c_void_p(h), inst, ct.c_void_p(_field(h, inst, psi)),
                                               ct.c_void_p(_field(h, inst, p, "p")), th,
                                               ct.c_void_p(_field(h, inst, out, "out"))))


def egpe_fft(h: int, inst: int, x, out, nfields: int, inverse: bool = False):
    _check("egpe_fft", load().egpe_fft(ct.c_void_p(h), inst, ct.c_void_p(_field(h, inst, x, "x", int(nfields))),
                                       ct.c_void_p(_field(h, inst, out, "out", int(nfields))),
                                       int(nfields), 1 if inverse else 0))


def egpe_profile_attempt(h: int, inst: int, engine: int, psi, precond: int, reps: int = 5, cap: int = 64):
    """[(name, mean ms, algorithmic bytes)] for every kernel of one solver attempt."""
    names = ct.create_string_buffer(48 * cap)
    ms = (ct.c_double * cap)()
    by = (ct.c_double * cap)()
    n = ct.c_int()
    _check("egpe_profile_attempt", load().egpe_profile_attempt(ct.c_void_p(h), inst, engine,
                                                               ct.c_void_p(_field(h, inst, psi, engine=engine)),
                                                               int(precond), int(reps), cap, names, ms, by,
                                                               ct.byref(n)))
    raw = names.raw
    out = []
    for k in range(n.value):
        nm = raw[48 * k:48 * (k + 1)].split(b"\0", 1)[0].decode()
        out.append((nm, ms[k], by[k]))
    return out


def egpe_default_solve_opts() -> egpe_solve_opts:
    o = egpe_solve_opts()
    load().egpe_default_solve_opts(ct.byref(o))
    return o


def egpe_ncg_solve(h: int, psis, opts: egpe_solve_opts, n_inst: int = 1, trace_cap: int = 0):
    """Runs the solver in place on psis (list of tensors/pointers).  Returns
    (status, [report dicts], [trace dicts of instance 0])."""
    lib = load()
    ptrs = (ct.c_void_p * n_inst)(*[ct.c_void_p(_field(h, i, x, on_host=bool(opts.psi_on_host)))
                                    for i, x in enumerate(psis)])
    reps = (egpe_report * n_inst)()
    tr = None
    if trace_cap > 0:
        tr = (egpe_trace_entry * trace_cap)()
        opts.trace = ct.cast(tr, ct.c_void_p)
        opts.trace_cap = trace_cap
    status = lib.egpe_ncg_solve(ct.c_void_p(h), ptrs, ct.byref(opts), reps)
    if status in (1, 2, 3):
        raise EgpeError("egpe_ncg_solve", status)
    out = [_report_dict(r) for r in reps]
    trace = []
    if tr is not None:
        for k in range(out[0]["trace_len"]):
            e = tr[k]
            trace.append(dict(n=e.n, kind=e.kind, armijo=e.armijo, flags=e.flags, E=e.E, E_trial=e.E_trial,
                              res=e.res, beta=e.beta, alpha=e.alpha, theta=(e.theta[0], e.theta[1]), Ep=e.Ep,
                              Epp=e.Epp))
    return status, out, trace


def egpe_default_ite_opts() -> egpe_ite_opts:
    o = egpe_ite_opts()
    load().egpe_default_ite_opts(ct.byref(o))
    return o


def egpe_ite_solve(h: int, psis, opts: egpe_ite_opts, n_inst: int = 1):
    """Imaginary-time evolution in place on psis.  Returns (status, [report dicts])."""
    lib = load()
    ptrs = (ct.c_void_p * n_inst)(*[ct.c_void_p(_field(h, i, x, on_host=bool(opts.psi_on_host)))
                                    for i, x in enumerate(psis)])
    reps = (egpe_report * n_inst)()
    status = lib.egpe_ite_solve(ct.c_void_p(h), ptrs, ct.byref(opts), reps)
    if status in (1, 2, 3):
        raise EgpeError("egpe_ite_solve", status)
    return status, [_report_dict(r) for r in reps]


def egpe_ncg_continuation(h: int, inst: int, path, psi, opts: egpe_solve_opts, psi_out=None):
    """Ground states along a parameter path (list of egpe_params), each solve
    warm-started from the previous one.  Returns (status, [report dicts])."""
    n = len(path)
    P = (egpe_params * n)(*path)
    outs = None
    if psi_out is not None:
        outs = (ct.c_void_p * n)(*[ct.c_void_p(_field(h, inst, x, "psi_out", on_host=bool(opts.psi_on_host)))
                                   for x in psi_out])
    reps = (egpe_report * n)()
    status = load().egpe_ncg_continuation(ct.c_void_p(h), inst, P, n,
                                          ct.c_void_p(_field(h, inst, psi, on_host=bool(opts.psi_on_host))), outs,
                                          ct.byref(opts),
                                          reps)
    if status in (1, 2, 3):
        raise EgpeError("egpe_ncg_continuation", status)
    return status, [_report_dict(r) for r in reps]


def egpe_param_grad(h: int, inst: int, psi) -> dict:
    """dE/dp at fixed psi for p in PARAM_NAMES."""
    out = (ct.c_double * len(PARAM_NAMES))()
    _check("egpe_param_grad", load().egpe_param_grad(ct.c_void_p(h), inst, ct.c_void_p(_field(h, inst, psi)), out))
    return {k: out[i] for i, k in enumerate(PARAM_NAMES)}


def egpe_set_params(h: int, inst: int, params: egpe_params) -> None:
    _check("egpe_set_params", load().egpe_set_params(ct.c_void_p(h), inst, ct.byref(params)))


def egpe_autotune(h: int, inst: int, engine: int, psi, precond: int, reps: int = 5, cap: int = 64):
    """Tunes the instance's launch shapes from psi; returns one dict per kernel."""
    arr = (egpe_tuning * cap)()
    n = ct.c_int(0)
    _check("egpe_autotune", load().egpe_autotune(ct.c_void_p(h), inst, engine,
                                                 ct.c_void_p(_field(h, inst, psi, engine=engine)), precond,
                                                 reps, arr, cap, ct.byref(n)))
    return [dict(key=t.key.decode(), name=t.name.decode(), L=t.L, kind=t.kind, choice=t.choice,
                 default_choice=t.default_choice, ms_best=t.ms_best, ms_default=t.ms_default)
            for t in arr[:n.value]]


def egpe_set_tuning(h: int, inst: int, engine: int, entries) -> None:
    """Applies tuned shapes (dicts with key and choice)."""
    arr = (egpe_tuning * max(1, len(entries)))()
    for k, e in enumerate(entries):
        arr[k].key = e["key"].encode()[:159]
        arr[k].choice = int(e["choice"])
    _check("egpe_set_tuning", load().egpe_set_tuning(ct.c_void_p(h), inst, engine, arr, len(entries)))


def egpe_lhy_table_eval(params: egpe_params, n1, n2, precision: int = 0):
    """The LHY interpolation tables of the engine of `precision` (EGPE_FP64 or
    EGPE_FP32), plus its exact nodes, evaluated on the host at points
    (n1[k], n2[k]): returns (mu (count, 2), hess (count, 3), (intervals per
    half, exact nodes))."""
    import numpy as np
    a = np.ascontiguousarray(n1, dtype=np.float64).ravel()
    b = np.ascontiguousarray(n2, dtype=np.float64).ravel()
    if a.shape != b.shape:
        raise ValueError("n1 and n2 must have the same size")
    mu = np.empty((a.size, 2))
    hs = np.empty((a.size, 3))
    info = (ct.c_int * 2)()
    _check("egpe_lhy_table_eval", load().egpe_lhy_table_eval(ct.byref(params), int(precision), a.size, a.ctypes.data,
                                                             b.ctypes.data, mu.ctypes.data, hs.ctypes.data, info))
    return mu, hs, (info[0], info[1])


def egpe_set_wait_limit(h: int, polls: int) -> None:
    """Poll budget of the device-side TMA waits of every engine of the handle."""
    _check("egpe_set_wait_limit", load().egpe_set_wait_limit(ct.c_void_p(h), int(polls)))


def _report_dict(r) -> dict:
    return dict(status=r.status, iters=r.iters, iters_fp32=r.iters_fp32, attempts=r.attempts, restarts=r.restarts,
                armijo_steps=r.armijo_steps, trace_len=r.trace_len, graph_launches=r.graph_launches, E=r.E,
                mu=(r.mu[0], r.mu[1]), res=r.res, seconds=r.seconds, ffts=r.ffts, kernels=r.kernels)


def egpe_solver_start(h: int, inst: int, engine: int, psi, opts: egpe_solve_opts):
    _check("egpe_solver_start", load().egpe_solver_start(ct.c_void_p(h), inst, engine,
                                                         ct.c_void_p(_field(h, inst, psi, engine=engine)),
                                                         ct.byref(opts)))


def egpe_solver_step(h: int, inst: int, engine: int, attempts: int):
    _check("egpe_solver_step", load().egpe_solver_step(ct.c_void_p(h), inst, engine, int(attempts)))


def egpe_solver_read(h: int, inst: int, engine: int, psi_out=None) -> dict:
    r = egpe_report()
    _check("egpe_solver_read", load().egpe_solver_read(ct.c_void_p(h), inst, engine, ct.byref(r),
                                                       ct.c_void_p(_field(h, inst, psi_out, "psi_out",
                                                                          engine=engine))))
    return _report_dict(r)


def egpe_status_string(s: int) -> str:
    return load().egpe_status_string(int(s)).decode()


def egpe_version() -> int:
    return load().egpe_version()


def params_from_workload(w) -> egpe_params:
    """C parameter struct of a workload from paper_2510_24543_gb300.inputs."""
    return make_params(w.g, w.gdd, w.kappa, w.eta_s, w.lhy_nodes, w.trap)
