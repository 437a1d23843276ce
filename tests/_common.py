"""Shared test helpers: oracle parameters and GPU handles built from the same
workload description (paper_2510_24543_gb300.inputs)."""
import math

import numpy as np

import oracle as O
from paper_2510_24543_gb300 import inputs as I


def oracle_case(w, nodes=None):
    g = O.Grid(w.n, w.L)
    prm = O.Params(w.g, w.gdd, w.kappa, w.eta_s, nodes or w.lhy_nodes, w.trap)
    return g, prm


def workload(name, n=None, L=None, nodes=None, seed=None, **kw):
    base = I.PRESETS[name]
    fields = dict(name=base.name, n=n or base.n, L=L or base.L, trap=base.trap, g=base.g, gdd=base.gdd,
                  lhy_c=base.lhy_c, seed=base.seed if seed is None else seed, precond=base.precond,
                  lhy_nodes=nodes or base.lhy_nodes)
    fields.update(kw)
    return I.Workload(**fields)


def mixed_workload(n, L=(4.0, 5.0, 3.0), seed=3):
    """Anisotropic grid and box with every coupling distinct (catches swapped
    indices and axes)."""
    return I.Workload("mixed", n, L, (1.0, 1.3, 1.9), ((310.0, 140.0), (140.0, 260.0)),
                      ((220.0, 90.0), (90.0, 180.0)), 35.0, seed, "kinetic", 12)


def gauge_fix(psi):
    """Multiply each component by the phase that makes it real and positive at
    its |psi|-argmax (ground states are compared up to a global phase)."""
    out = psi.copy()
    for i in range(psi.shape[0]):
        k = np.unravel_index(np.argmax(np.abs(psi[i])), psi[i].shape)
        out[i] *= np.exp(-1j * np.angle(psi[i][k]))
    return out


def rel(a, b):
    return abs(a - b) / max(abs(b), 1e-300)
