"""Seeded synthetic inputs and workload presets.

This module only *prepares* inputs: grid/box sizes, coupling constants and the
seeded initial wave functions of the workloads.  It holds none of the method's
arithmetic (no energy, no Hamiltonian, no FFT), so both the CUDA path and the
FP64 CPU oracle can be fed from it without sharing any computation.

Workloads (the paper's Cr/Dy parameter sets are incomplete, Sec. VI.A, so these
synthetic sets stand in for them; every array is generated from a seed):

* ``c1``  32^3 on [-8,8]^3, trap (1,1,2), g = 400/400/250, g_dd = 300, LHY c = 50
* ``c2``  64^3 on [-10,10]^3, trap (1,1,3), g = 200/200/150, g_dd = 350, c = 80
* ``c3``  128x128x64 on [-16,16]^2 x [-8,8], trap (0.5,1,2), g = 300/300/280,
          g_dd = 420/420/400, c = 100
* ``c3p`` the same physics on 128^3 (z resolution doubled) -- the headline size
* ``c5``  256x256x128 on [-24,24]^2 x [-12,12], trap (0.4,0.8,2), g = 350/350/300,
          g_dd = 450, c = 120
* ``scan`` 64 instances (16 each of 48^3, 64^3, 80^3, 96^3) on [-10,10]^3 with a
          seeded Latin hypercube over g12 in [100,350] and g_dd in [250,450].

Couplings are in per-particle normalised form (each component normalised to 1,
Eq. 1 with N_i -> 1).  ``g_dd`` is the k-space dipolar coefficient, i.e. the
dipolar kernel in Fourier space is g_dd (3 k_z^2/|k|^2 - 1).  The LHY strength
"c" of a workload is mapped to the functional's prefactor kappa = 2c/5 with
eta_s = g11 + g22, which makes the single-component, non-dipolar limit the
familiar mu_LHY = c n^{3/2} when g11 = g22 (Eq. 1 LHY term, Sec. II).
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Dict, List, Tuple

import numpy as np


@dataclass(frozen=True)
class Workload:
    """One eGPE instance: grid, box, couplings and the seeded start."""

    name: str
    n: Tuple[int, int, int]          # (nx, ny, nz); arrays are stored (2, nz, ny, nx)
    L: Tuple[float, float, float]    # periodic box [-L_a, L_a)
    trap: Tuple[float, float, float]  # (lambda_x, lambda_y, lambda_z)
    g: Tuple[Tuple[float, float], Tuple[float, float]]
    gdd: Tuple[Tuple[float, float], Tuple[float, float]]
    lhy_c: float
    seed: int
    precond: str = "kinetic"         # kinetic | diagonal | kinetic+diagonal | none
    lhy_nodes: int = 32

    @property
    def kappa(self) -> float:
        return 0.4 * self.lhy_c

    @property
    def eta_s(self) -> float:
        return self.g[0][0] + self.g[1][1]

    @property
    def points(self) -> int:
        return self.n[0] * self.n[1] * self.n[2]


def _sym(a11: float, a22: float, a12: float):
    return ((float(a11), float(a12)), (float(a12), float(a22)))


PRESETS: Dict[str, Workload] = {
    "c1": Workload("c1 32^3 plain FP64", (32, 32, 32), (8.0, 8.0, 8.0), (1.0, 1.0, 2.0),
                   _sym(400, 400, 250), _sym(300, 300, 300), 50.0, 1001, "kinetic"),
    "c2": Workload("c2 64^3 droplet", (64, 64, 64), (10.0, 10.0, 10.0), (1.0, 1.0, 3.0),
                   _sym(200, 200, 150), _sym(350, 350, 350), 80.0, 1002, "kinetic+diagonal"),
    "c3": Workload("c3 128x128x64 stripe/supersolid", (128, 128, 64), (16.0, 16.0, 8.0),
                   (0.5, 1.0, 2.0), _sym(300, 300, 280), _sym(420, 420, 400), 100.0, 1003,
                   "kinetic+diagonal"),
    "c3p": Workload("c3' 128^3 stripe/supersolid", (128, 128, 128), (16.0, 16.0, 8.0),
                    (0.5, 1.0, 2.0), _sym(300, 300, 280), _sym(420, 420, 400), 100.0, 1003,
                    "kinetic+diagonal"),
    "c5": Workload("c5 256x256x128 supersolid", (256, 256, 128), (24.0, 24.0, 12.0),
                   (0.4, 0.8, 2.0), _sym(350, 350, 300), _sym(450, 450, 450), 120.0, 1005,
                   "kinetic+diagonal"),
}


def scan_workloads(count: int = 64, seed: int = 4242) -> List[Workload]:
    """Latin-hypercube parameter scan: 16 each of 48^3, 64^3, 80^3, 96^3.

    Axis samples: an independent permutation pi of 0..count-1 per axis and
    sample_k = lo + (pi[k] + U_k)/count * (hi - lo).  Instance k gets grid
    index floor(k / (count/4)) and noise seed 2000 + k.
    """
    rng = np.random.default_rng(seed)
    out = []
    ranges = [(100.0, 350.0), (250.0, 450.0)]
    samples = []
    for lo, hi in ranges:
        perm = rng.permutation(count)
        u = rng.random(count)
        samples.append(lo + (perm + u) / count * (hi - lo))
    sizes = [48, 64, 80, 96]
    per = count // len(sizes)
    for k in range(count):
        s = sizes[min(k // per, len(sizes) - 1)]
        g12, gdd = float(samples[0][k]), float(samples[1][k])
        out.append(Workload(f"scan[{k}] {s}^3", (s, s, s), (10.0, 10.0, 10.0), (1.0, 1.0, 2.0),
                            _sym(400, 400, g12), _sym(gdd, gdd, gdd), 60.0, 2000 + k,
                            "kinetic+diagonal"))
    return out


def axes(n, L):
    """Grid coordinates x_a[j] = -L_a + j*2L_a/n_a for a = x, y, z."""
    return [(-L[a] + np.arange(n[a]) * (2.0 * L[a] / n[a])) for a in range(3)]


def gaussian_start(w: Workload, noise: float = 0.01, seed: int | None = None) -> np.ndarray:
    """Seeded start psi_j = G (1 + noise*xi_j), each component normalised.

    G is the product of the 1D harmonic-oscillator ground states of the trap,
    prod_a (lambda_a/pi)^{1/4} exp(-lambda_a x_a^2 / 2); xi ~ N(0,1) i.i.d. per
    point from numpy.random.default_rng(seed).standard_normal((2,nz,ny,nx)).
    Returns complex128 of shape (2, nz, ny, nx).
    """
    n, L = w.n, w.L
    xs = axes(n, L)
    gx = [(w.trap[a] / np.pi) ** 0.25 * np.exp(-0.5 * w.trap[a] * xs[a] ** 2) for a in range(3)]
    G = gx[2][:, None, None] * gx[1][None, :, None] * gx[0][None, None, :]
    rng = np.random.default_rng(w.seed if seed is None else seed)
    xi = rng.standard_normal((2, n[2], n[1], n[0]))
    psi = (G[None] * (1.0 + noise * xi)).astype(np.complex128)
    return normalise(psi, n, L)


def normalise(psi: np.ndarray, n, L) -> np.ndarray:
    dV = (2.0 * L[0] / n[0]) * (2.0 * L[1] / n[1]) * (2.0 * L[2] / n[2])
    out = psi.copy()
    for i in range(out.shape[0]):
        out[i] /= np.sqrt(dV * np.sum(np.abs(out[i]) ** 2))
    return out


def random_fields(shape, seed: int, complex_: bool = True, scale: float = 1.0) -> np.ndarray:
    """Seeded smooth-free random complex (or real) fields of the given shape."""
    rng = np.random.default_rng(seed)
    a = rng.standard_normal(shape)
    if complex_:
        a = a + 1j * rng.standard_normal(shape)
    return (scale * a).astype(np.complex128)


def random_state(n, L, seed: int, width=(1.0, 1.0, 1.0), phase: bool = True) -> np.ndarray:
    """Seeded complex test state: a Gaussian envelope times random amplitude and
    phase per point, normalised per component (exercises the complex arithmetic
    that real ground-state inputs never reach)."""
    xs = axes(n, L)
    env = (np.exp(-0.5 * (xs[2][:, None, None] / width[2]) ** 2)
           * np.exp(-0.5 * (xs[1][None, :, None] / width[1]) ** 2)
           * np.exp(-0.5 * (xs[0][None, None, :] / width[0]) ** 2))
    rng = np.random.default_rng(seed)
    amp = 1.0 + 0.3 * rng.standard_normal((2, n[2], n[1], n[0]))
    ph = rng.uniform(-np.pi, np.pi, (2, n[2], n[1], n[0])) if phase else 0.0
    psi = (env[None] * amp * np.exp(1j * ph)).astype(np.complex128)
    return normalise(psi, n, L)


def raw_direction(n, L, seed: int, ncomp: int = 2) -> np.ndarray:
    """Seeded random complex direction with a Gaussian envelope, shape (ncomp,nz,ny,nx).

    Not projected: tests make it tangent with the oracle's own projection before
    handing the same array to both sides."""
    xs = axes(n, L)
    env = np.exp(-0.25 * (xs[2][:, None, None] ** 2 + xs[1][None, :, None] ** 2
                          + xs[0][None, None, :] ** 2))
    rng = np.random.default_rng(seed)
    shape = (ncomp, n[2], n[1], n[0])
    p = env[None] * (rng.standard_normal(shape) + 1j * rng.standard_normal(shape))
    return p.astype(np.complex128)
