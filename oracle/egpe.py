"""Plain FP64 NumPy oracle of the eGPE energy, gradient, line search and NCG.

TEST INFRASTRUCTURE ONLY (see the package docstring): imported by tests, the
smoke check and the bench's CPU-baseline leg, never by the CUDA path.

Discretisation (the paper states spectral accuracy and FFT-based convolution,
Sec. I and Sec. VI.C; the grid itself is a reading):

* x_a[j] = -L_a + j h_a, h_a = 2 L_a / N_a, periodic box [-L_a, L_a)
* k_a[j] = (pi/L_a) * (j if j < N_a/2 else j - N_a)  (Nyquist kept as -N_a/2,
  so every multiplier is real and even)
* <a, b> = dV * sum(conj(a) b); arrays are (2, nz, ny, nx), x fastest.

Couplings are in per-particle normalised form: N_i -> 1 in Eq. 1 and in
mu_LHY, with dimensionless g_ij (contact) and g_dd_ij (the k-space dipolar
coefficient: U~_ij(k) = g_dd_ij (3 k_z^2/|k|^2 - 1), U~(0) := 0; dipoles along z).
The LHY energy density is kappa * eta_s^{-5/2} * int_0^1 du sum_+- max(V_+-,0)^{5/2}
(Eq. 1 with a selectable prefactor; kappa = sqrt(2)/(15 pi^2), eta_s = 1 is the
literal form) and the u-integral is a Q-point Gauss-Legendre rule on [0,1].
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Dict, List, Optional

import numpy as np

PRECOND_MODES = {"none": 0, "kinetic": 1, "diagonal": 2, "kinetic+diagonal": 3, "blend": 4}


# ----------------------------------------------------------------------------
# Grid, parameters, elementary operations
# ----------------------------------------------------------------------------
class Grid:
    """Periodic box [-L_a, L_a) with N_a points per axis (a = x, y, z)."""

    def __init__(self, n, L):
        self.n = tuple(int(v) for v in n)
        self.L = tuple(float(v) for v in L)
        self.h = [2.0 * self.L[a] / self.n[a] for a in range(3)]
        self.x = [-self.L[a] + np.arange(self.n[a]) * self.h[a] for a in range(3)]
        self.k = []
        for a in range(3):
            j = np.arange(self.n[a])
            self.k.append((np.pi / self.L[a]) * np.where(j < self.n[a] // 2, j, j - self.n[a]))
        self.dV = self.h[0] * self.h[1] * self.h[2]
        self.N = self.n[0] * self.n[1] * self.n[2]
        kx = self.k[0][None, None, :]
        ky = self.k[1][None, :, None]
        kz = self.k[2][:, None, None]
        self.k2 = kx ** 2 + ky ** 2 + kz ** 2
        # dipolar kernel 3 k_z^2/|k|^2 - 1 with the k = 0 mode set to 0 (reading 4)
        safe = np.where(self.k2 > 0, self.k2, 1.0)
        self.kdd = np.where(self.k2 > 0, 3.0 * kz ** 2 / safe - 1.0, 0.0)

    @property
    def shape(self):
        return (self.n[2], self.n[1], self.n[0])


@dataclass
class Params:
    """Couplings of Eq. 1 (per-particle normalised form)."""

    g: np.ndarray          # 2x2 contact couplings (symmetric)
    gdd: np.ndarray        # 2x2 k-space dipolar coefficients (symmetric)
    kappa: float           # LHY prefactor
    eta_s: float = 1.0     # LHY scale: density term is (V/eta_s)^{5/2}
    nodes: int = 32        # Gauss-Legendre nodes for the u-integral
    trap: tuple = (1.0, 1.0, 1.0)

    def __post_init__(self):
        self.g = np.asarray(self.g, dtype=np.float64).reshape(2, 2)
        self.gdd = np.asarray(self.gdd, dtype=np.float64).reshape(2, 2)

    @property
    def c5(self) -> float:
        return float(self.kappa) * float(self.eta_s) ** -2.5


def inner(grid: Grid, a: np.ndarray, b: np.ndarray) -> complex:
    """<a, b> = dV * sum conj(a) b  (the L^2 product of Sec. III)."""
    return grid.dV * np.sum(np.conj(a) * b)


# Transform backend: numpy.fft (pocketfft, one thread) unless set_fft_workers
# chose scipy.fft (the same pocketfft algorithm) with several threads, which
# only the host-baseline timing does.  The arithmetic is the same either way.
_FFT_WORKERS = None


def set_fft_workers(n: Optional[int]) -> None:
    """Run the oracle's transforms on n host threads (None: numpy.fft, one thread)."""
    global _FFT_WORKERS
    _FFT_WORKERS = int(n) if n else None


def dft(f):
    if _FFT_WORKERS:
        import scipy.fft
        return scipy.fft.fftn(f, workers=_FFT_WORKERS)
    return np.fft.fftn(f)


def idft(F):
    if _FFT_WORKERS:
        import scipy.fft
        return scipy.fft.ifftn(F, workers=_FFT_WORKERS)
    return np.fft.ifftn(F)


def kinetic_apply(grid: Grid, f: np.ndarray) -> np.ndarray:
    """T f = -1/2 Laplacian f, spectrally: IDFT(|k|^2/2 * DFT f) (Eq. 1 first term)."""
    return idft(0.5 * grid.k2 * dft(f))


def trap_potential(grid: Grid, trap) -> np.ndarray:
    """V_ext = 1/2 (lx^2 x^2 + ly^2 y^2 + lz^2 z^2) (Sec. II, trap equation)."""
    x, y, z = grid.x
    return 0.5 * (trap[0] ** 2 * x[None, None, :] ** 2
                  + trap[1] ** 2 * y[None, :, None] ** 2
                  + trap[2] ** 2 * z[:, None, None] ** 2)


def dipolar_potentials(grid: Grid, prm: Params, n: np.ndarray) -> np.ndarray:
    """Phi_i = sum_j U_ij * n_j, evaluated as IDFT(K(k) DFT(sum_j g_dd_ij n_j)).

    Eq. 1 dipolar term and the coupled eGPE (Sec. II): the convolution with
    (1 - 3cos^2 theta)/r^3 is taken in Fourier space, where it is
    g_dd_ij (3 k_z^2/|k|^2 - 1).  One transform pair per component (no packing).
    """
    Phi = np.empty(n.shape, dtype=np.float64)
    for i in range(2):
        src = prm.gdd[i, 0] * n[0] + prm.gdd[i, 1] * n[1]
        Phi[i] = idft(grid.kdd * dft(src)).real
    return Phi


def gauss_legendre_01(Q: int):
    """Q-point Gauss-Legendre nodes/weights mapped from [-1,1] to [0,1]."""
    t, w = np.polynomial.legendre.leggauss(int(Q))
    return 0.5 * (t + 1.0), 0.5 * w


def _eta(prm: Params, u: float) -> np.ndarray:
    """eta_ij(u) = G_ij + D_ij (3u^2 - 1) (Sec. II, LHY branch potentials)."""
    return prm.g + prm.gdd * (3.0 * u * u - 1.0)


def lhy_density_and_mu(prm: Params, n1: np.ndarray, n2: np.ndarray):
    """LHY energy density F(n1,n2) and mu_LHY^(i) = dF/dn_i (Eq. 1, Sec. II).

    V_+-(u) = eta11 n1 + eta22 n2 +- s, s = sqrt(delta^2 + 4 eta12 eta21 n1 n2),
    delta = eta11 n1 - eta22 n2.  The chemical potential follows the paper's
    mu_LHY formula: per node (5/2) V^{3/2} [eta_ii +- sigma_i / s] with
    sigma_1 = +eta11 delta + 2 eta12 eta21 n2, sigma_2 = -eta22 delta + 2 eta12 eta21 n1.
    Readings: negative V contributes max(V,0)^{5/2} (the real part of V^{5/2});
    where s = 0 the term sigma_i/s is taken as 0 (the +- branches coincide there).
    """
    u, w = gauss_legendre_01(prm.nodes)
    F = np.zeros_like(n1)
    mu1 = np.zeros_like(n1)
    mu2 = np.zeros_like(n1)
    for uq, wq in zip(u, w):
        eta = _eta(prm, uq)
        e11, e22, e1221 = eta[0, 0], eta[1, 1], eta[0, 1] * eta[1, 0]
        delta = e11 * n1 - e22 * n2
        s = np.sqrt(delta ** 2 + 4.0 * e1221 * n1 * n2)
        A = e11 * n1 + e22 * n2
        Vp = np.maximum(A + s, 0.0)
        Vm = np.maximum(A - s, 0.0)
        sig1 = e11 * delta + 2.0 * e1221 * n2
        sig2 = -e22 * delta + 2.0 * e1221 * n1
        with np.errstate(divide="ignore", invalid="ignore"):
            q1 = np.where(s > 0, sig1 / np.where(s > 0, s, 1.0), 0.0)
            q2 = np.where(s > 0, sig2 / np.where(s > 0, s, 1.0), 0.0)
        F += wq * (Vp ** 2.5 + Vm ** 2.5)
        mu1 += wq * 2.5 * (Vp ** 1.5 * (e11 + q1) + Vm ** 1.5 * (e11 - q1))
        mu2 += wq * 2.5 * (Vp ** 1.5 * (e22 + q2) + Vm ** 1.5 * (e22 - q2))
    c5 = prm.c5
    return c5 * F, c5 * mu1, c5 * mu2


# ----------------------------------------------------------------------------
# Energy and gradient (Eq. 1, coupled eGPE, Hamiltonian H_i, mu_i, residual)
# ----------------------------------------------------------------------------
@dataclass
class Evaluation:
    E: float
    terms: Dict[str, float]
    mu: np.ndarray          # mu_i = Re<psi_i, H_i psi_i>
    Hpsi: np.ndarray        # H_i psi_i  (gradient convention of the C ABI)
    n: np.ndarray           # densities |psi_i|^2
    V: np.ndarray           # trap
    Phi: np.ndarray         # dipolar potentials Phi_i
    muL: np.ndarray         # LHY chemical potentials mu_LHY^(i)(r)
    Tpsi: np.ndarray


def evaluate(grid: Grid, prm: Params, psi: np.ndarray) -> Evaluation:
    """E[psi1, psi2] of Eq. 1 and H_i psi_i of the coupled eGPE (Sec. II).

    E = sum_i Re<psi_i, T psi_i> + dV sum V (n1+n2) + 1/2 dV sum_ij g_ij n_i n_j
        + 1/2 dV sum_i n_i Phi_i + dV sum F_LHY
    H_i psi_i = T psi_i + (V + sum_j g_ij n_j + Phi_i + mu_LHY^(i)) psi_i
    mu_i = Re<psi_i, H_i psi_i>  (Sec. III, chemical potentials)
    """
    n = (np.abs(psi) ** 2).astype(np.float64)
    Tpsi = np.stack([kinetic_apply(grid, psi[i]) for i in range(2)])
    V = trap_potential(grid, prm.trap)
    Phi = dipolar_potentials(grid, prm, n)
    F, muL1, muL2 = lhy_density_and_mu(prm, n[0], n[1])
    muL = np.stack([muL1, muL2])
    dV = grid.dV
    kin = [inner(grid, psi[i], Tpsi[i]).real for i in range(2)]
    trap = dV * np.sum(V * (n[0] + n[1]))
    contact = 0.5 * dV * sum(prm.g[i, j] * np.sum(n[i] * n[j]) for i in range(2) for j in range(2))
    dip = 0.5 * dV * sum(np.sum(n[i] * Phi[i]) for i in range(2))
    lhy = dV * np.sum(F)
    E = kin[0] + kin[1] + trap + contact + dip + lhy
    Hpsi = np.empty_like(psi)
    for i in range(2):
        U = V + prm.g[i, 0] * n[0] + prm.g[i, 1] * n[1] + Phi[i] + muL[i]
        Hpsi[i] = Tpsi[i] + U * psi[i]
    mu = np.array([inner(grid, psi[i], Hpsi[i]).real for i in range(2)])
    terms = dict(kin1=kin[0], kin2=kin[1], trap=trap, contact=contact, dipolar=dip, lhy=lhy,
                 norm1=inner(grid, psi[0], psi[0]).real, norm2=inner(grid, psi[1], psi[1]).real)
    return Evaluation(E, terms, mu, Hpsi, n, V, Phi, muL, Tpsi)


def energy_grad(grid: Grid, prm: Params, psi: np.ndarray):
    """(E, mu, H psi): the energy of Eq. 1, mu_i and the gradient H_i psi_i.

    Gradient convention: d/de E(psi + e phi)|_0 = 2 sum_i Re<phi_i, H_i psi_i>.
    """
    ev = evaluate(grid, prm, psi)
    return ev.E, ev.mu, ev.Hpsi


PARAM_NAMES = ("g11", "g12", "g22", "gdd11", "gdd12", "gdd22", "kappa", "eta_s", "trap_x", "trap_y", "trap_z")


def lhy_eta_derivatives(prm: Params, n1: np.ndarray, n2: np.ndarray):
    """Partial derivatives of the LHY density F (Eq. 1) with respect to the
    entries of eta(u) = g + g_dd (3u^2 - 1), accumulated over the u-rule:
    returns dF/dg11, dF/dg22, dF/dg12 (the symmetric pair g12 = g21 moved
    together) and the same with the extra factor 3u^2 - 1 (dF/dgdd_ij).

    With A = eta11 n1 + eta22 n2, delta = eta11 n1 - eta22 n2,
    s^2 = delta^2 + 4 eta12 eta21 n1 n2 and V_+- = A +- s:
      dV_+-/deta11 = n1 +- delta n1 / s,   dV_+-/deta22 = n2 -+ delta n2 / s,
      dV_+-/deta12 (pair) = +- 4 eta12 n1 n2 / s,
    and d max(V,0)^{5/2} = (5/2) max(V,0)^{3/2} dV (terms / s taken as 0 where s = 0).
    """
    u, w = gauss_legendre_01(prm.nodes)
    out = [np.zeros_like(n1) for _ in range(6)]
    for uq, wq in zip(u, w):
        x = 3.0 * uq * uq - 1.0
        eta = _eta(prm, uq)
        e11, e22, e12 = eta[0, 0], eta[1, 1], eta[0, 1]
        delta = e11 * n1 - e22 * n2
        s = np.sqrt(delta ** 2 + 4.0 * eta[0, 1] * eta[1, 0] * n1 * n2)
        A = e11 * n1 + e22 * n2
        with np.errstate(divide="ignore", invalid="ignore"):
            inv_s = np.where(s > 0, 1.0 / np.where(s > 0, s, 1.0), 0.0)
        for sign in (1.0, -1.0):
            V = np.maximum(A + sign * s, 0.0)
            f = 2.5 * V ** 1.5
            d11 = n1 + sign * delta * n1 * inv_s
            d22 = n2 - sign * delta * n2 * inv_s
            d12 = sign * 4.0 * e12 * n1 * n2 * inv_s
            for k, d in enumerate((d11, d22, d12)):
                out[k] += wq * f * d
                out[3 + k] += wq * x * f * d
    c5 = prm.c5
    return [c5 * a for a in out]


def param_grad(grid: Grid, prm: Params, psi: np.ndarray) -> Dict[str, float]:
    """Partial derivatives of E (Eq. 1) with respect to its parameters at fixed psi.

    Contact: dE/dg_ii = 1/2 int n_i^2, dE/dg12 = int n1 n2 (g12 = g21 together).
    Dipolar: dE/dgdd_ii = 1/2 int n_i (K * n_i), dE/dgdd12 = int n1 (K * n2), K the
    k-space kernel 3k_z^2/|k|^2 - 1.  LHY: through eta(u) (lhy_eta_derivatives),
    dE/dkappa = E_LHY / kappa, dE/deta_s = -(5/2) E_LHY / eta_s.  Trap (V = 1/2
    sum lambda_a^2 x_a^2): dE/dlambda_a = lambda_a int x_a^2 (n1 + n2).
    At a normalised ground state these are dE0/dp (Hellmann-Feynman).
    """
    n = (np.abs(psi) ** 2).astype(np.float64)
    dV = grid.dV
    Kn = [idft(grid.kdd * dft(n[i])).real for i in range(2)]
    L = lhy_eta_derivatives(prm, n[0], n[1])
    F, _, _ = lhy_density_and_mu(prm, n[0], n[1])
    E_lhy = dV * np.sum(F)
    x, y, z = grid.x
    nt = n[0] + n[1]
    out = {
        "g11": dV * (0.5 * np.sum(n[0] * n[0]) + np.sum(L[0])),
        "g22": dV * (0.5 * np.sum(n[1] * n[1]) + np.sum(L[1])),
        "g12": dV * (np.sum(n[0] * n[1]) + np.sum(L[2])),
        "gdd11": dV * (0.5 * np.sum(n[0] * Kn[0]) + np.sum(L[3])),
        "gdd22": dV * (0.5 * np.sum(n[1] * Kn[1]) + np.sum(L[4])),
        "gdd12": dV * (np.sum(n[0] * Kn[1]) + np.sum(L[5])),
        "kappa": E_lhy / prm.kappa,
        "eta_s": -2.5 * E_lhy / prm.eta_s,
        "trap_x": prm.trap[0] * dV * np.sum(x[None, None, :] ** 2 * nt),
        "trap_y": prm.trap[1] * dV * np.sum(y[None, :, None] ** 2 * nt),
        "trap_z": prm.trap[2] * dV * np.sum(z[:, None, None] ** 2 * nt),
    }
    return {k: float(v) for k, v in out.items()}


# ----------------------------------------------------------------------------
# Analytic line-search coefficients (Sec. V)
# ----------------------------------------------------------------------------
def line_coeffs_detail(grid: Grid, prm: Params, psi: np.ndarray, p: np.ndarray,
                       ev: Optional[Evaluation] = None) -> Dict[str, float]:
    """First/second-order coefficients of the energy along the geodesic (Sec. V).

    Follows the paper's E'_i, E''_ii, E''_ij, E'_LHY, E''_LHY with auxiliaries
    gamma_i, w_ij, rho_k, V^1, V^2, n', n'', delta_1, delta_2.  Readings:
    * w_ij multiplies psi_i (the printed psi_j would not give the derivative of
      the cross term; Re<w_ij, p_i> = 2 int rho_i (g_ij rho_j + Phi_ij[rho_j]));
    * H_MF is H without mu_LHY;
    * the printed n'' and V^2 are half second derivatives, so the printed E''
      is the exact second derivative along psi(alpha) (no extra factor);
    * where s = 0 the +- terms divided by s are taken as 0.
    """
    if ev is None:
        ev = evaluate(grid, prm, psi)
    n, V, Phi = ev.n, ev.V, ev.Phi
    pnorm2 = np.array([inner(grid, p[i], p[i]).real for i in range(2)])  # 1/gamma_i^2
    HMF_psi, HMF_p = [], []
    for i in range(2):
        Umf = V + prm.g[i, 0] * n[0] + prm.g[i, 1] * n[1] + Phi[i]
        HMF_psi.append(ev.Tpsi[i] + Umf * psi[i])
        HMF_p.append(kinetic_apply(grid, p[i]) + Umf * p[i])
    rho = np.stack([np.real(psi[k] * np.conj(p[k])) for k in range(2)])
    # Phi_ij[rho_j] = D_ij U * rho_j  (Fourier kernel K(k))
    PhiRho = np.empty((2, 2) + rho.shape[1:])
    for i in range(2):
        for j in range(2):
            PhiRho[i, j] = idft(grid.kdd * dft(prm.gdd[i, j] * rho[j])).real
    w = np.empty((2, 2) + psi.shape[1:], dtype=np.complex128)
    for i in range(2):
        for j in range(2):
            w[i, j] = 2.0 * (prm.g[i, j] * rho[j] + PhiRho[i, j]) * psi[i]
    E1 = [2.0 * inner(grid, p[i], HMF_psi[i]).real for i in range(2)]
    E2 = np.zeros((2, 2))
    for i in range(2):
        E2[i, i] = 2.0 * (-pnorm2[i] * inner(grid, psi[i], HMF_psi[i]).real
                          + inner(grid, p[i], HMF_p[i]).real
                          + inner(grid, w[i, i], p[i]).real)
        j = 1 - i
        E2[i, j] = 2.0 * inner(grid, w[i, j], p[i]).real
    # LHY variations: n' = 2 Re(psi* p), n'' = |p|^2 - |psi|^2 / gamma^2
    n1p, n2p = 2.0 * rho[0], 2.0 * rho[1]
    n1pp = np.abs(p[0]) ** 2 - n[0] * pnorm2[0]
    n2pp = np.abs(p[1]) ** 2 - n[1] * pnorm2[1]
    n1, n2 = n[0], n[1]
    u, wq_all = gauss_legendre_01(prm.nodes)
    E1L = np.zeros_like(n1)
    E2L = np.zeros_like(n1)
    for uq, wq in zip(u, wq_all):
        eta = _eta(prm, uq)
        e11, e22, e1221 = eta[0, 0], eta[1, 1], eta[0, 1] * eta[1, 0]
        delta = e11 * n1 - e22 * n2
        s2 = delta ** 2 + 4.0 * e1221 * n1 * n2
        s = np.sqrt(s2)
        A = e11 * n1 + e22 * n2
        d1 = e11 * n1p - e22 * n2p
        d2 = e11 * n1pp - e22 * n2pp
        num1 = delta * d1 + 2.0 * e1221 * (n1 * n2p + n1p * n2)
        num2 = d1 ** 2 + 2.0 * delta * d2 + 4.0 * e1221 * (n1p * n2p + n1 * n2pp + n1pp * n2)
        # ds/dalpha = num1/s and 1/2 d2s/dalpha2 = num2/(2s) - num1^2/(2 s^3),
        # written as (num2 - (num1/s)^2)/(2s) so that s^3 cannot underflow
        pos = s > 0
        ss = np.where(pos, s, 1.0)
        t1 = np.where(pos, num1 / ss, 0.0)
        t2 = np.where(pos, (num2 - t1 * t1) / (2.0 * ss), 0.0)
        A1 = e11 * n1p + e22 * n2p
        A2 = e11 * n1pp + e22 * n2pp
        for sgn in (+1.0, -1.0):
            Vb = np.maximum(A + sgn * s, 0.0)
            V1 = A1 + sgn * t1
            V2 = A2 + sgn * t2
            E1L += wq * 2.5 * Vb ** 1.5 * V1
            E2L += wq * 2.5 * (2.0 * Vb ** 1.5 * V2 + 1.5 * Vb ** 0.5 * V1 ** 2)
    E1_lhy = prm.c5 * grid.dV * np.sum(E1L)
    E2_lhy = prm.c5 * grid.dV * np.sum(E2L)
    Ep = E1[0] + E1[1] + E1_lhy
    Epp = E2.sum() + E2_lhy
    return dict(E0=ev.E, Ep=Ep, Epp=Epp, E1=E1, E2=E2, E1_lhy=E1_lhy, E2_lhy=E2_lhy,
                pnorm2=pnorm2)


def line_coeffs(grid: Grid, prm: Params, psi: np.ndarray, p: np.ndarray,
                ev: Optional[Evaluation] = None):
    """(E0, E', E'') of the quadratic energy model along the geodesic (Sec. V)."""
    d = line_coeffs_detail(grid, prm, psi, p, ev)
    return d["E0"], d["Ep"], d["Epp"]


# ----------------------------------------------------------------------------
# Preconditioners (Sec. IV.B), projection and retraction (Sec. III, Sec. V)
# ----------------------------------------------------------------------------
def preconditioner_shift(grid: Grid, ev: Evaluation, psi: np.ndarray) -> np.ndarray:
    """alpha_i = Re<psi_i, (T + V + sum_j g_ij n_j + mu_LHY^(i)) psi_i> = mu_i - Re<psi_i, Phi_i psi_i>.

    Reading of the garbled integral in P_V and P_Delta (Sec. IV.B): the integral
    is the component-i energy density without the dipolar term.
    """
    return np.array([ev.mu[i] - inner(grid, psi[i], ev.Phi[i] * psi[i]).real for i in range(2)])


def precondition(grid: Grid, prm: Params, ev: Evaluation, psi: np.ndarray, r: np.ndarray,
                 mode: str, pv_floor: float = 1e-2, blend: float = 0.5) -> np.ndarray:
    """z = P^{-1} r with P^{-1} = P_Delta^{-1} P_V^{-1} (Sec. IV.B, composition formula).

    P_V,i(r) = max(|alpha_i| + V + sum_j g_ij n_j + mu_LHY^(i), pv_floor |alpha_i|):
    real-space diagonal, dipolar term excluded, with a positive floor (the
    paper's "small positive shift", value not given).
    P_Delta,i(k) = |alpha_i| + |k|^2/2 (the printed "+1/2 Laplacian" read as the
    positive kinetic operator).  Mode "none" returns r; "kinetic" applies P_Delta
    only; "diagonal" P_V only; "kinetic+diagonal" P_V first, then P_Delta, as the
    composition formula is written.  |alpha_i| keeps both operators positive.
    Mode "blend" is the weighted combination the paper names as possible (Sec.
    IV.B) and as an extension (Sec. VII), read as the convex combination
    z = blend P_V^{-1} r + (1 - blend) P_Delta^{-1} r.
    """
    if mode not in PRECOND_MODES:
        raise ValueError(mode)
    if mode == "blend":
        zv = precondition(grid, prm, ev, psi, r, "diagonal", pv_floor)
        zd = precondition(grid, prm, ev, psi, r, "kinetic", pv_floor)
        return blend * zv + (1.0 - blend) * zd
    alpha = np.abs(preconditioner_shift(grid, ev, psi))
    z = r.astype(np.complex128).copy()
    n = ev.n
    if mode in ("diagonal", "kinetic+diagonal"):
        for i in range(2):
            PV = alpha[i] + ev.V + prm.g[i, 0] * n[0] + prm.g[i, 1] * n[1] + ev.muL[i]
            PV = np.maximum(PV, pv_floor * alpha[i])
            z[i] = z[i] / PV
    if mode in ("kinetic", "kinetic+diagonal"):
        for i in range(2):
            z[i] = idft(dft(z[i]) / (alpha[i] + 0.5 * grid.k2))
    return z


def project(grid: Grid, psi: np.ndarray, d: np.ndarray) -> np.ndarray:
    """Rectified direction p_i = d_i - Re<d_i, psi_i> psi_i (Sec. V)."""
    p = d.astype(np.complex128).copy()
    for i in range(2):
        p[i] = d[i] - inner(grid, d[i], psi[i]).real * psi[i]
    return p


def retract(grid: Grid, psi: np.ndarray, p: np.ndarray, theta) -> np.ndarray:
    """psi_i(theta_i) = cos(theta_i) psi_i + sin(theta_i) p_i/||p_i||, renormalised.

    Great-circle geodesic of Sec. III and Algorithm 1; the explicit
    renormalisation follows the normalised update of Sec. V.
    """
    out = np.empty_like(psi)
    for i in range(2):
        pn = math.sqrt(inner(grid, p[i], p[i]).real)
        if pn > 0.0:
            q = math.cos(theta[i]) * psi[i] + math.sin(theta[i]) * (p[i] / pn)
        else:
            q = psi[i].copy()
        out[i] = q / math.sqrt(inner(grid, q, q).real)
    return out


# ----------------------------------------------------------------------------
# Preconditioned nonlinear CG on the product of spheres (Algorithm 1)
# ----------------------------------------------------------------------------
def cg_beta(grid: Grid, r: np.ndarray, z: np.ndarray, r_prev: np.ndarray, p_prev: np.ndarray,
            rz_prev: Optional[float], rule: str = "HS"):
    """Conjugacy coefficient of the preconditioned NCG direction (Sec. IV.C).

    With z = P^{-1} r and sums over both components (one global beta; Algorithm 1
    carries no component index on beta):
      HS+: beta = max( sum_i Re<r_i - r_prev_i, z_i> / sum_i Re<r_i - r_prev_i, p_prev_i>, 0 )
      PR+: beta = max( sum_i Re<r_i - r_prev_i, z_i> / rz_prev, 0 ),
           rz_prev = sum_i Re<r_prev_i, z_prev_i>
    Readings: the HS denominator takes the previous direction p^{n-1} (the printed
    p^{(n)} would be circular); the PR denominator is the stored value of the
    previous iteration, i.e. with the preconditioner of iteration n-1.
    Returns (beta, ok); ok is False when the denominator is zero or either sum is
    not finite, which the solver treats as a restart (beta = 0).
    """
    num = sum(inner(grid, r[i] - r_prev[i], z[i]).real for i in range(2))
    if rule == "PR":
        den = rz_prev
    else:
        den = sum(inner(grid, r[i] - r_prev[i], p_prev[i]).real for i in range(2))
    if den is None or den == 0.0 or not np.isfinite(den) or not np.isfinite(num):
        return 0.0, False
    return max(num / den, 0.0), True


@dataclass
class SolveOpts:
    precond: str = "kinetic"
    tol_res: float = 1e-8          # stop when ||r|| = sqrt(sum_i <r_i, r_i>) < tol_res
    tol_dE: float = 0.0            # optional: stop when |E^{n+1} - E^n| < tol_dE
    max_iter: int = 2000
    restart_period: int = 20       # K_r: beta = 0 when n mod K_r == 0
    armijo_c1: float = 1e-4
    armijo_max: int = 30
    theta_max: float = 0.5 * math.pi
    accept_rtol: float = 1e-13     # round-off allowance: accept if E_t < E + accept_rtol |E|
    pv_floor: float = 1e-2
    beta_rule: str = "HS"          # "HS" (Hestenes-Stiefel+) or "PR" (Polak-Ribiere+)
    blend: float = 0.5             # weight of P_V in the "blend" preconditioner


def ncg_solve(grid: Grid, prm: Params, psi0: np.ndarray, opts: SolveOpts = SolveOpts(),
              trace: Optional[List[dict]] = None):
    """Preconditioned NCG of Algorithm 1 with HS+ beta, analytic step, exact-path check.

    Per iteration n (Algorithm 1 order):
      r_i = H_i psi_i - mu_i psi_i                         (Sec. III / IV.A)
      z = P^{-1} r                                          (Sec. IV.B)
      beta = max(beta_HS, 0) (or max(beta_PR, 0) with beta_rule "PR"), HS denominator on
             p^{n-1}                                        (Sec. IV.C; reading: the
             printed p^{(n)} is the previous direction); beta = 0 when n mod K_r == 0,
             when the denominator is zero or non-finite, and when the resulting
             direction has Re<r, p> >= 0 (restart rule of Sec. IV.C)
      d = -z + beta p^{n-1};  p = d - Re<d, psi> psi        (Sec. IV.C, Sec. V)
      alpha = -E'/E'' from the quadratic model; theta_i = alpha ||p_i||   (Sec. V)
      psi(theta) on the exact normalised path; accept on a decrease (strict up to a
      round-off allowance accept_rtol |E|); otherwise, or when E'' <= 0, Armijo
      halving along the same path: E(alpha) <= E0 + c1 alpha E' (+ the allowance).
    Readings: the largest theta_i is capped at theta_max by scaling alpha; with
    E'' <= 0 the Armijo start is the previous accepted alpha (pi/(4 max||p_i||) at
    n = 0); if even the restarted direction is not a descent direction, the
    unpreconditioned residual is used for that iteration.
    Returns (psi, report dict).
    """
    psi = psi0.astype(np.complex128).copy()
    ev = evaluate(grid, prm, psi)
    r_prev = None
    p_prev = None
    rz_prev = None
    alpha_prev = None
    n_it = 0
    restarts = 0
    armijo_total = 0
    status = "not_converged"
    res = float("nan")
    while True:
        mu = ev.mu
        r = np.stack([ev.Hpsi[i] - mu[i] * psi[i] for i in range(2)])
        res = math.sqrt(sum(inner(grid, r[i], r[i]).real for i in range(2)))
        if not np.isfinite(res) or not np.isfinite(ev.E):
            status = "nonfinite"
            break
        if res < opts.tol_res:
            status = "converged"
            break
        if n_it >= opts.max_iter:
            status = "not_converged"
            break
        z = precondition(grid, prm, ev, psi, r, opts.precond, opts.pv_floor, opts.blend)
        restart = (n_it % opts.restart_period == 0) or p_prev is None
        beta = 0.0
        rz = sum(inner(grid, r[i], z[i]).real for i in range(2))
        if not restart:
            beta, ok = cg_beta(grid, r, z, r_prev, p_prev, rz_prev, opts.beta_rule)
            restart = not ok
        d = -z + beta * p_prev if beta != 0.0 else -z
        p = project(grid, psi, d)
        descent = sum(inner(grid, r[i], p[i]).real for i in range(2))
        if descent >= 0.0 and beta != 0.0:
            restart = True
            beta = 0.0
            p = project(grid, psi, -z)
            descent = sum(inner(grid, r[i], p[i]).real for i in range(2))
        fallback = False
        if descent >= 0.0:
            fallback = True
            p = project(grid, psi, -r)
        if beta == 0.0:
            restarts += 1
        E0, Ep, Epp = line_coeffs(grid, prm, psi, p, ev)
        pn = np.array([math.sqrt(inner(grid, p[i], p[i]).real) for i in range(2)])
        pmax = float(pn.max())
        if not pmax > 0.0:
            status = "stagnated"
            break
        if Epp > 0.0 and np.isfinite(Epp) and np.isfinite(Ep):
            alpha0 = -Ep / Epp
            kind = "analytic"
        else:
            alpha0 = alpha_prev if alpha_prev is not None else math.pi / (4.0 * pmax)
            kind = "armijo"
        if alpha0 * pmax > opts.theta_max:
            alpha0 = opts.theta_max / pmax
        tau = opts.accept_rtol * abs(ev.E)
        k = 0
        accepted = False
        while True:
            alpha = alpha0 / (2.0 ** k)
            theta = alpha * pn
            psi_t = retract(grid, psi, p, theta)
            ev_t = evaluate(grid, prm, psi_t)
            if kind == "analytic" and k == 0:
                ok = ev_t.E < ev.E + tau
            else:
                ok = ev_t.E <= ev.E + opts.armijo_c1 * alpha * Ep + tau
            if ok:
                accepted = True
                break
            k += 1
            armijo_total += 1
            if k > opts.armijo_max:
                break
        if trace is not None:
            trace.append(dict(n=n_it, E=ev.E, res=res, beta=beta, alpha=alpha, theta=theta.tolist(),
                              Ep=Ep, Epp=Epp, kind=kind, armijo=k, accepted=accepted,
                              restart=bool(beta == 0.0), fallback=fallback, E_new=ev_t.E))
        if not accepted:
            status = "stagnated"
            break
        dE = ev_t.E - ev.E
        r_prev, p_prev, rz_prev = r, p, rz
        psi, ev = psi_t, ev_t
        alpha_prev = alpha
        n_it += 1
        if opts.tol_dE > 0.0 and abs(dE) < opts.tol_dE:
            r_last = np.stack([ev.Hpsi[i] - ev.mu[i] * psi[i] for i in range(2)])
            res = math.sqrt(sum(inner(grid, r_last[i], r_last[i]).real for i in range(2)))
            status = "converged"
            break
    report = dict(status=status, iters=n_it, E=ev.E, mu=ev.mu.copy(), res=res,
                  restarts=restarts, armijo_steps=armijo_total, terms=ev.terms)
    return psi, report


# ----------------------------------------------------------------------------
# Imaginary-time evolution reference (the paper's baseline, Sec. I / VI)
# ----------------------------------------------------------------------------
def ite_solve(grid: Grid, prm: Params, psi0: np.ndarray, dtau: float = 1e-3,
              tol_dE: float = 1e-6, max_steps: int = 100000, tol_res: float = 0.0):
    """Strang-split imaginary-time evolution with per-component renormalisation.

    The paper compares against ITE with 8 FFTs per step (Sec. VI.B) but does not
    give its scheme; this reading uses
      psi <- e^{-dtau T/2} e^{-dtau H_pot[psi]} e^{-dtau T/2} psi,  psi_i <- psi_i/||psi_i||
    with H_pot = V + sum_j g_ij n_j + Phi_i + mu_LHY^(i) at the half-stepped density,
    stopping when |E^{k+1} - E^k| < tol_dE (the paper's ITE stopping rule, Sec. VI.A)
    or the residual is below tol_res.
    """
    psi = psi0.astype(np.complex128).copy()
    half = np.exp(-0.25 * dtau * grid.k2)   # exp(-dtau/2 * |k|^2/2)
    V = trap_potential(grid, prm.trap)
    E_prev = evaluate(grid, prm, psi).E
    steps = 0
    status = "not_converged"
    while steps < max_steps:
        for i in range(2):
            psi[i] = idft(half * dft(psi[i]))
        n = np.abs(psi) ** 2
        Phi = dipolar_potentials(grid, prm, n)
        _, muL1, muL2 = lhy_density_and_mu(prm, n[0], n[1])
        muL = (muL1, muL2)
        for i in range(2):
            U = V + prm.g[i, 0] * n[0] + prm.g[i, 1] * n[1] + Phi[i] + muL[i]
            psi[i] = np.exp(-dtau * U) * psi[i]
        for i in range(2):
            psi[i] = idft(half * dft(psi[i]))
            psi[i] /= math.sqrt(inner(grid, psi[i], psi[i]).real)
        steps += 1
        ev = evaluate(grid, prm, psi)
        if abs(ev.E - E_prev) < tol_dE:
            status = "converged"
            break
        if tol_res > 0.0:
            r = np.stack([ev.Hpsi[i] - ev.mu[i] * psi[i] for i in range(2)])
            if math.sqrt(sum(inner(grid, r[i], r[i]).real for i in range(2))) < tol_res:
                status = "converged"
                break
        E_prev = ev.E
    ev = evaluate(grid, prm, psi)
    return psi, dict(status=status, steps=steps, E=ev.E, mu=ev.mu.copy())
