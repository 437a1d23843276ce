"""Pins for the FP64 CPU oracle: closed forms, brute force, library routines and
invariants that do not come from the oracle itself.

Each test targets a plausible mistake (dropped term, wrong sign, wrong index,
transposed axis) in one oracle function.  Sizes are small so the whole file
runs in well under a minute.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2510_24543_gb300 import inputs as I

from . import _common as _cm


def _prm(g=((0, 0), (0, 0)), gdd=((0, 0), (0, 0)), kappa=0.0, eta_s=1.0, nodes=32, trap=(1, 1, 1)):
    return O.Params(np.array(g, float), np.array(gdd, float), kappa, eta_s, nodes, trap)


# ---------------------------------------------------------------- transforms
def test_fft_convention_matches_brute_force_dft():
    """numpy's 3D transform over (z,y,x) equals the O(N^2) DFT sum with x fastest."""
    nz, ny, nx = 3, 4, 5
    rng = np.random.default_rng(0)
    f = rng.standard_normal((nz, ny, nx)) + 1j * rng.standard_normal((nz, ny, nx))
    F = np.zeros_like(f)
    for kz in range(nz):
        for ky in range(ny):
            for kx in range(nx):
                acc = 0j
                for z in range(nz):
                    for y in range(ny):
                        for x in range(nx):
                            acc += f[z, y, x] * np.exp(-2j * np.pi * (kx * x / nx + ky * y / ny + kz * z / nz))
                F[kz, ky, kx] = acc
    assert np.max(np.abs(O.egpe.dft(f) - F)) < 1e-12
    assert np.max(np.abs(O.egpe.idft(F) - f)) < 1e-13


def test_parseval():
    g = O.Grid((8, 6, 10), (3.0, 2.0, 4.0))
    f = I.random_fields(g.shape, 3)
    lhs = O.inner(g, f, f).real
    rhs = g.dV / g.N * np.sum(np.abs(O.egpe.dft(f)) ** 2)
    assert abs(lhs - rhs) < 1e-12 * lhs


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_kinetic_plane_wave(axis):
    """T exp(i k.x) = |k|^2/2 exp(i k.x) on a non-cubic grid, for each axis and the
    Nyquist mode (pins the wavenumber convention and axis order)."""
    g = O.Grid((8, 12, 16), (2.0, 3.0, 5.0))
    X = [g.x[0][None, None, :], g.x[1][None, :, None], g.x[2][:, None, None]]
    for m in (1, 3, g.n[axis] // 2):
        k = math.pi / g.L[axis] * m
        f = np.exp(1j * k * X[axis]) * np.ones(g.shape)
        Tf = O.kinetic_apply(g, f)
        assert np.max(np.abs(Tf - 0.5 * k * k * f)) < 1e-10 * max(1.0, k * k)


# ---------------------------------------------------------------- harmonic closed forms
def _harmonic_gs(g, trap):
    X = [g.x[0][None, None, :], g.x[1][None, :, None], g.x[2][:, None, None]]
    G = np.ones(g.shape)
    for a in range(3):
        G = G * (trap[a] / np.pi) ** 0.25 * np.exp(-0.5 * trap[a] * X[a] ** 2)
    return np.stack([G, G]).astype(np.complex128)


def test_harmonic_energy_terms_closed_form():
    """Non-interacting Gaussian: E_kin = E_trap = sum_a lambda_a/4 per component,
    mu_i = sum_a lambda_a/2 and H psi = mu psi (Sec. II trap, Eq. 1)."""
    trap = (1.0, 1.5, 2.0)
    g = O.Grid((48, 56, 64), (8.0, 8.0, 8.0))
    psi = _harmonic_gs(g, trap)
    ev = O.evaluate(g, _prm(trap=trap), psi)
    q = sum(trap) / 4.0
    assert abs(ev.terms["kin1"] - q) < 1e-12 and abs(ev.terms["kin2"] - q) < 1e-12
    assert abs(ev.terms["trap"] - 2 * q) < 1e-12
    assert abs(ev.E - 4 * q) < 1e-12
    assert np.allclose(ev.mu, 2 * q, atol=1e-12, rtol=0)
    assert np.max(np.abs(ev.Hpsi - 2 * q * psi)) < 1e-10


def test_ncg_reaches_harmonic_ground_state():
    """g = g_dd = kappa = 0: NCG from a noisy start reaches E = sum_i (lx+ly+lz)/2 = 4."""
    trap = (1.0, 1.0, 2.0)
    # h_x = 0.39, h_z = 0.25: spectral and truncation errors of the Gaussian < 1e-13
    w = I.Workload("h", (36, 36, 48), (7.0, 7.0, 6.0), trap, ((0, 0), (0, 0)), ((0, 0), (0, 0)), 0.0, 11)
    g = O.Grid(w.n, w.L)
    psi0 = I.gaussian_start(w, noise=0.05)
    psi, rep = O.ncg_solve(g, _prm(trap=trap, nodes=1), psi0,
                           O.SolveOpts(precond="kinetic+diagonal", tol_res=1e-9))
    assert rep["status"] == "converged"
    assert abs(rep["E"] - 4.0) < 1e-12
    assert np.allclose(rep["mu"], 2.0, atol=1e-9, rtol=0)


# ---------------------------------------------------------------- dipolar kernel
@pytest.mark.parametrize("axis,mult", [(2, 2.0), (0, -1.0), (1, -1.0)])
def test_dipolar_plane_wave_multiplier(axis, mult):
    """A density modulated along z sees +2 g_dd, along x or y -g_dd (3cos^2-1 with
    dipoles along z); the uniform part has no dipolar potential (K(0) = 0)."""
    g = O.Grid((8, 10, 12), (3.0, 4.0, 5.0))
    X = [g.x[0][None, None, :], g.x[1][None, :, None], g.x[2][:, None, None]]
    k = math.pi / g.L[axis] * 2
    n1 = 0.7 + 0.1 * np.cos(k * X[axis]) * np.ones(g.shape)
    n2 = 0.2 * np.ones(g.shape)
    gdd = np.array([[300.0, 120.0], [120.0, 50.0]])
    Phi = O.dipolar_potentials(g, _prm(gdd=gdd), np.stack([n1, n2]))
    for i in range(2):
        expect = gdd[i, 0] * mult * 0.1 * np.cos(k * X[axis]) * np.ones(g.shape)
        assert np.max(np.abs(Phi[i] - expect)) < 1e-11


def test_dipolar_oblique_wave():
    """k along (1,0,1)/sqrt2: 3cos^2(45deg)-1 = 1/2."""
    g = O.Grid((8, 8, 8), (4.0, 4.0, 4.0))
    X = [g.x[0][None, None, :], g.x[1][None, :, None], g.x[2][:, None, None]]
    k = math.pi / 4.0 * 2
    n1 = 1.0 + 0.3 * np.cos(k * (X[0] + X[2]))
    n = np.stack([n1 * np.ones(g.shape), np.zeros(g.shape)])
    Phi = O.dipolar_potentials(g, _prm(gdd=((100.0, 0), (0, 0))), n)
    assert np.max(np.abs(Phi[0] - 100.0 * 0.5 * 0.3 * np.cos(k * (X[0] + X[2])))) < 1e-11


def test_isotropic_density_on_cubic_grid_has_zero_dipolar_energy():
    """Cubic symmetry of the lattice sum: sum_k (3kz^2/k^2 - 1)|n^(k)|^2 = 0."""
    g = O.Grid((16, 16, 16), (6.0, 6.0, 6.0))
    X = [g.x[0][None, None, :], g.x[1][None, :, None], g.x[2][:, None, None]]
    G = np.exp(-0.5 * (X[0] ** 2 + X[1] ** 2 + X[2] ** 2))
    psi = np.stack([G, 0.5 * G]).astype(np.complex128)
    ev = O.evaluate(g, _prm(gdd=((300.0, 200.0), (200.0, 100.0)), trap=(1, 1, 1)), psi)
    assert abs(ev.terms["dipolar"]) < 1e-12 * abs(ev.terms["kin1"]) * 300


# ---------------------------------------------------------------- LHY
def test_lhy_without_dipoles_is_node_independent_and_matches_eigenvalues():
    """g_dd = 0: eta does not depend on u, so any Q gives the same F; and
    V_+- = 2 * eigenvalues of [[g11 n1, g12 sqrt(n1 n2)], [g12 sqrt(n1 n2), g22 n2]]."""
    rng = np.random.default_rng(4)
    n1 = rng.uniform(0.0, 0.3, 50)
    n2 = rng.uniform(0.0, 0.3, 50)
    g = np.array([[400.0, 380.0], [380.0, 300.0]])
    F32, m1, m2 = O.lhy_density_and_mu(_prm(g=g, kappa=1.3, eta_s=2.0, nodes=32), n1, n2)
    F1, _, _ = O.lhy_density_and_mu(_prm(g=g, kappa=1.3, eta_s=2.0, nodes=1), n1, n2)
    assert np.max(np.abs(F32 - F1)) < 1e-12 * np.max(np.abs(F32))
    ref = np.empty_like(n1)
    for k in range(len(n1)):
        M = np.array([[g[0, 0] * n1[k], g[0, 1] * math.sqrt(n1[k] * n2[k])],
                      [g[0, 1] * math.sqrt(n1[k] * n2[k]), g[1, 1] * n2[k]]])
        lam = np.linalg.eigvalsh(M)
        ref[k] = 1.3 * 2.0 ** -2.5 * sum(max(2 * l, 0.0) ** 2.5 for l in lam)
    assert np.max(np.abs(F32 - ref)) < 1e-11 * np.max(np.abs(ref))


def _q5_closed_form(eps):
    """int_0^1 (1 + eps (3u^2 - 1))^{5/2} du, 0 < eps < 1, by the standard reduction
    of int (a + b u^2)^{m/2} du (a = 1 - eps, b = 3 eps)."""
    a, b = 1.0 - eps, 3.0 * eps
    f = lambda m: (a + b) ** (m / 2.0)  # value of (a + b u^2)^{m/2} at u = 1
    I1 = math.asinh(math.sqrt(b / a)) / math.sqrt(b)          # int du / sqrt(a + b u^2)
    I_half = f(1) / 2.0 + a / 2.0 * I1                         # int (a+bu^2)^{1/2}
    I_3half = f(3) / 4.0 + 3.0 * a / 4.0 * I_half              # int (a+bu^2)^{3/2}
    return f(5) / 6.0 + 5.0 * a / 6.0 * I_3half                # int (a+bu^2)^{5/2}


@pytest.mark.parametrize("eps", [0.2, 0.5, 0.75, 0.9])
def test_lhy_single_component_closed_form(eps):
    """n2 = 0: V_+ = 2 eta11 n1, so F = C (2 g n)^{5/2} int_0^1 (1+eps(3u^2-1))^{5/2} du,
    and (when g11 = g22, kappa = 2c/5, eta_s = g11+g22) mu = c n^{3/2} Q5(eps)."""
    g11 = 400.0
    gdd = eps * g11
    c = 50.0
    prm = _prm(g=((g11, 123.0), (123.0, g11)), gdd=((gdd, 77.0), (77.0, 9.0)),
               kappa=0.4 * c, eta_s=2 * g11, nodes=32)
    n1 = np.array([0.01, 0.1, 0.25])
    F, m1, _ = O.lhy_density_and_mu(prm, n1, np.zeros(3))
    q5 = _q5_closed_form(eps)
    assert np.allclose(F, 0.4 * c * (2 * g11) ** -2.5 * (2 * g11 * n1) ** 2.5 * q5, rtol=1e-13, atol=0)
    assert np.allclose(m1, c * n1 ** 1.5 * q5, rtol=1e-13, atol=0)


def test_lhy_mu_is_derivative_of_density():
    rng = np.random.default_rng(7)
    n1 = rng.uniform(0.02, 0.3, 40)
    n2 = rng.uniform(0.02, 0.3, 40)
    prm = _prm(g=((300, 280), (280, 300)), gdd=((420, 400), (400, 420)), kappa=40.0, eta_s=600.0)
    F, m1, m2 = O.lhy_density_and_mu(prm, n1, n2)
    h = 1e-6
    fd1 = (O.lhy_density_and_mu(prm, n1 + h, n2)[0] - O.lhy_density_and_mu(prm, n1 - h, n2)[0]) / (2 * h)
    fd2 = (O.lhy_density_and_mu(prm, n1, n2 + h)[0] - O.lhy_density_and_mu(prm, n1, n2 - h)[0]) / (2 * h)
    assert np.max(np.abs(fd1 - m1)) < 1e-7 * np.max(np.abs(m1))
    assert np.max(np.abs(fd2 - m2)) < 1e-7 * np.max(np.abs(m2))


def test_lhy_euler_identity():
    """V_+- are homogeneous of degree 1 in (n1, n2), so the LHY density F is of
    degree 5/2 and n1 mu1 + n2 mu2 = (5/2) F exactly (Euler's theorem), also where
    det eta(u) < 0 at some nodes (one branch clamped) and at zero density."""
    rng = np.random.default_rng(11)
    n1 = np.concatenate([rng.uniform(0.0, 0.3, 60), [0.0, 0.2, 0.0]])
    n2 = np.concatenate([rng.uniform(0.0, 0.3, 60), [0.0, 0.0, 0.15]])
    for g12, gdd12 in ((280.0, 400.0), (340.0, 150.0), (120.0, 60.0)):
        prm = _prm(g=((300, g12), (g12, 310)), gdd=((420, gdd12), (gdd12, 380)), kappa=40.0, eta_s=610.0)
        F, m1, m2 = O.lhy_density_and_mu(prm, n1, n2)
        assert np.max(np.abs(n1 * m1 + n2 * m2 - 2.5 * F)) < 1e-13 * np.max(np.abs(F))
        assert F[-3] == 0.0 and m1[-3] == 0.0 and m2[-3] == 0.0


def test_lhy_quadrature_against_adaptive_integral():
    """For smooth integrands (all V > 0) the 32-node rule matches scipy.quad."""
    from scipy.integrate import quad
    g = np.array([[300.0, 100.0], [100.0, 300.0]])
    gdd = np.array([[120.0, 40.0], [40.0, 120.0]])
    prm = _prm(g=g, gdd=gdd, kappa=1.0, eta_s=1.0, nodes=32)
    n1, n2 = 0.2, 0.1

    def integrand(u):
        e = g + gdd * (3 * u * u - 1)
        d = e[0, 0] * n1 - e[1, 1] * n2
        s = math.sqrt(d * d + 4 * e[0, 1] * e[1, 0] * n1 * n2)
        A = e[0, 0] * n1 + e[1, 1] * n2
        return max(A + s, 0) ** 2.5 + max(A - s, 0) ** 2.5
    ref = quad(integrand, 0.0, 1.0, epsabs=0, epsrel=1e-13)[0]
    F, _, _ = O.lhy_density_and_mu(prm, np.array([n1]), np.array([n2]))
    assert abs(F[0] - ref) < 1e-12 * ref


# ---------------------------------------------------------------- gradient and line search
def _full_params():
    return _prm(g=((400, 250), (250, 380)), gdd=((300, 280), (280, 260)), kappa=20.0, eta_s=780.0,
                nodes=16, trap=(1.0, 1.3, 2.0))


def test_gradient_matches_finite_differences():
    """d/de E(psi + e phi) = 2 sum_i Re<phi_i, H_i psi_i> with every term on (8^3, complex)."""
    n, L = (8, 8, 8), (3.0, 3.5, 2.5)
    g = O.Grid(n, L)
    prm = _full_params()
    psi = I.random_state(n, L, 5)
    phi = I.random_fields(psi.shape, 6, scale=0.1)
    _, _, H = O.energy_grad(g, prm, psi)
    eps = 1e-5
    fd = (O.evaluate(g, prm, psi + eps * phi).E - O.evaluate(g, prm, psi - eps * phi).E) / (2 * eps)
    an = 2 * sum(O.inner(g, phi[i], H[i]).real for i in range(2))
    assert abs(fd - an) < 1e-9 * abs(an)


def test_chemical_potential_and_tangent_residual():
    n, L = (8, 8, 8), (3.0, 3.0, 3.0)
    g = O.Grid(n, L)
    psi = I.random_state(n, L, 8)
    ev = O.evaluate(g, _full_params(), psi)
    for i in range(2):
        r = ev.Hpsi[i] - ev.mu[i] * psi[i]
        assert abs(O.inner(g, r, psi[i]).real) < 1e-12 * abs(ev.mu[i])


def test_line_coefficients_match_exact_geodesic():
    """E' and E'' (Sec. V formulas) against central differences of E along
    psi_i(alpha) = cos(alpha||p_i||) psi_i + sin(alpha||p_i||) p_i/||p_i||."""
    n, L = (8, 8, 8), (3.0, 3.0, 3.0)
    g = O.Grid(n, L)
    prm = _full_params()
    psi = I.random_state(n, L, 5)
    p = O.project(g, psi, I.raw_direction(n, L, 7))
    E0, Ep, Epp = O.line_coeffs(g, prm, psi, p)
    pn = np.array([math.sqrt(O.inner(g, p[i], p[i]).real) for i in range(2)])

    def E(a):
        return O.evaluate(g, prm, O.retract(g, psi, p, a * pn)).E
    def d1(h):
        return (E(h) - E(-h)) / (2 * h)

    def d2(h):
        return (E(h) - 2 * E0 + E(-h)) / (h * h)
    h = 2e-3  # Richardson extrapolation of the central differences: O(h^4)
    fd1 = (4 * d1(h / 2) - d1(h)) / 3
    fd2 = (4 * d2(h / 2) - d2(h)) / 3
    assert abs(fd1 - Ep) < 1e-8 * abs(Ep)
    assert abs(fd2 - Epp) < 1e-7 * abs(Epp)


def test_line_coefficients_cross_terms_needed():
    """Swapping the roles of the components (w_ij acting on psi_i) leaves E'' unchanged:
    the mixture's cross terms are symmetric under relabelling 1 <-> 2."""
    n, L = (8, 8, 8), (3.0, 3.0, 3.0)
    g = O.Grid(n, L)
    prm = _full_params()
    psi = I.random_state(n, L, 15)
    p = O.project(g, psi, I.raw_direction(n, L, 16))
    a = O.line_coeffs(g, prm, psi, p)
    prm_sw = O.Params(prm.g[::-1, ::-1], prm.gdd[::-1, ::-1], prm.kappa, prm.eta_s, prm.nodes, prm.trap)
    b = O.line_coeffs(g, prm_sw, psi[::-1].copy(), p[::-1].copy())
    assert np.allclose(a, b, rtol=1e-12, atol=0)


# ---------------------------------------------------------------- manifold
def test_retraction_projection_preserve_manifold():
    n, L = (8, 8, 8), (3.0, 3.0, 3.0)
    g = O.Grid(n, L)
    psi = I.random_state(n, L, 21)
    p = O.project(g, psi, I.raw_direction(n, L, 22))
    for i in range(2):
        assert abs(O.inner(g, p[i], psi[i]).real) < 1e-14
    out = O.retract(g, psi, p, [0.3, 1.1])
    for i in range(2):
        assert abs(O.inner(g, out[i], out[i]).real - 1.0) < 1e-14
    # exact geodesic without the renormalisation already has unit norm
    pn = math.sqrt(O.inner(g, p[0], p[0]).real)
    q = math.cos(0.3) * psi[0] + math.sin(0.3) * p[0] / pn
    assert abs(O.inner(g, q, q).real - 1.0) < 1e-13


def test_preconditioners_are_positive():
    """Re<r, P^{-1} r> > 0 for every mode (descent direction) on a random residual,
    and P_Delta acts on a plane wave as 1/(alpha + |k|^2/2)."""
    w = I.PRESETS["c1"]
    n, L = (16, 16, 16), w.L
    g = O.Grid(n, L)
    prm = O.Params(w.g, w.gdd, w.kappa, w.eta_s, 8, w.trap)
    psi = I.random_state(n, L, 30, width=(2.0, 2.0, 1.0))
    ev = O.evaluate(g, prm, psi)
    r = np.stack([ev.Hpsi[i] - ev.mu[i] * psi[i] for i in range(2)])
    for mode in O.PRECOND_MODES:
        z = O.precondition(g, prm, ev, psi, r, mode)
        assert sum(O.inner(g, r[i], z[i]).real for i in range(2)) > 0
    alpha = np.abs(O.preconditioner_shift(g, ev, psi))
    assert np.all(alpha > 0)
    k = math.pi / L[2] * 3
    wave = np.exp(1j * k * g.x[2][:, None, None]) * np.ones(g.shape)
    z = O.precondition(g, prm, ev, psi, np.stack([wave, wave]), "kinetic")
    for i in range(2):
        assert np.max(np.abs(z[i] - wave / (alpha[i] + 0.5 * k * k))) < 1e-13


def test_preconditioner_shift_and_pv_harmonic_closed_form():
    """g = g_dd = kappa = 0 at the harmonic ground state: alpha_i = mu_i =
    (lx+ly+lz)/2 exactly, P_V,i = alpha_i + V pointwise, so the diagonal mode is
    z = r/(alpha_i + V); the kinetic mode with that alpha acts on a plane wave
    as 1/(alpha + |k|^2/2); the composed mode is P_Delta^{-1}(P_V^{-1} r) (Sec. IV.B)."""
    trap = (1.0, 1.5, 2.0)
    g = O.Grid((32, 32, 40), (7.0, 7.0, 6.0))
    psi = _harmonic_gs(g, trap)
    prm = _prm(trap=trap)
    ev = O.evaluate(g, prm, psi)
    alpha = O.preconditioner_shift(g, ev, psi)
    assert np.allclose(alpha, sum(trap) / 2.0, atol=1e-12, rtol=0)
    X = [g.x[0][None, None, :], g.x[1][None, :, None], g.x[2][:, None, None]]
    V = 0.5 * sum(trap[a] ** 2 * X[a] ** 2 for a in range(3))
    r = I.random_fields(psi.shape, 31)
    z = O.precondition(g, prm, ev, psi, r, "diagonal")
    for i in range(2):
        assert np.max(np.abs(z[i] - r[i] / (sum(trap) / 2.0 + V))) < 1e-13 * np.max(np.abs(r[i]))
    k = math.pi / g.L[0] * 4
    wave = np.exp(1j * k * X[0]) * np.ones(g.shape)
    zk = O.precondition(g, prm, ev, psi, np.stack([wave, 2 * wave]), "kinetic")
    for i in range(2):
        assert np.max(np.abs(zk[i] - (i + 1) * wave / (sum(trap) / 2.0 + 0.5 * k * k))) < 1e-13
    zkd = O.precondition(g, prm, ev, psi, r, "kinetic+diagonal")
    assert np.max(np.abs(zkd - O.precondition(g, prm, ev, psi, z, "kinetic"))) < 1e-14 * np.max(np.abs(zkd))


@pytest.mark.parametrize("comp", [0, 1])
def test_preconditioner_shift_and_pv_plane_wave_closed_form(comp):
    """One occupied component psi_c = a + b cos(k z) (the other zero) with every
    coupling on.  Its terms have closed forms: T psi_c = b k^2/2 cos(kz); the
    density has modes 0, k, 2k along z, so Phi_c = 2 gdd_cc (density minus its
    mean) (kernel +2 g_dd along the dipoles, 0 at k = 0); with the other
    density zero the LHY chemical potential is the single-component
    mu_LHY = (5/2) kappa eta_s^{-5/2} (2 g_cc)^{5/2} n^{3/2} Q5(gdd_cc/g_cc).  Hence
    alpha_c = <psi,T psi> + int (V + g_cc n + mu_LHY) n (the dipolar energy
    excluded) and P_V,c = max(|alpha_c| + V + g_cc n + mu_LHY, 1e-2 |alpha_c|).
    Adding Phi to P_V, dropping mu_LHY or V, or taking mu_c for alpha_c fails."""
    g = O.Grid((8, 10, 16), (3.0, 3.5, 4.0))
    trap = (0.7, 0.9, 1.3)
    gm = np.array([[310.0, 140.0], [140.0, 260.0]])
    gdd = np.array([[220.0, 90.0], [90.0, 180.0]])
    prm = _prm(g=gm, gdd=gdd, kappa=21.0, eta_s=570.0, nodes=32, trap=trap)
    X = [g.x[0][None, None, :], g.x[1][None, :, None], g.x[2][:, None, None]]
    vol = 8.0 * g.L[0] * g.L[1] * g.L[2]
    k = math.pi / g.L[2] * 2
    a = 1.0 / math.sqrt(vol * (1.0 + 0.3 ** 2 / 2))
    b = 0.3 * a
    phi = (a + b * np.cos(k * X[2])) * np.ones(g.shape)
    psi = np.zeros((2,) + g.shape, dtype=np.complex128)
    psi[comp] = phi
    ev = O.evaluate(g, prm, psi)
    n = phi ** 2
    V = 0.5 * sum(trap[ax] ** 2 * X[ax] ** 2 for ax in range(3))
    gc, dc = gm[comp, comp], gdd[comp, comp]
    muL = 2.5 * prm.kappa * prm.eta_s ** -2.5 * (2 * gc) ** 2.5 * n ** 1.5 * _q5_closed_form(dc / gc)
    kin = vol * b * b * k * k / 4.0
    alpha = kin + g.dV * np.sum((V + gc * n + muL) * n)
    phi_dd = 2.0 * dc * (n - (a * a + b * b / 2.0))
    mu = alpha + g.dV * np.sum(phi_dd * n)
    assert abs(ev.mu[comp] - mu) < 1e-12 * abs(mu)
    sh = O.preconditioner_shift(g, ev, psi)
    assert abs(sh[comp] - alpha) < 1e-12 * abs(alpha)
    assert abs(alpha - mu) > 1e-3 * abs(alpha)  # the dipolar part is not negligible here
    r = I.random_fields(psi.shape, 32)
    z = O.precondition(g, prm, ev, psi, r, "diagonal")
    PV = np.maximum(abs(alpha) + V + gc * n + muL, 1e-2 * abs(alpha))
    assert np.max(np.abs(z[comp] - r[comp] / PV)) < 1e-12 * np.max(np.abs(r[comp] / PV))


def test_preconditioner_pv_floor_binds():
    """Where alpha + V + sum_j g_ij n_j + mu_LHY falls below 1e-2 |alpha| (an
    attractive contact coupling), P_V is the floor 1e-2 |alpha| (Sec. IV.B's
    small positive shift); elsewhere it is the unfloored value."""
    g = O.Grid((8, 8, 16), (3.0, 3.0, 4.0))
    prm = _prm(g=((-500.0, 0.0), (0.0, 100.0)), trap=(0.0, 0.0, 0.0))
    X = g.x[2][:, None, None]
    vol = 8.0 * g.L[0] * g.L[1] * g.L[2]
    k = math.pi / g.L[2] * 2
    a = 1.0 / math.sqrt(vol * (1.0 + 0.9 ** 2 / 2))
    phi = (a + 0.9 * a * np.cos(k * X)) * np.ones(g.shape)
    psi = np.stack([phi, phi]).astype(np.complex128)
    ev = O.evaluate(g, prm, psi)
    n = phi ** 2
    alpha = abs(O.preconditioner_shift(g, ev, psi)[0])
    raw = alpha + (-500.0) * n
    assert np.any(raw < 1e-2 * alpha) and np.any(raw > 1e-2 * alpha)
    r = I.random_fields(psi.shape, 33)
    z = O.precondition(g, prm, ev, psi, r, "diagonal")
    assert np.max(np.abs(z[0] - r[0] / np.maximum(raw, 1e-2 * alpha))) < 1e-12 * np.max(np.abs(z[0]))


def _beta_fields():
    """Hand-built fields on a grid with dV = 1, nonzero only at three points,
    so every inner product is an exact small rational:
      d = r - r_prev: comp 1 at A = 2, comp 2 at B = 1 - i
      z:              comp 1 at A = 3/2, comp 2 at B = 2 + 3i
      p_prev:         comp 1 at A = 1/4, comp 1 at C = 7, comp 2 at B = -i
      Re<d, z>      = 2 * 3/2 + Re((1 + i)(2 + 3i)) = 3 - 1 = 2
      Re<d, p_prev> = 2 * 1/4 + Re((1 + i)(-i))     = 1/2 + 1 = 3/2
    """
    g = O.Grid((4, 4, 4), (2.0, 2.0, 2.0))
    assert g.dV == 1.0
    A, B, C = (0, 1, 2), (3, 0, 1), (2, 2, 2)
    z0 = np.zeros((2,) + g.shape, dtype=np.complex128)
    r_prev, r, z, p_prev = z0.copy(), z0.copy(), z0.copy(), z0.copy()
    r_prev[0][A], r_prev[1][B] = 1.0, 2j
    r[0][A], r[1][B] = 3.0, 1.0 + 1j
    z[0][A], z[1][B] = 1.5, 2.0 + 3j
    p_prev[0][A], p_prev[0][C], p_prev[1][B] = 0.25, 7.0, -1j
    return g, r, z, r_prev, p_prev


def test_beta_hs_and_pr_hand_computed():
    """HS+ = 2 / (3/2) = 4/3; PR+ with Re<r_prev, z_prev> = 4/5 is 2 / (4/5) = 5/2
    (Sec. IV.C; sums over both components).  Component 1 alone would give 3/(1/2)
    = 6, a missing conjugate 8/(3/2), r in place of r - r_prev 19/2 / ..."""
    g, r, z, r_prev, p_prev = _beta_fields()
    b, ok = O.cg_beta(g, r, z, r_prev, p_prev, 0.8, "HS")
    assert ok and abs(b - 4.0 / 3.0) < 1e-15
    b, ok = O.cg_beta(g, r, z, r_prev, p_prev, 0.8, "PR")
    assert ok and abs(b - 2.5) < 1e-15


def test_beta_clamp_and_restarts():
    """max(., 0): with z at A negated the numerator is -3 - 1 = -4, so both
    rules give 0 without a restart; a zero or non-finite denominator is a
    restart (beta = 0, ok False)."""
    g, r, z, r_prev, p_prev = _beta_fields()
    zn = z.copy()
    zn[0][0, 1, 2] = -1.5
    for rule in ("HS", "PR"):
        b, ok = O.cg_beta(g, r, zn, r_prev, p_prev, 0.8, rule)
        assert ok and b == 0.0
    b, ok = O.cg_beta(g, r, z, r_prev, np.zeros_like(p_prev), 0.8, "HS")
    assert not ok and b == 0.0
    b, ok = O.cg_beta(g, r, z, r_prev, p_prev, 0.0, "PR")
    assert not ok and b == 0.0
    rn = r.copy()
    rn[1][3, 0, 1] = np.nan
    for rule in ("HS", "PR"):
        b, ok = O.cg_beta(g, rn, z, r_prev, p_prev, 0.8, rule)
        assert not ok and b == 0.0


# ---------------------------------------------------------------- solver invariants
@pytest.fixture(scope="module")
def c1_small():
    """C1 physics on 16^3 (same box): cheap enough for solver invariants."""
    w = I.PRESETS["c1"]
    g = O.Grid((16, 16, 16), w.L)
    prm = O.Params(w.g, w.gdd, w.kappa, w.eta_s, 16, w.trap)
    ww = I.Workload("c1/16", (16, 16, 16), w.L, w.trap, w.g, w.gdd, w.lhy_c, w.seed)
    return g, prm, I.gaussian_start(ww)


def test_ncg_monotone_descent_and_norms(c1_small):
    g, prm, psi0 = c1_small
    tr = []
    opts = O.SolveOpts(precond="kinetic+diagonal", tol_res=1e-9)
    psi, rep = O.ncg_solve(g, prm, psi0, opts, trace=tr)
    assert rep["status"] == "converged"
    tau = opts.accept_rtol * abs(tr[0]["E"])
    for t in tr:
        assert t["E_new"] <= t["E"] + tau
    for i in range(2):
        assert abs(O.inner(g, psi[i], psi[i]).real - 1.0) < 1e-13


def test_ncg_all_preconditioners_same_minimum(c1_small):
    g, prm, psi0 = c1_small
    Es = []
    for mode in O.PRECOND_MODES:
        _, rep = O.ncg_solve(g, prm, psi0, O.SolveOpts(precond=mode, tol_res=1e-9))
        assert rep["status"] == "converged", mode
        Es.append(rep["E"])
    assert max(Es) - min(Es) < 1e-11 * abs(Es[0])


def test_pr_plus_reaches_the_same_minimum(c1_small):
    """Polak-Ribiere+ beta (Sec. IV.C) converges to the HS+ minimum, descending monotonically."""
    g, prm, psi0 = c1_small
    _, rep_hs = O.ncg_solve(g, prm, psi0, O.SolveOpts(precond="kinetic+diagonal", tol_res=1e-9))
    tr = []
    opts = O.SolveOpts(precond="kinetic+diagonal", tol_res=1e-9, beta_rule="PR")
    _, rep_pr = O.ncg_solve(g, prm, psi0, opts, trace=tr)
    assert rep_pr["status"] == "converged"
    assert abs(rep_pr["E"] - rep_hs["E"]) < 1e-11 * abs(rep_hs["E"])
    assert any(t["beta"] > 0 for t in tr)
    tau = opts.accept_rtol * abs(tr[0]["E"])
    assert all(t["E_new"] <= t["E"] + tau for t in tr)


def test_periodic_restart(c1_small):
    """beta = 0 exactly at n mod K_r = 0 (short periodic restarts, Sec. IV.C), and
    the conjugate coefficient is used in between."""
    g, prm, psi0 = c1_small
    tr = []
    O.ncg_solve(g, prm, psi0, O.SolveOpts(precond="kinetic", tol_res=1e-9, restart_period=4, max_iter=14), trace=tr)
    acc = [t for t in tr if t["accepted"]]
    assert len(acc) >= 13
    for t in acc:
        if t["n"] % 4 == 0:
            assert t["beta"] == 0.0, t["n"]
    assert sum(t["beta"] > 0 for t in acc if t["n"] % 4) >= 6


def test_solver_failure_statuses(c1_small):
    """A non-finite start ends the solve as "nonfinite"; an acceptance rule no
    trial can meet ends it as "stagnated" after the first trial and armijo_max
    halvings (Sec. V, last paragraph)."""
    g, prm, psi0 = c1_small
    bad = psi0.copy()
    bad[1, 2, 3, 4] = np.inf
    with np.errstate(invalid="ignore"):
        _, rep = O.ncg_solve(g, prm, bad, O.SolveOpts(precond="kinetic", max_iter=3))
    assert rep["status"] == "nonfinite" and rep["iters"] == 0
    tr = []
    _, rep = O.ncg_solve(g, prm, psi0, O.SolveOpts(precond="kinetic", accept_rtol=-0.9, armijo_max=2), trace=tr)
    assert rep["status"] == "stagnated" and rep["armijo_steps"] == 3 and rep["iters"] == 0
    assert len(tr) == 1 and tr[0]["armijo"] == 3 and not tr[0]["accepted"]


def test_symmetric_mixture_keeps_components_equal():
    """Symmetric couplings and psi1 = psi2 at the start give psi1 = psi2 throughout;
    swapping the components leaves E unchanged."""
    w = I.PRESETS["c1"]
    g = O.Grid((16, 16, 16), w.L)
    prm = O.Params(w.g, w.gdd, w.kappa, w.eta_s, 16, w.trap)
    ww = I.Workload("sym", (16, 16, 16), w.L, w.trap, w.g, w.gdd, w.lhy_c, 3)
    psi0 = I.gaussian_start(ww)
    psi0[1] = psi0[0]
    psi, rep = O.ncg_solve(g, prm, psi0, O.SolveOpts(precond="kinetic", tol_res=1e-8, max_iter=60))
    assert np.max(np.abs(psi[0] - psi[1])) < 1e-12
    a = O.evaluate(g, prm, I.random_state((16, 16, 16), w.L, 9)).E
    b = O.evaluate(g, prm, I.random_state((16, 16, 16), w.L, 9)[::-1].copy()).E
    assert abs(a - b) < 1e-12 * abs(a)


def test_virial_identity_at_ground_state(c1_small):
    """Scaling psi -> lambda^{3/2} psi(lambda r) gives, at a minimiser,
    2 E_kin - 2 E_trap + 3 (E_c + E_dd) + 9/2 E_LHY = 0 (up to discretisation)."""
    w = I.PRESETS["c1"]
    g = O.Grid((32, 32, 48), w.L)
    prm = O.Params(w.g, w.gdd, w.kappa, w.eta_s, 16, w.trap)
    ww = I.Workload("vir", g.n, w.L, w.trap, w.g, w.gdd, w.lhy_c, 5)
    psi, rep = O.ncg_solve(g, prm, I.gaussian_start(ww), O.SolveOpts(precond="kinetic+diagonal", tol_res=1e-8))
    t = rep["terms"]
    vir = 2 * (t["kin1"] + t["kin2"]) - 2 * t["trap"] + 3 * (t["contact"] + t["dipolar"]) + 4.5 * t["lhy"]
    scale = 2 * (t["kin1"] + t["kin2"]) + 2 * t["trap"] + 3 * (t["contact"] + abs(t["dipolar"])) + 4.5 * t["lhy"]
    assert abs(vir) < 2e-3 * scale


def test_ite_and_ncg_reach_the_same_minimum():
    """Strang ITE has an O(dtau^2) fixed-point bias: Richardson-extrapolate two
    step sizes and compare with the NCG minimum."""
    w = I.Workload("ite", (16, 16, 16), (6.0, 6.0, 6.0), (1.0, 1.0, 2.0), ((60, 30), (30, 50)),
                   ((40, 30), (30, 40)), 5.0, 12)
    g = O.Grid(w.n, w.L)
    prm = O.Params(w.g, w.gdd, w.kappa, w.eta_s, 8, w.trap)
    psi0 = I.gaussian_start(w)
    _, rep = O.ncg_solve(g, prm, psi0, O.SolveOpts(precond="kinetic", tol_res=1e-10))
    E_cg = rep["E"]
    Es = []
    for dt in (0.02, 0.01):
        _, r = O.ite_solve(g, prm, psi0, dtau=dt, tol_dE=1e-13, max_steps=20000)
        Es.append(r["E"])
    E_extrap = (4 * Es[1] - Es[0]) / 3
    assert Es[1] >= E_cg - 1e-12
    assert abs(E_extrap - E_cg) < 0.05 * abs(Es[1] - E_cg) + 1e-9


# ---------------------------------------------------------------- stored regression values
def test_oracle_matches_stored_c1_values():
    """The oracle's C1 numbers stored by tests/golden/make_golden.py (oracle only)."""
    import json
    import os
    with open(os.path.join(os.path.dirname(__file__), "golden", "oracle_c1.json")) as f:
        gold = json.load(f)
    w = I.PRESETS["c1"]
    g = O.Grid(w.n, w.L)
    prm = O.Params(w.g, w.gdd, w.kappa, w.eta_s, w.lhy_nodes, w.trap)
    psi = I.gaussian_start(w)
    ev = O.evaluate(g, prm, psi)
    assert abs(ev.E - gold["initial"]["E"]) < 1e-12 * abs(ev.E)
    for k, v in gold["initial"]["terms"].items():
        assert abs(ev.terms[k] - v) < 1e-12 * max(1.0, abs(v))
    p = O.project(g, psi, I.raw_direction(w.n, w.L, gold["line_coeffs"]["direction_seed"]))
    E0, Ep, Epp = O.line_coeffs(g, prm, psi, p, ev)
    assert abs(Ep - gold["line_coeffs"]["Ep"]) < 1e-11 * abs(Ep)
    assert abs(Epp - gold["line_coeffs"]["Epp"]) < 1e-11 * abs(Epp)


# ---------------------------------------------------------------- parameter derivatives
def _with_param(prm, name, value):
    import copy
    q = copy.deepcopy(prm)
    if name in ("g11", "g22"):
        i = 0 if name == "g11" else 1
        q.g[i, i] = value
    elif name == "g12":
        q.g[0, 1] = q.g[1, 0] = value
    elif name in ("gdd11", "gdd22"):
        i = 0 if name == "gdd11" else 1
        q.gdd[i, i] = value
    elif name == "gdd12":
        q.gdd[0, 1] = q.gdd[1, 0] = value
    elif name == "kappa":
        q.kappa = value
    elif name == "eta_s":
        q.eta_s = value
    else:
        t = list(q.trap)
        t["xyz".index(name[-1])] = value
        q.trap = tuple(t)
    return q


def _param_value(prm, name):
    return {"g11": prm.g[0, 0], "g22": prm.g[1, 1], "g12": prm.g[0, 1], "gdd11": prm.gdd[0, 0],
            "gdd22": prm.gdd[1, 1], "gdd12": prm.gdd[0, 1], "kappa": prm.kappa, "eta_s": prm.eta_s,
            "trap_x": prm.trap[0], "trap_y": prm.trap[1], "trap_z": prm.trap[2]}[name]


def test_param_grad_matches_central_differences():
    """Every partial derivative against Richardson-extrapolated central
    differences of the energy, on a complex state with distinct couplings
    (a dropped LHY term or a wrong factor 1/2 fails by far more than 1e-6)."""
    w = _cm.mixed_workload((12, 10, 16))
    g, prm = _cm.oracle_case(w)
    psi = I.random_state(w.n, w.L, 5, width=(1.2, 1.5, 0.9))
    d = O.param_grad(g, prm, psi)
    for name in O.PARAM_NAMES:
        p0 = _param_value(prm, name)
        h = 1e-3 * abs(p0)

        def E(v):
            return O.evaluate(g, _with_param(prm, name, v), psi).E

        d1 = (E(p0 + h) - E(p0 - h)) / (2 * h)
        d2 = (E(p0 + h / 2) - E(p0 - h / 2)) / h
        fd = (4 * d2 - d1) / 3
        assert abs(d[name] - fd) < 1e-6 * max(abs(fd), 1e-3 * abs(O.evaluate(g, prm, psi).E)), name


def test_lhy_eta_derivatives_vanish_without_lhy_and_scale_with_kappa():
    w = _cm.mixed_workload((8, 8, 8))
    g, prm = _cm.oracle_case(w)
    psi = I.random_state(w.n, w.L, 6)
    n = np.abs(psi) ** 2
    a = O.lhy_eta_derivatives(prm, n[0], n[1])
    b = O.lhy_eta_derivatives(_with_param(prm, "kappa", 2 * prm.kappa), n[0], n[1])
    for x, y in zip(a, b):
        assert np.allclose(2 * x, y, rtol=1e-14, atol=0)
    z = O.lhy_eta_derivatives(_with_param(prm, "kappa", 0.0), n[0], n[1])
    assert all(np.all(v == 0) for v in z)


def test_hellmann_feynman_at_a_ground_state():
    """At a converged ground state dE0/dp equals the partial derivative at
    fixed psi (the normalisation does not depend on p): checked for g12,
    gdd12 and the z trap frequency against central differences of solved
    ground-state energies."""
    w = I.Workload("hf", (16, 16, 16), (6.0, 6.0, 6.0), (1.0, 1.0, 1.5), ((60.0, 25.0), (25.0, 50.0)),
                   ((40.0, 20.0), (20.0, 30.0)), 10.0, 7, "kinetic", 8)
    g, prm = _cm.oracle_case(w)
    psi0 = I.gaussian_start(w)
    opts = O.SolveOpts(precond="kinetic+diagonal", tol_res=1e-10, max_iter=4000)
    psi, rep = O.ncg_solve(g, prm, psi0, opts)
    assert rep["status"] == "converged"
    d = O.param_grad(g, prm, psi)
    for name in ("g12", "gdd12", "trap_z"):
        p0 = _param_value(prm, name)
        h = 1e-3 * abs(p0)
        Ep = O.ncg_solve(g, _with_param(prm, name, p0 + h), psi, opts)[1]["E"]
        Em = O.ncg_solve(g, _with_param(prm, name, p0 - h), psi, opts)[1]["E"]
        fd = (Ep - Em) / (2 * h)
        assert abs(fd - d[name]) < 1e-6 * max(1.0, abs(d[name])), name


# ---------------------------------------------------------------- blended preconditioner
def test_blend_limits_and_same_minimum():
    """The weighted combination reduces to P_V (weight 1) and P_Delta (weight
    0), is positive definite (Re<r, z> > 0), and the solver reaches the same
    minimum with it as with P_Delta alone."""
    w = _cm.mixed_workload((12, 10, 16))
    g, prm = _cm.oracle_case(w)
    psi = I.random_state(w.n, w.L, 8, width=(1.2, 1.5, 0.9))
    ev = O.evaluate(g, prm, psi)
    r = I.random_fields(psi.shape, 9)
    zv = O.precondition(g, prm, ev, psi, r, "diagonal")
    zd = O.precondition(g, prm, ev, psi, r, "kinetic")
    assert np.array_equal(O.precondition(g, prm, ev, psi, r, "blend", blend=1.0), zv)
    assert np.array_equal(O.precondition(g, prm, ev, psi, r, "blend", blend=0.0), zd)
    zb = O.precondition(g, prm, ev, psi, r, "blend", blend=0.3)
    for i in range(2):
        assert O.inner(g, r[i], zb[i]).real > 0
    w2 = I.Workload("bl", (16, 16, 16), (6.0, 6.0, 6.0), (1.0, 1.0, 1.5), ((60.0, 25.0), (25.0, 50.0)),
                    ((40.0, 20.0), (20.0, 30.0)), 10.0, 7, "kinetic", 8)
    g2, prm2 = _cm.oracle_case(w2)
    psi0 = I.gaussian_start(w2)
    _, ra = O.ncg_solve(g2, prm2, psi0, O.SolveOpts(precond="kinetic", tol_res=1e-10))
    _, rb = O.ncg_solve(g2, prm2, psi0, O.SolveOpts(precond="blend", blend=0.5, tol_res=1e-10))
    assert ra["status"] == rb["status"] == "converged"
    assert abs(ra["E"] - rb["E"]) < 1e-12 * abs(ra["E"])
