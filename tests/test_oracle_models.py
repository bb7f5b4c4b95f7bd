"""Pins of the oracle's model options (Table 1 and the viscous-term
specialisations of Section 3): the cubic-spline, quadratic and Gaussian
kernels, SPH formulation 2, the Morris / Monaghan / Espanol-Revenga viscous
models with the three averaging operators, and Molteni-Colagrossi density
diffusion.  Every pin is a fact of the mathematics (unit integral, continuum
limits of the lattice sums, exact antisymmetries, identities between means),
not the oracle's own formula retyped.

Lattice pins use h = 2.5 dp, where the lattice sums of the kernel moments
are within 0.7 % of their integrals for all four kernels (measured by
test_lattice_moments_converge); their tolerance is 2 %.
"""
import math

import numpy as np
import pytest
from scipy import integrate

import oracle
from paper_2207_11328_gb300 import scenes

H = 0.026
KERNELS = [(1, 2.0), (2, 2.0), (3, 3.0)]  # (type, radius in h)
DP = 0.01
RHO0 = 1000.0
HR = 2.5  # h / dp of the lattice pins


def _quad(f, a, b, points=()):
    val, _ = integrate.quad(f, a, b, epsabs=1e-15, epsrel=1e-13, limit=400, points=list(points) or None)
    return val


# ---------------------------------------------------------------- kernels
@pytest.mark.parametrize("kt,Q", KERNELS)
def test_kernel_unit_integral(kt, Q):
    # Section 2.1: int W dV = 1 over the support
    val = _quad(lambda r: 4 * math.pi * r * r * oracle.kernel_W(r, H, kt, Q), 0, Q * H, points=(H,))
    assert abs(val - 1.0) <= 1e-11


@pytest.mark.parametrize("kt,Q", KERNELS)
def test_kernel_F_is_dW_dr_over_r(kt, Q):
    for q in np.linspace(0.05, Q - 0.05, 47):
        if abs(q - 1.0) < 1e-3:
            continue
        r = q * H
        eps = 1e-6 * H
        dWdr = (oracle.kernel_W(r + eps, H, kt, Q) - oracle.kernel_W(r - eps, H, kt, Q)) / (2 * eps)
        F = oracle.kernel_F(r, H, kt, Q)
        assert abs(dWdr / r - F) <= 1e-7 * abs(F) + 1e-3


@pytest.mark.parametrize("kt,Q", KERNELS)
def test_kernel_F_moment(kt, Q):
    # integration by parts (W vanishes at the cut): 4 pi int r^4 F dr = -3
    val = _quad(lambda r: 4 * math.pi * r ** 4 * oracle.kernel_F(r, H, kt, Q), 0, Q * H, points=(H,))
    assert abs(val + 3.0) <= 1e-10


@pytest.mark.parametrize("kt,Q", KERNELS)
def test_kernel_support_and_continuity(kt, Q):
    for r in (Q * H, 1.0001 * Q * H, 2 * Q * H):
        assert oracle.kernel_W(r, H, kt, Q) == 0.0 and oracle.kernel_F(r, H, kt, Q) == 0.0
    # W continuous (and zero) at the cut and, for the piecewise cubic, W and F continuous at q = 1
    assert abs(oracle.kernel_W((Q - 1e-9) * H, H, kt, Q)) < 1e-6 * oracle.kernel_W(0.0, H, kt, Q)
    e = 1e-9
    for fn in (oracle.kernel_W, oracle.kernel_F):
        lo, hi = fn((1 - e) * H, H, kt, Q), fn((1 + e) * H, H, kt, Q)
        assert lo == pytest.approx(hi, rel=1e-7)


def test_kernel_shapes():
    # the shape functions named in Table 1 / the kernel listing, up to normalisation
    W0 = oracle.kernel_W(0.0, H, 2, 2.0)
    for q in (0.2, 0.9, 1.7):
        assert oracle.kernel_W(q * H, H, 2, 2.0) / W0 == pytest.approx((1 - q / 2) ** 2, rel=1e-13)
        # truncated Gaussian listing: f(q) = -exp(-q^2)
        assert oracle.kernel_F(q * H, H, 3, 3.0) / oracle.kernel_F(1e-300, H, 3, 3.0) == pytest.approx(
            math.exp(-q * q), rel=1e-13)
    # cubic spline: W(1)/W(0) = 1/4, W(1.5)/W(0) = (0.5)^3/4
    c0 = oracle.kernel_W(0.0, H, 1, 2.0)
    assert oracle.kernel_W(H, H, 1, 2.0) / c0 == pytest.approx(0.25, rel=1e-13)
    assert oracle.kernel_W(1.5 * H, H, 1, 2.0) / c0 == pytest.approx(0.125 / 4, rel=1e-13)


# ---------------------------------------------------------- lattice helpers
def _cube(Q):
    n = 2 * int(math.ceil(Q * HR)) + 3
    pos = scenes._lattice(n, n, n, DP)
    c = pos.mean(0)
    i = int(np.argmin(((pos - c) ** 2).sum(1)))
    return pos, pos[i].copy(), i


def _p(kt=0, Q=2.0, **kw):
    base = dict(dp=DP, h=HR * DP, kernel_radius=Q, kernel_type=kt, rho0=RHO0, c0=10.0, gamma=7.0,
                visc_model=1, alpha=0.0, nu=1e-3, origin=(0, 0, 0), size=(1, 1, 1), periodic_mask=0)
    base.update(kw)
    return oracle.params(**base)


def _centre_rhs(p, pos, vel, delta, mass, i):
    n = len(pos)
    a, drho, _, _ = oracle.rhs_sample(p, pos, vel, delta, mass, np.zeros(n, np.uint8), [i])
    return a[0], drho[0]


@pytest.mark.parametrize("kt,Q", [(0, 2.0)] + KERNELS)
def test_lattice_moments_converge(kt, Q):
    # at h = 2.5 dp the lattice sums of r^2 F, x^4 F/r^2 and x^2 y^2 F/r^2 are within
    # 0.7 % of -3, -3/5 and -1/5 (the isotropic integrals): the basis of the 2 % pins
    h = HR * DP
    n = int(math.ceil(Q * HR)) + 1
    g = np.arange(-n, n + 1) * DP
    X, Y, Z = [t.ravel() for t in np.meshgrid(g, g, g, indexing="ij")]
    r = np.sqrt(X * X + Y * Y + Z * Z)
    m = (r > 0) & (r < Q * h)
    F = np.array([oracle.kernel_F(t, h, kt, Q) for t in r[m]])
    V = DP ** 3
    x, y, rr = X[m], Y[m], r[m]
    assert (V * F * rr ** 2).sum() == pytest.approx(-3.0, rel=0.007)
    assert (V * F * x ** 4 / rr ** 2).sum() == pytest.approx(-0.6, rel=0.007)
    assert (V * F * x * x * y * y / rr ** 2).sum() == pytest.approx(-0.2, rel=0.007)


# --------------------------------------------------------- viscous models
# continuum limits (constant density): Morris nu lap u; Monaghan with K = d + 2
# nu (lap u + 2 grad div u); Espanol-Revenga nu lap u + (zeta + nu/3) grad div u
SHEAR = lambda d: np.stack([d[:, 1] ** 2, 0 * d[:, 0], 0 * d[:, 0]], 1)  # noqa: E731  lap u = 2 x^
STRETCH = lambda d: np.stack([d[:, 0] ** 2, 0 * d[:, 0], 0 * d[:, 0]], 1)  # noqa: E731  lap u = grad div u = 2 x^


@pytest.mark.parametrize("kt,Q", [(0, 2.0)] + KERNELS)
@pytest.mark.parametrize("model,field,expect", [
    (1, "shear", 2.0), (1, "stretch", 2.0),
    (2, "shear", 2.0), (2, "stretch", 6.0),
    (3, "shear", 2.0), (3, "stretch", 8.0 / 3.0)])
def test_viscous_models_continuum_limit(kt, Q, model, field, expect):
    pos, c, i = _cube(Q)
    n = len(pos)
    eps, nu = 0.5, 1e-3
    vel = eps * (SHEAR if field == "shear" else STRETCH)(pos - c)
    a, _ = _centre_rhs(_p(kt, Q, visc_model=model, nu=nu), pos, vel, np.zeros(n), np.full(n, RHO0 * DP ** 3), i)
    assert a[0] == pytest.approx(expect * nu * eps, rel=0.02)
    assert abs(a[1]) + abs(a[2]) < 1e-9 * abs(a[0])


@pytest.mark.parametrize("field,expect", [("shear", 0.0), ("stretch", 2.0)])
def test_bulk_viscosity_acts_on_divergence_only(field, expect):
    # Espanol-Revenga with zeta only: zeta grad div u (zero for the divergence-free shear)
    pos, c, i = _cube(2.0)
    n = len(pos)
    eps, zeta = 0.5, 2e-3
    vel = eps * (SHEAR if field == "shear" else STRETCH)(pos - c)
    a, _ = _centre_rhs(_p(visc_model=3, nu=0.0, zeta=zeta), pos, vel, np.zeros(n), np.full(n, RHO0 * DP ** 3), i)
    scale = 2.0 * zeta * eps
    assert a[0] == pytest.approx(expect * zeta * eps, abs=0.02 * scale)


def test_averaging_operators_are_the_three_means():
    # two particles of different density: the laminar force is linear in mubar, so
    # geometric^2 = arithmetic * harmonic and arithmetic > geometric > harmonic
    pos = np.array([[0.0, 0.0, 0.0], [0.013, 0.004, -0.002]])
    vel = np.array([[0.1, -0.2, 0.05], [-0.3, 0.1, 0.2]])
    delta = np.array([0.02, -0.03])
    mass = np.full(2, RHO0 * DP ** 3)
    a = {}
    for op in (0, 1, 2):
        p = _p(visc_model=1, visc_avg=op, c0=0.0, h=0.013)
        a[op] = oracle.rhs(p, pos, vel, delta, mass, np.zeros(2, np.uint8))[0][0]
    assert np.allclose(a[2] ** 2, a[1] * a[0], rtol=1e-12)
    assert np.all(np.abs(a[1]) > np.abs(a[2])) and np.all(np.abs(a[2]) > np.abs(a[0]))
    # equal densities: all three means coincide
    b = [oracle.rhs(_p(visc_model=1, visc_avg=op, c0=0.0, h=0.013), pos, vel, np.full(2, 0.01), mass,
                    np.zeros(2, np.uint8))[0][0] for op in (0, 1, 2)]
    assert np.allclose(b[0], b[1], rtol=1e-14) and np.allclose(b[0], b[2], rtol=1e-14)


# ------------------------------------------------------------ formulation 2
def _random_periodic(n=8, seed=1):
    s = scenes.periodic_box(n_per_axis=n, dp=0.02, jitter=0.3, seed=seed)
    rng = np.random.default_rng(seed)
    return s, rng


def test_formulation2_equals_formulation1_at_uniform_density():
    # rho_i = rho_j: (P_i + P_j)/(rho_i rho_j) = P_i/rho_i^2 + P_j/rho_j^2 and rho_i/rho_j = 1
    s, _ = _random_periodic()
    d = np.full(s.n, 0.012)
    r1 = oracle.rhs(oracle.params(s), s.pos, s.vel, d, s.mass, s.ptype)
    r2 = oracle.rhs(oracle.params(s, formulation=1), s.pos, s.vel, d, s.mass, s.ptype)
    for u, v in zip(r1, r2):
        assert np.allclose(u, v, rtol=1e-12, atol=1e-12 * np.abs(u).max())


def test_formulation2_conserves_momentum():
    # the pair force m_i m_j (P_i + P_j)/(rho_i rho_j) x_ij F_ij is antisymmetric
    s, rng = _random_periodic(seed=2)
    d = rng.uniform(-0.02, 0.02, s.n)
    a, _ = oracle.rhs(oracle.params(s, formulation=1, alpha=0.05), s.pos, s.vel, d, s.mass, s.ptype)
    tot = (s.mass[:, None] * a).sum(0)
    assert np.all(np.abs(tot) <= 1e-11 * (s.mass[:, None] * np.abs(a)).sum(0))
    a1, _ = oracle.rhs(oracle.params(s, alpha=0.05), s.pos, s.vel, d, s.mass, s.ptype)
    assert np.max(np.abs(a - a1)) > 1e-3 * np.max(np.abs(a1))  # the two formulations differ here


def test_formulation2_continuity_weights_volumes():
    # drho_i/rho_i = sum_j (m_j/rho_j) u_ij.x_ij F_ij: with m_j = rho_j dp^3 every
    # neighbour weighs dp^3 whatever its density, so for u = eps x the rate per unit
    # density equals the uniform-lattice rate of formulation 1 divided by rho0
    pos, c, i = _cube(2.0)
    n = len(pos)
    rng = np.random.default_rng(5)
    d = rng.uniform(-0.02, 0.02, n)
    mass = RHO0 * (1 + d) * DP ** 3
    vel = 1e-3 * (pos - c)
    _, r2 = _centre_rhs(_p(formulation=1, visc_model=0, nu=0.0), pos, vel, d, mass, i)
    _, r1 = _centre_rhs(_p(visc_model=0, nu=0.0), pos, vel, np.zeros(n), np.full(n, RHO0 * DP ** 3), i)
    assert r2 / (RHO0 * (1 + d[i])) == pytest.approx(r1 / RHO0, rel=1e-11)


# -------------------------------------------------------- density diffusion
def test_density_diffusion_laplacian():
    # xi h c0 sum_j psi_ij.grad W V_j -> xi h c0 lap rho: rho = rho0 (1 + eps x^2) gives 2 eps rho0
    pos, c, i = _cube(2.0)
    n = len(pos)
    eps = 50.0
    d = eps * ((pos - c)[:, 0]) ** 2
    mass = RHO0 * (1 + d) * DP ** 3  # V_j = dp^3
    xi, c0 = 0.1, 10.0
    p = _p(visc_model=0, nu=0.0, ddiff=1, ddiff_coef=xi, c0=c0)
    _, drho = _centre_rhs(p, pos, np.zeros((n, 3)), d, mass, i)
    assert drho == pytest.approx(xi * HR * DP * c0 * 2 * eps * RHO0, rel=0.02)


def test_density_diffusion_conserves_volume_weighted_mass():
    # sum_i V_i D_i = 2 xi h c0 sum_ij V_i V_j (rho_i - rho_j) F_ij = 0 (antisymmetric)
    s, rng = _random_periodic(seed=3)
    d = rng.uniform(-0.02, 0.02, s.n)
    base = oracle.rhs(oracle.params(s), s.pos, s.vel, d, s.mass, s.ptype)[1]
    dd = oracle.rhs(oracle.params(s, ddiff=1, ddiff_coef=0.1), s.pos, s.vel, d, s.mass, s.ptype)[1] - base
    V = s.mass / (RHO0 * (1 + d))
    assert abs((V * dd).sum()) <= 1e-11 * (V * np.abs(dd)).sum()
    assert np.max(np.abs(dd)) > 0
    # uniform density: no diffusion at all
    u = np.full(s.n, 0.01)
    b0 = oracle.rhs(oracle.params(s), s.pos, s.vel, u, s.mass, s.ptype)[1]
    b1 = oracle.rhs(oracle.params(s, ddiff=1, ddiff_coef=0.1), s.pos, s.vel, u, s.mass, s.ptype)[1]
    assert np.allclose(b0, b1, rtol=0, atol=1e-12 * np.abs(b0).max())


def test_density_diffusion_sign_and_fluid_pairs_only():
    # a light particle among denser fluid neighbours gains density; boundary
    # neighbours do not diffuse into the fluid (reading D1)
    pos = np.array([[0.0, 0.0, 0.0], [0.012, 0.0, 0.0], [-0.012, 0.0, 0.0]])
    mass = np.full(3, RHO0 * DP ** 3)
    d = np.array([0.0, 0.01, 0.01])
    p = _p(visc_model=0, nu=0.0, ddiff=1, ddiff_coef=0.1, h=0.013)
    q = _p(visc_model=0, nu=0.0, h=0.013)
    z = np.zeros((3, 3))
    fl = np.zeros(3, np.uint8)
    gain = oracle.rhs(p, pos, z, d, mass, fl)[1][0] - oracle.rhs(q, pos, z, d, mass, fl)[1][0]
    assert gain > 0
    bnd = np.array([0, 1, 1], np.uint8)
    assert oracle.rhs(p, pos, z, d, mass, bnd)[1][0] == oracle.rhs(q, pos, z, d, mass, bnd)[1][0]
