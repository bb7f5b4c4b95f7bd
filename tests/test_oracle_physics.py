"""Pins of the oracle's time derivatives (Section 2.1, golden-rule continuity
and momentum; readings C1-C5) against closed forms, exact symmetries and
invariants.  Each pin is chosen so a plausible mistake (sign, dropped m_j,
wrong coefficient, transposed operand) fails it."""
import numpy as np
import pytest

import oracle
from paper_2207_11328_gb300 import scenes

DP = 0.02
RHO0 = 1000.0


def _block(n):
    pos = scenes._lattice(n, n, n, DP)
    c = pos.mean(0)
    centre = int(np.argmin(((pos - c) ** 2).sum(1)))
    return pos, c, centre


def _params(**kw):
    base = dict(dp=DP, h=1.3 * DP, rho0=RHO0, c0=20.0, gamma=7.0, visc_model=0, alpha=0.0,
                origin=(0, 0, 0), size=(0.26, 0.26, 0.26), periodic_mask=0)
    base.update(kw)
    return oracle.params(**base)


def _lattice_moment():
    # sum_j V_j r_ij^2 F_ij over the full h = 1.3 dp lattice neighbourhood:
    # the quadrature of int r^2 F dV = -3 (used to state the lattice error bound)
    s = 0.0
    for i in range(-3, 4):
        for j in range(-3, 4):
            for k in range(-3, 4):
                r = DP * np.sqrt(i * i + j * j + k * k)
                if 0 < r < 2.6 * DP:
                    s += DP ** 3 * r * r * oracle.kernel_F(r, 1.3 * DP)
    return s


def test_lattice_quadrature_close_to_closed_form():
    m = _lattice_moment()
    assert abs(m / -3.0 - 1.0) < 0.03


def test_continuity_linear_field():
    # C1: for u = eps (x - c), drho/dt = -rho div u = -3 eps rho0 (closed form,
    # within the lattice quadrature error of the kernel moment)
    pos, c, i = _block(13)
    eps = 1e-3
    n = len(pos)
    a, drho = oracle.rhs(_params(), pos, eps * (pos - c), np.zeros(n), np.full(n, RHO0 * DP ** 3),
                         np.zeros(n, np.uint8))
    assert drho[i] / (-3 * eps * RHO0) == pytest.approx(_lattice_moment() / -3.0, rel=1e-9)
    assert drho[i] / (-3 * eps * RHO0) == pytest.approx(1.0, abs=0.03)


def test_continuity_sign_approaching_pair():
    # C1: two approaching particles compress (drho > 0); receding expand
    h = 1.3 * DP
    pos = np.array([[0.1, 0.1, 0.1], [0.1 + h, 0.1, 0.1]])
    m = np.full(2, RHO0 * DP ** 3)
    for v, sign in ((0.1, 1), (-0.1, -1)):
        vel = np.array([[v, 0, 0], [-v, 0, 0]])
        a, drho = oracle.rhs(_params(), pos, vel, np.zeros(2), m, np.zeros(2, np.uint8))
        assert np.all(np.sign(drho) == sign)


def test_pressure_gradient_linear_density():
    # C2: a = -grad P / rho for a linear density ramp (lattice with constant m):
    # the golden-rule sum gives rho0 grad(P/rho^2) -> -c0^2 kappa at delta ~ 0
    pos, c, i = _block(13)
    n = len(pos)
    kappa = 1e-3 / 0.26
    delta = kappa * (pos[:, 2] - c[2])
    a, drho = oracle.rhs(_params(), pos, np.zeros_like(pos), delta, np.full(n, RHO0 * DP ** 3),
                         np.zeros(n, np.uint8))
    assert abs(a[i, 0]) < 1e-9 and abs(a[i, 1]) < 1e-9
    assert a[i, 2] / (-400.0 * kappa) == pytest.approx(_lattice_moment() / -3.0, rel=2e-3)


def test_mass_factor_in_pressure_term():
    # C2: the pressure term scales with the neighbours' mass m_j
    pos, c, i = _block(9)
    n = len(pos)
    delta = 1e-3 * (pos[:, 2] - c[2]) / 0.18
    p = _params(size=(0.18,) * 3)
    a1, _ = oracle.rhs(p, pos, np.zeros_like(pos), delta, np.full(n, RHO0 * DP ** 3), np.zeros(n, np.uint8))
    a2, _ = oracle.rhs(p, pos, np.zeros_like(pos), delta, np.full(n, 2 * RHO0 * DP ** 3), np.zeros(n, np.uint8))
    assert a2[i, 2] == pytest.approx(2 * a1[i, 2], rel=1e-12)


def test_uniform_compression_at_rest_cancels():
    # exact special case: uniform periodic lattice, uniform delta, at rest, g = 0
    s = scenes.periodic_box(n_per_axis=10, dp=DP)
    p = oracle.params(s, alpha=0.02)
    delta = np.full(s.n, 3e-3)
    a, drho = oracle.rhs(p, s.pos, np.zeros((s.n, 3)), delta, s.mass, s.ptype)
    # scale of individual terms: m * 2 P/rho^2 * |x F| at r = h
    P = oracle.eos(p, 3e-3)
    term = s.mass[0] * 2 * P / (RHO0 * 1.003) ** 2 * 1.3 * DP * abs(oracle.kernel_F(1.3 * DP, 1.3 * DP))
    assert np.max(np.abs(a)) <= 1e-12 * 80 * term
    assert np.max(np.abs(drho)) == 0.0


@pytest.mark.parametrize("visc,alpha,nu", [(0, 0.02, 0.0), (0, 0.0, 0.0), (1, 0.0, 0.1)])
def test_momentum_conserved_periodic(visc, alpha, nu):
    # pair antisymmetry: sum_i m_i a_i = 0 with g = 0 in a periodic box
    s = scenes.periodic_box(n_per_axis=9, dp=DP, jitter=0.2, seed=11)
    rng = np.random.default_rng(3)
    delta = rng.uniform(-2e-3, 2e-3, s.n)
    p = oracle.params(s, visc_model=visc, alpha=alpha, nu=nu)
    a, drho = oracle.rhs(p, s.pos, s.vel, delta, s.mass, s.ptype)
    m = s.mass.astype(np.float64)[:, None]
    tot = np.abs((m * a).sum(0))
    scale = np.abs(m * a).sum()
    assert np.all(tot <= 1e-12 * scale)


def test_artificial_viscosity_switch():
    # C4: Pi acts only on approaching pairs and opposes the approach; alpha = 0 removes it
    h = 1.3 * DP
    pos = np.array([[0.1, 0.1, 0.1], [0.1 + h, 0.1, 0.1]])
    m = np.full(2, RHO0 * DP ** 3)
    t = np.zeros(2, np.uint8)
    app = np.array([[0.1, 0, 0], [-0.1, 0, 0]])
    a, _ = oracle.rhs(_params(alpha=0.1), pos, app, np.zeros(2), m, t)
    assert a[0, 0] < 0 < a[1, 0]
    a0, _ = oracle.rhs(_params(alpha=0.0), pos, app, np.zeros(2), m, t)
    assert np.all(a0 == 0.0)
    a2, _ = oracle.rhs(_params(alpha=0.1), pos, -app, np.zeros(2), m, t)
    assert np.all(a2 == 0.0)
    # linear in alpha (closed form Pi = -alpha h c0 mu / rhobar)
    a3, _ = oracle.rhs(_params(alpha=0.2), pos, app, np.zeros(2), m, t)
    assert a3[0, 0] == pytest.approx(2 * a[0, 0], rel=1e-12)


def test_laminar_shear_closed_form():
    # C3: Morris laminar term with harmonic kinematic mean -> nu * laplacian(u)
    n = 24
    s = scenes.periodic_box(n_per_axis=n, dp=DP)
    L = n * DP
    k = 2 * np.pi / L
    u = np.zeros((s.n, 3))
    u[:, 0] = 1e-3 * np.sin(k * s.pos[:, 1])
    p = oracle.params(s, visc_model=1, nu=0.1, alpha=0.0)
    a, _ = oracle.rhs(p, s.pos, u, np.zeros(s.n), s.mass, s.ptype)
    ref = -0.1 * k * k * u[:, 0]
    err = np.max(np.abs(a[:, 0] - ref)) / np.max(np.abs(ref))
    assert err < 0.03
    # uniform velocity: no viscous force
    u2 = np.tile([0.3, -0.2, 0.1], (s.n, 1))
    a2, _ = oracle.rhs(p, s.pos, u2, np.zeros(s.n), s.mass, s.ptype)
    assert np.max(np.abs(a2)) < 1e-12


def test_boundary_particles():
    # C5: boundary particles get no acceleration, see u = 0 whatever was given,
    # and obey continuity with the fluid's velocity
    h = 1.3 * DP
    pos = np.array([[0.1, 0.1, 0.1], [0.1 + h, 0.1, 0.1]])
    m = np.full(2, RHO0 * DP ** 3)
    t = np.array([0, 1], np.uint8)
    vel = np.array([[0.1, 0, 0], [5.0, 1.0, 2.0]])   # boundary velocity is ignored
    p = _params(alpha=0.05, g=(0, 0, -9.81))
    a, drho = oracle.rhs(p, pos, vel, np.zeros(2), m, t)
    assert np.all(a[1] == 0.0)
    vel0 = vel.copy(); vel0[1] = 0
    a0, drho0 = oracle.rhs(p, pos, vel0, np.zeros(2), m, t)
    assert np.array_equal(a, a0) and np.array_equal(drho, drho0)
    assert drho[1] > 0 and drho[0] > 0      # fluid approaching the wall compresses both
    assert a[0, 2] == pytest.approx(-9.81)  # gravity on the fluid only


def test_cfl_dt_branches():
    # C7: dt = min(cfl * min(sqrt(h/|a|max), h/c0), 0.125 h^2/nu)
    p = _params(cfl=0.3, c0=20.0)
    h = 1.3 * DP
    a = np.array([[0, 0, 0.0], [3.0, 4.0, 0.0]])
    t = np.zeros(2, np.uint8)
    assert oracle.cfl_dt(p, a, t) == pytest.approx(0.3 * min(np.sqrt(h / 5.0), h / 20.0))
    a_big = np.array([[0, 0, 1e6]])
    assert oracle.cfl_dt(p, a_big, np.zeros(1, np.uint8)) == pytest.approx(0.3 * np.sqrt(h / 1e6))
    # boundary accelerations are ignored
    assert oracle.cfl_dt(p, a_big, np.ones(1, np.uint8)) == pytest.approx(0.3 * h / 20.0)
    pl = _params(cfl=0.3, c0=1.0, visc_model=1, nu=0.1)
    assert oracle.cfl_dt(pl, np.zeros((1, 3)), np.zeros(1, np.uint8)) == pytest.approx(0.125 * h * h / 0.1)
    # the viscous limit does not scale with the CFL factor
    pl2 = _params(cfl=0.6, c0=1.0, visc_model=1, nu=0.1)
    assert oracle.cfl_dt(pl2, np.zeros((1, 3)), np.zeros(1, np.uint8)) == pytest.approx(0.125 * h * h / 0.1)


def test_viscous_time_step_is_within_the_stable_range():
    # The laminar (Morris) term's fastest mode on the lattice: u_x = eps (-1)^(i+j+k),
    # neighbours of odd parity move against the particle.  Its decay rate lambda = -a_x/u_x
    # comes from the oracle's own right-hand side.  The two-stage predictor-corrector
    # u* = u + dt/2 a(u), u' = u + dt a(u*) multiplies this mode by 1 - z + z^2/2 with
    # z = lambda dt, which stays within [-1, 1] only for 0 <= z <= 2.  The viscous
    # limit of the time step must keep z <= 2; the CFL factor 0.3 applied to h^2/nu
    # would not (it is the limit that made a 64-across channel blow up after ~2 s).
    n, nu = 12, 0.1
    s = scenes.periodic_box(n_per_axis=n, dp=DP)
    p = oracle.params(s, visc_model=1, nu=nu, alpha=0.0, c0=1.0, g=(0.0, 0.0, 0.0))
    ijk = np.round(s.pos / DP - 0.5).astype(int)
    sign = (-1.0) ** ijk.sum(1)
    vel = np.zeros((s.n, 3))
    vel[:, 0] = 1e-3 * sign
    a, _ = oracle.rhs(p, s.pos, vel, np.zeros(s.n), s.mass, s.ptype)
    lam = -a[:, 0] / vel[:, 0]
    assert np.allclose(lam, lam[0], rtol=1e-9) and lam[0] > 0      # an eigenmode of the lattice
    h = s.h
    assert 6.0 * nu / h ** 2 < lam[0] < 8.0 * nu / h ** 2            # ~ 4 nu sum_odd |F| dp^3 = 7 nu/h^2
    dt = oracle.cfl_dt(p, np.zeros((s.n, 3)), s.ptype)
    z = lam[0] * dt
    assert dt == pytest.approx(0.125 * h * h / nu) and abs(1 - z + z * z / 2) <= 1.0
    z_old = lam[0] * 0.3 * h * h / nu
    assert abs(1 - z_old + z_old * z_old / 2) > 1.0


def test_artificial_viscosity_shear_decay():
    # C4 magnitude: in the long-wave limit the Monaghan term with the approach
    # switch acts on a divergence-free shear as nu = alpha h c0 / 20 (the
    # unswitched term gives (alpha h c0/10)(lap u + 2 grad div u); the switch
    # keeps half of the fourth moment).  On the lattice the fourth moment is
    # the quadrature sum below (with the 0.01 h^2 regularisation).  A shear
    # wave u_x = A sin(k y) must decay at nu k^2 times that quadrature factor.
    n = 16
    s = scenes.periodic_box(n_per_axis=n, dp=DP)
    h = s.h
    k = 2 * np.pi / (n * DP)
    lat = 0.0
    for i in range(-3, 4):
        for j in range(-3, 4):
            for l in range(-3, 4):
                x = np.array([i, j, l]) * DP
                r2 = x @ x
                if 0 < r2 < (2 * h) ** 2:
                    lat += DP ** 3 * x[0] ** 2 * x[1] ** 2 * oracle.kernel_F(np.sqrt(r2), h) / (r2 + 0.01 * h * h)
    quad = lat / -0.2          # continuum value of the moment: (1/15) int r^2 F dV = -3/15
    alpha = 0.1
    u = np.zeros((s.n, 3))
    u[:, 0] = 1e-3 * np.sin(k * s.pos[:, 1])
    p = oracle.params(s, alpha=alpha, dt_fixed=3.9e-4)
    x, v, d = s.pos, u, s.delta.astype(float)
    ts, amps, t = [], [], 0.0
    for _ in range(5):
        x, v, d, _, _ = oracle.step(p, x, v, d, s.mass, s.ptype, 10)
        t += 10 * 3.9e-4
        ts.append(t)
        amps.append(2 * np.mean(v[:, 0] * np.sin(k * x[:, 1])))
    rate = -np.polyfit(ts, np.log(amps), 1)[0]
    nu = rate / k ** 2
    assert nu / (alpha * s.h * s.c0 / 20 * quad) == pytest.approx(1.0, abs=0.03)
