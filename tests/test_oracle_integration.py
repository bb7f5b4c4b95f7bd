"""Pins of the oracle's time integration and flows (readings C6, C7 of the
predictor-corrector scheme; resting-tank pressure rho0*g*depth; plane
Poiseuille closed form; forward-mode derivatives vs central differences)."""
import numpy as np
import pytest

import oracle
from paper_2207_11328_gb300 import scenes


def _run(p, s, nsteps, dt=0.0, x=None, u=None, d=None):
    x = s.pos if x is None else x
    u = s.vel if u is None else u
    d = s.delta if d is None else d
    return oracle.step(p, x, u, d, s.mass, s.ptype, nsteps, dt)


def test_energy_non_increasing_with_artificial_viscosity():
    # Monaghan viscosity only dissipates: E(t) decreases step after step
    s = scenes.periodic_box(n_per_axis=8, dp=0.02)
    p = oracle.params(s, alpha=0.02)
    x, u, d = s.pos, s.vel.astype(float), s.delta.astype(float)
    E = [oracle.energy(p, x, u, d, s.mass, s.ptype)]
    dt = 0.0
    for _ in range(30):
        x, u, d, dt, _ = oracle.step(p, x, u, d, s.mass, s.ptype, 1, dt)
        E.append(oracle.energy(p, x, u, d, s.mass, s.ptype))
    assert np.all(np.diff(E) < 0)


def test_energy_drift_vanishes_with_dt():
    # alpha = 0: the semi-discrete system conserves E; the integrator's drift
    # over a fixed time falls at least as dt^2 (measured: ~dt^3)
    s = scenes.periodic_box(n_per_axis=8, dp=0.02)
    drifts = []
    for dtf in (4e-4, 2e-4, 1e-4):
        p = oracle.params(s, alpha=0.0, dt_fixed=dtf)
        E0 = oracle.energy(p, s.pos, s.vel, s.delta, s.mass, s.ptype)
        x, u, d, _, _ = _run(p, s, int(round(0.016 / dtf)))
        drifts.append(abs(oracle.energy(p, x, u, d, s.mass, s.ptype) - E0))
    assert drifts[0] / drifts[1] > 3.5 and drifts[1] / drifts[2] > 3.5


def test_predictor_corrector_second_order():
    # C6: halving dt divides the error at fixed time by ~4
    s = scenes.periodic_box(n_per_axis=8, dp=0.02)
    res = {}
    for dtf in (4e-4, 2e-4, 1e-4, 2.5e-5):
        p = oracle.params(s, alpha=0.02, dt_fixed=dtf)
        res[dtf] = _run(p, s, int(round(0.016 / dtf)))
    ref = res[2.5e-5]
    err = []
    for dtf in (4e-4, 2e-4, 1e-4):
        dx = res[dtf][0] - ref[0]
        dx -= 0.16 * np.round(dx / 0.16)
        err.append(np.abs(dx).max())
    assert 3.5 < err[0] / err[1] < 4.8 and 3.5 < err[1] / err[2] < 4.8


def test_first_dt_from_initial_forces_and_cfl():
    # C7: dt0 comes from one forces call on the initial state; later dts from
    # the corrector-stage accelerations; all bounded by cfl*h/c0
    s = scenes.periodic_box(n_per_axis=8, dp=0.02)
    p = oracle.params(s)
    a, _ = oracle.rhs(p, s.pos, s.vel, s.delta, s.mass, s.ptype)
    dt0 = oracle.cfl_dt(p, a, s.ptype)
    _, _, _, dtn, dts = _run(p, s, 3)
    assert dts[0] == dt0
    assert np.all(dts <= 0.3 * s.h / s.c0 + 1e-15) and dtn <= 0.3 * s.h / s.c0 + 1e-15


def test_hydrostatic_tank_pressure():
    # resting tank: time-averaged P(z) = rho0 g (H - z) within 5% of rho0 g H
    # away from the walls (band of the resting-tank check), rms within 2%
    s = scenes.hydrostatic_tank(dp=0.02, width=0.2, depth=0.2, height=0.4, fill=0.3, alpha=0.1)
    p = oracle.params(s)
    H, rho0, g = 0.3, 1000.0, 9.81
    f = s.ptype == 0
    x = s.pos
    inner = f & (x[:, 0] > 0.052) & (x[:, 0] < 0.148) & (x[:, 1] > 0.052) & (x[:, 1] < 0.148) & (x[:, 2] > 0.052)
    x, u, d, dt, t = s.pos, s.vel.astype(float), s.delta.astype(float), 0.0, 0.0
    accP = np.zeros(s.n); accz = np.zeros(s.n); cnt = 0
    while t < 0.27:
        x, u, d, dt, dts = oracle.step(p, x, u, d, s.mass, s.ptype, 5, dt)
        t += dts.sum()
        if t > 0.09:
            accP += np.array([oracle.eos(p, v) for v in d]); accz += x[:, 2]; cnt += 1
        inst = np.array([oracle.eos(p, v) for v in d[inner]])
        assert np.max(np.abs(inst - rho0 * g * (H - x[inner, 2]))) < 0.06 * rho0 * g * H
    P = accP / cnt; z = accz / cnt
    err = P[inner] - rho0 * g * (H - z[inner])
    assert np.max(np.abs(err)) < 0.05 * rho0 * g * H
    assert np.sqrt(np.mean(err ** 2)) < 0.02 * rho0 * g * H


def poiseuille_profile(y, t, F=0.01, nu=0.1, a=0.5, nterms=60):
    """Start-up plane Poiseuille flow between plates at y = +-a (series solution)."""
    u = F * (a * a - y * y) / (2 * nu)
    for n in range(nterms):
        k = 2 * n + 1
        u -= (16 * F * a * a * (-1) ** n / (nu * np.pi ** 3 * k ** 3) * np.cos(k * np.pi * y / (2 * a))
              * np.exp(-k * k * np.pi ** 2 * nu * t / (4 * a * a)))
    return u


def test_poiseuille_series_itself():
    # the series starts from rest and tends to the parabola
    y = np.linspace(-0.49, 0.49, 9)
    assert np.max(np.abs(poiseuille_profile(y, 0.0))) < 2e-6
    assert np.allclose(poiseuille_profile(y, 50.0), 0.01 * (0.25 - y * y) / 0.2, rtol=1e-9)


@pytest.fixture(scope="module")
def channel_runs():
    # the plane channel at 16 and 32 particles across (nx = nz = 8), stepped by the
    # oracle from rest to t = 5 s; the states at t = 1 s and t = 5 s are kept
    out = {}
    for ny in (16, 32):
        s = scenes.poiseuille(dp=1.0 / ny, nx=8, ny=ny, nz=8)
        p = oracle.params(s)
        x, u, d, dt, t = s.pos, s.vel.astype(float), s.delta.astype(float), 0.0, 0.0
        for t_end in (1.0, 5.0):
            while t < t_end - 1e-12:
                x, u, d, dt, dts = oracle.step(p, x, u, d, s.mass, s.ptype, 1, dt)
                t += dts[0]
            out[(ny, t_end)] = (s, x.copy(), u.copy(), t)
    return out


def test_poiseuille_converges_to_closed_form(channel_runs):
    # laminar channel at t = 1 s: L2 error vs the closed form <= 3.5% of u_max
    # at 32 particles across and falling at first order in dp (16 -> 32)
    errs = []
    for ny in (16, 32):
        s, x, u, t = channel_runs[(ny, 1.0)]
        f = s.ptype == 0
        ref = poiseuille_profile(x[f, 1], t)
        errs.append(np.sqrt(np.mean((u[f, 0] - ref) ** 2)) / 0.0125)
        assert np.max(np.abs(u[f, 1:])) < 1e-3 * 0.0125   # no cross-flow
    assert errs[1] < 0.035
    assert 1.5 < errs[0] / errs[1] < 2.5


def test_poiseuille_steady_state(channel_runs):
    # the same channel at t = 5 s (five time constants 4a^2/(pi^2 nu)): the profile has
    # reached the parabola u = F (a^2 - y^2)/(2 nu).  Dynamic boundary particles hold
    # u = 0 at their own positions, so the no-slip plane is the first boundary layer
    # y = +-(a + dp/2): against it the L2 error is <= 2.5% of u_max at 16 and 32 across;
    # against the plates at +-a the error is the O(dp) offset of that plane, falling at
    # first order (16 -> 32).
    errs_a, errs_w = [], []
    for ny in (16, 32):
        s, x, u, t = channel_runs[(ny, 5.0)]
        f = s.ptype == 0
        for errs, aw in ((errs_a, 0.5), (errs_w, 0.5 + 0.5 / ny)):
            ref = poiseuille_profile(x[f, 1], t, a=aw)
            errs.append(np.sqrt(np.mean((u[f, 0] - ref) ** 2)) / (0.01 * aw * aw / 0.2))
        # the series at t = 5 s is the parabola to 0.8% of u_max
        assert np.max(np.abs(poiseuille_profile(x[f, 1], t) - 0.01 * (0.25 - x[f, 1] ** 2) / 0.2)) < 0.008 * 0.0125
        assert np.max(np.abs(u[f, 1:])) < 2e-3 * 0.0125   # no cross-flow
    assert max(errs_w) <= 0.025
    assert 1.5 < errs_a[0] / errs_a[1] < 2.5


@pytest.fixture(scope="module")
def box8():
    s = scenes.periodic_box(n_per_axis=8, dp=0.02)
    tgt = s.pos + scenes.seeded_normal(s.pos.shape, 0.1 * 0.02, 7)
    return s, tgt


def test_jvp_matches_central_differences_smooth(box8):
    # alpha = 0: the step map is smooth (Wendland F and F' vanish at q = 2),
    # so dual-number derivatives equal central differences (eps = 1e-4) to 1e-6
    s, tgt = box8
    p = oracle.params(s, alpha=0.0, dt_fixed=3.9e-4)
    for v in scenes.seeded_directions(3 * s.n, 3):
        v = v.reshape(-1, 3)
        L, dL = oracle.loss_jvp(p, s.pos, s.vel, s.delta, s.mass, s.ptype, 8, 3.9e-4, tgt, v)
        Lp, _ = oracle.loss_jvp(p, s.pos, s.vel + 1e-4 * v, s.delta, s.mass, s.ptype, 8, 3.9e-4, tgt)
        Lm, _ = oracle.loss_jvp(p, s.pos, s.vel - 1e-4 * v, s.delta, s.mass, s.ptype, 8, 3.9e-4, tgt)
        assert abs(dL - (Lp - Lm) / 2e-4) <= 1e-6 * abs(dL)


def test_jvp_alpha_and_viscosity_kink(box8):
    # d/dalpha is smooth; velocity directions with alpha > 0 cross the
    # switch u.x = 0 of the artificial viscosity, where central differences
    # are only O(eps) accurate: the gap shrinks ~10x when eps does
    s, tgt = box8
    p = oracle.params(s, alpha=0.02, dt_fixed=3.9e-4)
    L, dL = oracle.loss_jvp(p, s.pos, s.vel, s.delta, s.mass, s.ptype, 8, 3.9e-4, tgt, None, 1.0)
    e = 1e-4
    Lp, _ = oracle.loss_jvp(oracle.params(s, alpha=0.02 + e, dt_fixed=3.9e-4), s.pos, s.vel, s.delta,
                            s.mass, s.ptype, 8, 3.9e-4, tgt)
    Lm, _ = oracle.loss_jvp(oracle.params(s, alpha=0.02 - e, dt_fixed=3.9e-4), s.pos, s.vel, s.delta,
                            s.mass, s.ptype, 8, 3.9e-4, tgt)
    assert abs(dL - (Lp - Lm) / (2 * e)) <= 1e-6 * abs(dL)
    v = scenes.seeded_directions(3 * s.n, 1)[0].reshape(-1, 3)
    L, dL = oracle.loss_jvp(p, s.pos, s.vel, s.delta, s.mass, s.ptype, 8, 3.9e-4, tgt, v)
    gaps = []
    for eps in (1e-4, 1e-5):
        Lp, _ = oracle.loss_jvp(p, s.pos, s.vel + eps * v, s.delta, s.mass, s.ptype, 8, 3.9e-4, tgt)
        Lm, _ = oracle.loss_jvp(p, s.pos, s.vel - eps * v, s.delta, s.mass, s.ptype, 8, 3.9e-4, tgt)
        gaps.append(abs(dL - (Lp - Lm) / (2 * eps)) / abs(dL))
    assert gaps[0] < 1e-4 and gaps[1] < gaps[0] / 5
