"""Multi-step runs on the GPU judged by invariants and closed forms (marked
gpu): mass exact, momentum drift, energy dissipation, resting-tank pressure,
plane Poiseuille profile."""
import numpy as np
import pytest

import oracle
from paper_2207_11328_gb300 import scenes
from tests.gpu_common import require_gpu, sim_for
from tests.test_oracle_integration import poiseuille_profile

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True, scope="module")
def _gpu():
    require_gpu()


def test_periodic_box_100_steps_invariants():
    # periodic box, 16^3 lattice, dp 0.02, c0 20, alpha 0.02, no gravity, 100 steps
    s = scenes.periodic_box(n_per_axis=16)
    p = oracle.params(s)
    sim = sim_for(s)
    m = s.mass.astype(np.float64)
    P0 = (m[:, None] * s.vel).sum(0)
    scale = (m[:, None] * np.abs(s.vel)).sum()
    E = [oracle.energy(p, s.pos, s.vel, s.delta, s.mass, s.ptype)]
    for _ in range(10):
        sim.step(10)
        pos, vel, delta = sim.download()
        E.append(oracle.energy(p, pos, vel, delta, s.mass, s.ptype))
    st = sim.stats()
    assert st["n_active"] == s.n and st["n_removed"] == 0 and st["steps"] == 100
    assert np.all(np.isfinite(pos))
    # momentum: pair antisymmetry holds up to FP32 rounding of each half-pair
    P1 = (m[:, None] * vel).sum(0)
    assert np.all(np.abs(P1 - P0) <= 1e-5 * scale)
    # artificial viscosity dissipates
    assert np.all(np.diff(E) < 0)
    # trajectory stays close to the FP64 oracle's over 100 steps
    x1, u1, d1, _, _ = oracle.step(p, s.pos, s.vel, s.delta, s.mass, s.ptype, 100)
    L = np.array(s.size)
    dx = pos - x1
    dx -= L * np.round(dx / L)
    assert np.max(np.abs(dx)) < 1e-3 * s.dp
    assert np.max(np.abs(vel - u1)) < 1e-3 * 0.05


def test_hydrostatic_tank_pressure_gpu():
    s = scenes.hydrostatic_tank(dp=0.02, width=0.2, depth=0.2, height=0.4, fill=0.3, alpha=0.1)
    p = oracle.params(s)
    H, rho0, g = 0.3, 1000.0, 9.81
    f = s.ptype == 0
    x = s.pos
    inner = f & (x[:, 0] > 0.052) & (x[:, 0] < 0.148) & (x[:, 1] > 0.052) & (x[:, 1] < 0.148) & (x[:, 2] > 0.052)
    sim = sim_for(s)
    accP = np.zeros(s.n); accz = np.zeros(s.n); cnt = 0
    t = 0.0
    while t < 0.27:
        sim.step(5)
        t = sim.stats()["time"]
        if t > 0.09:
            pos, vel, d = sim.download()
            accP += np.array([oracle.eos(p, v) for v in d]); accz += pos[:, 2]; cnt += 1
    P = accP / cnt; z = accz / cnt
    err = P[inner] - rho0 * g * (H - z[inner])
    assert np.max(np.abs(err)) < 0.05 * rho0 * g * H
    assert np.sqrt(np.mean(err ** 2)) < 0.02 * rho0 * g * H
    assert sim.stats()["n_removed"] == 0


def test_poiseuille_profile_gpu():
    # plane Poiseuille, 128 x 64 x 8 fluid (65,536) at dp = 1/64, nu = 0.1,
    # body force 0.01: profile at t = 1 s vs the start-up series solution
    s = scenes.poiseuille()
    sim = sim_for(s)
    t = 0.0
    while t < 1.0:
        sim.step(20)
        t = sim.stats()["time"]
    pos, vel, _ = sim.download()
    f = s.ptype == 0
    ref = poiseuille_profile(pos[f, 1], t)
    err = np.sqrt(np.mean((vel[f, 0] - ref) ** 2)) / 0.0125
    print(f"Poiseuille t={t:.3f} L2 err / u_max = {err:.4f}")
    assert err < 0.02
    assert np.max(np.abs(vel[f, 1:])) < 1e-3 * 0.0125
