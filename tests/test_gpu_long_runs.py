"""Long GPU runs judged by invariants and closed forms (marked gpu).

  dam_break_1M, 1000 steps (the benchmark's ~1M-fluid dam break, dp 4.3 mm,
      1,647,828 particles): particle count and total mass exact, no removal,
      no non-finite value, total energy (kinetic + internal + gravity
      potential, Section 2.1 with the Cole equation of state) non-increasing
      within the integration-error band, and, on the late (collapsing) state,
      sampled forces against the oracle and sampled neighbour sets equal to
      the oracle's.
  Poiseuille to steady state (the 128 x 64 x 8 channel, t = 5 s, about five
      time constants 4a^2/(pi^2 nu)): L2 error against the closed-form
      profile, and first-order convergence toward it from 32 to 64 across.
"""
import dataclasses

import numpy as np
import pytest

import oracle
from paper_2207_11328_gb300 import scenes
from tests.gpu_common import compare_neighbor_sets_sample, rel_check, require_gpu, sim_for
from tests.test_oracle_integration import poiseuille_profile

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True, scope="module")
def _gpu():
    require_gpu()


def _energy_change(s, sim, chunks, chunk):
    p = oracle.params(s)
    E = [oracle.energy(p, s.pos, s.vel, s.delta, s.mass, s.ptype)]
    state = None
    for _ in range(chunks):
        sim.step(chunk)
        st = sim.stats()
        assert st["n_active"] == s.n and st["n_removed"] == 0 and st["error_bits"] == 0
        state = sim.download()
        assert all(np.all(np.isfinite(a)) for a in state)
        E.append(oracle.energy(p, *state, s.mass, s.ptype))
    return np.array(E), state


def test_dam_break_1m_1000_steps():
    s = scenes.dam_break(dp=4.3e-3)
    sim = sim_for(s)
    m0 = sim.conservation()["mass"]
    # FP64 sum of identical FP32 masses: exact in any order (k m fits 53 bits for k < 2^29)
    assert m0 == float(np.sum(s.mass.astype(np.float64)))
    E, (pos, vel, delta) = _energy_change(s, sim, 10, 100)
    st = sim.stats()
    assert st["steps"] == 1000
    dt0 = st["dt"]
    # the same simulated time at half the time step: the predictor-corrector is second
    # order, so the integration error of the first run is ~4/3 of their difference
    s_half = dataclasses.replace(s, dt_fixed=0.5 * dt0)
    sim_h = sim_for(s_half)
    T = st["time"]
    sim_h.step(int(round(T / (0.5 * dt0))))
    Eh = oracle.energy(oracle.params(s), *sim_h.download(), s.mass, s.ptype)
    dE, dEh = E[-1] - E[0], Eh - E[0]
    band = 4.0 / 3.0 * abs(dE - dEh)
    print(f"dam 1M: E0 {E[0]:.6f} J, change over 1000 steps {dE:.4e} J (half dt {dEh:.4e} J), "
          f"integration band {band:.2e} J; increments {np.diff(E)}")
    # artificial viscosity dissipates: no interval gains more than the integration band,
    # and the change is dissipation, not integration error
    assert np.all(np.diff(E) <= band)
    assert dEh < 0 and abs(dE - dEh) <= 0.25 * abs(dEh)
    # total mass bitwise after 1000 steps of sorting and reordering
    cons = sim.conservation()
    assert cons["mass"] == m0
    # the late state: forces and neighbour sets of sampled particles against the oracle
    late = dataclasses.replace(s, pos=pos, vel=vel, delta=delta, name="dam_break_1M_t1000")
    moved = np.linalg.norm(pos - s.pos, axis=1)
    assert moved.max() > 2 * s.dp        # the column front has moved: not the initial lattice
    sim.build_neighbors()
    sim.forces()
    acc, drho = sim.download_forces()
    sample = np.sort(np.random.default_rng(31).choice(s.n, size=3000, replace=False)).astype(np.int32)
    # half the sample where the flow is (particles that moved most)
    front = np.argsort(moved)[-1500:].astype(np.int32)
    sample = np.unique(np.concatenate([sample[:1500], front]))
    a_ref, d_ref, nnb, mag = oracle.rhs_sample(oracle.params(late), late.pos, late.vel, late.delta, late.mass,
                                               late.ptype, sample)
    ra, fa = rel_check(acc[sample], a_ref, 1e-5, "late acceleration", mag[:, 0])
    rd, fd = rel_check(drho[sample], d_ref, 1e-5, "late density rate", mag[:, 1])
    print(f"late state: acceleration max rel {ra:.2e} ({100 * fa:.2f}% within 1e-5), "
          f"density rate max rel {rd:.2e} ({100 * fd:.2f}%)")
    counts, ids = sim.download_neighbors()
    pairs = compare_neighbor_sets_sample(late, sample, counts, ids)
    assert pairs > 0.9 * 40 * len(sample)


def _poiseuille_run(ny, t_end=5.0):
    s = scenes.poiseuille(dp=1.0 / ny, nx=2 * ny, ny=ny, nz=8)
    sim = sim_for(s)
    t = 0.0
    while t < t_end:
        sim.step(100)
        t = sim.stats()["time"]
    pos, vel, _ = sim.download()
    f = s.ptype == 0
    y, u = pos[f, 1], vel[f, 0].astype(np.float64)
    out = {"t": t, "cross": float(np.max(np.abs(vel[f, 1:]))) / 0.0125}
    for key, aw in (("wall_a", 0.5), ("wall_first_layer", 0.5 + 0.5 / ny)):
        ref = poiseuille_profile(y, t, a=aw)
        out[key] = float(np.sqrt(np.mean((u - ref) ** 2))) / (0.01 * aw * aw / 0.2)
    return out


def test_poiseuille_steady_state_gpu():
    # plates at y = +-a = +-0.5 m, nu = 0.1, body force 0.01: u(y) = F (a^2 - y^2) / (2 nu)
    # at steady state, u_max = 0.0125 m/s.  Dynamic boundary particles hold u = 0 at their
    # own positions: the no-slip plane is the first boundary layer, y = +-(a + dp/2)
    # (reading of the wall location); against the plates at +-a the error is the
    # O(dp) offset of that plane and falls at first order with dp.
    r32 = _poiseuille_run(32)
    r64 = _poiseuille_run(64)
    print(f"Poiseuille steady state: 32 across {r32}, 64 across {r64}")
    assert r64["t"] >= 5.0
    assert r64["wall_first_layer"] <= 0.02
    assert 1.5 <= r32["wall_a"] / r64["wall_a"] <= 2.5
    assert r64["cross"] < 2e-3
