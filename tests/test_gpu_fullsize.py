"""Parity at the benchmark's full sizes, in the launch configuration the
benchmark times (marked gpu).  The oracle computes sampled particles one by
one: forces of a seeded sample of 3000 particles, neighbour counts, and the
state after one full step.

  dam_break_1M : tank 1.6 x 0.67 x 0.6 m, column 0.4 x 0.67 x 0.3 m, dp 4.3 mm (1.65M particles)
  dam_break_16M: same at dp 4.3 mm / 16^(1/3)                             (~20.5M particles)
"""
import dataclasses

import numpy as np
import pytest

import oracle
from paper_2207_11328_gb300 import scenes
from tests.gpu_common import compare_neighbor_sets_of, rel_check, require_gpu, sim_for

pytestmark = pytest.mark.gpu
TOL_RHS = 1e-5


@pytest.fixture(autouse=True, scope="module")
def _gpu():
    require_gpu()


def _sample(n, k, seed):
    return np.sort(np.random.default_rng(seed).choice(n, size=min(k, n), replace=False)).astype(np.int32)


def _check_sample(s, sim, sample):
    sim.forces()
    acc, drho = sim.download_forces()
    a_ref, d_ref, nnb, mag = oracle.rhs_sample(oracle.params(s), s.pos, s.vel, s.delta, s.mass, s.ptype, sample)
    ra, fa = rel_check(acc[sample], a_ref, TOL_RHS, f"{s.name} acceleration", mag[:, 0])
    rd, fd = rel_check(drho[sample], d_ref, TOL_RHS, f"{s.name} density rate", mag[:, 1])
    cond = mag[:, 0] / np.maximum(np.linalg.norm(a_ref, axis=1), 1e-300)
    print(f"{s.name}: acceleration max rel {ra:.2e} ({100 * fa:.2f}% within 1e-5, max condition {cond.max():.0f}); "
          f"density rate max rel {rd:.2e} ({100 * fd:.2f}%)")
    return nnb


@pytest.mark.parametrize("dp,name", [(4.3e-3, "dam_break_1M"), (4.3e-3 / 16 ** (1 / 3), "dam_break_16M")])
def test_fullsize_forces_sampled(dp, name):
    s = scenes.dam_break(dp=dp, name=name)
    sim = sim_for(s)
    st = sim.stats()
    assert st["n_active"] == s.n and st["error_bits"] == 0
    sample = _sample(s.n, 3000, 11)
    nnb = _check_sample(s, sim, sample)
    # fluid particles: the GPU list holds every neighbour (no pair sits in the
    # cutoff band on this lattice: |r - 2h| >= 0.1 dp for all lattice pairs)
    counts = sim.download_neighbors()[0] if s.n < 5_000_000 else None
    if counts is not None:
        f = s.ptype[sample] == 0
        assert np.array_equal(counts[sample][f].sum(1), nnb[f])


def test_fullsize_one_step_sampled():
    s = scenes.dam_break(dp=4.3e-3)
    sim = sim_for(s)
    sim.step(1)
    pos, vel, delta = sim.download()
    x1, u1, d1, _, dts = oracle.step(oracle.params(s), s.pos, s.vel, s.delta, s.mass, s.ptype, 1)
    assert sim.stats()["dt"] == pytest.approx(dts[0], rel=1e-5)
    du, du_ref = vel - s.vel, u1 - s.vel
    scale = np.max(np.abs(du_ref))
    assert np.max(np.abs(du - du_ref)) <= 1e-4 * scale + 4 * np.spacing(np.float32(scale))
    dd, dd_ref = delta - s.delta, d1 - s.delta
    assert np.max(np.abs(dd - dd_ref)) <= 1e-4 * np.max(np.abs(dd_ref)) + 4 * np.spacing(np.float32(0.02))
    half_cell = 0.5 * max(s.size[a] / np.floor(s.size[a] / (2 * s.h)) for a in range(3))
    assert np.max(np.abs(pos - x1)) <= 1e-4 * np.max(np.abs(x1 - s.pos)) + 2 * np.spacing(np.float32(half_cell))


def _dam_moving(dp=4.3e-3):
    # the benchmark's dam break with a seeded velocity field and density perturbation,
    # so that the continuity sum, the switched viscosity and the diffusion are all active
    s = scenes.dam_break(dp=dp, name="dam_break_1M_moving" if dp >= 4e-3 else "dam_break_16M_moving")
    f = s.ptype == 0
    vel = s.vel.copy()
    vel[f] = scenes.seeded_normal((int(f.sum()), 3), 0.2, 23).astype(np.float32)
    delta = s.delta + scenes.seeded_normal((s.n,), 2e-3, 24).astype(np.float32)
    return dataclasses.replace(s, vel=vel, delta=delta.astype(np.float32))


@pytest.mark.parametrize("model", ["default", "density_diffusion", "all_options", "skin_list", "skin_list_16M"])
def test_fullsize_moving_state_sampled(model):
    s = _dam_moving(4.3e-3 / 16 ** (1 / 3)) if model.endswith("16M") else _dam_moving()
    kw = {}
    if model == "density_diffusion":
        s = dataclasses.replace(s, ddiff=1, ddiff_coef=0.1)
    elif model == "all_options":
        s = dataclasses.replace(s, kernel_type=1, formulation=1, visc=3, visc_avg=1, alpha=0.0, nu=1e-6, zeta=1e-6,
                                ddiff=1, ddiff_coef=0.1)
    elif model.startswith("skin_list"):
        kw = dict(rebuild_every=10, skin=0.3 * s.h, max_neibs=192)
    sim = sim_for(s, **kw)
    assert sim.stats()["error_bits"] == 0
    _check_sample(s, sim, _sample(s.n, 3000, 12))


@pytest.mark.parametrize("dp,name", [(4.3e-3, "dam_break_1M_jitter"), (4.3e-3 / 16 ** (1 / 3), "dam_break_16M_jitter")])
def test_fullsize_disordered_lists_and_forces_sampled(dp, name):
    # a disordered full-size state: fluid positions jittered by a seeded U(-0.15, 0.15) dp per
    # component, seeded velocities and densities; the lists of 3000 sampled particles (half of
    # them fluid next to the walls, where both list parts are used) against the oracle's
    # sampled search, bit for bit outside the 1e-6 h band, and their forces within P3
    s = scenes.dam_break(dp=dp, name=name)
    f = s.ptype == 0
    pos = s.pos.copy()
    pos[f] += scenes.seeded_uniform((int(f.sum()), 3), -0.15 * s.dp, 0.15 * s.dp, 31)
    vel = s.vel.copy()
    vel[f] = scenes.seeded_normal((int(f.sum()), 3), 0.1, 32).astype(np.float32)
    delta = (s.delta + scenes.seeded_normal((s.n,), 1e-3, 33)).astype(np.float32)
    s = dataclasses.replace(s, pos=pos, vel=vel, delta=delta)
    sim = sim_for(s)
    assert sim.stats()["error_bits"] == 0
    rng = np.random.default_rng(34)
    nearwall = np.nonzero(f & ((pos[:, 0] < 3 * s.dp) | (pos[:, 2] < 3 * s.dp)))[0]
    sample = np.unique(np.concatenate([rng.choice(s.n, 1500, replace=False),
                                       rng.choice(nearwall, 1500, replace=False)])).astype(np.int32)
    counts, ids = sim.download_neighbors_of(sample)
    pairs = compare_neighbor_sets_of(s, sample, counts, ids)
    assert np.any(counts[:, 1] > 0) and pairs > 40 * len(sample)
    _check_sample(s, sim, sample)
