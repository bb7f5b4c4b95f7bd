"""Neighbour list rebuilt every k steps with a skin (the paper's default mode:
GPUSPH rebuilds every 10 steps with an enlarged search radius), marked gpu.
The list then holds every pair within 2h as long as no particle moved more
than skin/2 since the build; the device checks that and reports SPH_ERR_SKIN."""
import numpy as np
import pytest

import oracle
from paper_2207_11328_gb300 import SphError, scenes
from tests.gpu_common import rel_check, require_gpu, sim_for

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True, scope="module")
def _gpu():
    require_gpu()


def _box(seed=3):
    s = scenes.periodic_box(n_per_axis=16, jitter=0.3, seed=seed)
    s.delta = np.random.default_rng(seed).uniform(-2e-3, 2e-3, s.n).astype(np.float32)
    return s


def test_skin_list_forces_match_oracle():
    s = _box()
    sim = sim_for(s, rebuild_every=10, skin=0.4 * s.h, max_neibs=192)
    assert sim.stats()["error_bits"] == 0
    sim.forces()
    acc, drho = sim.download_forces()
    a_ref, d_ref, mag = oracle.rhs(oracle.params(s), s.pos, s.vel, s.delta, s.mass, s.ptype, with_mag=True)
    rel_check(acc, a_ref, 1e-5, "acceleration", mag[:, 0])
    rel_check(drho, d_ref, 1e-5, "density rate", mag[:, 1])
    # the skin list holds the exact set plus the shell out to 2h + skin
    counts, _ = sim.download_neighbors()
    off, _ = oracle.neighbors(oracle.params(s), s.pos)
    assert np.all(counts.sum(1) >= np.diff(off))


@pytest.mark.parametrize("k,skin", [(10, 0.3), (5, 0.2)])
def test_skin_mode_follows_the_oracle(k, skin):
    s = _box(seed=9)
    sim = sim_for(s, rebuild_every=k, skin=skin * s.h, max_neibs=192)
    sim.step(30)
    pos, vel, delta = sim.download()
    st = sim.stats()
    assert st["steps"] == 30 and st["error_bits"] == 0
    # the upload's build, then one at least every k steps (earlier when a particle moved skin/4)
    assert 1 + (30 - 1) // k <= st["builds"] <= 31
    # 30 steps x the first pass's pairs within 2h
    off, _ = oracle.neighbors(oracle.params(s), s.pos)
    assert st["interactions"] == pytest.approx(30 * off[-1], rel=0.01)
    x1, u1, d1, _, _ = oracle.step(oracle.params(s), s.pos, s.vel, s.delta, s.mass, s.ptype, 30)
    L = np.array(s.size)
    dx = pos - x1
    dx -= L * np.round(dx / L)
    assert np.max(np.abs(dx)) < 1e-4 * s.dp
    assert np.max(np.abs(vel - u1)) < 1e-4 * 0.05


def test_skin_exceeded_is_reported():
    s = scenes.periodic_box(n_per_axis=16, vel_amp=0.5, seed=4)
    sim = sim_for(s, rebuild_every=200, skin=1e-3 * s.h)
    sim.step(20)
    st = sim.stats(check=False)
    assert st["rc"] == -9
    with pytest.raises(SphError):
        sim.sync()


def test_dam_skin_mode_matches_every_step_build():
    s = scenes.dam_break(dp=0.03)
    a = sim_for(s)
    b = sim_for(s, rebuild_every=10, skin=0.4 * s.h, max_neibs=192)
    a.step(40)
    b.step(40)
    pa, va, da = a.download()
    pb, vb, db = b.download()
    assert b.stats()["error_bits"] == 0
    assert a.stats()["builds"] == 40  # the upload's build serves the first step
    assert 1 + (40 - 1) // 10 <= b.stats()["builds"] < 41
    f = s.ptype == 0
    assert np.max(np.abs(pa - pb)) < 1e-6 * s.dp
    assert np.max(np.abs(va[f] - vb[f])) <= 1e-4 * np.max(np.abs(va[f])) + 1e-6


def test_explicit_build_in_skin_mode_runs_the_pipeline():
    s = _box(seed=5)
    sim = sim_for(s, rebuild_every=10, skin=0.3 * s.h, max_neibs=192)
    sim.step(3)
    b0 = sim.stats()["builds"]
    sim.build_neighbors()
    sim.forces()
    assert sim.stats()["builds"] == b0 + 1
    pos, vel, delta = sim.download()
    acc, drho = sim.download_forces()
    a_ref, d_ref, mag = oracle.rhs(oracle.params(s), pos, vel, delta, s.mass, s.ptype, with_mag=True)
    rel_check(acc, a_ref, 1e-5, "acceleration", mag[:, 0])
    rel_check(drho, d_ref, 1e-5, "density rate", mag[:, 1])


def test_record_rejects_skin_mode():
    s = _box(seed=6)
    sim = sim_for(s, rebuild_every=10, skin=0.3 * s.h, max_neibs=192)
    with pytest.raises(SphError):
        sim.record(4, 2)
