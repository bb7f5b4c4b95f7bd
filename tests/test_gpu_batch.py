"""Batched scenes (marked gpu): many independent tanks stepped in one context
(one graph per step) give bit-identical results to each tank stepped alone,
with per-scene dt and time."""
import dataclasses

import numpy as np
import pytest

import oracle
from paper_2207_11328_gb300 import scenes
from tests.gpu_common import rel_check, require_gpu, sim_for

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True, scope="module")
def _gpu():
    require_gpu()


def _alone(batch, s):
    m = batch.scene == s
    d = batch.scenes[s]
    one = scenes.subset(batch, m, name=f"tank{s}")
    return dataclasses.replace(one, scenes=None, scene=np.zeros(int(m.sum()), np.uint32), origin=d["origin"],
                               size=d["size"], periodic=d["periodic"], c0=d["c0"])


def test_batch_equals_scenes_alone():
    b = scenes.sloshing_batch(n_scenes=6, nmin=2000, nmax=8000, seed=77)
    sim = sim_for(b)
    sim.autotune()
    sim.step(25)
    pos, vel, delta = sim.download()
    dts, times = sim.scene_times()
    assert len(set(np.round(dts, 12))) > 1          # scenes keep their own dt
    for s in range(6):
        one = _alone(b, s)
        so = sim_for(one)
        so.step(25)
        p1, v1, d1 = so.download()
        m = b.scene == s
        assert np.array_equal(pos[m], p1) and np.array_equal(vel[m], v1) and np.array_equal(delta[m], d1)
        dt1, t1 = so.scene_times()
        assert dt1[0] == dts[s] and t1[0] == times[s]


def test_batch_256_tanks_runs():
    b = scenes.sloshing_batch()
    sim = sim_for(b)
    sim.step(5)
    st = sim.stats()
    assert st["n_active"] == b.n and st["n_removed"] == 0 and st["error_bits"] == 0
    dts, times = sim.scene_times()
    assert np.all(dts > 0) and np.all(times > 0)


def test_batch_model_options_match_the_oracle_per_scene():
    # per-scene sound speed enters the viscosity and the density diffusion: each tank's
    # forces against the oracle run on that tank alone with its own c0
    b = dataclasses.replace(scenes.sloshing_batch(n_scenes=5, nmin=2000, nmax=6000, seed=78), kernel_type=1,
                            formulation=1, ddiff=1, ddiff_coef=0.1)
    f = b.ptype == 0
    b.vel[f] = scenes.seeded_normal((int(f.sum()), 3), 0.05, 79).astype(np.float32)
    sim = sim_for(b)
    sim.forces()
    acc, drho = sim.download_forces()
    for s in range(5):
        one = _alone(b, s)
        m = b.scene == s
        a_ref, d_ref, mag = oracle.rhs(oracle.params(one), one.pos, one.vel, one.delta, one.mass, one.ptype,
                                       with_mag=True)
        rel_check(acc[m], a_ref, 1e-5, f"tank {s} acceleration", mag[:, 0])
        rel_check(drho[m], d_ref, 1e-5, f"tank {s} density rate", mag[:, 1])


def test_batch_with_a_skin_list_follows_the_every_step_run():
    b = scenes.sloshing_batch(n_scenes=6, nmin=2000, nmax=8000, seed=80)
    a = sim_for(b)
    k = sim_for(b, rebuild_every=10, skin=0.3 * b.h, max_neibs=192)
    a.step(30)
    k.step(30)
    assert k.stats()["error_bits"] == 0 and k.stats()["builds"] < 31
    pa, va, _ = a.download()
    pk, vk, _ = k.download()
    assert np.max(np.abs(pa - pk)) < 1e-5 * b.dp
    f = b.ptype == 0
    assert np.max(np.abs(va[f] - vk[f])) <= 1e-4 * np.max(np.abs(va[f])) + 1e-6
