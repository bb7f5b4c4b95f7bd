"""Batched scenes (marked gpu): many independent tanks stepped in one context
(one graph per step) give bit-identical results to each tank stepped alone,
with per-scene dt and time."""
import dataclasses

import numpy as np
import pytest

from paper_2207_11328_gb300 import scenes
from tests.gpu_common import require_gpu, sim_for

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
