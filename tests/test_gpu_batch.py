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


def test_batch_256_tanks_forces_and_dt_match_the_oracle_sampled():
    # the full batch of 256 tanks (8.6M particles): forces of 200 sampled particles in each
    # of 12 seeded tanks, and the first time step of the three smallest tanks, against the
    # oracle run on each tank alone with its own grid and sound speed
    b = scenes.sloshing_batch()
    sim = sim_for(b)
    sim.forces()
    acc, drho = sim.download_forces()
    rng = np.random.default_rng(85)
    for s in rng.choice(len(b.scenes), 12, replace=False):
        one = _alone(b, int(s))
        ids = np.nonzero(b.scene == s)[0]
        sample = np.sort(rng.choice(len(ids), min(200, len(ids)), replace=False)).astype(np.int32)
        a_ref, d_ref, _, mag = oracle.rhs_sample(oracle.params(one), one.pos, one.vel, one.delta, one.mass,
                                                 one.ptype, sample)
        rel_check(acc[ids[sample]], a_ref, 1e-5, f"tank {s} acceleration", mag[:, 0])
        rel_check(drho[ids[sample]], d_ref, 1e-5, f"tank {s} density rate", mag[:, 1])
    sim.step(1)
    dts, _ = sim.scene_times()
    sizes = np.bincount(b.scene, minlength=len(b.scenes))
    for s in np.argsort(sizes)[:3]:
        one = _alone(b, int(s))
        p = oracle.params(one)
        a, _ = oracle.rhs(p, one.pos, one.vel, one.delta, one.mass, one.ptype)
        assert dts[s] == pytest.approx(oracle.cfl_dt(p, a, one.ptype), rel=1e-5)


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


@pytest.mark.parametrize("case", ["batch", "box", "dam", "laminar_channel"])
def test_persistent_step_kernel_equals_the_graph(case):
    # the whole step as one persistent kernel (grid-wide barriers between the phases) gives
    # the graph of per-phase kernels' results to the bit: states, per-scene dt and time,
    # list counters; over step() calls of several lengths (odd and even buffer parities)
    if case == "batch":
        s = scenes.sloshing_batch(n_scenes=8, nmin=2000, nmax=12000, seed=81)
    elif case == "box":
        s = scenes.periodic_box(n_per_axis=16, jitter=0.2, seed=82)
    elif case == "dam":
        s = scenes.dam_break(dp=0.03)
    else:
        s = scenes.poiseuille(dp=1.0 / 16, nx=8, ny=16, nz=8)
    g = sim_for(s)
    p = sim_for(s)
    p.set_persistent(True)
    for n in (1, 4, 7, 2):
        g.step(n)
        p.step(n)
    sg, sp = g.stats(), p.stats()
    for k in ("n_active", "n_removed", "steps", "list_entries", "builds", "max_neibs_seen", "error_bits"):
        assert sg[k] == sp[k], k
    assert sp["kernels_per_step"] == 1
    for a, b in zip(g.download(), p.download()):
        assert np.array_equal(a, b)
    dg, tg = g.scene_times()
    dp_, tp = p.scene_times()
    assert np.array_equal(dg, dp_) and np.array_equal(tg, tp)
    # back to the graph: the context carries on from the persistent kernel's state
    p.set_persistent(False)
    g.step(3)
    p.step(3)
    for a, b in zip(g.download(), p.download()):
        assert np.array_equal(a, b)


def test_persistent_mode_refuses_a_skin_list_and_model_options():
    from paper_2207_11328_gb300 import SphError
    b = scenes.sloshing_batch(n_scenes=2, nmin=2000, nmax=3000, seed=83)
    k = sim_for(b, rebuild_every=10, skin=0.3 * b.h, max_neibs=192)
    with pytest.raises(SphError):
        k.set_persistent(True)
    m = sim_for(dataclasses.replace(b, kernel_type=1))
    with pytest.raises(SphError):
        m.set_persistent(True)


@pytest.mark.parametrize("case", ["batch", "box", "dam", "laminar_channel"])
def test_fused_build_and_predictor_equal_the_two_kernels(case):
    # the list build and the predictor pass as one kernel: the same list, states, dt and
    # counters as the two kernels, to the bit
    if case == "batch":
        s = scenes.sloshing_batch(n_scenes=8, nmin=2000, nmax=12000, seed=84)
    elif case == "box":
        s = scenes.periodic_box(n_per_axis=16, jitter=0.2, seed=85)
    elif case == "dam":
        s = scenes.dam_break(dp=0.03)
    else:
        s = scenes.poiseuille(dp=1.0 / 16, nx=8, ny=16, nz=8)
    a = sim_for(s)
    f = sim_for(s)
    a.set_fused_predict(False)
    f.set_fused_predict(True)
    assert f.step_options()["fused_predict"] and not a.step_options()["fused_predict"]
    for n in (1, 5, 2):
        a.step(n)
        f.step(n)
    sa, sf = a.stats(), f.stats()
    for k in ("n_active", "steps", "list_entries", "builds", "max_neibs_seen", "error_bits"):
        assert sa[k] == sf[k], k
    for x, y in zip(a.download(), f.download()):
        assert np.array_equal(x, y)
    ca, ia = a.download_neighbors()
    cf, if_ = f.download_neighbors()
    assert np.array_equal(ca, cf) and np.array_equal(ia, if_)
    # step_profiled (kernel by kernel) runs the fused kernel too
    a.step_profiled(2)
    ph = f.step_profiled(2)
    assert ph["forces_predict"] == 0.0 and ph["build"] > 0.0
    for x, y in zip(a.download(), f.download()):
        assert np.array_equal(x, y)
