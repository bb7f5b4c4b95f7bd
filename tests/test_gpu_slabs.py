"""Slab decomposition on the GPU (marked gpu): the ranks of a decomposed run
share the one device, each with its own library context on its slab (halo
copies left out of the CFL reduction, the minimum dt passed back with
sph_set_dt), exchanging halos and migrants in-process between steps.  The
owned particles must follow the undivided run on the same device: the same
time steps and the same states (to FP32 rounding), with particles changing
owner during the run."""
import dataclasses

import numpy as np
import pytest

from paper_2207_11328_gb300 import scenes, slabs
from tests.gpu_common import require_gpu, sim_for

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True, scope="module")
def _gpu():
    require_gpu()


def _dam_moving(dp=0.02):
    s = scenes.dam_break(dp=dp)
    f = s.ptype == 0
    vel = s.vel.copy()
    vel[f] = scenes.seeded_normal((int(f.sum()), 3), 0.05, 92).astype(np.float32)
    vel[f, 0] += 1.0
    return dataclasses.replace(s, vel=vel)


@pytest.mark.parametrize("world", [2, 3])
def test_decomposed_gpu_run_follows_the_undivided_run(world):
    s = _dam_moving()
    steps = 40
    ref = sim_for(s)
    dts_ref = []
    for _ in range(steps):
        ref.step(1)
        dts_ref.append(ref.stats()["dt"])
    pos_ref, vel_ref, d_ref = ref.download()
    cut = np.linspace(0.0, 0.4, world + 1)[1:-1]    # cuts through the moving column
    initial = None

    def engine(sl, r):
        nonlocal initial
        if initial is None:
            initial = [p.gid.copy() for p in slabs.initial_parts(s, sl)]
        return slabs.GpuEngine(s, sl, r, capacity=s.n)

    orig = slabs.make_slabs
    slabs.make_slabs = lambda sc, w, **kw: orig(sc, w, at=cut, **kw)
    try:
        parts, dts, sl = slabs.run_local(s, world, steps, engine)
    finally:
        slabs.make_slabs = orig
    gid = np.concatenate([p.gid for p in parts])
    assert np.array_equal(np.sort(gid), np.arange(s.n))
    moved = sum(len(set(p.gid.tolist()) - set(g.tolist())) for p, g in zip(parts, initial))
    assert moved > 0
    pos = np.empty_like(pos_ref); vel = np.empty_like(vel_ref); d = np.empty_like(d_ref)
    for p in parts:
        pos[p.gid], vel[p.gid], d[p.gid] = p.pos, p.vel, p.delta
    rel_dt = np.max(np.abs(np.array(dts) - np.array(dts_ref)) / np.array(dts_ref))
    dx = np.max(np.abs(pos - pos_ref))
    du = np.max(np.abs(vel - vel_ref)) / np.max(np.abs(vel_ref))
    dd = np.max(np.abs(d - d_ref))
    print(f"{world} slabs, {moved} migrants: dt rel {rel_dt:.1e}, |dx| {dx:.2e} m, |du|/umax {du:.1e}, |ddelta| {dd:.1e}")
    assert rel_dt <= 1e-6
    assert dx <= 1e-6 * s.dp
    assert du <= 1e-5
    assert dd <= 1e-6
