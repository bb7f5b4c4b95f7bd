"""Edge cases and error paths of the C ABI on the GPU (marked gpu).  Every
failure is made on the host (bad arguments, tiny capacity, a particle placed
outside the domain, NaN in the uploaded state): nothing here faults the GPU."""
import numpy as np
import pytest

from paper_2207_11328_gb300 import Simulation, SphError, params_from_scene, scenes
from tests.gpu_common import require_gpu, sim_for

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True, scope="module")
def _gpu():
    require_gpu()
    from paper_2207_11328_gb300 import _build
    _build.build()


def test_empty_upload_and_step():
    s = scenes.periodic_box(n_per_axis=8)
    sim = Simulation(params_from_scene(s, max_particles=1000))
    sim.upload(pos=np.zeros((0, 3)), vel=np.zeros((0, 3)), delta=np.zeros(0), mass=np.zeros(0),
               ptype=np.zeros(0))
    sim.step(3)
    st = sim.stats()
    assert st["n_active"] == 0 and st["steps"] == 3
    pos, vel, delta = sim.download()
    assert pos.shape == (0, 3)


def test_single_particle_free_fall():
    s = scenes.dam_break(dp=0.05)
    one = scenes.subset(s, np.arange(s.n) == 5)
    one.vel[:] = 0
    sim = sim_for(one)
    sim.step(10)
    pos, vel, _ = sim.download()
    st = sim.stats()
    # no neighbours: a = g exactly; predictor-corrector is exact for constant a
    assert vel[0, 2] == pytest.approx(-9.81 * st["time"], rel=1e-5)
    assert pos[0, 2] == pytest.approx(one.pos[0, 2] - 0.5 * 9.81 * st["time"] ** 2, abs=1e-7)


def test_capacity_error():
    s = scenes.periodic_box(n_per_axis=8)
    sim = Simulation(params_from_scene(s, max_particles=100))
    with pytest.raises(SphError) as e:
        sim.upload(s)
    assert e.value.code == -3


def test_out_of_domain_upload_rejected():
    s = scenes.dam_break(dp=0.05)
    s.pos = s.pos.copy()
    s.pos[0, 0] = s.origin[0] - 1.0
    with pytest.raises(SphError) as e:
        sim_for(s)
    assert e.value.code == -5


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_domain_faces_decided_exactly(axis):
    # positions on and next to the faces of the domain [origin, origin + size) of a non-periodic
    # axis: inside the FP32 estimate's margin of a face (1e-6 of the magnitudes) the upload
    # decides in FP64.  (A particle within FP32 resolution below the upper face is re-based
    # out of the domain by the first sort, so the inside case there keeps 1e-6 of the size.)
    base = scenes.dam_break(dp=0.05)
    lo, size = base.origin[axis], base.size[axis]
    cases = [(lo, True), (np.nextafter(lo, -np.inf), False), (lo + 1e-9 * size, True), (lo - 1e-9 * size, False),
             (lo + size - 1e-6 * size, True), (lo + size + 1e-9 * size, False), (lo + 0.5 * size, True)]
    for x, inside in cases:
        s = scenes.dam_break(dp=0.05)
        s.pos = s.pos.copy()
        s.pos[0, axis] = x
        if inside:
            sim = sim_for(s)
            assert sim.stats()["n_active"] == s.n
        else:
            with pytest.raises(SphError) as e:
                sim_for(s)
            assert e.value.code == -5


def test_nonfinite_upload_rejected():
    s = scenes.periodic_box(n_per_axis=8)
    s.vel = s.vel.copy()
    s.vel[3, 1] = np.nan
    with pytest.raises(SphError) as e:
        sim_for(s)
    assert e.value.code == -6


def test_bad_type_rejected():
    s = scenes.periodic_box(n_per_axis=8)
    s.ptype = s.ptype.copy()
    s.ptype[0] = 7
    with pytest.raises(SphError) as e:
        sim_for(s)
    assert e.value.code == -1


def test_step_before_upload_is_state_error():
    s = scenes.periodic_box(n_per_axis=8)
    sim = Simulation(params_from_scene(s))
    with pytest.raises(SphError) as e:
        sim.step(1)
    assert e.value.code == -8


def test_periodic_axis_needs_three_cells():
    s = scenes.periodic_box(n_per_axis=5)   # 0.1 m box, 2h = 0.052: 1 cell
    with pytest.raises(SphError) as e:
        Simulation(params_from_scene(s))
    assert e.value.code == -1


def test_neighbor_overflow_reported():
    s = scenes.periodic_box(n_per_axis=10)
    sim = sim_for(s, max_neibs=16)
    st = sim.stats(check=False)
    assert st["rc"] == -4 and st["max_neibs_seen"] == 80
    counts, ids = sim.download_neighbors()
    assert np.all(counts.sum(1) == 16)
    sim.clear_error()
    assert sim.stats(check=False)["rc"] == 0


def test_particle_leaving_domain_is_removed():
    s = scenes.dam_break(dp=0.05)
    s.vel = s.vel.copy()
    top = int(np.argmax(np.where(s.ptype == 0, s.pos[:, 2], -1)))
    s.vel[top] = (0.0, 0.0, 40.0)      # leaves through the top within a few steps
    sim = sim_for(s)
    sim.step(40)
    st = sim.stats()
    assert st["n_removed"] == 1 and st["n_active"] == s.n - 1
    pos, vel, delta = sim.download()
    assert np.all(np.isnan(pos[top])) and np.isfinite(pos[np.arange(s.n) != top]).all()


def test_boundary_velocity_ignored():
    s = scenes.dam_break(dp=0.05)
    s.vel = s.vel.copy()
    s.vel[s.ptype == 1] = 3.0
    sim = sim_for(s)
    _, vel, _ = sim.download()
    assert np.all(vel[s.ptype == 1] == 0)
