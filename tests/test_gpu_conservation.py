"""Conservation sums of the GPU path (sph_conservation, marked gpu): the pair
forces of Section 2.1 are antisymmetric, so in a periodic box without walls or
gravity the force sum vanishes to rounding; the sums agree with the oracle's
FP64 sums and with the state, and are bitwise reproducible."""
import numpy as np
import pytest

import oracle
from paper_2207_11328_gb300 import scenes
from tests.gpu_common import require_gpu, sim_for

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True, scope="module")
def _gpu():
    require_gpu()


def _box(seed=41):
    s = scenes.periodic_box(n_per_axis=14, jitter=0.3, seed=seed)
    s.delta = np.random.default_rng(seed).uniform(-5e-3, 5e-3, s.n).astype(np.float32)
    return s


def test_force_sum_vanishes_in_a_periodic_box():
    s = _box()
    sim = sim_for(s)
    c = sim.conservation()
    acc, _ = sim.download_forces()
    scale = float(np.sum(np.abs(s.mass)[:, None] * np.abs(acc.astype(np.float64))))
    assert np.all(np.abs(c["force"]) <= 1e-6 * scale)
    # momentum and kinetic energy are sums of the state
    u = s.vel.astype(np.float64)
    m = s.mass.astype(np.float64)
    assert np.allclose(c["momentum"], (m[:, None] * u).sum(0), rtol=1e-12, atol=1e-15)
    assert c["kinetic"] == pytest.approx(0.5 * float((m * (u * u).sum(1)).sum()), rel=1e-12)


def test_sums_match_the_oracle_on_the_dam_break():
    s = scenes.dam_break(dp=0.03)
    f = s.ptype == 0
    s.vel[f] = scenes.seeded_normal((int(f.sum()), 3), 0.2, 42).astype(np.float32)
    sim = sim_for(s)
    c = sim.conservation()
    a, d = oracle.rhs(oracle.params(s), s.pos, s.vel, s.delta, s.mass, s.ptype)
    m = np.abs(s.mass.astype(np.float64))
    ref_force = (m[:, None] * a).sum(0)
    ref_rate = float((m * d).sum())
    scale = float((m[:, None] * np.abs(a)).sum())
    assert np.all(np.abs(c["force"] - ref_force) <= 1e-5 * scale)
    assert abs(c["mass_rate"] - ref_rate) <= 1e-5 * float((m * np.abs(d)).sum())


def test_sums_are_bitwise_reproducible():
    s = _box(seed=43)
    sim = sim_for(s)
    sim.step(3)
    a, b = sim.conservation(), sim.conservation()
    for k in a:
        assert np.array_equal(np.asarray(a[k]), np.asarray(b[k]))
