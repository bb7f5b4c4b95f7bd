"""GPU path vs the FP64 oracle, through the C ABI (marked gpu).

Neighbour sets: bit-exact outside a 1e-6 h band around the cutoff.
Density rates and accelerations of one forces call: relative 1e-5 per
particle, relative to max(|oracle_i|, rms over particles), or 4 units of
FP32 roundoff of the summed pair-term magnitudes where the sum is
ill-conditioned (see tests/gpu_common.rel_check).
One full step: increments within 1e-4 of the increment plus the FP32
representation error of the stored state.
"""
import numpy as np
import pytest

import oracle
from paper_2207_11328_gb300 import build_variant_names, forces_variant_names, scenes
from tests.gpu_common import compare_neighbor_sets, rel_check, require_gpu, sim_for

pytestmark = pytest.mark.gpu

TOL_RHS = 1e-5


@pytest.fixture(autouse=True, scope="module")
def _gpu():
    require_gpu()


def _state_box(n=16, seed=21, jitter=0.3, dmax=2e-3):
    s = scenes.periodic_box(n_per_axis=n, dp=0.02, jitter=jitter, seed=seed)
    rng = np.random.default_rng(seed)
    s.delta = rng.uniform(-dmax, dmax, s.n).astype(np.float32)
    return s


def _small_dam(dp=0.03):
    s = scenes.dam_break(dp=dp)
    return s


CASES = {
    "box_lattice": lambda: scenes.periodic_box(n_per_axis=16),
    "box_jitter": lambda: _state_box(),
    "box_ragged": lambda: _state_box(n=11, seed=4),          # 1331 particles: ragged tail
    "dam_small": lambda: _small_dam(),
    "poiseuille_small": lambda: scenes.poiseuille(dp=1 / 32, nx=8, ny=32, nz=8),
}


@pytest.mark.parametrize("case", list(CASES))
def test_neighbor_sets_exact(case):
    s = CASES[case]()
    sim = sim_for(s)
    counts, ids = sim.download_neighbors()
    st = sim.stats()
    assert st["n_active"] == s.n and st["error_bits"] == 0
    npairs = compare_neighbor_sets(s, counts, ids)
    assert npairs > 0
    assert st["max_neibs_seen"] == int(counts.sum(1).max())


def _laminar_shear_box():
    s = _state_box(n=12, seed=8)
    s.visc, s.nu, s.alpha = 1, 0.1, 0.0
    return s


FORCE_CASES = dict(CASES, box_laminar=_laminar_shear_box)


@pytest.mark.parametrize("case", list(FORCE_CASES))
def test_forces_match_oracle(case):
    s = FORCE_CASES[case]()
    sim = sim_for(s)
    sim.forces()
    acc, drho = sim.download_forces()
    a_ref, d_ref, mag = oracle.rhs(oracle.params(s), s.pos, s.vel, s.delta, s.mass, s.ptype, with_mag=True)
    ra, fa = rel_check(acc, a_ref, TOL_RHS, f"{case} acceleration", mag[:, 0])
    rd, fd = rel_check(drho, d_ref, TOL_RHS, f"{case} density rate", mag[:, 1])
    print(f"{case}: max rel err a {ra:.2e} ({100 * fa:.2f}% within 1e-5) drho {rd:.2e} ({100 * fd:.2f}%)")


def test_one_step_matches_oracle():
    s = _state_box(seed=3)
    sim = sim_for(s)
    sim.step(1)
    pos, vel, delta = sim.download()
    st = sim.stats()
    p = oracle.params(s)
    x1, u1, d1, dt_next, dts = oracle.step(p, s.pos, s.vel, s.delta, s.mass, s.ptype, 1)
    assert st["dt"] == pytest.approx(dts[0], rel=1e-5)
    L = np.array(s.size)
    dx_ref = x1 - s.pos
    dx_ref -= L * np.round(dx_ref / L)
    dx = pos - s.pos
    dx -= L * np.round(dx / L)
    ulp_pos = np.spacing(np.float32(0.5 * 0.0534)) * 4
    assert np.max(np.abs(dx - dx_ref)) <= 1e-4 * np.max(np.abs(dx_ref)) + ulp_pos
    du, du_ref = vel - s.vel, u1 - s.vel
    assert np.max(np.abs(du - du_ref)) <= 1e-4 * np.max(np.abs(du_ref)) + 4 * np.spacing(np.float32(0.05))
    dd, dd_ref = delta - s.delta, d1 - s.delta
    assert np.max(np.abs(dd - dd_ref)) <= 1e-4 * np.max(np.abs(dd_ref)) + 4 * np.spacing(np.float32(2e-3))


def test_dam_step_matches_oracle():
    s = _small_dam(dp=0.04)
    sim = sim_for(s)
    sim.step(2)
    pos, vel, delta = sim.download()
    x1, u1, d1, _, dts = oracle.step(oracle.params(s), s.pos, s.vel, s.delta, s.mass, s.ptype, 2)
    assert sim.stats()["dt"] == pytest.approx(dts[1], rel=1e-5)
    f = s.ptype == 0
    du, du_ref = vel - s.vel, u1 - s.vel
    assert np.max(np.abs(du - du_ref)) <= 1e-4 * np.max(np.abs(du_ref)) + 4 * np.spacing(np.float32(0.01))
    # boundary particles do not move: only the FP32 cell-offset rounding of the upload remains
    half_cell = 0.5 * max(s.size[a] / np.floor(s.size[a] / (2 * s.h)) for a in range(3))
    assert np.max(np.abs(pos[~f] - s.pos[~f])) <= np.spacing(np.float32(half_cell))
    dd, dd_ref = delta - s.delta, d1 - s.delta
    assert np.max(np.abs(dd - dd_ref)) <= 1e-4 * np.max(np.abs(dd_ref)) + 4 * np.spacing(np.float32(0.02))


def test_deterministic_bitwise():
    s = _state_box(seed=5)
    outs = []
    for _ in range(2):
        sim = sim_for(s)
        sim.step(5)
        outs.append(sim.download())
        sim.close()
    for a, b in zip(*outs):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("case", ["dam_small", "box_lattice"])
def test_resort_is_idempotent(case):
    # sorting an unchanged state again moves no particle between cells (a particle on a
    # cell face keeps its cell), so lists and sums are bitwise the same after any number
    # of re-sorts
    s = CASES[case]()
    sim = sim_for(s)
    outs = []
    for _ in range(3):
        sim.forces()
        outs.append((*sim.download_forces(), *sim.download_neighbors()))
        sim.build_neighbors()
    for o in outs[1:]:
        for a, b in zip(outs[0], o):
            assert np.array_equal(a, b)


@pytest.mark.parametrize("bv", range(5))
def test_every_variant_gives_the_same_bits(bv):
    # every neighbour-build variant writes the same list, every force launch shape the same sums
    s = _small_dam(dp=0.03)
    ref = sim_for(s)
    ref.step(3)
    r = ref.download()
    for fv in range(5):
        sim = sim_for(s)
        sim.set_variants(bv, fv)
        sim.build_neighbors()
        sim.step(3)
        for a, b in zip(sim.download(), r):
            assert np.array_equal(a, b), (bv, fv)


@pytest.mark.parametrize("case", ["dam_small", "box_jitter"])
def test_first_step_after_a_build_skips_the_pipeline_bitwise(case):
    # the first step after an upload reuses the upload's list and its dt0 forces pass as
    # the predictor's forces; stepping through the full pipeline instead gives the same bits
    s = CASES[case]()
    a = sim_for(s)
    a.step(4)
    b = sim_for(s)
    b.step_profiled(1)  # kernel by kernel, the whole pipeline
    b.step(3)
    for x, y in zip(a.download(), b.download()):
        assert np.array_equal(x, y)
    sa, sb = a.stats(), b.stats()
    assert sa["steps"] == sb["steps"] == 4 and sa["dt"] == sb["dt"]
    assert sa["builds"] == 4 and sb["builds"] == 5  # the upload's build serves the first step of a


def test_autotune_keeps_results_bitwise():
    # every build variant writes the same list, every block size the same sums
    s = _small_dam(dp=0.03)
    sim = sim_for(s)
    sim.forces()
    a0, d0 = sim.download_forces()
    c0 = sim.download_neighbors()
    variant, fvariant = sim.autotune()
    assert variant and fvariant and "?" not in variant + fvariant
    sim.build_neighbors()
    sim.forces()
    a1, d1 = sim.download_forces()
    c1 = sim.download_neighbors()
    assert np.array_equal(a0, a1) and np.array_equal(d0, d1)
    assert np.array_equal(c0[0], c1[0]) and np.array_equal(c0[1], c1[1])
    sim.step(3)
    assert sim.stats()["steps"] == 3


@pytest.mark.parametrize("skin", [0.0, 0.3])
def test_autotune_leaves_the_run_unchanged(skin):
    # the corrector shapes are timed on a scratch copy of the state: a run after the
    # autotuner steps bit for bit like a run with the same shapes set by hand
    s = _small_dam(dp=0.03)
    kw = dict(rebuild_every=10, skin=skin * s.h, max_neibs=224) if skin else {}
    a = sim_for(s, **kw)
    a.autotune()
    v = a.variants()
    names = forces_variant_names()
    b = sim_for(s, **kw)
    b.set_variants(build=build_variant_names().index(v["build"]))
    b.set_forces_variants(names.index(v["forces_predict"]), names.index(v["forces_correct"]))
    assert b.variants() == v
    a.step(6)
    b.step(6)
    for x, y in zip(a.download(), b.download()):
        assert np.array_equal(x, y)
    assert a.stats()["dt"] == b.stats()["dt"]
    assert a.stats()["error_bits"] == 0
