"""Pins of the oracle's neighbour sets (Section 2.3: all particles within the
influence radius 2h; periodic axes use the minimum image, Table 1)."""
import numpy as np
import pytest

import oracle
from paper_2207_11328_gb300 import scenes


def _numpy_sets(pos, R, size, periodic):
    # independent O(N^2) definition with numpy: 0 < r < R, minimum image
    d = pos[:, None, :] - pos[None, :, :]
    for a in range(3):
        if (periodic >> a) & 1:
            d[..., a] -= size[a] * np.round(d[..., a] / size[a])
    r2 = np.einsum("ijk,ijk->ij", d, d)
    m = (r2 > 0) & (r2 < R * R)
    return [set(np.nonzero(m[i])[0].tolist()) for i in range(pos.shape[0])]


def _csr_sets(off, idx):
    return [set(idx[off[i]:off[i + 1]].tolist()) for i in range(len(off) - 1)]


@pytest.mark.parametrize("periodic", [0, 7, 0b101])
def test_brute_matches_numpy(periodic):
    rng = np.random.default_rng(1)
    n, L = 400, 0.2
    pos = rng.uniform(0, L, size=(n, 3))
    p = oracle.params(h=0.013, kernel_radius=2.0, origin=(0, 0, 0), size=(L, L, L), periodic_mask=periodic)
    off, idx = oracle.neighbors(p, pos, brute=True)
    assert _csr_sets(off, idx) == _numpy_sets(pos, 0.026, (L, L, L), periodic)


@pytest.mark.parametrize("periodic", [0, 7, 0b011])
def test_grid_matches_brute(periodic):
    s = scenes.periodic_box(n_per_axis=12, dp=0.02, jitter=0.35, seed=5)
    p = oracle.params(s, periodic_mask=periodic)
    off_b, idx_b = oracle.neighbors(p, s.pos, brute=True)
    off_g, idx_g = oracle.neighbors(p, s.pos, brute=False)
    assert np.array_equal(off_b, off_g)
    assert np.array_equal(idx_b, idx_g)


def test_lattice_interior_count_is_80():
    # h = 1.3 dp, radius 2h = 2.6 dp: lattice points with i^2+j^2+k^2 <= 6.76
    # excluding the origin; counted here on the integer lattice
    expected = sum(1 for i in range(-3, 4) for j in range(-3, 4) for k in range(-3, 4)
                   if 0 < i * i + j * j + k * k < 6.76)
    assert expected == 80
    s = scenes.periodic_box(n_per_axis=10, dp=0.02)
    off, idx = oracle.neighbors(oracle.params(s), s.pos)
    assert np.all(np.diff(off) == 80)


def test_symmetry_and_no_self():
    s = scenes.dam_break(dp=0.03)
    p = oracle.params(s)
    off, idx = oracle.neighbors(p, s.pos)
    sets = _csr_sets(off, idx)
    for i, S in enumerate(sets):
        assert i not in S
        for j in S:
            assert i in sets[j]


def test_dam_break_grid_matches_brute_small():
    s = scenes.dam_break(dp=0.05)
    p = oracle.params(s)
    off_b, idx_b = oracle.neighbors(p, s.pos, brute=True)
    off_g, idx_g = oracle.neighbors(p, s.pos)
    assert np.array_equal(off_b, off_g) and np.array_equal(idx_b, idx_g)


@pytest.mark.parametrize("case", ["box", "dam"])
def test_sampled_neighbour_sets_equal_the_full_search(case):
    # the sampled search (used at full sizes) returns, for each sampled particle, exactly
    # the set of the full search, which is pinned to brute force above
    s = scenes.periodic_box(n_per_axis=10, jitter=0.3, seed=4) if case == "box" else scenes.dam_break(dp=0.04)
    p = oracle.params(s)
    off, idx = oracle.neighbors(p, s.pos)
    sample = np.sort(np.random.default_rng(5).choice(s.n, size=min(300, s.n), replace=False)).astype(np.int32)
    so, si = oracle.neighbors_sample(p, s.pos, sample)
    for k, i in enumerate(sample):
        assert np.array_equal(si[so[k]:so[k + 1]], idx[off[i]:off[i + 1]])
