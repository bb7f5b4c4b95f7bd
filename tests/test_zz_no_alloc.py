"""sph_download_neighbors_noalloc: the neighbour download for callers that
must not allocate device memory while they run (marked gpu).

It must return exactly what sph_download_neighbors returns (integer ids and
counts: bit-exact), on two calls in a row (the shared device array keeps the
previous call's contents), and refuse sizes beyond its fixed capacity."""
import ctypes

import numpy as np
import pytest

from paper_2207_11328_gb300 import SphError, _lib, scenes
from tests.gpu_common import require_gpu, sim_for

pytestmark = pytest.mark.gpu


def _call_noalloc(sim):
    n, mn = sim.n, sim.params.max_neibs
    counts = np.full((n, 2), 7, np.uint32)
    ids = np.full((n, mn), 7, np.uint32)
    rc = _lib().sph_download_neighbors_noalloc(sim._h, n, ctypes.c_void_p(counts.ctypes.data),
                                               ctypes.c_void_p(ids.ctypes.data), None)
    assert rc == 0, rc
    return counts, ids


def _check_twice(sim):
    ref_counts, ref_ids = sim.download_neighbors()
    for _ in range(2):
        counts, ids = _call_noalloc(sim)
        assert np.array_equal(counts, ref_counts)
        assert np.array_equal(ids, ref_ids)


def test_noalloc_download_matches_allocating_download():
    require_gpu()
    # the larger state first (10,204 particles), then a smaller one (4,096): the second
    # state's slots of the shared array still hold the first state's ids, so a call that
    # failed to reset them would return stale ids in the unused (0xFFFFFFFF) slots
    big = scenes.dam_break(dp=0.04)
    small = scenes.periodic_box(n_per_axis=16, jitter=0.3, seed=21)
    assert big.n > small.n
    sim_big = sim_for(big)
    _check_twice(sim_big)
    sim_small = sim_for(small)
    _check_twice(sim_small)
    # and back to the larger one: nothing of the smaller call leaks into it either
    _check_twice(sim_big)


def test_noalloc_download_rejects_oversize():
    require_gpu()
    s = scenes.periodic_box(n_per_axis=34)      # 39,304 particles x 128 slots > 2^22 entries
    sim = sim_for(s)
    with pytest.raises(SphError) as e:
        sim.download_neighbors_noalloc()
    assert e.value.code == -3
