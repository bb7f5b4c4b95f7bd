"""The neighbour list's two-entry-chunk layout (fluid part from the front,
boundary part from the back) at every list size (marked gpu): truncated lists
keep a prefix of each part in candidate order, every build variant writes the
same list, and an odd list size changes no result bit."""
import numpy as np
import pytest

from paper_2207_11328_gb300 import N_BUILD_VARIANTS, scenes
from tests.gpu_common import require_gpu, sim_for

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True, scope="module")
def _gpu():
    require_gpu()


def _dam():
    return scenes.dam_break(dp=0.03)


def _lists(sim):
    counts, ids = sim.download_neighbors()
    return counts, ids


@pytest.mark.parametrize("max_neibs", [17, 24, 33, 47])
def test_truncated_lists_keep_prefixes_of_both_parts(max_neibs):
    s = _dam()
    full = sim_for(s, max_neibs=128)
    cf, idf = _lists(full)
    assert full.stats()["error_bits"] == 0 and cf.sum(1).max() > max_neibs
    ref = None
    for v in range(N_BUILD_VARIANTS):
        sim = sim_for(s, max_neibs=max_neibs)
        sim.set_variants(build=v)
        sim.build_neighbors()
        st = sim.stats(check=False)
        assert st["rc"] == -4  # overflow reported, lists truncated
        c, ids = _lists(sim)
        nf, nb = c[:, 0].astype(int), c[:, 1].astype(int)
        assert np.all(nf + nb == np.minimum(cf.sum(1), max_neibs))
        for i in range(s.n):
            # each part is a prefix of the untruncated part, in candidate order
            assert np.array_equal(ids[i, :nf[i]], idf[i, :nf[i]])
            assert np.array_equal(ids[i, nf[i]:nf[i] + nb[i]], idf[i, cf[i, 0]:cf[i, 0] + nb[i]])
        if ref is None:
            ref = (c, ids)
        else:  # every variant keeps the same entries
            assert np.array_equal(c, ref[0]) and np.array_equal(ids, ref[1])


@pytest.mark.parametrize("skin", [0.0, 0.3])
def test_odd_list_size_changes_no_bit(skin):
    s = _dam()
    kw = dict(rebuild_every=10, skin=skin * s.h) if skin else {}
    out = []
    for mn in (193, 224):  # odd: a last chunk half empty in both parts
        sim = sim_for(s, max_neibs=mn, **kw)
        sim.forces()
        a, d = sim.download_forces()
        sim.step(4)
        assert sim.stats()["error_bits"] == 0
        out.append((a, d) + tuple(sim.download()))
    for x, y in zip(*out):
        assert np.array_equal(x, y)
