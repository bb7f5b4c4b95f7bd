"""Upload -> download with no step in between (marked gpu): the device holds each
position as a cell plus an FP32 offset from the cell's FP64 centre (reading P1), so
the downloaded FP64 position must equal the uploaded one to half an FP32 ulp of a
half-cell offset plus FP64 rounding.  The cases reach every path of the conversion:
positions across the domain, exactly on cell faces and at cell centres, a domain that
straddles the coordinate origin (where a position and its cell centre can differ in
sign or binade, and the conversion falls back to an FP64 subtraction), a periodic
domain, and positions just inside the faces of the domain."""
import dataclasses

import numpy as np
import pytest

from paper_2207_11328_gb300 import scenes
from tests.gpu_common import require_gpu, sim_for

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True, scope="module")
def _gpu():
    require_gpu()


def _cells(s):
    R = s.kernel_radius * s.h
    nc = np.floor(np.array(s.size) / R)
    return np.array(s.size) / nc, nc


def _check_roundtrip(s):
    sim = sim_for(s)
    assert sim.stats()["n_active"] == s.n
    pos, _, _ = sim.download()
    cell, _ = _cells(s)
    d = pos - s.pos
    size = np.array(s.size)
    for a in range(3):
        if (s.periodic >> a) & 1:    # a position on the upper face comes back on the lower one
            d[:, a] -= size[a] * np.round(d[:, a] / size[a])
    bound = cell * 2.0 ** -25 + 4 * np.spacing(np.abs(s.pos) + cell)
    assert np.all(np.abs(d) <= bound), np.max(np.abs(d) / bound)
    return np.max(np.abs(d) / cell)


def test_roundtrip_dam_break_jittered():
    s = scenes.dam_break(dp=0.02)
    f = s.ptype == 0
    pos = s.pos.copy()
    pos[f] += scenes.seeded_uniform((int(f.sum()), 3), -0.3 * s.dp, 0.3 * s.dp, 71)
    _check_roundtrip(dataclasses.replace(s, pos=pos))


def test_roundtrip_domain_across_the_coordinate_origin():
    # a periodic box whose domain is [-L/2, L/2)^3: cells around x = 0, positions of both
    # signs, some exactly at 0 and within 1e-9 of it
    s = scenes.periodic_box(n_per_axis=12, jitter=0.3)
    L = s.size[0]
    pos = s.pos - L / 2
    pos[:6] = [[0.0, 0.0, 0.0], [1e-9, -1e-9, 0.0], [-1e-12, 2e-12, 1e-15], [np.nextafter(0.0, 1.0), 0.0, 0.0],
               [-0.5 * L, 0.0, 0.0], [0.25 * L, -0.25 * L, 1e-7]]
    _check_roundtrip(dataclasses.replace(s, pos=pos, origin=(-L / 2, -L / 2, -L / 2)))


def test_roundtrip_cell_faces_and_centres():
    # one coordinate of every particle moved onto the nearest cell face (first half) or cell
    # centre (second half), the axis chosen per particle, the other two left on the lattice
    s = scenes.periodic_box(n_per_axis=12, jitter=0.3)
    cell, nc = _cells(s)
    rng = np.random.default_rng(72)
    pos = s.pos.copy()
    axis = rng.integers(0, 3, size=s.n)
    half = s.n // 2
    for i in range(s.n):
        a = axis[i]
        u = (pos[i, a] - s.origin[a]) / cell[a]
        k = np.floor(u + 0.5) if i < half else np.floor(u) + 0.5
        pos[i, a] = s.origin[a] + (k % nc[a]) * cell[a]
    _check_roundtrip(dataclasses.replace(s, pos=pos))


def test_roundtrip_just_inside_the_domain_faces():
    s = scenes.dam_break(dp=0.05)
    pos = s.pos.copy()
    lo = np.array(s.origin)
    hi = lo + np.array(s.size)
    for a in range(3):
        pos[2 * a, a] = lo[a]
        pos[2 * a + 1, a] = hi[a] - 1e-6 * s.size[a]
    _check_roundtrip(dataclasses.replace(s, pos=pos))
