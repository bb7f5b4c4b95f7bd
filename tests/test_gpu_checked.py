"""The checked build (compiled with SPH_CHECKED: list, cell and slot indices are
tested before use and every device buffer carries a canary tail) runs the
pipeline, the model kernels, the skin list, batched scenes and the adjoint on
small cases without recording a violation (marked gpu).  It stands in for a
memory checker: a bad index is reported as SPH_ERR_BOUNDS, never dereferenced."""
import json
import os
import subprocess
import sys

import pytest

from tests.gpu_common import require_gpu

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r'''
import dataclasses, json, os, sys
sys.path.insert(0, os.getcwd())
import numpy as np
import paper_2207_11328_gb300 as P
from paper_2207_11328_gb300 import Simulation, scenes
assert P.LIB_PATH.endswith("libsph_gb300_checked.so"), P.LIB_PATH
res = {}

def run(name, s, steps, **kw):
    sim = Simulation.from_scene(s, **kw)
    sim.autotune()
    sim.step(steps)
    sim.forces()
    sim.download_neighbors()
    sim.conservation()
    res[name] = sim.stats(check=False)["error_bits"]
    return sim

run("box", scenes.periodic_box(n_per_axis=12, jitter=0.3), 20)
run("dam", scenes.dam_break(dp=0.03), 20)
run("dam_skin", scenes.dam_break(dp=0.03), 25, rebuild_every=10, skin=0.3 * scenes.dam_break(dp=0.03).h, max_neibs=192)
run("dam_models", dataclasses.replace(scenes.dam_break(dp=0.03), kernel_type=1, formulation=1, visc=3, visc_avg=2,
                                      alpha=0.0, nu=1e-3, zeta=1e-3, ddiff=1, ddiff_coef=0.1), 10)
run("batch", scenes.sloshing_batch(n_scenes=4, nmin=2000, nmax=6000, seed=81), 10)
import torch
sim = Simulation.from_scene(scenes.periodic_box(n_per_axis=10, jitter=0.2))
sim.record(8, 4)
sim.backward(torch.ones((sim.n, 3), dtype=torch.float32, device="cuda"))
res["adjoint"] = sim.stats(check=False)["error_bits"]
print(json.dumps(res))
'''


@pytest.fixture(autouse=True, scope="module")
def _gpu():
    require_gpu()


def test_checked_build_finds_no_violation():
    from paper_2207_11328_gb300 import _build
    _build.build(checked=True)
    out = subprocess.run([sys.executable, "-c", SCRIPT], cwd=ROOT, capture_output=True, text=True, timeout=600,
                         env=dict(os.environ, SPH_GB300_CHECKED="1"))
    assert out.returncode == 0, out.stderr[-3000:]
    res = json.loads(out.stdout.strip().splitlines()[-1])
    assert res and all(v == 0 for v in res.values()), res
