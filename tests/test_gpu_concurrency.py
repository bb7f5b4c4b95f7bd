"""Independent contexts driven from several host threads at once (marked gpu):
each thread owns one context and one CUDA stream and runs the public calls a
user makes per batch (upload from pinned host arrays, steps, download, the
counters), as the benchmark's end-to-end leg does.  The contexts share nothing
on the device, and graph capture is thread-local, so every thread's results
must equal, to the bit, those of the same calls made by one thread alone."""
import threading

import numpy as np
import pytest

from paper_2207_11328_gb300 import scenes
from tests.gpu_common import require_gpu, sim_for

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True, scope="module")
def _gpu():
    require_gpu()


def _batch(sim, stream, scene, steps, rounds, out):
    for _ in range(rounds):
        sim.upload(pos=scene.pos, vel=scene.vel, delta=scene.delta, mass=scene.mass, ptype=scene.ptype,
                   stream=stream)
        sim.step(steps, stream=stream)
        pos, vel, delta = sim.download(stream=stream)
        st = sim.stats(stream=stream)
        out.append((pos, vel, delta, st["list_entries"], st["dt"]))


@pytest.mark.parametrize("workers", [2, 3])
def test_threads_with_their_own_contexts_give_the_single_thread_bits(workers):
    import torch
    s = scenes.dam_break(dp=0.012)
    steps, rounds = 5, 4
    alone = []
    ref = sim_for(s)
    _batch(ref, torch.cuda.current_stream(), s, steps, rounds, alone)
    ref.close()
    sims = [sim_for(s) for _ in range(workers)]
    streams = [torch.cuda.Stream() for _ in range(workers)]
    outs = [[] for _ in range(workers)]
    errors = []

    def run(k):
        try:
            _batch(sims[k], streams[k], s, steps, rounds, outs[k])
        except Exception as e:  # reported below, on the main thread
            errors.append(e)

    threads = [threading.Thread(target=run, args=(k,)) for k in range(workers)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    torch.cuda.synchronize()
    assert not errors, errors
    for k in range(workers):
        assert len(outs[k]) == rounds
        for got, want in zip(outs[k], alone):
            for a, b in zip(got[:3], want[:3]):
                assert np.array_equal(a, b)
            assert got[3] == want[3] and got[4] == want[4]
    for sim in sims:
        sim.close()
