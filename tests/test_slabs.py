"""Slab decomposition (paper Section "Multi-GPU": halo copies of the
neighbouring devices' particles, migration across boundaries, a minimum
reduction of the time step) on CPU: the partition and exchange logic, and a
world_size-2 gloo run whose ranks step their slabs with the FP64 oracle,
checked against the oracle on the undivided scene (neighbour sets of the owned
particles exactly, states to FP64 rounding)."""
import dataclasses
import multiprocessing as mp
import os
import socket

import numpy as np
import pytest

import oracle
from paper_2207_11328_gb300 import scenes, slabs


def _dam():
    return scenes.dam_break(dp=0.03)


def _dam_moving():
    # the column given a seeded velocity field with a mean of 1 m/s along the cut
    # axis, so that particles cross the slab boundary within the run (migration)
    s = _dam()
    f = s.ptype == 0
    vel = s.vel.copy()
    vel[f] = scenes.seeded_normal((int(f.sum()), 3), 0.05, 91).astype(np.float32)
    vel[f, 0] += 1.0
    return dataclasses.replace(s, vel=vel)


def test_partition_owns_each_particle_once_and_keeps_halo_depth():
    s = _dam()
    for world in (2, 3):
        sl = slabs.make_slabs(s, world)
        assert sl.axis == 0 and sl.cuts[0] == 0 and sl.cuts[-1] == sl.ncell
        parts = slabs.initial_parts(s, sl)
        gids = np.concatenate([p.gid for p in parts])
        assert np.array_equal(np.sort(gids), np.arange(s.n))
        # the cells of a slab are whole cells of the grid the library lays out
        R = s.kernel_radius * s.h
        assert sl.cell >= R and sl.ncell == int(np.floor(s.size[0] / R))
        kept, outs, mig = zip(*[slabs.migrate_and_halo(sl, r, parts[r]) for r in range(world)])
        assert all(m.n == 0 for m in mig)
        inbox = slabs.LocalComm(world).exchange(list(outs))
        for r in range(world):
            local, n_own = slabs.assemble(sl, r, kept[r], inbox[r], mig[r])
            assert n_own == parts[r].n and np.array_equal(local.gid[:n_own], parts[r].gid)
            # every particle within two cells (>= twice the influence radius) of an owned
            # particle along the cut axis is in the local set
            x = s.pos[:, 0]
            xo = x[parts[r].gid]
            near = (x >= xo.min() - 2 * sl.cell) & (x < xo.max() + 2 * sl.cell)
            assert set(np.nonzero(near)[0]) <= set(local.gid.tolist())
            # and nothing beyond the halo cells of the slab's edges
            lo, hi = sl.edge(r) - sl.layers * sl.cell, sl.edge(r + 1) + sl.layers * sl.cell
            assert np.all((x[local.gid] >= lo - 1e-12) & (x[local.gid] < hi + 1e-12))


def test_migrants_change_owner_and_stay_as_halo():
    s = _dam()
    sl = slabs.make_slabs(s, 2)
    parts = slabs.initial_parts(s, sl)
    # push the rank-0 particles of its last cell a third of a cell across the cut
    edge = sl.edge(1)
    p0 = parts[0]
    m = p0.pos[:, 0] > edge - sl.cell
    moved = p0.pos.copy()
    moved[m, 0] += sl.cell / 3
    crossed = m & (moved[:, 0] >= edge)
    assert crossed.sum() > 0
    parts[0] = dataclasses.replace(p0, pos=moved)
    kept, outs, mig = zip(*[slabs.migrate_and_halo(sl, r, parts[r]) for r in range(2)])
    assert mig[0].n == int(crossed.sum()) and mig[1].n == 0
    inbox = slabs.LocalComm(2).exchange(list(outs))
    l0, n0 = slabs.assemble(sl, 0, kept[0], inbox[0], mig[0])
    l1, n1 = slabs.assemble(sl, 1, kept[1], inbox[1], mig[1])
    g = p0.gid[crossed]
    assert set(g) <= set(l1.gid[:n1].tolist())          # owned by rank 1 now
    assert set(g) <= set(l0.gid[n0:].tolist())          # and a halo copy on rank 0
    assert not set(g) & set(l0.gid[:n0].tolist())
    assert n0 + n1 == s.n


def test_dt_is_the_minimum_of_the_ranks_proposals():
    comm = slabs.LocalComm(3)
    assert comm.min([3e-4, 1e-4, 2e-4]) == [1e-4] * 3


class OracleEngine:
    """A rank's step on its local set with the FP64 oracle (test engine)."""

    def __init__(self, scene, sl, r, dt):
        origin, size = sl.local_domain(scene, r)
        self.p = oracle.params(dataclasses.replace(scene, origin=origin, size=size), dt_fixed=dt)
        self.dt = dt

    def load(self, part, n_owned):
        self.part, self.n_owned = part, n_owned

    def cfl_dt(self):
        return self.dt

    def step(self, dt):
        q = self.part
        x, u, d, _, _ = oracle.step(self.p, q.pos, q.vel.astype(np.float64), q.delta.astype(np.float64),
                                    q.mass, q.ptype, 1, dt)
        return x, u, d, self.dt

    def neighbour_sets(self):
        off, idx = oracle.neighbors(self.p, self.part.pos)
        g = self.part.gid
        return {int(g[i]): set(g[idx[off[i]:off[i + 1]]].tolist()) for i in range(self.n_owned)}


def _free_port():
    with socket.socket() as so:
        so.bind(("127.0.0.1", 0))
        return so.getsockname()[1]


def _rank(rank, world, port, dt, steps, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    s = _dam_moving()
    sl = slabs.make_slabs(s, world, at=[0.2])    # the cut through the moving column
    comm = slabs.TorchComm()
    part = slabs.initial_parts(s, sl)[rank]
    eng = OracleEngine(s, sl, rank, dt)
    nsets = None
    dt_used = []
    next_dt = None
    for k in range(steps):
        part, used, next_dt = slabs.step_rank(comm, sl, rank, part, eng, next_dt)
        dt_used.append(used)
        if k == 0:
            nsets = eng.neighbour_sets()
    q.put((rank, part.gid, part.pos, part.vel, part.delta, nsets, dt_used, slabs.initial_parts(s, sl)[rank].gid))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_reproduce_the_undivided_oracle():
    s = _dam_moving()
    dt, steps = 5e-4, 40
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, dt, steps, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=600) for _ in procs]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    gid = np.concatenate([o[1] for o in out])
    assert np.array_equal(np.sort(gid), np.arange(s.n))       # every particle owned once
    moved = sum(len(set(o[1].tolist()) - set(o[7].tolist())) for o in out)
    assert moved > 0                                           # particles changed owner
    pos = np.empty((s.n, 3)); vel = np.empty((s.n, 3)); delta = np.empty(s.n)
    for o in out:
        pos[o[1]], vel[o[1]], delta[o[1]] = o[2], o[3], o[4]
        assert o[6] == [dt] * steps
    p = oracle.params(s, dt_fixed=dt)
    # neighbour sets of the first step (state 0), owned particles of both ranks: exactly
    off, idx = oracle.neighbors(p, s.pos)
    for o in out:
        for i, js in o[5].items():
            assert js == set(idx[off[i]:off[i + 1]].tolist()), f"particle {i}"
    x, u, d, _, _ = oracle.step(p, s.pos, s.vel.astype(np.float64), s.delta.astype(np.float64), s.mass, s.ptype,
                                steps, dt)
    assert np.max(np.abs(pos - x)) < 1e-12
    assert np.max(np.abs(vel - u)) < 1e-12 * max(1.0, np.max(np.abs(u)))
    assert np.max(np.abs(delta - d)) < 1e-12
