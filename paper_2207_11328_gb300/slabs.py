"""Slab decomposition of one scene over several ranks (paper Section
"Multi-GPU": each device holds the particles of its part of the domain plus
copies of its neighbours' particles near the shared boundary, the halo, which
are refreshed between steps; particles that cross a boundary move to the
device that now owns them; the time step is the minimum over all particles).

The domain is cut along one axis (the longest non-periodic one) into slabs of
whole cells of the scene's grid (cells of side >= the influence radius, as the
library lays them out), so every rank's grid is the global grid restricted to
its slab and the neighbour candidates of a particle are the same cells as in
the undivided run.  Each rank holds two cell layers of halo beyond each inner
boundary: a predictor-corrector step of its own particles reads neighbours
within one layer at the predicted state, and those neighbours' predicted
states read one more layer, so with two layers the whole step of the owned
particles runs locally and is exact; the halo copies' own updates are
discarded.  One exchange per step (halo refresh plus migration) and one
minimum-reduction of dt.

The arithmetic of the step is the engine's (``GpuEngine``: the CUDA library on
this rank's GPU); this module only partitions, exchanges and reduces.  The
exchange goes through a ``Comm`` (``TorchComm``: torch.distributed, any
backend; ``LocalComm``: all ranks in one process, for a single device).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

FIELDS = ("pos", "vel", "delta", "mass", "ptype", "gid")


@dataclasses.dataclass
class Part:
    """Particles of one rank, in the scene's layouts plus the global id."""
    pos: np.ndarray      # (n,3) float64
    vel: np.ndarray      # (n,3) float32
    delta: np.ndarray    # (n,)  float32
    mass: np.ndarray     # (n,)  float32
    ptype: np.ndarray    # (n,)  uint8
    gid: np.ndarray      # (n,)  uint32 id in the undivided scene

    @property
    def n(self):
        return int(self.pos.shape[0])

    def take(self, mask_or_idx):
        return Part(*(getattr(self, f)[mask_or_idx] for f in FIELDS))

    @staticmethod
    def cat(parts):
        return Part(*(np.concatenate([getattr(p, f) for p in parts], 0) for f in FIELDS))

    def sorted_by_gid(self):
        return self.take(np.argsort(self.gid, kind="stable"))


def _empty_like(p):
    return p.take(np.zeros(0, np.int64))


@dataclasses.dataclass
class Slabs:
    axis: int            # decomposition axis
    cell: float          # cell side along it (the library's grid)
    lo: float            # domain start along the axis
    ncell: int           # cells along the axis
    cuts: list           # rank r owns cells [cuts[r], cuts[r+1])
    layers: int = 2      # halo depth in cells

    @property
    def world(self):
        return len(self.cuts) - 1

    def edge(self, k):
        return self.lo + self.cuts[k] * self.cell

    def owner(self, x):
        """Rank owning positions x along the axis (cells cut at the slab edges)."""
        c = np.floor((x - self.lo) / self.cell).astype(np.int64)
        c = np.clip(c, 0, self.ncell - 1)
        return np.searchsorted(np.asarray(self.cuts[1:-1]), c, side="right")

    def local_domain(self, scene, r):
        """origin, size of rank r's grid: its slab plus `layers` halo cells on each inner side,
        cell-aligned with the undivided grid (outer sides keep the scene's margins)."""
        c0 = max(0, self.cuts[r] - self.layers)
        c1 = min(self.ncell, self.cuts[r + 1] + self.layers)
        origin, size = list(scene.origin), list(scene.size)
        origin[self.axis] = self.lo + c0 * self.cell
        size[self.axis] = (c1 - c0) * self.cell
        return tuple(origin), tuple(size)


def make_slabs(scene, world, axis=None, kernel_radius=None, layers=2, at=None):
    """Cut the scene's grid into `world` slabs of whole cells with about equal particle
    counts (or at the cells holding the positions `at`, world - 1 of them).  The axis must
    not be periodic (a periodic axis would need a wrapped halo)."""
    R = (kernel_radius or scene.kernel_radius) * scene.h
    if axis is None:
        cand = [a for a in range(3) if not (scene.periodic >> a) & 1]
        if not cand:
            raise ValueError("slab decomposition needs a non-periodic axis")
        axis = max(cand, key=lambda a: scene.size[a])
    if (scene.periodic >> axis) & 1:
        raise ValueError("the decomposition axis must not be periodic")
    ncell = max(1, int(math.floor(scene.size[axis] / R)))
    cell = scene.size[axis] / ncell
    lo = scene.origin[axis]
    c = np.clip(np.floor((scene.pos[:, axis] - lo) / cell).astype(np.int64), 0, ncell - 1)
    counts = np.bincount(c, minlength=ncell)
    cum = np.cumsum(counts)
    cuts = [0]
    for r in range(1, world):
        if at is not None:
            k = int(np.floor((at[r - 1] - lo) / cell))
        else:
            k = int(np.searchsorted(cum, r * cum[-1] / world)) + 1
        cuts.append(min(max(k, cuts[-1] + 2 * layers), ncell - 2 * layers * (world - r)))
    cuts.append(ncell)
    if any(b - a < 2 * layers for a, b in zip(cuts[:-1], cuts[1:])):
        raise ValueError("slabs thinner than their halo: fewer ranks or a finer grid needed")
    return Slabs(axis=axis, cell=cell, lo=lo, ncell=ncell, cuts=cuts, layers=layers)


def initial_parts(scene, slabs):
    """The scene's particles split by owner (each part sorted by global id)."""
    gid = np.arange(scene.n, dtype=np.uint32)
    allp = Part(scene.pos, scene.vel, scene.delta.astype(np.float32), scene.mass, scene.ptype, gid)
    own = slabs.owner(scene.pos[:, slabs.axis])
    return [allp.take(own == r) for r in range(slabs.world)]


class LocalComm:
    """All ranks in one process (a single device): exchange is a hand-over."""

    def __init__(self, world):
        self.world = world

    def exchange(self, outboxes):
        """outboxes[r][q]: what rank r sends to rank q -> inboxes[q][r]."""
        return [[outboxes[r][q] for r in range(self.world)] for q in range(self.world)]

    def min(self, values):
        m = min(values)
        return [m] * len(values)


class TorchComm:
    """One rank per process through torch.distributed (gloo on CPU, nccl on GPUs)."""

    def __init__(self):
        import torch.distributed as dist
        self.dist = dist
        self.world = dist.get_world_size()
        self.rank = dist.get_rank()

    def exchange(self, outbox):
        """outbox[q]: what this rank sends to rank q -> inbox[r]: what rank r sent here."""
        gathered = [None] * self.world
        self.dist.all_gather_object(gathered, outbox)
        return [gathered[r][self.rank] for r in range(self.world)]

    def min(self, value):
        out = [None] * self.world
        self.dist.all_gather_object(out, float(value))
        return min(out)


def migrate_and_halo(slabs, r, own):
    """Outbox of rank r: particles that left its slab (to their new owner) and the
    halo copies of its boundary layers (to each neighbour).  A particle moves by less
    than a cell per step, so a migrant lands in the neighbour's first cell, inside
    rank r's own halo: r keeps its current copy there (the new owner's halo copies are
    taken from what it owned before the exchange).  Returns (kept, outbox, own halo)."""
    x = own.pos[:, slabs.axis]
    owner = slabs.owner(x)
    kept = own.take(owner == r)
    migrants = own.take(owner != r)
    out = [_empty_like(own) for _ in range(slabs.world)]
    for q in range(slabs.world):
        if q != r:
            out[q] = own.take(owner == q)
    xk = kept.pos[:, slabs.axis]
    halo = slabs.layers * slabs.cell
    if r > 0:
        lo = slabs.edge(r)
        out[r - 1] = Part.cat([out[r - 1], kept.take(xk < lo + halo)])
    if r < slabs.world - 1:
        hi = slabs.edge(r + 1)
        out[r + 1] = Part.cat([out[r + 1], kept.take(xk >= hi - halo)])
    return kept, out, migrants


def assemble(slabs, r, kept, inbox, own_halo):
    """Rank r's local set: its owned particles (arrived migrants included) first, then the
    halo copies (received, and its own departed migrants), each sorted by global id;
    returns (local part, n_owned)."""
    arrivals, halos = [kept], [own_halo]
    for q, box in enumerate(inbox):
        if q == r or box.n == 0:
            continue
        own = slabs.owner(box.pos[:, slabs.axis]) == r
        arrivals.append(box.take(own))
        halos.append(box.take(~own))
    owned = Part.cat(arrivals).sorted_by_gid()
    halo = Part.cat(halos).sorted_by_gid()
    return Part.cat([owned, halo]), owned.n


class GpuEngine:
    """The CUDA library on this rank's slab: one context sized for the local set."""

    def __init__(self, scene, slabs, r, capacity, max_neibs=128, stream=None):
        from . import Simulation
        origin, size = slabs.local_domain(scene, r)
        local = dataclasses.replace(scene, origin=origin, size=size, scenes=None)
        self.sim = Simulation.from_scene(local, max_particles=capacity, max_neibs=max_neibs, upload=False)
        self.stream = stream
        self.capacity = capacity

    def load(self, part, n_owned):
        if part.n > self.capacity:
            raise RuntimeError(f"local set of {part.n} particles exceeds the rank's capacity {self.capacity}")
        self.sim.upload(pos=part.pos, vel=part.vel, delta=part.delta, mass=part.mass, ptype=part.ptype,
                        stream=self.stream)
        self.sim.set_owned(n_owned)

    def cfl_dt(self):
        return self.sim.cfl_dt(stream=self.stream)

    def step(self, dt):
        """One step with the given dt; returns the new (pos, vel, delta) in upload order
        and this rank's proposal for the next dt (owned particles only)."""
        self.sim.set_dt(dt)
        self.sim.step(1, stream=self.stream)
        pos, vel, delta = self.sim.download(stream=self.stream)
        return pos, vel, delta, self.sim.next_dt(stream=self.stream)

    def close(self):
        self.sim.close()


def run_local(scene, world, steps, make_engine, layers=2):
    """All ranks in one process (LocalComm): `steps` steps of the decomposed scene,
    each rank stepped by make_engine(slabs, r).  Returns the owned particles of every
    rank after the last step (a list of Part) and the time steps used."""
    slabs = make_slabs(scene, world, layers=layers)
    comm = LocalComm(world)
    parts = initial_parts(scene, slabs)
    engines = [make_engine(slabs, r) for r in range(world)]
    dts = []
    dt = None
    for _ in range(steps):
        kept, outs, mig = zip(*[migrate_and_halo(slabs, r, parts[r]) for r in range(world)])
        inboxes = comm.exchange(list(outs))
        local = [assemble(slabs, r, kept[r], inboxes[r], mig[r]) for r in range(world)]
        for r in range(world):
            engines[r].load(*local[r])
        if dt is None:  # the first step's dt: the minimum of every rank's CFL value
            dt = comm.min([engines[r].cfl_dt() for r in range(world)])[0]
        proposals = []
        for r in range(world):
            part, n_own = local[r]
            pos, vel, delta, prop = engines[r].step(dt)
            parts[r] = Part(pos[:n_own], vel[:n_own], delta[:n_own], part.mass[:n_own], part.ptype[:n_own],
                            part.gid[:n_own])
            proposals.append(prop)
        dts.append(dt)
        dt = comm.min(proposals)[0]
    for e in engines:
        if hasattr(e, "close"):
            e.close()
    return parts, dts, slabs


def step_rank(comm, slabs, r, part, engine, dt):
    """One decomposed step of rank r under a TorchComm: exchange, load, (first dt),
    step, dt reduction.  Returns (owned part after the step, dt used, next dt)."""
    kept, out, mig = migrate_and_halo(slabs, r, part)
    inbox = comm.exchange(out)
    local, n_own = assemble(slabs, r, kept, inbox, mig)
    engine.load(local, n_own)
    if dt is None:
        dt = comm.min(engine.cfl_dt())
    pos, vel, delta, prop = engine.step(dt)
    owned = Part(pos[:n_own], vel[:n_own], delta[:n_own], local.mass[:n_own], local.ptype[:n_own], local.gid[:n_own])
    return owned, dt, comm.min(prop)
