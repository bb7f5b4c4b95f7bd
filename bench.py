"""Benchmark of the GB300 WCSPH hot path.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--workload NAME]

A step is one pass of the whole hot path: neighbour pipeline (hash, sort,
reorder, cell start/end, split neighbour list), forces at n + predictor,
forces at the predicted state + corrector, CFL dt.  The default workload is
the 3D dam break refined to ~16M fluid particles (tank 1.6 x 0.67 x 0.6 m,
column 0.4 x 0.67 x 0.3 m, dp = 4.3 mm / 16^(1/3) = 1.71 mm, 3 layers of
dynamic boundary particles, 20.1M particles in total), synthetic and seeded,
with the list rebuilt every step; its arrays (~16 GB with the neighbour
list) exceed the 126 MB L2 many times over, so no flush is needed between
steps.  `--workload dam1m` runs the ~1M-fluid-particle version (dp 4.3 mm,
1.65M particles).

The timed region is exactly --steps steps after --warmup steps from the
initial column at rest; the line also carries the same measurement taken
after --flow-steps further steps (`flowing`: the column collapsing), the
per-kernel roofline (the dominant kernel first), the clocks sampled through
NVML every 10 ms inside the timed region, the end-to-end figure through the
C ABI with host buffers, and the FP64 oracle on the host cores.

Metric: particle-interactions/s = (neighbour-list entries of each step's
build x 2 force passes) / time; particle-steps/s is reported beside it.
Rank 0 prints one JSON line.  Under torchrun each rank runs an independent
replica (the single scene does not shard; "replicas only") and value is the
whole-job aggregate over the max-over-ranks time.
"""
from __future__ import annotations

import argparse
import csv
import io
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "particle-interactions/s and particle-steps/s at 1 GB300, % HBM roofline"
UNIT = "particle-interactions/s"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM_GBS = 6800.0


def make_workload(name):
    from paper_2207_11328_gb300 import scenes
    if name == "dam1m":
        return scenes.dam_break(dp=4.3e-3), "dam_break_1M: tank 1.6x0.67x0.6 m, column 0.4x0.67x0.3 m, dp 4.3 mm"
    if name == "dam16m":
        return (scenes.dam_break(dp=4.3e-3 / 16 ** (1 / 3)),
                "dam_break_16M: tank 1.6x0.67x0.6 m, column 0.4x0.67x0.3 m, dp 1.71 mm")
    if name == "box":
        return scenes.periodic_box(n_per_axis=16), "periodic_box_4096: 16^3 lattice, dp 0.02 m"
    if name == "box2m":
        return (scenes.periodic_box(n_per_axis=128, jitter=0.1),
                "periodic_box_2M: 128^3 lattice (jitter 0.1 dp), dp 0.02 m, all fluid, 80 neighbours")
    raise SystemExit(f"unknown workload {name}")


def kernel_traffic(kernel, workload):
    """Measured DRAM bytes (read + write) per launch of `kernel` on `workload`
    from a committed ncu summary (profiles/traffic_*.md: lines `kernel:`,
    `workload:`, `sources:`, `source_sha256:`, `dram_bytes_per_launch:`), or
    None when no summary matches or a listed source changed since the capture."""
    import glob
    import hashlib
    for path in sorted(glob.glob(os.path.join(ROOT, "profiles", "traffic_*.md"))):
        kv = {}
        for line in open(path):
            if ":" in line and not line.startswith(("#", "|", " ", "`")):
                k, v = line.split(":", 1)
                kv.setdefault(k.strip(), v.strip())
        if kv.get("kernel") != kernel or kv.get("workload") != workload:
            continue
        h = hashlib.sha256()
        for f in kv.get("sources", "").split(","):
            h.update(open(os.path.join(ROOT, "paper_2207_11328_gb300", "csrc", f.strip()), "rb").read())
        if kv.get("source_sha256") == h.hexdigest():
            return float(kv["dram_bytes_per_launch"])
    return None


KERNELS = {"wendland": 0, "cubic": 1, "quadratic": 2, "gaussian": 3}
VISC = {"artificial": 0, "morris": 1, "monaghan": 2, "espanol-revenga": 3}


def apply_physics(scene, args):
    """Model options of Table 1 on top of the workload's own (default: the
    workload as generated).  Returns the scene and a description."""
    import dataclasses
    kw = {}
    if args.kernel != "wendland":
        kw["kernel_type"] = KERNELS[args.kernel]
        if args.kernel == "gaussian":
            kw["kernel_radius"] = 3.0
    if args.formulation == 2:
        kw["formulation"] = 1
    if args.visc is not None:
        kw["visc"] = VISC[args.visc]
        if kw["visc"] != 0:
            kw.update(alpha=0.0, nu=args.nu)
    if args.ddiff > 0:
        kw.update(ddiff=1, ddiff_coef=args.ddiff)
    desc = {"kernel": args.kernel, "formulation": args.formulation,
            "viscosity": args.visc or ("artificial" if scene.visc == 0 else "morris"),
            "density_diffusion": f"Molteni-Colagrossi xi={args.ddiff}" if args.ddiff > 0 else "none"}
    return (dataclasses.replace(scene, **kw) if kw else scene), desc


def load_peaks():
    try:
        with open(PEAKS_FILE) as f:
            pk = json.load(f)
        return float(pk["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


class _Nvml:
    """The few NVML queries the clock record needs, through ctypes (libnvidia-ml
    ships with the driver; no Python NVML package is assumed).  Read-only."""
    SM = 1  # NVML_CLOCK_SM
    REASONS = {0x8: "hw_slowdown", 0x40: "hw_thermal_slowdown", 0x20: "sw_thermal_slowdown",
               0x4: "sw_power_cap", 0x80: "hw_power_brake_slowdown"}

    def __init__(self, local_index):
        import ctypes
        self.c = ctypes
        self.lib = ctypes.CDLL("libnvidia-ml.so.1")
        if self.lib.nvmlInit_v2() != 0:
            raise OSError("nvmlInit failed")
        self.dev = ctypes.c_void_p()
        uuid = None
        try:
            import torch
            u = getattr(torch.cuda.get_device_properties(local_index), "uuid", None)
            uuid = ("GPU-" + str(u)) if u is not None else None
        except Exception:
            uuid = None
        rc = -1
        if uuid:
            rc = self.lib.nvmlDeviceGetHandleByUUID(uuid.encode(), ctypes.byref(self.dev))
        if rc != 0:
            vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
            ids = [v for v in vis.split(",") if v.strip()]
            idx = int(ids[local_index]) if ids and ids[local_index].strip().isdigit() else local_index
            rc = self.lib.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(idx), ctypes.byref(self.dev))
        if rc != 0:
            raise OSError("no NVML handle for the device")
        fn = getattr(self.lib, "nvmlDeviceGetCurrentClocksEventReasons", None)
        self.reasons_fn = fn or self.lib.nvmlDeviceGetCurrentClocksThrottleReasons
        mx = ctypes.c_uint()
        self.max_sm = float(mx.value) if self.lib.nvmlDeviceGetMaxClockInfo(self.dev, self.SM,
                                                                             ctypes.byref(mx)) == 0 else None

    def sample(self):
        c = self.c
        sm, pw, rs = c.c_uint(), c.c_uint(), c.c_ulonglong()
        ok = self.lib.nvmlDeviceGetClockInfo(self.dev, self.SM, c.byref(sm)) == 0
        self.lib.nvmlDeviceGetPowerUsage(self.dev, c.byref(pw))
        self.reasons_fn(self.dev, c.byref(rs))
        return (float(sm.value) if ok else None), pw.value / 1e3, int(rs.value)


class ClockSampler:
    """SM clock, power and throttle reasons sampled every 10 ms (NVML) while the
    timed region runs; mark() brackets the region and summary() keeps only the
    samples taken inside it.  Falls back to nvidia-smi at 200 ms without NVML."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    PERIOD_S = 0.010

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.nvml = None
        self.rows = []          # (t, sm_mhz, power_w, reasons bits)
        self.t0 = self.t1 = None
        self.out = ""

    def _loop(self):
        while not self._stop.is_set():
            t = time.perf_counter()
            try:
                self.rows.append((t,) + self.nvml.sample())
            except Exception:
                pass
            self._stop.wait(self.PERIOD_S)

    def __enter__(self):
        import threading
        try:
            self.nvml = _Nvml(self.index)
        except Exception:
            self.nvml = None
        if self.nvml is not None:
            self._stop = threading.Event()
            self._th = threading.Thread(target=self._loop, daemon=True)
            self._th.start()
        else:
            try:
                self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                              "--format=csv,noheader,nounits", "-lms", "200"],
                                             stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            except Exception:
                self.proc = None
            time.sleep(0.3)
        return self

    def mark(self, start):
        """Host time at the start (start=True, after the synchronize before the
        region) or the end (after the synchronize that closes it)."""
        if start:
            self.t0 = time.perf_counter()
        else:
            self.t1 = time.perf_counter()

    def __exit__(self, *a):
        if self.nvml is not None:
            self._stop.set()
            self._th.join(timeout=5)
        elif self.proc:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
        return False

    def summary(self):
        if self.nvml is not None:
            inside = [r for r in self.rows if self.t0 is not None and self.t1 is not None and self.t0 <= r[0] <= self.t1]
            sm = [r[1] for r in inside if r[1] is not None]
            bits = 0
            for r in inside:
                bits |= r[3]
            reasons = sorted(name for b, name in _Nvml.REASONS.items() if bits & b)
            return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": self.nvml.max_sm,
                    "sm_mhz_min": min(sm) if sm else None, "power_w_max": max((r[2] for r in inside), default=None),
                    "reasons": reasons, "samples": len(inside), "source": "NVML every 10 ms inside the timed region",
                    "region_s": (self.t1 - self.t0) if self.t0 is not None and self.t1 is not None else None}
        rows = [r for r in csv.reader(io.StringIO(self.out or "")) if len(r) >= 9]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].strip().lower() == "active"})
        load = sorted(sm)[len(sm) // 2:] if sm else []   # upper half: samples under load
        return {"sm_mhz": float(np.median(load)) if load else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows), "source": "nvidia-smi every 200 ms around the region"}


def dist_setup(n_gpus):
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    elif torch.cuda.is_available():
        torch.cuda.set_device(0)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def _reduce(world, v, op):
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=op)
    return float(t.item())


def allmax(world, v):
    import torch.distributed as dist
    return _reduce(world, v, dist.ReduceOp.MAX if world > 1 else None)


def allsum(world, v):
    import torch.distributed as dist
    return _reduce(world, v, dist.ReduceOp.SUM if world > 1 else None)


def aggregate(world, interactions_local, particle_steps_local, seconds_local):
    """Whole-job throughput of independent replicas: work summed over ranks
    divided by the slowest rank's time (max over ranks)."""
    t_max = allmax(world, seconds_local)
    return allsum(world, interactions_local) / t_max, allsum(world, particle_steps_local) / t_max, t_max


# ---------------------------------------------------------------------------
# oracle timing (the CPU baseline and the reference arm)
# ---------------------------------------------------------------------------
def oracle_window(scene, target_n):
    """Bounded sample of a workload: the particles in the corner cube
    x, y, z < w of the tank (fluid and walls alike), w chosen so that about
    target_n particles fall inside."""
    from paper_2207_11328_gb300 import scenes
    if target_n >= scene.n:
        return scene, None
    # a particle is inside the cube iff its largest coordinate is below w: w just above
    # the target_n-th smallest of those maxima (one selection pass)
    top = np.max(scene.pos, axis=1)
    w = float(np.nextafter(np.partition(top, target_n - 1)[target_n - 1], np.inf))
    mask = top < w
    sub = scenes.subset(scene, mask, name=scene.name + f"_corner{w:.4f}")
    # the sample's own domain on the non-periodic axes: its extent twice over plus two
    # influence radii (room to move during a run), within the workload's, so that the
    # oracle bins the sample rather than the whole tank at the workload's resolution
    import dataclasses
    origin, size = np.asarray(scene.origin, np.float64), np.asarray(scene.size, np.float64)
    ext = 2.0 * (w - origin) + 2.0 * scene.kernel_radius * scene.h
    per = np.array([(scene.periodic >> a) & 1 for a in range(3)], bool)
    size = np.where(per, size, np.minimum(size, ext))
    return dataclasses.replace(sub, size=tuple(float(v) for v in size)), w


def interactions_of(p, sub, x):
    """Pairs a step evaluates twice: all neighbours of fluid particles, fluid
    neighbours of boundary particles (boundary-boundary pairs carry nothing), as
    ordered pairs at distance 0 < r < 2h.  Bookkeeping for the metric, counted
    with a k-d tree over the sample (the oracle's own search bins the whole
    domain of the workload on every call); periodic axes by minimum image."""
    from scipy.spatial import cKDTree
    per = np.array([(sub.periodic >> a) & 1 for a in range(3)], bool)
    R = float(np.nextafter(sub.kernel_radius * sub.h, 0.0))        # r < 2h
    pts = np.array(x, np.float64) - np.asarray(sub.origin, np.float64)
    if per.any():
        size = np.asarray(sub.size, np.float64)
        pts[:, per] = np.mod(pts[:, per], size[per])
        pts[:, per] = np.where(pts[:, per] >= size[per], 0.0, pts[:, per])
        pts[:, ~per] -= pts[:, ~per].min(axis=0)
        box = np.where(per, size, pts.max(axis=0) + 2.0 * R + 1.0)   # no wrap on the other axes
        tree = lambda q: cKDTree(q, boxsize=box)  # noqa: E731
    else:
        tree = cKDTree
    b = sub.ptype != 0
    t_all, t_b = tree(pts), tree(pts[b])
    n_all = int(t_all.count_neighbors(t_all, R)) - sub.n            # ordered pairs, self-pairs removed
    n_bb = int(t_b.count_neighbors(t_b, R)) - int(np.count_nonzero(b))
    return n_all - n_bb


def time_oracle_steps(sub, steps, warmup=0):
    """The FP64 oracle as it stands, single-threaded, on a bounded sample:
    warm-up steps untimed, then `steps` predictor-corrector steps timed.
    Returns (interactions, particle_steps, seconds)."""
    import oracle
    p = oracle.params(sub)
    x, u, d = sub.pos, sub.vel.astype(np.float64), sub.delta.astype(np.float64)
    a, _ = oracle.rhs(p, x, u, d, sub.mass, sub.ptype)
    dt = oracle.cfl_dt(p, a, sub.ptype)
    if warmup:
        x, u, d, dt, _ = oracle.step(p, x, u, d, sub.mass, sub.ptype, warmup, dt)
    inter = 0
    t = 0.0
    for _ in range(steps):
        inter += 2 * interactions_of(p, sub, x)      # untimed: the pairs this step will use
        t0 = time.perf_counter()
        x, u, d, dt, _ = oracle.step(p, x, u, d, sub.mass, sub.ptype, 1, dt)
        t += time.perf_counter() - t0
    return inter, sub.n * steps, t


_POOL_STATE = None


def _pool_init(pkw, x, u, d, m, t):
    global _POOL_STATE
    import oracle
    _POOL_STATE = (oracle.params(None, **pkw), x, u, d, m, t)


def _pool_rhs(idx):
    import oracle
    p, x, u, d, m, t = _POOL_STATE
    oracle.rhs_sample(p, x, u, d, m, t, idx)
    return len(idx)


def _params_kw(p):
    return {k: (list(getattr(p, k)) if k in ("g", "origin", "size") else getattr(p, k))
            for k, _ in p._fields_ if not k.startswith("pad")}


def time_oracle_parallel(sub, cores, passes=2):
    """The same oracle, unchanged, on every host core: `cores` spawned worker
    processes each evaluate the force pass (ora_rhs_sample, neighbours
    searched among all particles) for their share of the particles.  The
    state is handed to the workers once, before the timed passes.
    Returns (interactions, seconds)."""
    import multiprocessing as mp
    import oracle
    p = oracle.params(sub)
    x, u, d = sub.pos, sub.vel.astype(np.float64), sub.delta.astype(np.float64)
    chunks = [c.astype(np.int32) for c in np.array_split(np.arange(sub.n), cores)]
    inter = passes * interactions_of(p, sub, x)
    ctx = mp.get_context("spawn")
    with ctx.Pool(cores, initializer=_pool_init, initargs=(_params_kw(p), x, u, d, sub.mass, sub.ptype)) as pool:
        pool.map(_pool_rhs, [c[:16] for c in chunks[:cores]])  # warm: workers started, bins code paged in
        t0 = time.perf_counter()
        for _ in range(passes):
            pool.map(_pool_rhs, chunks, chunksize=1)
        t = time.perf_counter() - t0
    return inter, t


def cpu_baseline(scene, workload, target_n=600_000):
    sub, w = oracle_window(scene, target_n)
    inter, psteps, t = time_oracle_steps(sub, 1)
    where = f"the corner cube x, y, z < {w:.4f} m" if w is not None else "all particles"
    cores = max(1, os.cpu_count() or 1)
    passes = 6   # ~1 s on 16 cores: 10-20 s of CPU work with the single-thread step
    pinter, pt = time_oracle_parallel(sub, cores, passes)
    return {"value": pinter / pt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{passes} force passes of the FP64 oracle on the {sub.n} particles of the workload in "
                      f"{where}, split over {cores} worker processes ({pinter} interactions, {pt:.1f} s)",
            "single_thread": {"value": inter / t, "unit": UNIT, "cores": 1, "particle_steps_per_s": psteps / t,
                              "sample": f"1 predictor-corrector step (neighbour search + 2 force passes + dt) "
                                        f"of the same oracle, one thread, same particles ({inter} interactions, "
                                        f"{t:.1f} s)"}}


def run_reference(args, world, rank):
    if rank != 0:
        return
    scene, wdesc = make_workload(args.workload)
    # size the sample so the whole --steps/--warmup run stays within a few minutes: ~75 s of
    # timed oracle steps, and about as much again for each step's untimed pair count
    budget = 75.0 / max(1, args.steps + args.warmup)
    probe, _ = oracle_window(scene, 20_000)
    _, pn, pt = time_oracle_steps(probe, 1)
    rate = pn / max(pt, 1e-9)                     # particle-steps/s of the oracle
    sub, w = oracle_window(scene, max(2000, int(rate * budget)))
    where = f"the corner cube x, y, z < {w:.4f} m of the workload" if w is not None else "the whole workload"
    inter, psteps, t = time_oracle_steps(sub, args.steps, args.warmup)
    value = inter / t
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": wdesc, "n_particles": scene.n},
            "particle_steps_per_s": psteps / t,
            "cpu_baseline": {"value": value, "unit": UNIT, "kind": "oracle", "cores": 1,
                             "sample": f"each step: one FP64 oracle step (single thread) on the {sub.n} particles "
                                       f"of {where}"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# Algorithmic bytes per launch of each kernel of a step (what the method must move;
# neighbour candidates and gathers are served by L1/L2/shared memory by construction of
# the cell sort), with n particles and e list entries of the step's build:
#   hash      read pos4 16 + cell 4 + scene 4, write key 4 + slot 4              32 n
#   reorder   read unsorted 4 + pos4 16 + vel4 16 + P/rho^2 4 + scene 4 + id 4,
#             write the same five arrays + cell 4                                96 n
#   build     read pos4 16 + cell 4 + scene 4, write count 4 + list 4 e           28 n + 4 e
#   forces + predictor   read pos4 16 + vel4 16 + scene 4 + count 4 + list 4 e,
#                        write pos*, vel* 32                                      72 n + 4 e
#   forces + corrector   the same reads at the predicted state, read and write
#                        the state n (64)                                         104 n + 4 e
#   build + forces + predictor (one kernel)  read pos4 16 + vel4 16 + cell 4 + scene 4,
#                        write count 4 + list 4 e + pos*, vel* 32 + P*/rho*^2 4   80 n + 4 e
def algorithmic_bytes(phase, n, e):
    return {"hash": 32 * n, "reorder": 96 * n, "build": 28 * n + 4 * e, "forces_predict": 72 * n + 4 * e,
            "forces_correct": 104 * n + 4 * e, "build_predict": 80 * n + 4 * e}.get(phase)


KERNEL_NAMES = {"build": "k_build_tpp", "forces_predict": "k_forces<predictor>",
                "forces_correct": "k_forces<corrector>", "reorder": "k_reorder", "hash": "k_hash",
                "build_predict": "k_tile_predict"}


def timed_region(sim, steps, stream, world, local):
    """Exactly `steps` steps between CUDA events on the launch stream, bracketed
    by a barrier and a synchronize on both sides; clocks sampled inside.
    Returns (ms, stats before, stats after, clock summary)."""
    import torch
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    st0 = sim.stats(stream=stream)
    with ClockSampler(local) as clk:
        barrier(world)
        torch.cuda.synchronize()
        clk.mark(True)
        ev0.record(stream)
        sim.step(steps, stream=stream)
        ev1.record(stream)
        torch.cuda.synchronize()
        clk.mark(False)
        barrier(world)
    ms = ev0.elapsed_time(ev1)
    st1 = sim.stats(stream=stream)
    return ms, st0, st1, clk.summary()


def run_ours(args, world, rank, local):
    import torch
    from paper_2207_11328_gb300 import Simulation, _build, fp32_peak

    if rank == 0 or not os.path.exists(_build.LIB):
        _build.build()
    barrier(world)
    scene, wdesc = make_workload(args.workload)
    scene, physics = apply_physics(scene, args)
    if args.kernel == "gaussian":  # support 3h: ~3.4x the neighbours of 2h
        args.max_neibs = max(args.max_neibs, 352)
    stream = torch.cuda.current_stream()
    skin_mode = args.rebuild_every > 1
    if skin_mode:  # the skin shell adds ~(1 + skin/2h)^3 - 1 of the pairs to the list
        args.max_neibs = max(args.max_neibs, int(128 * (1 + args.skin / 2) ** 3) // 32 * 32 + 32)
    sim = Simulation.from_scene(scene, max_neibs=args.max_neibs, stream=stream, rebuild_every=args.rebuild_every,
                                skin=args.skin * scene.h)
    if args.variants:
        # shapes given (profiling under ncu, whose launch interception skews the tuner's timings)
        vb, vp, vc = (int(x) for x in args.variants.split(","))
        sim.set_variants(build=vb)
        sim.set_forces_variants(vp, vc)
    else:
        sim.autotune(stream=stream)
    tuned = sim.variants()
    sim.step(args.warmup, stream=stream)

    def pairs_of(st0, st1):
        # interactions: 2 force passes x pairs within 2h (the list itself when it is rebuilt
        # every step; counted by the first force pass when the list carries a skin)
        return 2.0 * ((st1["interactions"] - st0["interactions"]) if skin_mode
                      else (st1["list_entries"] - st0["list_entries"]))

    ms, st0, st1, clocks = timed_region(sim, args.steps, stream, world, local)
    inter_local = pairs_of(st0, st1)
    psteps_local = float(st1["n_active"]) * args.steps
    value, psteps, t_max = aggregate(world, inter_local, psteps_local, ms / 1e3)
    kernels = st1["kernels_per_step"]

    # per-kernel durations (same work, launched one by one with events on the launch stream)
    phases = sim.step_profiled(args.profile_steps, stream=stream)
    st2 = sim.stats(stream=stream)
    n = float(st2["n_active"])
    nbuilds = max(1, st2["builds"] - st1["builds"]) if skin_mode else args.profile_steps
    # list entries read per force launch: the list of the step (rebuilt every step), or the
    # skin list (its entries per build, read by every step until the next build)
    e_step = (st2["list_entries"] - st1["list_entries"]) / max(1, st2["builds"] - st1["builds"])
    hbm, peak_src = load_peaks()
    launches = {p: (nbuilds if p in ("hash", "scan", "scatter", "reorder", "build") and skin_mode
                    else args.profile_steps) for p in phases}
    per_launch_ms = {p: phases[p] / max(1, launches[p]) for p in phases if phases[p] > 0}
    step_ms = {p: phases[p] / args.profile_steps for p in phases}
    kernels_rf = {}
    for p in ("build_predict", "build", "forces_predict", "forces_correct", "reorder", "hash"):
        if p not in per_launch_ms:
            continue
        e_p = e_step
        if skin_mode and p in ("forces_correct",):
            e_p = (st2["interactions"] - st1["interactions"]) / args.profile_steps
        byts = algorithmic_bytes(p, n, e_p)
        if skin_mode and p == "forces_predict":  # reads the skin list, writes the exact list and counts
            byts = 76 * n + 4 * e_step + 4 * (st2["interactions"] - st1["interactions"]) / args.profile_steps
        t = per_launch_ms[p] / 1e3
        kernels_rf[p] = {"kernel": KERNEL_NAMES.get(p, p), "achieved": byts / t / 1e9, "unit": "GB/s",
                         "frac": byts / t / 1e9 / hbm, "algorithmic_bytes_per_launch": byts,
                         "ms_per_launch": 1e3 * t, "share_of_step": step_ms[p] / max(1e-12, sum(step_ms.values())),
                         "traffic": None if skin_mode else kernel_traffic(KERNEL_NAMES.get(p, p), args.workload)}
    dom = max(kernels_rf, key=lambda p: kernels_rf[p]["share_of_step"])
    d = kernels_rf[dom]
    roofline = {"bound": "hbm", "kernel": d["kernel"], "achieved": d["achieved"], "peak": hbm,
                "peak_source": f"{peak_src} HBM copy bandwidth (of {peak_src})", "unit": "GB/s",
                "frac": d["frac"], "traffic": d["traffic"],
                "algorithmic_bytes_per_launch": d["algorithmic_bytes_per_launch"], "ms_per_launch": d["ms_per_launch"],
                "note": "dominant kernel by share of the step; it is bound by instruction issue, not by HBM "
                        "(see kernels[*] and the ncu summaries)",
                "kernels": kernels_rf, "phase_ms_per_step": step_ms}
    # the ALU view of the force passes: FP32 flops of a pair term (FMA = 2): separation 3,
    # r^2 5, r 2, q - 2 2, m (q-2)^3 3, u_ij 3, u.x 5, continuity 2, pressure bracket 1,
    # coefficient 1, a 6 = 33 (+9 on approaching pairs for the artificial viscosity, not counted)
    pairs_step = 2 * ((st2["interactions"] - st1["interactions"]) / args.profile_steps if skin_mode else e_step)
    t_forces = (phases.get("forces_predict", 0.0) + phases.get("forces_correct", 0.0)
                + phases.get("build_predict", 0.0)) / args.profile_steps / 1e3
    alu_peak = fp32_peak(stream)
    alu = 33.0 * pairs_step / max(t_forces, 1e-12) / 1e12
    roofline["alu"] = {"kernel": "force passes", "achieved": alu, "peak": alu_peak, "unit": "TFLOP/s",
                       "frac": alu / alu_peak, "peak_source": "measured FP32 FMA throughput (sph_fp32_peak)",
                       "flops_per_pair": 33}
    if skin_mode:
        roofline["profiled_steps"] = {"steps": args.profile_steps, "list_builds": nbuilds,
                                      "build_ms_per_list_build": phases["build"] / nbuilds}

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": wdesc, "n_particles": scene.n, "n_fluid": scene.n_fluid, "dp": scene.dp,
                       "h": scene.h, "max_neibs": args.max_neibs,
                       "physics": physics,
                       "rebuild": "every step" if not skin_mode else
                                  f"every {args.rebuild_every} steps, list radius 2h + {args.skin}h",
                       "state": f"initial column at rest after {args.warmup} warm-up steps",
                       "l2": "inputs larger than L2 (no flush)", "parallelism": f"replicas x{world}",
                       "variants": dict(tuned, autotuned=not args.variants,
                                        fused_build_predict=bool(sim.step_options()["fused_predict"]))},
            "particle_steps_per_s": psteps, "mean_neighbours": inter_local / 2 / max(1.0, psteps_local),
            "list_builds": st1["builds"] - st0["builds"],
            "roofline": roofline, "gpu_launches": int(kernels * args.steps),
            "clocks": clocks}
    line["clocks"]["time_x_median_mhz"] = (1e3 * t_max / args.steps * clocks["sm_mhz"]
                                           if clocks.get("sm_mhz") else None)

    # the same measurement on a flowing state: the column collapses for flow_steps more steps
    if args.flow_steps > 0:
        sim.step(args.flow_steps, stream=stream)
        ms_f, sf0, sf1, clk_f = timed_region(sim, args.steps, stream, world, local)
        inter_f = pairs_of(sf0, sf1)
        ps_f = float(sf1["n_active"]) * args.steps
        v_f, p_f, t_f = aggregate(world, inter_f, ps_f, ms_f / 1e3)
        line["flowing"] = {"value": v_f, "unit": UNIT, "ms_per_step": 1e3 * t_f / args.steps,
                           "particle_steps_per_s": p_f, "steps": args.steps,
                           "steps_before": args.warmup + args.steps + args.profile_steps + args.flow_steps,
                           "simulated_time_s": sf1["time"], "mean_neighbours": inter_f / 2 / max(1.0, ps_f),
                           "n_removed": sf1["n_removed"], "clocks": clk_f}

    # end to end through the public API with host buffers (upload, one step, download), by
    # --e2e-workers host threads, each with its own context and stream (the first is the
    # benchmark's), so that one worker's copies run beside another's kernels
    if args.e2e_steps > 0:
        import threading
        from paper_2207_11328_gb300 import build_variant_names, forces_variant_names
        pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()  # noqa: E731
        hp = {k: pin(v) for k, v in dict(pos=scene.pos, vel=scene.vel, delta=scene.delta.astype(np.float32),
                                          mass=scene.mass, ptype=scene.ptype).items()}
        nw = max(1, args.e2e_workers)
        workers = [(sim, torch.cuda.Stream())]   # every worker on a stream of its own
        for _ in range(nw - 1):
            s_k = torch.cuda.Stream()
            sim_k = Simulation.from_scene(scene, max_neibs=args.max_neibs, stream=s_k,
                                          rebuild_every=args.rebuild_every, skin=args.skin * scene.h)
            sim_k.set_variants(build=build_variant_names().index(tuned["build"]))
            sim_k.set_forces_variants(forces_variant_names().index(tuned["forces_predict"]),
                                      forces_variant_names().index(tuned["forces_correct"]))
            sim_k.set_fused_predict(bool(sim.step_options()["fused_predict"]))
            workers.append((sim_k, s_k))
        outs = [{"pos": pin(np.empty_like(scene.pos)), "vel": pin(np.empty_like(scene.vel)),
                 "delta": pin(np.empty(scene.n, np.float32))} for _ in workers]
        h2d = sum(v.nbytes for v in hp.values())
        d2h = sum(v.nbytes for v in outs[0].values())
        counts = [0.0] * nw

        def e2e_steps(k, nsteps):
            sim_k, s_k = workers[k]
            for _ in range(nsteps):
                sim_k.upload(pos=hp["pos"], vel=hp["vel"], delta=hp["delta"], mass=hp["mass"],
                             ptype=hp["ptype"], stream=s_k)
                sim_k.step(1, stream=s_k)
                sim_k.download(stream=s_k, out=(outs[k]["pos"], outs[k]["vel"], outs[k]["delta"]))
                # the upload resets the counters: the list entries of its build (the list the
                # step uses), or the pairs the step's first pass found within 2h (skin list)
                counts[k] += 2.0 * sim_k.stats(stream=s_k, check=False)[
                    "interactions" if skin_mode else "list_entries"]

        torch.cuda.synchronize()
        for k in range(nw):   # each worker's first step (graph capture on its stream) outside the timing
            e2e_steps(k, 1)
        counts = [0.0] * nw
        share = [args.e2e_steps // nw + (1 if k < args.e2e_steps % nw else 0) for k in range(nw)]
        torch.cuda.synchronize()
        barrier(world)
        t0 = time.perf_counter()
        threads = [threading.Thread(target=e2e_steps, args=(k, share[k])) for k in range(nw)]
        for th in threads:
            th.start()
        for th in threads:
            th.join()
        torch.cuda.synchronize()
        t_e2e = allmax(world, time.perf_counter() - t0)
        line["e2e"] = {"value": allsum(world, sum(counts)) / t_e2e, "unit": UNIT, "h2d_bytes_per_step": h2d,
                       "d2h_bytes_per_step": d2h, "steps": args.e2e_steps, "workers": nw,
                       "ms_per_step": 1e3 * t_e2e / args.e2e_steps,
                       "note": "per step: sph_upload from pinned host arrays (incl. its sort and neighbour "
                               "build), sph_step(1) (dt0 forces pass doubling as the predictor's, "
                               "corrector), sph_download to pinned host arrays and the counters read back; "
                               "the steps shared by `workers` host threads, each with its own context and "
                               "stream"}
        for sim_k, _ in workers[1:]:
            sim_k.close()
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(scene, args.workload)
    if rank == 0:
        print(json.dumps(line), flush=True)
    sim.close()


def run_batch(args):
    """256 sloshing tanks: one context stepped by one captured graph per step,
    against one context per tank stepped scene by scene (per-scene launches)."""
    import torch
    from paper_2207_11328_gb300 import Simulation, _build, scenes
    _build.build()
    b = scenes.sloshing_batch()
    stream = torch.cuda.current_stream()
    sim = Simulation.from_scene(b, stream=stream)
    sim.autotune(stream=stream)
    tuned = sim.variants()
    sim.step(args.warmup, stream=stream)
    torch.cuda.synchronize()
    st0 = sim.stats(stream=stream)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(0) as clk:
        torch.cuda.synchronize()
        clk.mark(True)
        ev0.record(stream)
        sim.step(args.steps, stream=stream)
        ev1.record(stream)
        torch.cuda.synchronize()
        clk.mark(False)
    t_b = ev0.elapsed_time(ev1) / 1e3
    st1 = sim.stats(stream=stream)
    inter_b = 2.0 * (st1["list_entries"] - st0["list_entries"])
    # the same steps as one persistent kernel launch (grid-wide barriers between the phases)
    sim.set_persistent(True)
    sim.step(args.warmup, stream=stream)
    torch.cuda.synchronize()
    sp0 = sim.stats(stream=stream)
    with ClockSampler(0) as clk_p:
        torch.cuda.synchronize()
        clk_p.mark(True)
        ev0.record(stream)
        sim.step(args.steps, stream=stream)
        ev1.record(stream)
        torch.cuda.synchronize()
        clk_p.mark(False)
    t_pk = ev0.elapsed_time(ev1) / 1e3
    inter_pk = 2.0 * (sim.stats(stream=stream)["list_entries"] - sp0["list_entries"])
    sim.set_persistent(False)
    # per-scene contexts, each tank launched on its own
    per = []
    for k, d in enumerate(b.scenes):
        m = b.scene == k
        one = scenes.subset(b, m)
        import dataclasses
        one = dataclasses.replace(one, scenes=None, scene=np.zeros(int(m.sum()), np.uint32), origin=d["origin"],
                                  size=d["size"], periodic=d["periodic"], c0=d["c0"])
        ps = Simulation.from_scene(one, stream=stream)
        ps.step(args.warmup, stream=stream)
        per.append(ps)
    torch.cuda.synchronize()
    e0 = sum(ps.stats(stream=stream)["list_entries"] for ps in per)
    ps_steps = max(1, args.steps // 5)
    with ClockSampler(0) as clk_s:
        torch.cuda.synchronize()
        clk_s.mark(True)
        ev0.record(stream)
        for _ in range(ps_steps):
            for ps in per:
                ps.step(1, stream=stream)
        ev1.record(stream)
        torch.cuda.synchronize()
        clk_s.mark(False)
    t_p = ev0.elapsed_time(ev1) / 1e3
    inter_p = 2.0 * (sum(ps.stats(stream=stream)["list_entries"] for ps in per) - e0)
    line = {"metric": METRIC, "value": inter_b / t_b, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t_b / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"sloshing_batch: {len(b.scenes)} tanks, {b.n} particles "
                                   f"({b.n_fluid} fluid), dp 0.01 m",
                                   "variants": dict(tuned, autotuned=True,
                                                    fused_build_predict=bool(sim.step_options()["fused_predict"]))},
            "particle_steps_per_s": b.n * args.steps / t_b,
            "per_scene_launches": {"value": inter_p / t_p, "ms_per_step": 1e3 * t_p / ps_steps,
                                   "particle_steps_per_s": b.n * ps_steps / t_p, "steps": ps_steps,
                                   "clocks": clk_s.summary()},
            "persistent_kernel": {"value": inter_pk / t_pk, "ms_per_step": 1e3 * t_pk / args.steps,
                                  "particle_steps_per_s": b.n * args.steps / t_pk, "steps": args.steps,
                                  "launches": 1, "clocks": clk_p.summary(),
                                  "note": "every phase of the step in one cooperative kernel with grid-wide "
                                          "barriers, all steps of the timed region in one launch; same bits"},
            "batched_speedup": (inter_b / t_b) / (inter_p / t_p), "gpu_launches": int(st1["kernels_per_step"] * args.steps),
            "clocks": clk.summary()}
    print(json.dumps(line), flush=True)


def run_adjoint(args):
    """Differentiable run: 32^3 periodic box, T = 64 steps, checkpoint every 8:
    forward record, backward, and a plain 64-step forward for comparison."""
    import torch
    from paper_2207_11328_gb300 import Simulation, _build, scenes
    _build.build()
    s = scenes.periodic_box(n_per_axis=32)
    s.dt_fixed = 3.9e-4
    stream = torch.cuda.current_stream()
    sim = Simulation.from_scene(s, stream=stream)
    sim.autotune(stream=stream)
    xbar = torch.randn((s.n, 3), device="cuda", dtype=torch.float32)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    times = []
    with ClockSampler(0) as clk:   # clocks sampled over the measured repetitions
        for rep in range(args.warmup + 3):
            sim.upload(s, stream=stream)
            torch.cuda.synchronize()
            if rep == args.warmup:
                clk.mark(True)
            ev[0].record(stream)
            sim.record(64, 8, stream=stream)
            ev[1].record(stream)
            sim.backward(xbar_T=xbar, stream=stream)
            ev[2].record(stream)
            sim.upload(s, stream=stream)
            sim.step(64, stream=stream)
            ev[3].record(stream)
            torch.cuda.synchronize()
            if rep >= args.warmup:
                times.append([ev[0].elapsed_time(ev[1]), ev[1].elapsed_time(ev[2]), ev[2].elapsed_time(ev[3])])
        clk.mark(False)
    t = np.median(np.array(times), axis=0)
    line = {"metric": "forward+backward time, 32^3 periodic box, T=64, checkpoint every 8", "value": t[0] + t[1],
            "unit": "ms", "higher_is_better": False, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "periodic_box_32768, T=64, K=8, dt frozen 3.9e-4 s"},
            "record_ms": t[0], "backward_ms": t[1], "plain_forward_64_steps_ms_incl_upload": t[2],
            "backward_over_forward": t[1] / t[0], "clocks": clk.summary()}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="dam16m", choices=["dam1m", "dam16m", "box", "box2m", "batch", "adjoint"])
    ap.add_argument("--max-neibs", type=int, default=128)
    ap.add_argument("--profile-steps", type=int, default=20)
    ap.add_argument("--flow-steps", type=int, default=2000,
                    help="steps taken after the timed region before timing --steps again on the flowing state "
                         "(0: skip)")
    ap.add_argument("--variants", default="",
                    help="build,predictor,corrector variant indices (0..4) instead of autotuning")
    ap.add_argument("--e2e-steps", type=int, default=40)
    ap.add_argument("--e2e-workers", type=int, default=2,
                    help="host threads (one context and stream each) sharing the end-to-end steps")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--rebuild-every", type=int, default=1,
                    help="neighbour pipeline every k steps with a skin (paper default: 10)")
    ap.add_argument("--skin", type=float, default=0.0, help="list skin in units of h (with --rebuild-every > 1)")
    ap.add_argument("--kernel", choices=list(KERNELS), default="wendland", help="smoothing kernel (Table 1)")
    ap.add_argument("--formulation", type=int, choices=(1, 2), default=1, help="SPH formulation (Section 2.1)")
    ap.add_argument("--visc", choices=list(VISC), default=None, help="viscous model (default: the workload's)")
    ap.add_argument("--nu", type=float, default=1e-6, help="kinematic viscosity of the laminar models")
    ap.add_argument("--ddiff", type=float, default=0.0,
                    help="Molteni-Colagrossi density-diffusion coefficient (0: off; the paper's runs use it)")
    args = ap.parse_args()
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")
    if args.impl == "reference":
        # the oracle on the host cores: rank 0 only, no GPU work
        rank = int(os.environ.get("RANK", "0"))
        run_reference(args, int(os.environ.get("WORLD_SIZE", "1")), rank)
        return
    world, rank, local = dist_setup(args.gpus)
    if args.workload == "batch":
        run_batch(args)
        return
    if args.workload == "adjoint":
        run_adjoint(args)
        return
    run_ours(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
