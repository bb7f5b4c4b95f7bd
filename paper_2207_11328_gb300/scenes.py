"""Seeded synthetic scene generators (initial particle sets).

This module only lays particles out and draws seeded random numbers: it holds
none of the SPH method's arithmetic (no kernel, no equation of state, no
neighbour search, no integration).  Both the CUDA path and the FP64 oracle
consume the arrays it returns; neither imports the other.

Every generator returns a :class:`Scene`: particle arrays in upload order plus
the physical parameters of the run.  Positions are FP64 (the library converts
them to cell-relative FP32 on the device); velocities and the relative density
``delta = rho/rho0 - 1`` are FP32, which is the precision the state is kept in.

Scenes follow the test cases of the paper (Section 2 for the method, the 3D
dam break of the compiler analysis): a periodic lattice box, the dam break
tank with dynamic boundary walls, a plane Poiseuille channel and a batch of
sloshing tanks.  Sizes are stated in each generator.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

FLUID = 0
BOUNDARY = 1
VISC_ARTIFICIAL = 0
VISC_LAMINAR = 1

SEED_BASE = 2207_11328


@dataclasses.dataclass
class Scene:
    name: str
    pos: np.ndarray        # (n,3) float64
    vel: np.ndarray        # (n,3) float32
    delta: np.ndarray      # (n,)  float32, rho/rho0 - 1
    mass: np.ndarray       # (n,)  float32
    ptype: np.ndarray      # (n,)  uint8, 0 fluid / 1 boundary
    scene: np.ndarray      # (n,)  uint32 scene index (0 for single scenes)
    dp: float
    h: float
    rho0: float
    c0: float
    gamma: int
    visc: int
    alpha: float
    nu: float
    g: tuple
    cfl: float
    origin: tuple
    size: tuple
    periodic: int          # bit0 x, bit1 y, bit2 z
    dt_fixed: float = 0.0
    kernel_radius: float = 2.0
    # model options (Table 1): kernel 0 Wendland C2 / 1 cubic spline / 2 quadratic /
    # 3 Gaussian; formulation 0 or 1 (the paper's second form); laminar averaging
    # 0 harmonic / 1 arithmetic / 2 geometric; density diffusion 0 none / 1 Molteni-Colagrossi
    kernel_type: int = 0
    formulation: int = 0
    visc_avg: int = 0
    ddiff: int = 0
    ddiff_coef: float = 0.0
    zeta: float = 0.0
    # batched scenes: per-scene geometry and sound speed (None for a single scene)
    scenes: list | None = None

    @property
    def n(self) -> int:
        return int(self.pos.shape[0])

    @property
    def n_fluid(self) -> int:
        return int(np.count_nonzero(self.ptype == FLUID))


def _lattice(nx, ny, nz, dp, x0=0.0, y0=0.0, z0=0.0):
    i, j, k = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    p = np.stack([x0 + (i.ravel() + 0.5) * dp,
                  y0 + (j.ravel() + 0.5) * dp,
                  z0 + (k.ravel() + 0.5) * dp], axis=1)
    return p.astype(np.float64)


def periodic_box(n_per_axis=16, dp=0.02, vel_amp=0.05, alpha=0.02, c0=20.0,
                 seed=SEED_BASE + 0, jitter=0.0, name="periodic_box"):
    """Cubic lattice of n^3 fluid particles in a fully periodic cube of side n*dp.

    16^3 = 4096 particles at dp = 0.02 m is the small periodic box; 32^3 is the
    differentiable run's box.  Velocities are uniform in [-vel_amp, vel_amp]
    per component; delta = 0; no gravity.  ``jitter`` displaces positions by
    a seeded uniform amount (fraction of dp) for neighbour-set tests.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    L = n_per_axis * dp
    pos = _lattice(n_per_axis, n_per_axis, n_per_axis, dp)
    vel = rng.uniform(-vel_amp, vel_amp, size=pos.shape)
    if jitter:
        pos = pos + rng.uniform(-jitter * dp, jitter * dp, size=pos.shape)
        pos = np.mod(pos, L)
    n = pos.shape[0]
    rho0 = 1000.0
    return Scene(name=name, pos=pos, vel=vel.astype(np.float32),
                 delta=np.zeros(n, np.float32),
                 mass=np.full(n, rho0 * dp ** 3, np.float32),
                 ptype=np.zeros(n, np.uint8), scene=np.zeros(n, np.uint32),
                 dp=dp, h=1.3 * dp, rho0=rho0, c0=c0, gamma=7,
                 visc=VISC_ARTIFICIAL, alpha=alpha, nu=0.0, g=(0.0, 0.0, 0.0),
                 cfl=0.3, origin=(0.0, 0.0, 0.0), size=(L, L, L), periodic=7)


def _hydrostatic_delta(z, H, rho0, c0, gamma, g):
    """Initial relative density of a fluid column at rest (inverted Tait relation).

    This is an initial condition of the dam-break scene (rho at depth H - z
    such that P(rho) = rho0*g*(H - z)), clamped at zero above the surface.
    """
    B = rho0 * c0 * c0 / gamma
    depth = np.maximum(H - z, 0.0)
    return (1.0 + rho0 * g * depth / B) ** (1.0 / gamma) - 1.0


def _walls(lo, hi, dp, layers, floor=True, sides=(True, True, True, True), top_z=None):
    """Boundary particles: `layers` lattice layers at dp spacing outside the
    box [lo, hi] (x, y from the sides, z from the floor), up to height top_z."""
    lo = np.asarray(lo, float); hi = np.asarray(hi, float)
    top_z = hi[2] if top_z is None else top_z
    nxi = int(round((hi[0] - lo[0]) / dp)); nyi = int(round((hi[1] - lo[1]) / dp))
    nzi = int(round((top_z - lo[2]) / dp))
    pts = []
    # x index range including wall layers
    xs = np.arange(-layers, nxi + layers); ys = np.arange(-layers, nyi + layers)
    if floor:
        i, j, k = np.meshgrid(xs, ys, np.arange(-layers, 0), indexing="ij")
        pts.append(np.stack([i.ravel(), j.ravel(), k.ravel()], 1))
    zs = np.arange(0, nzi)
    if sides[0]:  # x = lo wall
        i, j, k = np.meshgrid(np.arange(-layers, 0), ys, zs, indexing="ij")
        pts.append(np.stack([i.ravel(), j.ravel(), k.ravel()], 1))
    if sides[1]:  # x = hi wall
        i, j, k = np.meshgrid(np.arange(nxi, nxi + layers), ys, zs, indexing="ij")
        pts.append(np.stack([i.ravel(), j.ravel(), k.ravel()], 1))
    xin = np.arange(0, nxi)
    if sides[2]:  # y = lo wall
        i, j, k = np.meshgrid(xin, np.arange(-layers, 0), zs, indexing="ij")
        pts.append(np.stack([i.ravel(), j.ravel(), k.ravel()], 1))
    if sides[3]:  # y = hi wall
        i, j, k = np.meshgrid(xin, np.arange(nyi, nyi + layers), zs, indexing="ij")
        pts.append(np.stack([i.ravel(), j.ravel(), k.ravel()], 1))
    ijk = np.concatenate(pts, 0).astype(np.float64)
    return lo[None, :] + (ijk + 0.5) * dp


def dam_break(dp=4.3e-3, tank=(1.6, 0.67, 0.6), column=(0.4, 0.67, 0.3), layers=3,
              alpha=0.01, g=9.81, name="dam_break", max_fluid=None):
    """3D dam break: tank 1.6 x 0.67 x 0.6 m, water column 0.4 x 0.67 x 0.3 m at
    x in [0, 0.4] at rest with hydrostatic initial density, `layers` layers of
    dynamic boundary particles on the floor and the four side walls.

    dp = 4.3e-3 m gives ~1.0M fluid + ~0.63M boundary particles; dp divided
    by 16^(1/3) gives ~16M fluid.  c0 = 10*sqrt(g*H_column).
    """
    H = column[2]
    c0 = 10.0 * math.sqrt(g * H)
    rho0 = 1000.0
    gamma = 7
    nx = int(round(column[0] / dp)); ny = int(round(tank[1] / dp)); nz = int(round(H / dp))
    fluid = _lattice(nx, ny, nz, dp)
    # tank interior in whole dp cells so the walls sit on the lattice
    tx = int(round(tank[0] / dp)); tz = int(round(tank[2] / dp))
    hi = (tx * dp, ny * dp, tz * dp)
    walls = _walls((0.0, 0.0, 0.0), hi, dp, layers)
    Hs = nz * dp  # free surface of the lattice column
    df = _hydrostatic_delta(fluid[:, 2], Hs, rho0, c0, gamma, g)
    db = _hydrostatic_delta(walls[:, 2], Hs, rho0, c0, gamma, g)
    pos = np.concatenate([fluid, walls], 0)
    nf, nb = fluid.shape[0], walls.shape[0]
    ptype = np.concatenate([np.zeros(nf, np.uint8), np.ones(nb, np.uint8)])
    delta = np.concatenate([df, db]).astype(np.float32)
    n = nf + nb
    margin = 2.6 * dp
    origin = (-layers * dp - margin, -layers * dp - margin, -layers * dp - margin)
    size = (hi[0] + 2 * (layers * dp + margin), hi[1] + 2 * (layers * dp + margin),
            hi[2] + layers * dp + 2 * margin)
    return Scene(name=name, pos=pos, vel=np.zeros((n, 3), np.float32), delta=delta,
                 mass=np.full(n, rho0 * dp ** 3, np.float32), ptype=ptype,
                 scene=np.zeros(n, np.uint32), dp=dp, h=1.3 * dp, rho0=rho0, c0=c0,
                 gamma=gamma, visc=VISC_ARTIFICIAL, alpha=alpha, nu=0.0,
                 g=(0.0, 0.0, -g), cfl=0.3, origin=origin, size=size, periodic=0)


def hydrostatic_tank(dp=0.02, width=0.2, depth=0.1, height=0.4, fill=0.3, layers=3,
                     alpha=0.02, g=9.81, name="hydrostatic_tank"):
    """Small closed tank filled to `fill` m, at rest with hydrostatic density:
    the resting-tank check of the pressure profile rho0*g*depth."""
    s = dam_break(dp=dp, tank=(width, depth, height), column=(width, depth, fill),
                  layers=layers, alpha=alpha, g=g, name=name)
    return s


def poiseuille(dp=1.0 / 64, nx=128, ny=64, nz=8, layers=3, nu=0.1, force=0.01, c0=1.0,
               name="poiseuille"):
    """Plane Poiseuille channel: fluid between plates at y = -a and y = +a
    (a = ny*dp/2 = 0.5 m), periodic in x and z, `layers` layers of boundary
    particles beyond each plate, laminar viscosity nu, body force `force`
    along x.  128 x 64 x 8 = 65,536 fluid particles at dp = 1/64."""
    a = ny * dp / 2
    fluid = _lattice(nx, ny, nz, dp, 0.0, -a, 0.0)
    lo = _lattice(nx, layers, nz, dp, 0.0, -a - layers * dp, 0.0)
    hi = _lattice(nx, layers, nz, dp, 0.0, a, 0.0)
    pos = np.concatenate([fluid, lo, hi], 0)
    nf = fluid.shape[0]; nb = lo.shape[0] + hi.shape[0]
    n = nf + nb
    rho0 = 1000.0
    ptype = np.concatenate([np.zeros(nf, np.uint8), np.ones(nb, np.uint8)])
    Ly = 2 * a + 2 * layers * dp
    margin = 2.6 * dp
    return Scene(name=name, pos=pos, vel=np.zeros((n, 3), np.float32),
                 delta=np.zeros(n, np.float32), mass=np.full(n, rho0 * dp ** 3, np.float32),
                 ptype=ptype, scene=np.zeros(n, np.uint32), dp=dp, h=1.3 * dp,
                 rho0=rho0, c0=c0, gamma=7, visc=VISC_LAMINAR, alpha=0.0, nu=nu,
                 g=(force, 0.0, 0.0), cfl=0.3, origin=(0.0, -Ly / 2 - margin, 0.0),
                 size=(nx * dp, Ly + 2 * margin, nz * dp), periodic=0b101)


def sloshing_batch(n_scenes=256, dp=0.01, nmin=2000, nmax=64000, layers=3, alpha=0.01,
                   g=9.81, tilt_deg=5.0, seed=SEED_BASE + 4, name="sloshing_batch"):
    """Batch of independent 3D sloshing tanks concatenated in one particle set.

    Per tank (seeded): fluid count N ~ logU[nmin, nmax]; aspect L/W ~ U[1,3];
    fill f ~ U[0.3, 0.6] of the tank height H = W; W from N*dp^3 = L*W*f*H;
    free surface tilted `tilt_deg` about y; `layers` wall layers on the floor
    and the four sides; c0 = 10*sqrt(g*f*H).  Each tank is its own scene with
    its own grid; scenes never interact.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    rho0 = 1000.0
    gamma = 7
    pos_l, type_l, delta_l, scene_l = [], [], [], []
    scenes = []
    cursor_x = 0.0
    tan_t = math.tan(math.radians(tilt_deg))
    for s in range(n_scenes):
        N = math.exp(rng.uniform(math.log(nmin), math.log(nmax)))
        aspect = rng.uniform(1.0, 3.0)
        fill = rng.uniform(0.3, 0.6)
        W = (N * dp ** 3 / (aspect * fill)) ** (1.0 / 3.0)
        L = aspect * W
        H = W
        nx = max(3, int(round(L / dp))); ny = max(3, int(round(W / dp)))
        nzt = max(3, int(round(H / dp)))
        Lx, Wy, Hz = nx * dp, ny * dp, nzt * dp
        hf = fill * Hz
        # fluid lattice below a free surface tilted about y through the tank centre
        full = _lattice(nx, ny, nzt, dp)
        surf = hf + (full[:, 0] - 0.5 * Lx) * tan_t
        fluid = full[full[:, 2] < surf]
        walls = _walls((0.0, 0.0, 0.0), (Lx, Wy, Hz), dp, layers)
        c0 = 10.0 * math.sqrt(g * hf)
        B = rho0 * c0 * c0 / gamma
        zs_f = hf + (fluid[:, 0] - 0.5 * Lx) * tan_t
        zs_b = hf + (walls[:, 0] - 0.5 * Lx) * tan_t
        df = (1.0 + rho0 * g * np.maximum(zs_f - fluid[:, 2], 0.0) / B) ** (1.0 / gamma) - 1.0
        db = (1.0 + rho0 * g * np.maximum(zs_b - walls[:, 2], 0.0) / B) ** (1.0 / gamma) - 1.0
        margin = 2.6 * dp
        off = np.array([cursor_x + layers * dp + margin, 0.0, 0.0])
        p = np.concatenate([fluid, walls], 0) + off[None, :]
        origin = (cursor_x, -layers * dp - margin, -layers * dp - margin)
        size = (Lx + 2 * (layers * dp + margin), Wy + 2 * (layers * dp + margin),
                Hz + layers * dp + 2 * margin)
        cursor_x += size[0] + 1.0
        pos_l.append(p)
        type_l.append(np.concatenate([np.zeros(len(fluid), np.uint8), np.ones(len(walls), np.uint8)]))
        delta_l.append(np.concatenate([df, db]))
        scene_l.append(np.full(len(p), s, np.uint32))
        scenes.append(dict(origin=origin, size=size, periodic=0, c0=c0,
                           n_fluid=len(fluid), n=len(p)))
    pos = np.concatenate(pos_l, 0)
    n = pos.shape[0]
    return Scene(name=name, pos=pos, vel=np.zeros((n, 3), np.float32),
                 delta=np.concatenate(delta_l).astype(np.float32),
                 mass=np.full(n, rho0 * dp ** 3, np.float32),
                 ptype=np.concatenate(type_l), scene=np.concatenate(scene_l),
                 dp=dp, h=1.3 * dp, rho0=rho0, c0=scenes[0]["c0"], gamma=gamma,
                 visc=VISC_ARTIFICIAL, alpha=alpha, nu=0.0, g=(0.0, 0.0, -g), cfl=0.3,
                 origin=scenes[0]["origin"], size=scenes[0]["size"], periodic=0,
                 scenes=scenes)


def subset(scene: Scene, mask: np.ndarray, name=None) -> Scene:
    """A scene restricted to the particles where `mask` is true (same physics)."""
    return dataclasses.replace(scene, name=name or scene.name + "_subset",
                               pos=scene.pos[mask].copy(), vel=scene.vel[mask].copy(),
                               delta=scene.delta[mask].copy(), mass=scene.mass[mask].copy(),
                               ptype=scene.ptype[mask].copy(), scene=scene.scene[mask].copy())


def seeded_directions(n, count, seed=SEED_BASE + 3):
    """`count` seeded unit directions in R^n (float64), for directional-derivative checks."""
    rng = np.random.Generator(np.random.PCG64(seed))
    v = rng.standard_normal((count, n))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def seeded_normal(shape, scale, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.normal(0.0, scale, size=shape)


def seeded_uniform(shape, lo, hi, seed):
    """Seeded U[lo, hi) samples (float64), e.g. to jitter positions of a lattice."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.uniform(lo, hi, size=shape)
