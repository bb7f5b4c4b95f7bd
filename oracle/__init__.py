"""FP64 CPU oracle for the WCSPH hot path (ctypes wrapper of sph_oracle.cpp).

TEST INFRASTRUCTURE: only the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import this package.  The CUDA library never
calls it and shares no code with it.

Functions and the passages they follow (arXiv 2207.11328):
  kernel_W / kernel_F   kernel-templates listing (Section 4), Table 1 kernels + unit integral (Section 2.1)
  eos                   Cole equation of state (Section 2.1), binomial form
  neighbors             neighbour sets 0 < r < 2h (Section 2.3), brute force or binning
  rhs / rhs_sample      golden-rule continuity + momentum (Section 2.1, readings C1-C5), with the
                        Table 1 options: formulation 2, Morris / Monaghan / Espanol-Revenga
                        viscosity and averaging operators (Section 3), Molteni-Colagrossi
                        density diffusion (reading D1)
  step                  predictor-corrector + CFL dt (readings C6, C7)
  energy                kinetic + internal + potential energy (invariant check)
  loss_jvp              loss after T steps and its directional derivative (dual numbers)

Parity is pinned by the tests in tests/test_oracle_*.py (normalisation,
brute-force sets, exact lattice cancellation, momentum, energy, hydrostatic
tank, Poiseuille closed form, convergence order, finite differences).
"""
from __future__ import annotations

import contextlib
import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sph_oracle.cpp")
_LIB = os.path.join(_HERE, "libsph_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with g++ (FP64, no fast-math, no FMA contraction so
    x86 and Arm hosts give the same results)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-fPIC", "-shared",
                               "-fno-fast-math", "-ffp-contract=off", _SRC, "-o", tmp])
        os.replace(tmp, _LIB)
    return _LIB


class Params(ctypes.Structure):
    _fields_ = [("dp", ctypes.c_double), ("h", ctypes.c_double), ("kernel_radius", ctypes.c_double),
                ("rho0", ctypes.c_double), ("c0", ctypes.c_double), ("gamma", ctypes.c_double),
                ("visc_model", ctypes.c_int32), ("pad0", ctypes.c_int32),
                ("alpha", ctypes.c_double), ("nu", ctypes.c_double),
                ("g", ctypes.c_double * 3), ("cfl", ctypes.c_double), ("dt_fixed", ctypes.c_double),
                ("origin", ctypes.c_double * 3), ("size", ctypes.c_double * 3),
                ("periodic_mask", ctypes.c_uint32), ("pad1", ctypes.c_uint32),
                ("kernel_type", ctypes.c_int32), ("formulation", ctypes.c_int32),
                ("visc_avg", ctypes.c_int32), ("ddiff", ctypes.c_int32),
                ("ddiff_coef", ctypes.c_double), ("zeta", ctypes.c_double)]


def _configure(lib):
    P = ctypes.POINTER(Params)
    dp_ = ctypes.POINTER(ctypes.c_double)
    i64p = ctypes.POINTER(ctypes.c_int64)
    i32p = ctypes.POINTER(ctypes.c_int32)
    u8p = ctypes.POINTER(ctypes.c_uint8)
    lib.ora_kernel_W.restype = ctypes.c_double
    lib.ora_kernel_W.argtypes = [ctypes.c_double, ctypes.c_double]
    lib.ora_kernel_F.restype = ctypes.c_double
    lib.ora_kernel_F.argtypes = [ctypes.c_double, ctypes.c_double]
    for f in (lib.ora_kernel_Wk, lib.ora_kernel_Fk):
        f.restype = ctypes.c_double
        f.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double]
    lib.ora_eos.restype = ctypes.c_double
    lib.ora_eos.argtypes = [P, ctypes.c_double]
    lib.ora_neighbors.restype = ctypes.c_int64
    lib.ora_neighbors.argtypes = [P, ctypes.c_int, dp_, ctypes.c_int, ctypes.c_int64, i64p, i32p]
    lib.ora_neighbors_sample.restype = ctypes.c_int64
    lib.ora_neighbors_sample.argtypes = [P, ctypes.c_int, dp_, ctypes.c_int, i32p, ctypes.c_int64, i64p, i32p]
    lib.ora_rhs.restype = ctypes.c_int
    lib.ora_rhs.argtypes = [P, ctypes.c_int, dp_, dp_, dp_, dp_, u8p, dp_, dp_, dp_]
    lib.ora_rhs_sample.restype = ctypes.c_int
    lib.ora_rhs_sample.argtypes = [P, ctypes.c_int, dp_, dp_, dp_, dp_, u8p, ctypes.c_int,
                                   i32p, dp_, dp_, i32p, dp_]
    lib.ora_cfl_dt.restype = ctypes.c_double
    lib.ora_cfl_dt.argtypes = [P, ctypes.c_int, dp_, u8p]
    lib.ora_step.restype = ctypes.c_int
    lib.ora_step.argtypes = [P, ctypes.c_int, dp_, dp_, dp_, dp_, u8p, ctypes.c_int, dp_, dp_]
    lib.ora_energy.restype = ctypes.c_double
    lib.ora_energy.argtypes = [P, ctypes.c_int, dp_, dp_, dp_, dp_, u8p]
    lib.ora_loss_jvp.restype = ctypes.c_int
    lib.ora_loss_jvp.argtypes = [P, ctypes.c_int, dp_, dp_, dp_, dp_, u8p, ctypes.c_int,
                                 ctypes.c_double, dp_, dp_, ctypes.c_double, dp_, dp_]
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = _configure(ctypes.CDLL(build()))
    return _lib


@contextlib.contextmanager
def using(lib_path):
    """Run the wrapper against another build of the oracle (used by the tests
    that plant mistakes in copies of the oracle to show the pins catch them)."""
    global _lib
    with _lock:
        saved = _lib
        _lib = _configure(ctypes.CDLL(lib_path))
    try:
        yield
    finally:
        with _lock:
            _lib = saved


def _d(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _u8(a):
    a = np.ascontiguousarray(a, dtype=np.uint8)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))


def params(scene=None, **kw) -> Params:
    """Oracle parameters from a Scene (any field overridable by keyword)."""
    src = {}
    if scene is not None:
        src = dict(dp=scene.dp, h=scene.h, kernel_radius=scene.kernel_radius, rho0=scene.rho0,
                   c0=scene.c0, gamma=float(scene.gamma), visc_model=scene.visc, alpha=scene.alpha,
                   nu=scene.nu, g=scene.g, cfl=scene.cfl, dt_fixed=scene.dt_fixed,
                   origin=scene.origin, size=scene.size, periodic_mask=scene.periodic,
                   kernel_type=scene.kernel_type, formulation=scene.formulation, visc_avg=scene.visc_avg,
                   ddiff=scene.ddiff, ddiff_coef=scene.ddiff_coef, zeta=scene.zeta)
    src.update(kw)
    p = Params()
    for k, v in src.items():
        if k in ("g", "origin", "size"):
            getattr(p, k)[:] = [float(t) for t in v]
        else:
            setattr(p, k, v)
    if p.kernel_radius == 0.0:
        p.kernel_radius = 2.0
    return p


def kernel_W(r, h, kernel=0, radius=2.0):
    """W(r) of a Table-1 kernel (0 Wendland C2, 1 cubic spline, 2 quadratic, 3 Gaussian cut at radius*h)."""
    if kernel == 0:
        return _load().ora_kernel_W(float(r), float(h))
    return _load().ora_kernel_Wk(int(kernel), float(radius), float(r), float(h))


def kernel_F(r, h, kernel=0, radius=2.0):
    """F(r) = (1/r) dW/dr of the same kernels."""
    if kernel == 0:
        return _load().ora_kernel_F(float(r), float(h))
    return _load().ora_kernel_Fk(int(kernel), float(radius), float(r), float(h))


def eos(p: Params, delta):
    return _load().ora_eos(ctypes.byref(p), float(delta))


def neighbors(p: Params, pos, brute=False):
    """CSR neighbour sets (offsets int64[n+1], indices int32[...]), ascending per particle."""
    lib = _load()
    pos, pp = _d(pos)
    n = pos.shape[0]
    off = np.zeros(n + 1, np.int64)
    cap = max(1, n * 64)
    while True:
        idx = np.zeros(cap, np.int32)
        tot = lib.ora_neighbors(ctypes.byref(p), n, pp, int(brute), cap,
                                off.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                idx.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
        if tot >= 0:
            return off, idx[:tot].copy()
        cap = -tot


def neighbors_sample(p: Params, pos, sample):
    """CSR neighbour sets of the particles in `sample` only (searched among all):
    offsets int64[len(sample)+1], indices int32[...], ascending per particle."""
    lib = _load()
    pos, pp = _d(pos)
    n = pos.shape[0]
    smp = np.ascontiguousarray(sample, np.int32)
    off = np.zeros(len(smp) + 1, np.int64)
    cap = max(1, len(smp) * 128)
    while True:
        idx = np.zeros(cap, np.int32)
        tot = lib.ora_neighbors_sample(ctypes.byref(p), n, pp, len(smp),
                                       smp.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), cap,
                                       off.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                       idx.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
        if tot >= 0:
            return off, idx[:tot].copy()
        cap = -tot


def rhs(p: Params, pos, vel, delta, mass, ptype, with_mag=False):
    """(a[n,3], drho[n]) at the given state (FP64); with_mag adds mag[n,2],
    the summed magnitudes of the momentum and continuity pair terms."""
    lib = _load()
    pos, pp = _d(pos); vel, vp = _d(vel); delta, dp_ = _d(delta); mass, mp = _d(mass)
    ptype, tp = _u8(ptype)
    n = pos.shape[0]
    a = np.zeros((n, 3)); drho = np.zeros(n)
    mag = np.zeros((n, 2)) if with_mag else None
    rc = lib.ora_rhs(ctypes.byref(p), n, pp, vp, dp_, mp, tp,
                     a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                     drho.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                     None if mag is None else mag.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    if rc != 0:
        raise RuntimeError("ora_rhs failed")
    return (a, drho, mag) if with_mag else (a, drho)


def rhs_sample(p: Params, pos, vel, delta, mass, ptype, sample):
    """(a[s,3], drho[s], n_neighbours[s], mag[s,2]) for particles `sample` only."""
    lib = _load()
    pos, pp = _d(pos); vel, vp = _d(vel); delta, dp_ = _d(delta); mass, mp = _d(mass)
    ptype, tp = _u8(ptype)
    sample = np.ascontiguousarray(sample, np.int32)
    ns = sample.shape[0]
    a = np.zeros((ns, 3)); drho = np.zeros(ns); nnb = np.zeros(ns, np.int32); mag = np.zeros((ns, 2))
    rc = lib.ora_rhs_sample(ctypes.byref(p), pos.shape[0], pp, vp, dp_, mp, tp, ns,
                            sample.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                            a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                            drho.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                            nnb.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                            mag.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    if rc != 0:
        raise RuntimeError("ora_rhs_sample failed")
    return a, drho, nnb, mag


def cfl_dt(p: Params, a, ptype):
    a, ap = _d(a); ptype, tp = _u8(ptype)
    return _load().ora_cfl_dt(ctypes.byref(p), a.shape[0], ap, tp)


def step(p: Params, pos, vel, delta, mass, ptype, nsteps=1, dt=0.0):
    """Run nsteps predictor-corrector steps on copies of the state.
    Returns (pos, vel, delta, dt_next, dts)."""
    lib = _load()
    pos = np.array(pos, np.float64, copy=True); vel = np.array(vel, np.float64, copy=True)
    delta = np.array(delta, np.float64, copy=True)
    mass, mp = _d(mass); ptype, tp = _u8(ptype)
    dt_io = ctypes.c_double(dt)
    dts = np.zeros(max(nsteps, 1))
    rc = lib.ora_step(ctypes.byref(p), pos.shape[0], pos.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                      vel.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                      delta.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), mp, tp, int(nsteps),
                      ctypes.byref(dt_io), dts.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    if rc != 0:
        raise RuntimeError("ora_step failed")
    return pos, vel, delta, dt_io.value, dts[:nsteps]


def energy(p: Params, pos, vel, delta, mass, ptype):
    pos, pp = _d(pos); vel, vp = _d(vel); delta, dp_ = _d(delta); mass, mp = _d(mass)
    ptype, tp = _u8(ptype)
    return _load().ora_energy(ctypes.byref(p), pos.shape[0], pp, vp, dp_, mp, tp)


def loss_jvp(p: Params, pos0, vel0, delta0, mass, ptype, T, dt, target, du0=None, dalpha=0.0):
    """(L, dL) with dL the derivative of L along (du0, dalpha)."""
    lib = _load()
    pos0, pp = _d(pos0); vel0, vp = _d(vel0); delta0, dp_ = _d(delta0); mass, mp = _d(mass)
    ptype, tp = _u8(ptype); target, tg = _d(target)
    if du0 is None:
        dup = None
    else:
        du0, dup = _d(du0)
    L = ctypes.c_double(); dL = ctypes.c_double()
    rc = lib.ora_loss_jvp(ctypes.byref(p), pos0.shape[0], pp, vp, dp_, mp, tp, int(T), float(dt),
                          tg, dup, float(dalpha), ctypes.byref(L), ctypes.byref(dL))
    if rc != 0:
        raise RuntimeError("ora_loss_jvp failed")
    return L.value, dL.value
