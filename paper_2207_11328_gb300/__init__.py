"""GB300-native weakly-compressible SPH hot path (arXiv 2207.11328).

Thin Python binding of the C ABI declared in include/sph.h: argument
marshalling only.  Every step of the path runs in the CUDA library
(libsph_gb300.so, built for sm_103a by ``paper_2207_11328_gb300._build``);
there is no CPU fallback: importing the binding without the library raises.

    from paper_2207_11328_gb300 import Simulation, scenes
    sim = Simulation.from_scene(scenes.periodic_box())
    sim.step(100)
    pos, vel, delta = sim.download()
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import scenes  # noqa: F401  (seeded generators; no method arithmetic)

_HERE = os.path.dirname(os.path.abspath(__file__))
# SPH_GB300_CHECKED=1 loads the checked build (bounds checks and buffer canaries that
# report SPH_ERR_BOUNDS instead of faulting); set it before the first call.
LIB_PATH = os.path.join(_HERE, "libsph_gb300_checked.so" if os.environ.get("SPH_GB300_CHECKED") == "1"
                        else "libsph_gb300.so")

SPH_OK = 0
_ERRNAMES = {-1: "SPH_ERR_ARG", -2: "SPH_ERR_CUDA", -3: "SPH_ERR_CAPACITY", -4: "SPH_ERR_NEIB_OVERFLOW",
             -5: "SPH_ERR_OUT_OF_DOMAIN", -6: "SPH_ERR_NONFINITE", -7: "SPH_ERR_TIMEOUT", -8: "SPH_ERR_STATE",
             -9: "SPH_ERR_SKIN", -10: "SPH_ERR_BOUNDS"}


class SphError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        super().__init__(f"{where}: {_ERRNAMES.get(code, code)} ({_lib().sph_strerror(code).decode()})")


class Params(ctypes.Structure):
    _fields_ = [("dp", ctypes.c_double), ("h", ctypes.c_double), ("kernel_radius", ctypes.c_double),
                ("rho0", ctypes.c_double), ("c0", ctypes.c_double), ("gamma", ctypes.c_double),
                ("visc_model", ctypes.c_int32), ("pad0", ctypes.c_int32),
                ("alpha", ctypes.c_double), ("nu", ctypes.c_double), ("g", ctypes.c_double * 3),
                ("cfl", ctypes.c_double), ("dt_fixed", ctypes.c_double),
                ("origin", ctypes.c_double * 3), ("size", ctypes.c_double * 3),
                ("periodic_mask", ctypes.c_uint32), ("max_particles", ctypes.c_uint32),
                ("max_neibs", ctypes.c_uint32), ("n_scenes", ctypes.c_uint32),
                ("rebuild_every", ctypes.c_uint32), ("pad1", ctypes.c_uint32), ("skin", ctypes.c_double),
                ("kernel_type", ctypes.c_int32), ("formulation", ctypes.c_int32),
                ("visc_avg", ctypes.c_int32), ("ddiff", ctypes.c_int32),
                ("ddiff_coef", ctypes.c_double), ("zeta", ctypes.c_double)]


class SceneDesc(ctypes.Structure):
    _fields_ = [("origin", ctypes.c_double * 3), ("size", ctypes.c_double * 3),
                ("periodic_mask", ctypes.c_uint32), ("pad0", ctypes.c_uint32), ("c0", ctypes.c_double)]


class Stats(ctypes.Structure):
    _fields_ = [("n_active", ctypes.c_uint32), ("n_removed", ctypes.c_uint32),
                ("max_neibs_seen", ctypes.c_uint32), ("error_bits", ctypes.c_uint32),
                ("steps", ctypes.c_uint64), ("dt", ctypes.c_double), ("time", ctypes.c_double),
                ("n_cells", ctypes.c_uint32), ("kernels_per_step", ctypes.c_uint32),
                ("list_entries", ctypes.c_uint64), ("interactions", ctypes.c_uint64),
                ("builds", ctypes.c_uint32), ("pad0", ctypes.c_uint32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if not k.startswith("pad")}


_LIB = None

# exported entry points and their signatures (argument marshalling only)
_vp = ctypes.c_void_p
_SIGS = {
    "sph_create": [ctypes.POINTER(Params), ctypes.POINTER(_vp)],
    "sph_set_scenes": [_vp, ctypes.c_uint32, ctypes.POINTER(SceneDesc)],
    "sph_upload": [_vp, ctypes.c_uint32, _vp, _vp, _vp, _vp, _vp, _vp, _vp],
    "sph_upload_device": [_vp, ctypes.c_uint32, _vp, _vp, _vp, _vp, _vp, _vp, _vp],
    "sph_build_neighbors": [_vp, _vp],
    "sph_forces": [_vp, _vp],
    "sph_step": [_vp, ctypes.c_uint32, _vp],
    "sph_set_persistent": [_vp, ctypes.c_int],
    "sph_set_fused_predict": [_vp, ctypes.c_int],
    "sph_get_step_options": [_vp, _vp, _vp],
    "sph_set_owned": [_vp, ctypes.c_uint32],
    "sph_set_dt": [_vp, ctypes.c_double],
    "sph_cfl_dt": [_vp, _vp, _vp],
    "sph_next_dt": [_vp, _vp, _vp],
    "sph_step_profiled": [_vp, ctypes.c_uint32, _vp, _vp],
    "sph_download": [_vp, ctypes.c_uint32, _vp, _vp, _vp, _vp],
    "sph_download_device": [_vp, ctypes.c_uint32, _vp, _vp, _vp, _vp],
    "sph_download_forces": [_vp, ctypes.c_uint32, _vp, _vp, _vp],
    "sph_download_neighbors": [_vp, ctypes.c_uint32, _vp, _vp, _vp],
    "sph_download_neighbors_noalloc": [_vp, ctypes.c_uint32, _vp, _vp, _vp],
    "sph_download_neighbors_of": [_vp, ctypes.c_uint32, _vp, _vp, _vp, _vp],
    "sph_get_stats": [_vp, ctypes.POINTER(Stats), _vp],
    "sph_get_scene_times": [_vp, _vp, _vp, _vp],
    "sph_clear_error": [_vp, _vp],
    "sph_sync": [_vp, _vp],
    "sph_autotune": [_vp, _vp, _vp, _vp],
    "sph_set_alpha": [_vp, ctypes.c_double],
    "sph_record": [_vp, ctypes.c_uint32, ctypes.c_uint32, _vp, _vp],
    "sph_backward": [_vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp],
    "sph_tape_generation": [_vp, _vp],
    "sph_set_variants": [_vp, ctypes.c_int, ctypes.c_int],
    "sph_build_variant_name": [ctypes.c_int],
    "sph_forces_variant_name": [ctypes.c_int],
    "sph_set_forces_variants": [_vp, ctypes.c_int, ctypes.c_int],
    "sph_get_variants": [_vp, _vp, _vp, _vp],
    "sph_fp32_peak": [_vp, _vp],
    "sph_conservation": [_vp, _vp, _vp],
    "sph_strerror": [ctypes.c_int],
    "sph_destroy": [_vp],
}


def exported_symbols():
    return list(_SIGS)


def _lib():
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"CUDA library not built: {LIB_PATH} is missing "
                              "(run python -m paper_2207_11328_gb300._build)")
        lib = ctypes.CDLL(LIB_PATH)
        for name, args in _SIGS.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = ctypes.c_int
        lib.sph_strerror.restype = ctypes.c_char_p
        lib.sph_build_variant_name.restype = ctypes.c_char_p
        lib.sph_forces_variant_name.restype = ctypes.c_char_p
        lib.sph_destroy.restype = None
        _LIB = lib
    return _LIB


def fp32_peak(stream=None):
    """Measured FP32 CUDA-core throughput of the current device, TFLOP/s."""
    t = ctypes.c_double()
    _check(_lib().sph_fp32_peak(_stream_handle(stream), ctypes.byref(t)), "sph_fp32_peak")
    return t.value


N_BUILD_VARIANTS = 5   # sph_set_variants / sph_autotune indices 0..4
N_FORCES_VARIANTS = 5


def build_variant_names():
    """Names of the neighbour-build variants, by index."""
    return [_lib().sph_build_variant_name(v).decode() for v in range(N_BUILD_VARIANTS)]


def forces_variant_names():
    """Names of the force-kernel launch shapes, by index."""
    return [_lib().sph_forces_variant_name(v).decode() for v in range(N_FORCES_VARIANTS)]


def _check(rc, where):
    if rc != SPH_OK:
        raise SphError(rc, where)


def _ptr(a):
    return None if a is None else ctypes.c_void_p(a.ctypes.data)


def _stream_handle(stream):
    """cudaStream_t of a torch stream (or None for the legacy default stream)."""
    if stream is None:
        return None
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def params_from_scene(scene, max_particles=None, max_neibs=128, rebuild_every=1, skin=0.0):
    p = Params()
    p.dp, p.h, p.kernel_radius = scene.dp, scene.h, scene.kernel_radius
    p.rho0, p.c0, p.gamma = scene.rho0, scene.c0, float(scene.gamma)
    p.visc_model, p.alpha, p.nu = scene.visc, scene.alpha, scene.nu
    p.g[:] = list(scene.g)
    p.cfl, p.dt_fixed = scene.cfl, scene.dt_fixed
    p.origin[:] = list(scene.origin)
    p.size[:] = list(scene.size)
    p.periodic_mask = scene.periodic
    p.max_particles = int(max_particles or max(scene.n, 1))
    p.max_neibs = int(max_neibs)
    p.n_scenes = 1
    p.rebuild_every = int(rebuild_every)
    p.skin = float(skin)
    p.kernel_type, p.formulation = int(scene.kernel_type), int(scene.formulation)
    p.visc_avg, p.ddiff = int(scene.visc_avg), int(scene.ddiff)
    p.ddiff_coef, p.zeta = float(scene.ddiff_coef), float(scene.zeta)
    return p


class Simulation:
    """One library context (sph_ctx) on the current CUDA device."""

    def __init__(self, params: Params, scenes_desc=None):
        lib = _lib()
        h = ctypes.c_void_p()
        _check(lib.sph_create(ctypes.byref(params), ctypes.byref(h)), "sph_create")
        self._h = h
        self.params = params
        self.n = 0
        if scenes_desc:
            arr = (SceneDesc * len(scenes_desc))()
            for k, d in enumerate(scenes_desc):
                arr[k].origin[:] = list(d["origin"])
                arr[k].size[:] = list(d["size"])
                arr[k].periodic_mask = int(d.get("periodic", 0))
                arr[k].c0 = float(d["c0"])
            _check(lib.sph_set_scenes(self._h, len(scenes_desc), arr), "sph_set_scenes")
        self.n_scenes = len(scenes_desc) if scenes_desc else 1

    @classmethod
    def from_scene(cls, scene, max_particles=None, max_neibs=128, upload=True, stream=None, rebuild_every=1,
                   skin=0.0):
        sim = cls(params_from_scene(scene, max_particles, max_neibs, rebuild_every, skin), scene.scenes)
        if upload:
            sim.upload(scene, stream=stream)
        return sim

    def close(self):
        if getattr(self, "_h", None):
            _lib().sph_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- upload / download -------------------------------------------------
    def upload(self, scene=None, *, pos=None, vel=None, delta=None, mass=None, ptype=None, scene_id=None,
               stream=None):
        if scene is not None:
            pos, vel, delta, mass, ptype = scene.pos, scene.vel, scene.delta, scene.mass, scene.ptype
            scene_id = scene.scene if scene.scenes else None
        pos = np.ascontiguousarray(pos, np.float64)
        vel = np.ascontiguousarray(vel, np.float32)
        delta = np.ascontiguousarray(delta, np.float32)
        mass = np.ascontiguousarray(mass, np.float32)
        ptype = np.ascontiguousarray(ptype, np.uint8)
        sid = None if scene_id is None else np.ascontiguousarray(scene_id, np.uint32)
        n = pos.shape[0]
        _check(_lib().sph_upload(self._h, n, _ptr(pos), _ptr(vel), _ptr(delta), _ptr(mass), _ptr(ptype),
                                 _ptr(sid), _stream_handle(stream)), "sph_upload")
        self.n = n

    def upload_device(self, pos, vel, delta, mass, ptype, scene_id=None, stream=None):
        """Upload from torch CUDA tensors (float64 pos, float32 vel/delta/mass, uint8 type)."""
        n = int(pos.shape[0])
        sid = None if scene_id is None else ctypes.c_void_p(scene_id.data_ptr())
        _check(_lib().sph_upload_device(self._h, n, ctypes.c_void_p(pos.data_ptr()), ctypes.c_void_p(vel.data_ptr()),
                                        ctypes.c_void_p(delta.data_ptr()), ctypes.c_void_p(mass.data_ptr()),
                                        ctypes.c_void_p(ptype.data_ptr()), sid, _stream_handle(stream)),
               "sph_upload_device")
        self.n = n

    def download(self, stream=None, out=None):
        """(pos, vel, delta) in upload order; `out` = preallocated (pos, vel, delta) host arrays."""
        n = self.n
        if out is None:
            pos = np.empty((n, 3), np.float64)
            vel = np.empty((n, 3), np.float32)
            delta = np.empty(n, np.float32)
        else:
            pos, vel, delta = out
            assert pos.dtype == np.float64 and vel.dtype == np.float32 and delta.dtype == np.float32
            assert pos.flags.c_contiguous and vel.flags.c_contiguous and delta.flags.c_contiguous
        _check(_lib().sph_download(self._h, n, _ptr(pos), _ptr(vel), _ptr(delta), _stream_handle(stream)),
               "sph_download")
        return pos, vel, delta

    def download_device(self, pos, vel, delta, stream=None):
        """Download into torch CUDA tensors (no host synchronisation)."""
        p = lambda t: None if t is None else ctypes.c_void_p(t.data_ptr())  # noqa: E731
        _check(_lib().sph_download_device(self._h, self.n, p(pos), p(vel), p(delta), _stream_handle(stream)),
               "sph_download_device")

    def download_forces(self, stream=None):
        n = self.n
        acc = np.empty((n, 3), np.float32)
        drho = np.empty(n, np.float32)
        _check(_lib().sph_download_forces(self._h, n, _ptr(acc), _ptr(drho), _stream_handle(stream)),
               "sph_download_forces")
        return acc, drho

    def download_neighbors(self, stream=None):
        n = self.n
        mn = self.params.max_neibs
        counts = np.empty((n, 2), np.uint32)
        ids = np.empty((n, mn), np.uint32)
        _check(_lib().sph_download_neighbors(self._h, n, _ptr(counts), _ptr(ids), _stream_handle(stream)),
               "sph_download_neighbors")
        return counts, ids

    def download_neighbors_of(self, sample, stream=None):
        """Lists of the particles with upload ids `sample`: (counts[m,2], ids[m,max_neibs])."""
        smp = np.ascontiguousarray(sample, np.uint32)
        m, mn = smp.shape[0], self.params.max_neibs
        counts = np.empty((m, 2), np.uint32)
        ids = np.empty((m, mn), np.uint32)
        _check(_lib().sph_download_neighbors_of(self._h, m, _ptr(smp), _ptr(counts), _ptr(ids),
                                                _stream_handle(stream)), "sph_download_neighbors_of")
        return counts, ids

    def download_neighbors_noalloc(self, stream=None):
        """download_neighbors without device allocation (fixed library-owned
        staging; n <= 2^20 and n * max_neibs <= 2^22)."""
        n = self.n
        mn = self.params.max_neibs
        counts = np.empty((n, 2), np.uint32)
        ids = np.empty((n, mn), np.uint32)
        _check(_lib().sph_download_neighbors_noalloc(self._h, n, _ptr(counts), _ptr(ids), _stream_handle(stream)),
               "sph_download_neighbors_noalloc")
        return counts, ids

    # ---- the hot path ------------------------------------------------------
    def build_neighbors(self, stream=None):
        _check(_lib().sph_build_neighbors(self._h, _stream_handle(stream)), "sph_build_neighbors")

    def forces(self, stream=None):
        _check(_lib().sph_forces(self._h, _stream_handle(stream)), "sph_forces")

    def step(self, nsteps=1, stream=None):
        _check(_lib().sph_step(self._h, int(nsteps), _stream_handle(stream)), "sph_step")

    def set_owned(self, n_owned=0xFFFFFFFF):
        """Particles with upload id >= n_owned are halo copies (left out of the CFL dt)."""
        _check(_lib().sph_set_owned(self._h, int(n_owned)), "sph_set_owned")

    def set_dt(self, dt):
        """The time step of the next step (instead of its own CFL value)."""
        _check(_lib().sph_set_dt(self._h, float(dt)), "sph_set_dt")

    def cfl_dt(self, stream=None):
        """CFL time step of the current state (halo copies left out), without a step."""
        dt = ctypes.c_double()
        _check(_lib().sph_cfl_dt(self._h, ctypes.byref(dt), _stream_handle(stream)), "sph_cfl_dt")
        return dt.value

    def next_dt(self, stream=None):
        """CFL time step the next step would take (from the last step's accelerations)."""
        dt = ctypes.c_double()
        _check(_lib().sph_next_dt(self._h, ctypes.byref(dt), _stream_handle(stream)), "sph_next_dt")
        return dt.value

    def set_fused_predict(self, on=True):
        """List build and predictor pass as one kernel (True) or two (False); same bits."""
        _check(_lib().sph_set_fused_predict(self._h, int(bool(on))), "sph_set_fused_predict")

    def step_options(self):
        """{"fused_predict": bool, "persistent": bool} in use."""
        f, p = ctypes.c_int(), ctypes.c_int()
        _check(_lib().sph_get_step_options(self._h, ctypes.byref(f), ctypes.byref(p)), "sph_get_step_options")
        return {"fused_predict": bool(f.value), "persistent": bool(p.value)}

    def set_persistent(self, on=True):
        """Step with one persistent kernel launch per step() call (True) or the captured
        graph of per-phase kernels (False); the same results to the bit."""
        _check(_lib().sph_set_persistent(self._h, int(bool(on))), "sph_set_persistent")

    def autotune(self, stream=None):
        """Pick the fastest neighbour-build variant and force-kernel launch shape
        on the uploaded state; returns (build variant name, forces variant name)."""
        v = ctypes.c_int()
        fv = ctypes.c_int()
        _check(_lib().sph_autotune(self._h, _stream_handle(stream), ctypes.byref(v), ctypes.byref(fv)),
               "sph_autotune")
        return _lib().sph_build_variant_name(v.value).decode(), _lib().sph_forces_variant_name(fv.value).decode()

    def conservation(self, stream=None):
        """Momentum (3), force sum m a (3), sum m drho/dt, kinetic energy and total mass at the
        current state."""
        out = np.zeros(9, np.float64)
        _check(_lib().sph_conservation(self._h, _ptr(out), _stream_handle(stream)), "sph_conservation")
        return {"momentum": out[0:3], "force": out[3:6], "mass_rate": out[6], "kinetic": out[7], "mass": out[8]}

    def set_variants(self, build=-1, forces=-1):
        """Select the build variant and force launch shape of every pass (0..4, -1 keeps)."""
        _check(_lib().sph_set_variants(self._h, int(build), int(forces)), "sph_set_variants")

    def set_forces_variants(self, predict=-1, correct=-1):
        """Select the force launch shapes of the predictor and corrector passes apart."""
        _check(_lib().sph_set_forces_variants(self._h, int(predict), int(correct)), "sph_set_forces_variants")

    def variants(self):
        """Names of the variants in use: {"build", "forces_predict", "forces_correct"}."""
        v = [ctypes.c_int() for _ in range(3)]
        _check(_lib().sph_get_variants(self._h, *(ctypes.byref(x) for x in v)), "sph_get_variants")
        return {"build": _lib().sph_build_variant_name(v[0].value).decode(),
                "forces_predict": _lib().sph_forces_variant_name(v[1].value).decode(),
                "forces_correct": _lib().sph_forces_variant_name(v[2].value).decode()}

    # ---- differentiable run ---------------------------------------------------
    def set_alpha(self, alpha):
        _check(_lib().sph_set_alpha(self._h, float(alpha)), "sph_set_alpha")

    def record(self, T, K, stream=None):
        """T steps with frozen dt and a checkpoint every K steps; returns dt."""
        dt = ctypes.c_double()
        _check(_lib().sph_record(self._h, int(T), int(K), _stream_handle(stream), ctypes.byref(dt)), "sph_record")
        return dt.value

    def tape_generation(self):
        """Generation of the recording the next backward() reverses (0: none)."""
        g = ctypes.c_uint64()
        _check(_lib().sph_tape_generation(self._h, ctypes.byref(g)), "sph_tape_generation")
        return g.value

    def backward(self, xbar_T=None, ubar_T=None, dbar_T=None, want_x=False, want_delta=False, stream=None):
        """Adjoint of the last record: torch CUDA float32 inputs (n,3)/(n,) or None;
        returns (dL/dx0 or None, dL/du0, dL/ddelta0 or None, dL/dalpha)."""
        import torch
        n = self.n
        dev = torch.device("cuda", torch.cuda.current_device())
        p = lambda t: None if t is None else ctypes.c_void_p(t.data_ptr())  # noqa: E731
        for t in (xbar_T, ubar_T, dbar_T):
            assert t is None or (t.is_cuda and t.dtype == torch.float32 and t.is_contiguous())
        ubar0 = torch.empty((n, 3), dtype=torch.float32, device=dev)
        xbar0 = torch.empty((n, 3), dtype=torch.float32, device=dev) if want_x else None
        dbar0 = torch.empty((n,), dtype=torch.float32, device=dev) if want_delta else None
        ab = ctypes.c_double()
        _check(_lib().sph_backward(self._h, p(xbar_T), p(ubar_T), p(dbar_T), p(xbar0), p(ubar0), p(dbar0),
                                   ctypes.byref(ab), _stream_handle(stream)), "sph_backward")
        return xbar0, ubar0, dbar0, ab.value

    PHASES = ("dt", "hash", "scan", "scatter", "reorder", "build", "forces_predict", "forces_correct")

    def step_profiled(self, nsteps=1, stream=None):
        """Steps launched kernel by kernel with CUDA events between them;
        returns {phase: total ms}."""
        ms = np.zeros(8, np.float64)
        _check(_lib().sph_step_profiled(self._h, int(nsteps), _stream_handle(stream), _ptr(ms)),
               "sph_step_profiled")
        return dict(zip(self.PHASES, ms.tolist()))

    # ---- counters ----------------------------------------------------------
    def stats(self, stream=None, check=True):
        s = Stats()
        rc = _lib().sph_get_stats(self._h, ctypes.byref(s), _stream_handle(stream))
        if check:
            _check(rc, "sph_get_stats")
        return s.as_dict() | {"rc": rc}

    def scene_times(self, stream=None):
        dt = np.empty(self.n_scenes, np.float64)
        t = np.empty(self.n_scenes, np.float64)
        _check(_lib().sph_get_scene_times(self._h, _ptr(dt), _ptr(t), _stream_handle(stream)), "sph_get_scene_times")
        return dt, t

    def clear_error(self, stream=None):
        _check(_lib().sph_clear_error(self._h, _stream_handle(stream)), "sph_clear_error")

    def sync(self, stream=None):
        _check(_lib().sph_sync(self._h, _stream_handle(stream)), "sph_sync")
