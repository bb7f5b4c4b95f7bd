"""Helpers shared by the GPU parity tests (comparison logic only)."""
import numpy as np
import pytest

import oracle


def require_gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU test run without a CUDA device")


def sim_for(scene, **kw):
    from paper_2207_11328_gb300 import Simulation, _build
    _build.build()
    return Simulation.from_scene(scene, **kw)


def compare_neighbor_sets(scene, counts, ids, band=1e-6):
    """GPU lists vs the oracle's sets, excluding pairs with |r - 2h| < band*h.
    Boundary particles keep only fluid neighbours (boundary-boundary pairs
    carry no interaction).  Returns the number of compared pairs."""
    p = oracle.params(scene)
    R = scene.kernel_radius * scene.h
    # oracle sets with a slightly larger radius so the band around R is visible
    p_out = oracle.params(scene, kernel_radius=(R + band * scene.h) / scene.h)
    off, idx = oracle.neighbors(p_out, scene.pos)
    pos = scene.pos
    size = np.array(scene.size)
    fluid = scene.ptype == 0
    n = scene.n
    total = 0
    for i in range(n):
        js = idx[off[i]:off[i + 1]]
        d = pos[i][None, :] - pos[js]
        for a in range(3):
            if (scene.periodic >> a) & 1:
                d[:, a] -= size[a] * np.round(d[:, a] / size[a])
        r = np.sqrt((d * d).sum(1))
        sure = js[r < R - band * scene.h]
        near = set(js[np.abs(r - R) <= band * scene.h].tolist())
        if not fluid[i]:
            sure = sure[fluid[sure]]
        nf, nb = int(counts[i, 0]), int(counts[i, 1])
        got = ids[i, :nf + nb]
        assert len(set(got.tolist())) == nf + nb, f"duplicate neighbours of {i}"
        assert np.all(fluid[got[:nf]]), f"non-fluid in the fluid part of {i}"
        assert not np.any(fluid[got[nf:nf + nb]]), f"fluid in the boundary part of {i}"
        g = set(got.tolist()) - near
        assert g == set(sure.tolist()), f"particle {i}: gpu-oracle {sorted(g - set(sure.tolist()))} " \
                                        f"oracle-gpu {sorted(set(sure.tolist()) - g)}"
        assert np.all(ids[i, nf + nb:] == 0xFFFFFFFF)
        total += len(sure)
    return total


U32 = 2.0 ** -24     # FP32 unit roundoff


def rel_check(gpu, ref, tol, what, mag=None, c_round=4.0):
    """Per particle |gpu - ref| <= max(tol * max(|ref_i|, rms_i |ref|),
    c_round * u * mag_i) (vector norm per row for vectors).

    tol is the relative tolerance (1e-5).  mag_i, when given, is the oracle's
    summed magnitude of the pair terms of particle i: a sum whose terms
    cancel to far below their magnitude (hydrostatic pressure: ~300x at 1M
    particles, ~700x at 16M) cannot be evaluated in FP32 to a relative 1e-5
    in any order; there the bound is c_round units of FP32 roundoff of the
    term magnitudes.  Returns (max relative error, fraction within tol)."""
    gpu = np.asarray(gpu, np.float64)
    ref = np.asarray(ref, np.float64)
    if ref.ndim == 1:
        err = np.abs(gpu - ref)
        mag_ref = np.abs(ref)
    else:
        err = np.linalg.norm(gpu - ref, axis=1)
        mag_ref = np.linalg.norm(ref, axis=1)
    rms = np.sqrt(np.mean(mag_ref ** 2)) if mag_ref.size else 0.0
    scale = np.maximum(mag_ref, rms)
    bound = tol * scale
    if mag is not None:
        bound = np.maximum(bound, c_round * U32 * np.asarray(mag, np.float64))
    bad = err > bound
    rel = err / np.maximum(scale, 1e-300)
    if np.any(bad):
        k = int(np.argmax(err / np.maximum(bound, 1e-300)))
        raise AssertionError(f"{what}: {int(bad.sum())}/{bad.size} outside the bound; worst i={k} "
                             f"gpu={gpu[k]} ref={ref[k]} rel={rel[k]:.3e} bound={bound[k] / scale[k]:.3e}")
    return (float(np.max(rel)) if rel.size else 0.0), (float(np.mean(rel <= tol)) if rel.size else 1.0)


def oracle_jvp_task(args):
    """One oracle directional derivative (for a spawn pool): returns (L, dL)."""
    import oracle as _o
    pkw, pos, vel, delta, mass, ptype, T, dt, tgt, du, dalpha = args
    p = _o.params(None, **pkw)
    return _o.loss_jvp(p, pos, vel, delta, mass, ptype, T, dt, tgt, du, dalpha)


def oracle_params_kw(scene, **kw):
    d = dict(dp=scene.dp, h=scene.h, kernel_radius=scene.kernel_radius, rho0=scene.rho0, c0=scene.c0,
             gamma=float(scene.gamma), visc_model=scene.visc, alpha=scene.alpha, nu=scene.nu, g=scene.g,
             cfl=scene.cfl, dt_fixed=scene.dt_fixed, origin=scene.origin, size=scene.size,
             periodic_mask=scene.periodic, kernel_type=scene.kernel_type, formulation=scene.formulation,
             visc_avg=scene.visc_avg, ddiff=scene.ddiff, ddiff_coef=scene.ddiff_coef, zeta=scene.zeta)
    d.update(kw)
    return d


def compare_neighbor_sets_sample(scene, sample, counts, ids, band=1e-6):
    """compare_neighbor_sets restricted to the particles in `sample` (the
    oracle's sets of all particles are computed, those of the sample
    compared).  Returns the number of compared pairs."""
    R = scene.kernel_radius * scene.h
    p_out = oracle.params(scene, kernel_radius=(R + band * scene.h) / scene.h)
    off, idx = oracle.neighbors(p_out, scene.pos)
    pos = scene.pos
    size = np.array(scene.size)
    fluid = scene.ptype == 0
    total = 0
    for i in sample:
        js = idx[off[i]:off[i + 1]]
        d = pos[i][None, :] - pos[js]
        for a in range(3):
            if (scene.periodic >> a) & 1:
                d[:, a] -= size[a] * np.round(d[:, a] / size[a])
        r = np.sqrt((d * d).sum(1))
        sure = js[r < R - band * scene.h]
        near = set(js[np.abs(r - R) <= band * scene.h].tolist())
        if not fluid[i]:
            sure = sure[fluid[sure]]
        nf, nb = int(counts[i, 0]), int(counts[i, 1])
        got = ids[i, :nf + nb]
        assert len(set(got.tolist())) == nf + nb, f"duplicate neighbours of {i}"
        assert np.all(fluid[got[:nf]]) and not np.any(fluid[got[nf:nf + nb]]), f"list parts of {i}"
        g = set(got.tolist()) - near
        assert g == set(sure.tolist()), f"particle {i}: gpu-oracle {sorted(g - set(sure.tolist()))} " \
                                        f"oracle-gpu {sorted(set(sure.tolist()) - g)}"
        total += len(sure)
    return total


def compare_neighbor_sets_of(scene, sample, counts, ids, band=1e-6):
    """GPU lists of the sampled particles (rows of sph_download_neighbors_of) against the
    oracle's sampled search, excluding pairs within band*h of the cutoff.  Returns the
    number of compared pairs."""
    R = scene.kernel_radius * scene.h
    p_out = oracle.params(scene, kernel_radius=(R + band * scene.h) / scene.h)
    off, idx = oracle.neighbors_sample(p_out, scene.pos, sample)
    fluid = scene.ptype == 0
    size = np.array(scene.size)
    total = 0
    for k, i in enumerate(sample):
        js = idx[off[k]:off[k + 1]]
        d = scene.pos[i][None, :] - scene.pos[js]
        for a in range(3):
            if (scene.periodic >> a) & 1:
                d[:, a] -= size[a] * np.round(d[:, a] / size[a])
        r = np.sqrt((d * d).sum(1))
        sure = js[r < R - band * scene.h]
        near = set(js[np.abs(r - R) <= band * scene.h].tolist())
        if not fluid[i]:
            sure = sure[fluid[sure]]
        nf, nb = int(counts[k, 0]), int(counts[k, 1])
        got = ids[k, :nf + nb]
        assert len(set(got.tolist())) == nf + nb, f"duplicate neighbours of {i}"
        assert np.all(fluid[got[:nf]]) and not np.any(fluid[got[nf:nf + nb]]), f"list parts of {i}"
        g = set(got.tolist()) - near
        assert g == set(sure.tolist()), f"particle {i}: gpu-oracle {sorted(g - set(sure.tolist()))} " \
                                        f"oracle-gpu {sorted(set(sure.tolist()) - g)}"
        assert np.all(ids[k, nf + nb:] == 0xFFFFFFFF)
        total += len(sure)
    return total
