// Pieces shared by the interaction kernels (forces.cu: the tuned kernels of
// the default model; forces_models.cu: the other model options of Table 1):
// the central particle's shifted offsets, and the per-particle epilogue that
// fuses the predictor or corrector update (reading C6) and the per-scene
// max |a|^2 reduction for the CFL time step (reading C7).  forces.cu writes
// the same epilogue out inline (faster there, measured).
#pragma once

#include "sph_internal.cuh"

namespace sphg {

struct Acc {
    float ax, ay, az, drho;
};

// The central particle's offset seen from a neighbour cell: o_i - d*cell for
// d = -1, 0, +1 per axis (list entries carry d + 1 in two bits per axis).
struct Central {
    float xm, x0, xp, ym, y0, yp, zm, z0, zp;
};

__device__ __forceinline__ Central central_of(const float4& pi, float cx, float cy, float cz) {
    return Central{pi.x + cx, pi.x, pi.x - cx, pi.y + cy, pi.y, pi.y - cy, pi.z + cz, pi.z, pi.z - cz};
}

__device__ __forceinline__ float pick(uint32_t b, float m, float z, float p) {
    return (b & 1u) ? z : ((b & 2u) ? p : m);
}

// The exact list of a skin-list step (written by the predictor pass, read by the
// corrector): entries in chunks of four, chunk g of particle i at uint4 index
// g * stride + i, fluid entries from chunk 0 and boundary entries from chunk
// exact_bnd_chunk(max_neibs).  A lane writes a chunk with one 16-byte store once
// it holds four entries (the entries of a list are found at different times in
// different lanes, so 4-byte stores would scatter); the corrector reads four
// entries per coalesced 16-byte load.  Unused slots of the last chunk hold kMarker.

struct ChunkWriter {
    uint4 buf;      // the last entries, newest in .w
    uint32_t n;     // entries written
    uint4* base;    // chunk 0 of particle 0 of this part
    size_t stride;
    uint32_t i;
    __device__ __forceinline__ void put(uint32_t e) {
        buf.x = buf.y;
        buf.y = buf.z;
        buf.z = buf.w;
        buf.w = e;
        if ((++n & 3u) == 0u) base[(size_t)((n >> 2) - 1u) * stride + i] = buf;
    }
    __device__ __forceinline__ void flush() {
        const uint32_t r = n & 3u;  // the last r entries sit in the top r slots
        if (r) {
            uint4 o;
            o.x = r == 1u ? buf.w : (r == 2u ? buf.z : buf.y);
            o.y = r == 1u ? kMarker : (r == 2u ? buf.w : buf.z);
            o.z = r == 3u ? buf.w : kMarker;
            o.w = kMarker;
            base[(size_t)(n >> 2) * stride + i] = o;
        }
    }
};

// Epilogue of particle i with its summed rates acc (a and drho/dt).
//   kForcesOnly: store (a, drho/dt);
//   kPredict:    u* = u + dt/2 a, delta* = delta + dt/2 drho/rho0, x* = x + dt/2 u  -> io_*
//   kCorrect:    state n in io_*: u' = u + dt a*, delta' = delta + dt drho*/rho0,
//                x' = x + dt (u + u')/2, overwritten in io_*;
// boundary particles integrate delta only.  pos_ref (skin list, corrector):
// displacement since the build, checked against skin/2 and reduced for the
// rebuild decision.  The corrector (or acc_dt) reduces max |a|^2 per scene.
template <int MODE>
__device__ __forceinline__ void finish_particle(uint32_t i, uint32_t s, const SceneDev& sc, const float4& pi,
                                                const float4& vi, bool fluid_i, const Acc& acc, float4* io_pos,
                                                float4* io_vel, float* io_phat, float4* __restrict__ force_out,
                                                SceneDyn* __restrict__ dyn, DevStatus* __restrict__ st, const Phys& ph,
                                                int acc_dt, const float4* __restrict__ pos_ref,
                                                const uint32_t* __restrict__ pid) {
    if (MODE == kForcesOnly) {
        force_out[i] = make_float4(acc.ax, acc.ay, acc.az, acc.drho);
    } else {
        const float dt = dyn[s].dt;
        if (MODE == kPredict) {
            const float hd = 0.5f * dt;
            float4 po = pi, vo = vi;
            vo.w = fmaf(hd * ph.inv_rho0, acc.drho, vi.w);
            if (fluid_i) {
                vo.x = fmaf(hd, acc.ax, vi.x);
                vo.y = fmaf(hd, acc.ay, vi.y);
                vo.z = fmaf(hd, acc.az, vi.z);
                po.x = fmaf(hd, vi.x, pi.x);
                po.y = fmaf(hd, vi.y, pi.y);
                po.z = fmaf(hd, vi.z, pi.z);
            }
            io_pos[i] = po;
            io_vel[i] = vo;
            io_phat[i] = eos_phat(vo.w, ph, sc.phat_coef);
        } else {  // kCorrect: state n in io_*, overwritten by n+1
            float4 po = io_pos[i], vo = io_vel[i];
            const float un_x = vo.x, un_y = vo.y, un_z = vo.z;
            vo.w = fmaf(dt * ph.inv_rho0, acc.drho, vo.w);
            if (fluid_i) {
                vo.x = fmaf(dt, acc.ax, un_x);
                vo.y = fmaf(dt, acc.ay, un_y);
                vo.z = fmaf(dt, acc.az, un_z);
                const float hd = 0.5f * dt;
                po.x = fmaf(hd, un_x + vo.x, po.x);
                po.y = fmaf(hd, un_y + vo.y, po.y);
                po.z = fmaf(hd, un_z + vo.z, po.z);
            }
            io_pos[i] = po;
            io_vel[i] = vo;
            io_phat[i] = eos_phat(vo.w, ph, sc.phat_coef);
            const float chk = po.x + po.y + po.z + vo.x + vo.y + vo.z + vo.w;
            if (!isfinite(chk)) atomicOr(&st->error_bits, SPH_EBIT_NONFINITE);
            if (pos_ref) {
                // the list (built with a skin) covers the cutoff while no particle has
                // moved more than skin/2 since the build; the largest displacement
                // decides the next rebuild (k_dt)
                const float4 r0 = pos_ref[i];
                const float dx = po.x - r0.x, dy = po.y - r0.y, dz = po.z - r0.z;
                const float d2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                if (d2 > ph.skin_lim2) atomicOr(&st->error_bits, SPH_EBIT_SKIN);
                const unsigned mk = __activemask();
                const uint32_t m = __reduce_max_sync(mk, __float_as_uint(d2));
                if ((threadIdx.x & 31) == (uint32_t)(__ffs(mk) - 1)) atomicMax(&st->maxdisp2_bits, m);
            }
        }
    }
    if (MODE == kCorrect || acc_dt) {
        const float a2 = fluid_i && cfl_counts(ph, pid, i)
                             ? fmaf(acc.ax, acc.ax, fmaf(acc.ay, acc.ay, acc.az * acc.az)) : 0.f;
        const uint32_t bits = __float_as_uint(a2);
        const unsigned mask = __activemask();
        const unsigned same = __match_any_sync(mask, s);
        if (same == mask) {
            const uint32_t m = __reduce_max_sync(mask, bits);
            if ((threadIdx.x & 31) == (uint32_t)(__ffs(mask) - 1) && m) atomicMax(&dyn[s].amax2_bits, m);
        } else if (bits) {
            atomicMax(&dyn[s].amax2_bits, bits);
        }
    }
}

}  // namespace sphg
