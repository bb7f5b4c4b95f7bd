// Particle interactions and time integration (paper Section 2.1; readings
// of the passages the paper leaves to its references are stated inline).
//
//   drho_i/dt = sum_j m_j (u_i - u_j).x_ij F_ij                        (C1)
//   du_i/dt   = -sum_j m_j (P_i/rho_i^2 + P_j/rho_j^2 + Pi_ij) x_ij F_ij  (C2)
//               + sum_j 4 nu m_j/(rho_i + rho_j) F_ij (u_i - u_j) + g     (C3)
//   Pi_ij = -alpha h c0 mu_ij / rhobar_ij for u_ij.x_ij < 0,
//   mu_ij = u_ij.x_ij/(r^2 + 0.01 h^2), rhobar = (rho_i + rho_j)/2          (C4)
//   F = (1/r) dW/dr = aF (q - 2)^3 for q = r/h < 2 (Wendland C2, Section 4)
//   Dynamic boundary particles: zero velocity, continuity only      (C5)
//
// One thread per particle, sorted order.  The neighbour list is read
// neighbour-major (a warp reads 256 contiguous bytes per two-entry chunk),
// fluid chunks from the front and boundary chunks from the back (split list,
// Section 4), each with its own loop.  Per neighbour the kernel gathers pos4 + vel4
// (32 bytes, served by L1/L2: neighbours of consecutive particles are the
// same cell-sorted particles) and P_j/rho_j^2, which the passes over a list
// built at this step recompute from delta_j instead (see fluid_pair).
// The predictor (dt/2) and corrector (dt) updates of reading C6 are fused
// into the epilogues of the two force passes; the corrector pass reduces
// max |a|^2 per scene (warp reduction + one atomic) for the CFL dt (C7).
#include <cooperative_groups.h>

#include "forces_common.cuh"
#include "pipeline.cuh"

namespace cg = cooperative_groups;

namespace sphg {

namespace {

// One neighbour of a fluid particle.  BND: the neighbour is a boundary
// particle (mass stored negated, velocity zero).  The kernel constant aF is
// factored out of every term (all terms are linear in F) and applied once.
// RECOMP: P_j/rho_j^2 from delta_j (the function that stores the per-particle
// value, so bit-identical to it) in place of a third gather.  Faster in every
// pass over the pairs within the cutoff; slower in the passes that filter a
// skin list (more registers live beside the exact-list writers), which keep
// the gather.
template <int VISC, bool BND, bool FILTER, bool RECOMP>
__device__ __forceinline__ bool fluid_pair(uint32_t e, const Central& ci, const float4& vi, float phat_i,
                                           const float4* __restrict__ pos, const float4* __restrict__ vel,
                                           const float* __restrict__ phat, float phat_coef, float pi_coef,
                                           const Phys& ph, Acc& acc, uint32_t& npairs) {
    const uint32_t j = e >> kCodeBits;
    const float4 pj = pos[j];
    const float4 vj = vel[j];  // all gathers issued together
    const float phat_j = RECOMP ? eos_phat(vj.w, ph, phat_coef) : phat[j];
    const float rx = pick(e, ci.xm, ci.x0, ci.xp) - pj.x;
    const float ry = pick(e >> 2, ci.ym, ci.y0, ci.yp) - pj.y;
    const float rz = pick(e >> 4, ci.zm, ci.z0, ci.zp) - pj.z;
    const float r2 = fmaxf(fmaf(rx, rx, fmaf(ry, ry, rz * rz)), 1e-30f);
    if (FILTER) {
        // list with a skin: pairs beyond the influence radius (F = 0) skip the arithmetic
        if (!(r2 < ph.R2)) return false;
        ++npairs;
    }
    const float r = r2 * rsqrtf(r2);
    const float t = fminf(fmaf(r, ph.inv_h, -2.0f), 0.0f);
    const float mj = BND ? -pj.w : pj.w;
    const float mF = mj * (t * t * t);  // m_j F / aF
    const float ux = BND ? vi.x : vi.x - vj.x;
    const float uy = BND ? vi.y : vi.y - vj.y;
    const float uz = BND ? vi.z : vi.z - vj.z;
    const float udx = fmaf(ux, rx, fmaf(uy, ry, uz * rz));
    acc.drho = fmaf(mF, udx, acc.drho);
    float bracket = phat_i + phat_j;
    if (VISC == SPH_VISC_ARTIFICIAL) {
        // approaching pairs only (u.x < 0), without a branch: receding pairs add -pi*0
        const float den = (r2 + ph.eps_h2) * fmaf(0.5f, vi.w + vj.w, 1.0f);
        bracket = fmaf(-pi_coef, __fdividef(fminf(udx, 0.f), den), bracket);
    }
    const float coef = mF * bracket;
    acc.ax = fmaf(-coef, rx, acc.ax);
    acc.ay = fmaf(-coef, ry, acc.ay);
    acc.az = fmaf(-coef, rz, acc.az);
    if (VISC == SPH_VISC_LAMINAR) {
        const float lam = ph.nu4 * ph.inv_rho0 * __fdividef(mF, 2.0f + vi.w + vj.w);
        acc.ax = fmaf(lam, ux, acc.ax);
        acc.ay = fmaf(lam, uy, acc.ay);
        acc.az = fmaf(lam, uz, acc.az);
    }
    return true;
}

// SKIN: the list carries a skin (rebuild every k steps).  The predictor pass
// (and sph_forces) skip pairs beyond the cutoff and count the pairs within it;
// the predictor also writes those pairs, the step's exact list, to
// nlist_x/ncount_x (same split layout), which the corrector pass reads as its
// list (so both passes use the pairs within R at x^n, as with a list built
// every step) before checking the displacement since the build.
// (the forces-only pass keeps the |a|^2 reduction for dt0 live beside the sums: it gets
// a looser register cap than the step's passes, so that no shape spills)
// One particle of a force pass (one iteration of the pass's particle loop): its pair sums
// over its list and the epilogue of the pass (store, predictor or corrector update).
__device__ __forceinline__ uint32_t ld_count_fresh(const uint32_t* p) {
    uint32_t v;
    asm volatile("ld.global.cg.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// List chunk loads: through the read-only path, or (FRESH: the list was written earlier in
// the same kernel, by this thread) through L2 only, coherent with those stores.
template <bool FRESH>
__device__ __forceinline__ uint2 ld_chunk(const uint2* p) {
    if (!FRESH) return __ldg(p);
    uint2 v;
    asm volatile("ld.global.cg.v2.u32 {%0, %1}, [%2];" : "=r"(v.x), "=r"(v.y) : "l"(p) : "memory");
    return v;
}

template <int VISC, int MODE, bool SKIN, bool FRESH = false>
__device__ __forceinline__ void particle_pass(
    uint32_t i, uint32_t n, const float4* __restrict__ pos, const float4* __restrict__ vel,
    const float* __restrict__ phat, float4* io_pos, float4* io_vel, float* io_phat, float4* __restrict__ force_out,
    const uint32_t* __restrict__ pinfo, const uint32_t* __restrict__ nlist, const uint32_t* __restrict__ ncount,
    const SceneDev* __restrict__ scenes, SceneDyn* __restrict__ dyn, DevStatus* __restrict__ st, const Phys& ph,
    int acc_dt, const float4* __restrict__ pos_ref, uint32_t* __restrict__ nlist_x,
    uint32_t* __restrict__ ncount_x, const uint32_t* __restrict__ pid, uint32_t& npairs, uint32_t cnt_fresh = 0) {
    static_assert(!(FRESH && SKIN), "a list written in the same kernel is a list built at this step");
    constexpr bool FILTER = SKIN && MODE != kCorrect;
    constexpr bool COMPACT = SKIN && MODE == kPredict;
    constexpr bool CHUNKED = SKIN && MODE == kCorrect;  // nlist/ncount: the exact list in chunks
    constexpr bool RECOMP = !FILTER;  // P_j/rho_j^2 recomputed (see fluid_pair)
    const uint32_t s = pinfo[i];
    const SceneDev& sc = scenes[s];
    const float4 pi = pos[i];
    const float4 vi = vel[i];
    const uint32_t cnt = FRESH ? cnt_fresh : ncount[i];
    uint32_t nf = cnt & 0xffffu, nb = cnt >> 16;
    SPH_GUARD(nf + nb <= ph.max_neibs, st, nf = nb = 0)
    const bool fluid_i = pi.w > 0.f;
    const float cx = sc.cell_f[0], cy = sc.cell_f[1], cz = sc.cell_f[2];
    Acc acc{0.f, 0.f, 0.f, 0.f};
    const size_t S = ph.stride;
    const uint32_t kxb = exact_bnd_chunk(ph.max_neibs);
    ChunkWriter xf{make_uint4(0u, 0u, 0u, 0u), 0u, reinterpret_cast<uint4*>(nlist_x), S, i};
    ChunkWriter xb{make_uint4(0u, 0u, 0u, 0u), 0u, reinterpret_cast<uint4*>(nlist_x) + (size_t)kxb * S, S, i};
    if (fluid_i && CHUNKED) {
        const float phat_i = phat[i];
        const float pic = sc.pi_coef;
        const Central ci = central_of(pi, cx, cy, cz);
        // full chunks: four pairs with no test between them (their gathers issue together);
        // then the last chunk of each part (1 to 3 entries, the rest kMarker)
#define SPH_PAIR(BND, e) fluid_pair<VISC, BND, false, RECOMP>(e, ci, vi, phat_i, pos, vel, phat, sc.phat_coef, pic, ph, acc, npairs)
#define SPH_OK_E(e) (((e) >> kCodeBits) < n)
        const uint4* cp = reinterpret_cast<const uint4*>(nlist) + i;
        uint32_t k = 0;
        uint4 qn = make_uint4(0u, 0u, 0u, 0u);
        if (nf >= 4) qn = __ldg(cp);
        for (; k + 4 <= nf; k += 4, cp += S) {
            const uint4 q = qn;
            if (k + 8 <= nf) qn = __ldg(cp + S);  // the next full chunk, one iteration ahead
            SPH_GUARD(SPH_OK_E(q.x) && SPH_OK_E(q.y) && SPH_OK_E(q.z) && SPH_OK_E(q.w), st, break)
            SPH_PAIR(false, q.x);
            SPH_PAIR(false, q.y);
            SPH_PAIR(false, q.z);
            SPH_PAIR(false, q.w);
        }
        do {
            if (k >= nf) break;
            const uint4 q = __ldg(cp);
            SPH_GUARD(SPH_OK_E(q.x) && (k + 1 >= nf || SPH_OK_E(q.y)) && (k + 2 >= nf || SPH_OK_E(q.z)), st, break)
            SPH_PAIR(false, q.x);
            if (k + 1 < nf) SPH_PAIR(false, q.y);
            if (k + 2 < nf) SPH_PAIR(false, q.z);
        } while (0);
        cp = reinterpret_cast<const uint4*>(nlist) + (size_t)kxb * S + i;
        for (k = 0; k + 4 <= nb; k += 4, cp += S) {
            const uint4 q = __ldg(cp);
            SPH_GUARD(SPH_OK_E(q.x) && SPH_OK_E(q.y) && SPH_OK_E(q.z) && SPH_OK_E(q.w), st, break)
            SPH_PAIR(true, q.x);
            SPH_PAIR(true, q.y);
            SPH_PAIR(true, q.z);
            SPH_PAIR(true, q.w);
        }
        do {
            if (k >= nb) break;
            const uint4 q = __ldg(cp);
            SPH_GUARD(SPH_OK_E(q.x) && (k + 1 >= nb || SPH_OK_E(q.y)) && (k + 2 >= nb || SPH_OK_E(q.z)), st, break)
            SPH_PAIR(true, q.x);
            if (k + 1 < nb) SPH_PAIR(true, q.y);
            if (k + 2 < nb) SPH_PAIR(true, q.z);
        } while (0);
#undef SPH_PAIR
#undef SPH_OK_E
        acc.ax = fmaf(ph.aF, acc.ax, ph.g[0]);
        acc.ay = fmaf(ph.aF, acc.ay, ph.g[1]);
        acc.az = fmaf(ph.aF, acc.az, ph.g[2]);
        acc.drho *= ph.aF;
    } else if (fluid_i) {
        const float phat_i = phat[i];
        const float pic = sc.pi_coef;
        const Central ci = central_of(pi, cx, cy, cz);
        // list chunks come from DRAM: two chunks (four entries) per iteration, loaded one
        // iteration ahead so that their latency is not on the path to the gathers
        const uint2* lp = reinterpret_cast<const uint2*>(nlist) + i;
        uint32_t k = 0;
// keep a pair of the exact list (COMPACT only)
#define SPH_KEEP_F(e) if (COMPACT) xf.put(e);
#define SPH_KEEP_B(e) if (COMPACT) xb.put(e);
        uint2 an = make_uint2(0u, 0u), bn = make_uint2(0u, 0u);
        if (nf >= 4) {
            an = ld_chunk<FRESH>(lp);
            bn = ld_chunk<FRESH>(lp + S);
        }
        for (; k + 4 <= nf; k += 4, lp += 2 * S) {
            const uint2 a = an, b = bn;
            if (k + 8 <= nf) {  // the next iteration's chunks (within the fluid part)
                an = ld_chunk<FRESH>(lp + 2 * S);
                bn = ld_chunk<FRESH>(lp + 3 * S);
            }
            SPH_GUARD((max(max(a.x, a.y), max(b.x, b.y)) >> kCodeBits) < n, st, break)
            if (fluid_pair<VISC, false, FILTER, RECOMP>(a.x, ci, vi, phat_i, pos, vel, phat, sc.phat_coef, pic, ph, acc, npairs)) SPH_KEEP_F(a.x)
            if (fluid_pair<VISC, false, FILTER, RECOMP>(a.y, ci, vi, phat_i, pos, vel, phat, sc.phat_coef, pic, ph, acc, npairs)) SPH_KEEP_F(a.y)
            if (fluid_pair<VISC, false, FILTER, RECOMP>(b.x, ci, vi, phat_i, pos, vel, phat, sc.phat_coef, pic, ph, acc, npairs)) SPH_KEEP_F(b.x)
            if (fluid_pair<VISC, false, FILTER, RECOMP>(b.y, ci, vi, phat_i, pos, vel, phat, sc.phat_coef, pic, ph, acc, npairs)) SPH_KEEP_F(b.y)
        }
        for (; k < nf; k += 2, lp += S) {
            const uint2 a = ld_chunk<FRESH>(lp);
            const bool two = k + 1 < nf;
            SPH_GUARD((a.x >> kCodeBits) < n && (!two || (a.y >> kCodeBits) < n), st, break)
            if (fluid_pair<VISC, false, FILTER, RECOMP>(a.x, ci, vi, phat_i, pos, vel, phat, sc.phat_coef, pic, ph, acc, npairs)) SPH_KEEP_F(a.x)
            if (two && fluid_pair<VISC, false, FILTER, RECOMP>(a.y, ci, vi, phat_i, pos, vel, phat, sc.phat_coef, pic, ph, acc, npairs)) SPH_KEEP_F(a.y)
        }
        lp = reinterpret_cast<const uint2*>(nlist) + (size_t)(list_chunks(ph.max_neibs) - 1u) * S + i;
        for (k = 0; k < nb; k += 2, lp -= S) {
            const uint2 a = ld_chunk<FRESH>(lp);
            const bool two = k + 1 < nb;
            SPH_GUARD((a.x >> kCodeBits) < n && (!two || (a.y >> kCodeBits) < n), st, break)
            if (fluid_pair<VISC, true, FILTER, RECOMP>(a.x, ci, vi, phat_i, pos, vel, phat, sc.phat_coef, pic, ph, acc, npairs)) SPH_KEEP_B(a.x)
            if (two && fluid_pair<VISC, true, FILTER, RECOMP>(a.y, ci, vi, phat_i, pos, vel, phat, sc.phat_coef, pic, ph, acc, npairs)) SPH_KEEP_B(a.y)
        }
        acc.ax = fmaf(ph.aF, acc.ax, ph.g[0]);
        acc.ay = fmaf(ph.aF, acc.ay, ph.g[1]);
        acc.az = fmaf(ph.aF, acc.az, ph.g[2]);
        acc.drho *= ph.aF;
    } else {
        // boundary particle: continuity over its fluid neighbours, u_i = 0
        const Central ci = central_of(pi, cx, cy, cz);
        const uint2* lp = reinterpret_cast<const uint2*>(nlist) + i;  // list of the build
        const uint4* cp = reinterpret_cast<const uint4*>(nlist) + i;  // chunked exact list
        uint4 q = make_uint4(0u, 0u, 0u, 0u);
        uint2 q2 = make_uint2(0u, 0u);
#pragma unroll 2
        for (uint32_t k = 0; k < nf; ++k) {
            uint32_t e;
            if (CHUNKED) {
                if ((k & 3u) == 0u) {
                    q = __ldg(cp);
                    cp += S;
                }
                e = (k & 3u) == 0u ? q.x : ((k & 3u) == 1u ? q.y : ((k & 3u) == 2u ? q.z : q.w));
            } else {
                if ((k & 1u) == 0u) {
                    q2 = ld_chunk<FRESH>(lp);
                    lp += S;
                }
                e = (k & 1u) ? q2.y : q2.x;
            }
            const uint32_t j = e >> kCodeBits;
            SPH_GUARD(j < n, st, continue)
            const float4 pj = pos[j];
            const float4 vj = vel[j];
            const float rx = pick(e, ci.xm, ci.x0, ci.xp) - pj.x;
            const float ry = pick(e >> 2, ci.ym, ci.y0, ci.yp) - pj.y;
            const float rz = pick(e >> 4, ci.zm, ci.z0, ci.zp) - pj.z;
            const float r2 = fmaxf(fmaf(rx, rx, fmaf(ry, ry, rz * rz)), 1e-30f);
            if (FILTER) {
                if (!(r2 < ph.R2)) continue;
                ++npairs;
            }
            SPH_KEEP_F(e)
            const float r = r2 * rsqrtf(r2);
            const float t = fminf(fmaf(r, ph.inv_h, -2.0f), 0.0f);
            const float mF = pj.w * (t * t * t);
            const float udx = -fmaf(vj.x, rx, fmaf(vj.y, ry, vj.z * rz));
            acc.drho = fmaf(mF, udx, acc.drho);
        }
        acc.drho *= ph.aF;
    }
#undef SPH_KEEP_F
#undef SPH_KEEP_B
    if (COMPACT) {
        xf.flush();
        xb.flush();
        ncount_x[i] = xf.n | (xb.n << 16);
    }

    // epilogue written out here rather than through finish_particle() of
    // forces_common.cuh (same operations): measured 7 % faster in these kernels
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
            if (SKIN) {
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

template <int VISC, int MODE, bool SKIN>
__device__ __forceinline__ void forces_body(
    const float4* __restrict__ pos, const float4* __restrict__ vel, const float* __restrict__ phat,
    float4* io_pos, float4* io_vel, float* io_phat, float4* __restrict__ force_out,
    const uint32_t* __restrict__ pinfo, const uint32_t* __restrict__ nlist, const uint32_t* __restrict__ ncount,
    const SceneDev* __restrict__ scenes, SceneDyn* __restrict__ dyn, DevStatus* __restrict__ st, const Phys& ph,
    int acc_dt, const float4* __restrict__ pos_ref, uint32_t* __restrict__ nlist_x,
    uint32_t* __restrict__ ncount_x, const uint32_t* __restrict__ pid) {
    const uint32_t n = st->n_active;
    uint32_t npairs = 0;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        particle_pass<VISC, MODE, SKIN>(i, n, pos, vel, phat, io_pos, io_vel, io_phat, force_out, pinfo, nlist, ncount,
                                        scenes, dyn, st, ph, acc_dt, pos_ref, nlist_x, ncount_x, pid, npairs);
    if (SKIN && MODE == kPredict) {
        const uint32_t w = __reduce_add_sync(0xffffffffu, npairs);
        if ((threadIdx.x & 31) == 0 && w) atomicAdd(&st->interactions, (unsigned long long)w);
    }
}

template <int VISC, int MODE, int kBlock, int kMinBlocks, bool SKIN>
__global__ void __launch_bounds__(kBlock, MODE == kForcesOnly ? (kMinBlocks * 2 + 2) / 3 : kMinBlocks) k_forces(
    const float4* __restrict__ pos, const float4* __restrict__ vel, const float* __restrict__ phat,
    float4* io_pos, float4* io_vel, float* io_phat, float4* __restrict__ force_out,
    const uint32_t* __restrict__ pinfo, const uint32_t* __restrict__ nlist, const uint32_t* __restrict__ ncount,
    const SceneDev* __restrict__ scenes, SceneDyn* __restrict__ dyn, DevStatus* __restrict__ st, const Phys ph,
    int acc_dt, const float4* __restrict__ pos_ref, uint32_t* __restrict__ nlist_x,
    uint32_t* __restrict__ ncount_x, const uint32_t* __restrict__ pid) {
    forces_body<VISC, MODE, SKIN>(pos, vel, phat, io_pos, io_vel, io_phat, force_out, pinfo, nlist, ncount, scenes, dyn,
                                  st, ph, acc_dt, pos_ref, nlist_x, ncount_x, pid);
}

// Predictor update (reading C6) from forces already stored by a
// forces-only pass at the same state: the same operations as the predictor
// pass's epilogue, so the result is the same to the bit.  Used by the first
// step after a list build, whose dt0 forces pass is also its predictor's.
__global__ void k_predict_from_forces(const float4* __restrict__ pos, const float4* __restrict__ vel,
                                      const float4* __restrict__ force, const uint32_t* __restrict__ pinfo,
                                      const SceneDev* __restrict__ scenes, const SceneDyn* __restrict__ dyn,
                                      const DevStatus* __restrict__ st, const Phys ph, float4* __restrict__ pos_o,
                                      float4* __restrict__ vel_o, float* __restrict__ phat_o) {
    const uint32_t n = st->n_active;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const uint32_t s = pinfo[i];
        const float4 pi = pos[i], vi = vel[i], a = force[i];
        const float hd = 0.5f * dyn[s].dt;
        float4 po = pi, vo = vi;
        vo.w = fmaf(hd * ph.inv_rho0, a.w, vi.w);
        if (pi.w > 0.f) {
            vo.x = fmaf(hd, a.x, vi.x);
            vo.y = fmaf(hd, a.y, vi.y);
            vo.z = fmaf(hd, a.z, vi.z);
            po.x = fmaf(hd, vi.x, pi.x);
            po.y = fmaf(hd, vi.y, pi.y);
            po.z = fmaf(hd, vi.z, pi.z);
        }
        pos_o[i] = po;
        vel_o[i] = vo;
        phat_o[i] = eos_phat(vo.w, ph, scenes[s].phat_coef);
    }
}

// One thread per scene: dt for the coming step (reading C7), simulated
// time, reset of the |a|^2 accumulator.
// The CFL time step of a scene from the largest |a|^2 of the last reduction (reading C7)
__device__ __forceinline__ double cfl_dt_of(const SceneDev& sc, const SceneDyn& d, double h, double cfl,
                                            double dt_fixed) {
    if (dt_fixed > 0.0) return dt_fixed;
    double dt = sc.dt_cap;
    const double a2 = (double)__uint_as_float(d.amax2_bits);
    if (a2 > 0.0) dt = fmin(dt, cfl * sqrt(h / sqrt(a2)));
    return dt;
}

__device__ __forceinline__ void dt_body(const SceneDev* __restrict__ scenes, SceneDyn* __restrict__ dyn,
                                        DevStatus* __restrict__ st, uint32_t n_scenes, double h, double cfl,
                                        double dt_fixed, int advance, uint32_t rebuild_every, float trig2,
                                        uint32_t builds_inc) {
    const double dt_host = st->dt_next;  // the host's time step for this step (sph_set_dt), or <= 0
    __syncthreads();
    for (uint32_t s = threadIdx.x; s < n_scenes; s += blockDim.x) {
        const double dt = dt_host > 0.0 ? dt_host : cfl_dt_of(scenes[s], dyn[s], h, cfl, dt_fixed);
        dyn[s].dt = (float)dt;
        dyn[s].dt_d = dt;
        if (advance) dyn[s].time += dt;
        dyn[s].amax2_bits = 0u;
    }
    if (threadIdx.x == 0 && dt_host > 0.0) st->dt_next = 0.0;
    if (threadIdx.x == 0 && advance) {
        st->steps += 1ull;
        if (rebuild_every > 1) {
            // skin list: rebuild when a particle has moved skin/4 (the predicted state of
            // the step then stays within skin/2: a CFL step moves less than 0.3 h) or after
            // rebuild_every steps
            const bool rb = st->since >= rebuild_every || __uint_as_float(st->maxdisp2_bits) > trig2;
            st->rebuild = rb ? 1u : 0u;
            st->since = rb ? 1u : st->since + 1u;
            if (rb) st->maxdisp2_bits = 0u;
            st->builds += rb ? 1u : 0u;
        } else {
            st->builds += builds_inc;
        }
    }
}

// the CFL dt the next step of scene 0 would take, without changing any state
__global__ void k_dt_peek(const SceneDev* __restrict__ scenes, const SceneDyn* __restrict__ dyn,
                          DevStatus* __restrict__ st, double h, double cfl, double dt_fixed) {
    if (threadIdx.x == 0) st->dt_peek = cfl_dt_of(scenes[0], dyn[0], h, cfl, dt_fixed);
}

__global__ void k_dt(const SceneDev* __restrict__ scenes, SceneDyn* __restrict__ dyn, DevStatus* __restrict__ st,
                     uint32_t n_scenes, double h, double cfl, double dt_fixed, int advance, uint32_t rebuild_every,
                     float trig2, uint32_t builds_inc) {
    dt_body(scenes, dyn, st, n_scenes, h, cfl, dt_fixed, advance, rebuild_every, trig2, builds_inc);
}

// ---------------------------------------------------------------------
// The neighbour build and the predictor pass in one kernel: each thread writes
// its particle's list (the thread-per-particle build) and evaluates the
// predictor pass over it at once, while the list and the candidates it has
// just loaded are in cache; no separate pass re-reads the list.  The same
// list and, pair for pair in the same order, the same sums and update as the
// two kernels.  List rebuilt every step (no skin), default model.
// ---------------------------------------------------------------------
template <int VISC>
__global__ void __launch_bounds__(kPipeBlock, 4) k_build_predict(const Buffers b, int cur, const Phys ph) {
    DevStatus* st = b.status;
    const uint32_t n = st->n_active;
    const uint32_t r2lim = __float_as_uint(ph.R2_list) - 1u;
    uint32_t npairs = 0;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        uint32_t nfound;
        const uint32_t nent = build_particle(i, b.pos[cur], b.cell[cur], b.pinfo[cur], b.start, b.cell_nfluid, b.scenes,
                                             b.nlist, b.ncount, r2lim, ph.max_neibs, ph.stride, &nfound, st, n);
        build_stats(st, nfound, nent, ph.max_neibs, __activemask());
        asm volatile("" ::: "memory");  // the list stores above precede its loads below
        const uint32_t cnt = ld_count_fresh(b.ncount + i);
        particle_pass<VISC, kPredict, false, true>(i, n, b.pos[cur], b.vel[cur], b.phat[cur], b.pos_s, b.vel_s,
                                                   b.phat_s, nullptr, b.pinfo[cur], b.nlist, b.ncount, b.scenes,
                                                   b.dyn, st, ph, 0, nullptr, nullptr, nullptr, b.pid[cur], npairs,
                                                   cnt);
    }
}

// ---------------------------------------------------------------------
// The whole step as one persistent kernel (batched scenes, north of the
// per-kernel graph): every block runs each phase of the step over its share
// of the particles (grid-stride loops), with a grid-wide barrier between
// phases, for nsteps steps.  A cooperative launch keeps every block resident,
// so the barriers always complete.  Phases and their arithmetic are the
// kernels of the captured step (dt, hash, scan, scatter, reorder,
// thread-per-particle list build, predictor pass, corrector pass), so the
// result is the same to the bit.  List rebuilt every step, default model.
// ---------------------------------------------------------------------
// 4 resident blocks of 256 threads per SM (64 registers): measured faster than 3 (80
// registers) and 2 (128): 12.5 / 13.9 / 16.3 ms per step on the 256-tank batch
constexpr int kPersistMinBlocks = 4;
template <int VISC>
__global__ void __launch_bounds__(kPipeBlock, kPersistMinBlocks) k_step_persistent(const Buffers b, const Geometry g, const Phys ph,
                                                                    int cur0, uint32_t nsteps) {
    cg::grid_group grid = cg::this_grid();
    const uint32_t nb = g.n_cells + 1;  // buckets: cells + the sentinel of removed particles
    const uint32_t ntiles = (nb + kScanTile - 1) / kScanTile;
    for (uint32_t s = 0; s < nsteps; ++s) {
        const int cur = (cur0 + (int)s) & 1, nxt = cur ^ 1;
        if (blockIdx.x == 0)
            dt_body(b.scenes, b.dyn, b.status, g.n_scenes, ph.h_d, ph.cfl, ph.dt_fixed, 1, ph.rebuild_every,
                    ph.skin_trig2, 1u);
        hash_body(b.pos[cur], b.cell[cur], b.pinfo[cur], b.scenes, b.status, b.key, b.slot, b.count, g.n_cells);
        grid.sync();
        for (uint32_t t = blockIdx.x; t < ntiles; t += gridDim.x) scan_reduce_tile(b.count, nb, b.bsum, t);
        grid.sync();
        if (blockIdx.x == 0) scan_bsums_body(b.bsum, ntiles);
        grid.sync();
        for (uint32_t t = blockIdx.x; t < ntiles; t += gridDim.x)
            scan_down_tile(b.count, nb, b.bsum, b.start, b.status, t);
        grid.sync();
        scatter_body(b.key, b.slot, b.start, b.status, b.unsorted, nb);
        grid.sync();
        reorder_body(b.pos[cur], b.vel[cur], b.phat[cur], b.pinfo[cur], b.pid[cur], b.start, b.unsorted, b.scenes,
                     g.n_cells, b.status, b.cell_nfluid, b.pos[nxt], b.vel[nxt], b.phat[nxt], b.cell[nxt],
                     b.pinfo[nxt], b.pid[nxt]);
        grid.sync();
        build_tpp_body(b.pos[nxt], b.cell[nxt], b.pinfo[nxt], b.start, b.cell_nfluid, b.scenes, b.status, b.nlist,
                       b.ncount, ph.R2_list, ph.max_neibs, ph.stride);
        grid.sync();
        forces_body<VISC, kPredict, false>(b.pos[nxt], b.vel[nxt], b.phat[nxt], b.pos_s, b.vel_s, b.phat_s, nullptr,
                                           b.pinfo[nxt], b.nlist, b.ncount, b.scenes, b.dyn, b.status, ph, 0,
                                           nullptr, nullptr, nullptr, b.pid[nxt]);
        grid.sync();
        forces_body<VISC, kCorrect, false>(b.pos_s, b.vel_s, b.phat_s, b.pos[nxt], b.vel[nxt], b.phat[nxt], nullptr,
                                           b.pinfo[nxt], b.nlist, b.ncount, b.scenes, b.dyn, b.status, ph, 0,
                                           nullptr, nullptr, nullptr, b.pid[nxt]);
        grid.sync();
    }
}

template <int VISC, int B, int MB, bool SKIN>
void launch_forces_s(const Buffers& b, int cur, const Geometry& g, const Phys& ph, ForceMode mode, int acc_dt,
                     cudaStream_t st) {
    const unsigned grid = g.cap ? (g.cap + B - 1) / B : 1;
    switch (mode) {
        case kForcesOnly:
            k_forces<VISC, kForcesOnly, B, MB, SKIN><<<grid, B, 0, st>>>(
                b.pos[cur], b.vel[cur], b.phat[cur], nullptr, nullptr, nullptr, b.force, b.pinfo[cur], b.nlist,
                b.ncount, b.scenes, b.dyn, b.status, ph, acc_dt, nullptr, nullptr, nullptr, b.pid[cur]);
            break;
        case kPredict:
            k_forces<VISC, kPredict, B, MB, SKIN><<<grid, B, 0, st>>>(
                b.pos[cur], b.vel[cur], b.phat[cur], b.pos_s, b.vel_s, b.phat_s, nullptr, b.pinfo[cur], b.nlist,
                b.ncount, b.scenes, b.dyn, b.status, ph, 0, nullptr, b.nlist_x, b.ncount_x, b.pid[cur]);
            break;
        case kCorrect:  // a skin list: the exact list the predictor wrote
            k_forces<VISC, kCorrect, B, MB, SKIN><<<grid, B, 0, st>>>(
                b.pos_s, b.vel_s, b.phat_s, b.pos[cur], b.vel[cur], b.phat[cur], nullptr, b.pinfo[cur],
                SKIN ? b.nlist_x : b.nlist, SKIN ? b.ncount_x : b.ncount, b.scenes, b.dyn, b.status, ph, 0,
                b.pos_ref, nullptr, nullptr, b.pid[cur]);
            break;
    }
}

template <int VISC, int B, int MB>
void launch_forces_b(const Buffers& b, int cur, const Geometry& g, const Phys& ph, ForceMode mode, int acc_dt,
                     cudaStream_t st, bool skin) {
    if (skin)
        launch_forces_s<VISC, B, MB, true>(b, cur, g, ph, mode, acc_dt, st);
    else
        launch_forces_s<VISC, B, MB, false>(b, cur, g, ph, mode, acc_dt, st);
}

// launch shapes of the force kernels (autotuned, the corrector pass on its own):
// threads per block and the register cap implied by a minimum of resident blocks per SM
template <int VISC>
void launch_forces_v(const Buffers& b, int cur, const Geometry& g, const Phys& ph, ForceMode mode, int acc_dt,
                     cudaStream_t st, bool skin) {
    switch (mode == kCorrect ? ph.forces_variant_c : ph.forces_variant) {
        case 0: launch_forces_b<VISC, 64, 16>(b, cur, g, ph, mode, acc_dt, st, skin); break;
        case 2: launch_forces_b<VISC, 256, 4>(b, cur, g, ph, mode, acc_dt, st, skin); break;
        case 3: launch_forces_b<VISC, 128, 6>(b, cur, g, ph, mode, acc_dt, st, skin); break;
        case 4: launch_forces_b<VISC, 128, 4>(b, cur, g, ph, mode, acc_dt, st, skin); break;
        default: launch_forces_b<VISC, 128, 8>(b, cur, g, ph, mode, acc_dt, st, skin); break;
    }
}

// Conservation sums (Section 2.1 invariants) over particles: momentum sum m u,
// force sum m a, sum m drho/dt, kinetic energy, total mass; |m| (boundary masses
// are stored negated).  Deterministic: a fixed grid, a fixed particle order per thread and
// fixed-order tree reductions in FP64 (per block, then over blocks).
constexpr int kConsBlocks = 304, kConsThreads = 256, kConsQ = kConservationSums;

__global__ void __launch_bounds__(kConsThreads) k_cons_partial(const float4* __restrict__ pos,
                                                               const float4* __restrict__ vel,
                                                               const float4* __restrict__ force,
                                                               const DevStatus* __restrict__ st,
                                                               double* __restrict__ part) {
    __shared__ double red[kConsQ][kConsThreads];
    double q[kConsQ] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    const uint32_t n = st->n_active;
    for (uint32_t i = blockIdx.x * kConsThreads + threadIdx.x; i < n; i += kConsBlocks * kConsThreads) {
        const double m = fabs((double)pos[i].w);
        const float4 v = vel[i], a = force[i];
        const bool fluid = pos[i].w > 0.f;
        const double ux = fluid ? v.x : 0.0, uy = fluid ? v.y : 0.0, uz = fluid ? v.z : 0.0;
        q[0] += m * ux;
        q[1] += m * uy;
        q[2] += m * uz;
        q[3] += m * a.x;
        q[4] += m * a.y;
        q[5] += m * a.z;
        q[6] += m * a.w;
        q[7] += 0.5 * m * (ux * ux + uy * uy + uz * uz);
        q[8] += m;
    }
#pragma unroll
    for (int k = 0; k < kConsQ; ++k) red[k][threadIdx.x] = q[k];
    __syncthreads();
    for (int w = kConsThreads / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w)
#pragma unroll
            for (int k = 0; k < kConsQ; ++k) red[k][threadIdx.x] += red[k][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x < kConsQ) part[blockIdx.x * kConsQ + threadIdx.x] = red[threadIdx.x][0];
}

__global__ void k_cons_final(const double* __restrict__ part, double* __restrict__ out) {
    if (threadIdx.x < kConsQ) {
        double s = 0.0;
        for (int b = 0; b < kConsBlocks; ++b) s += part[b * kConsQ + threadIdx.x];
        out[threadIdx.x] = s;
    }
}

}  // namespace

size_t conservation_scratch_bytes() { return sizeof(double) * kConsQ * (kConsBlocks + 1); }

void launch_conservation(const Buffers& b, int cur, double* scratch, cudaStream_t st) {
    k_cons_partial<<<kConsBlocks, kConsThreads, 0, st>>>(b.pos[cur], b.vel[cur], b.force, b.status, scratch);
    k_cons_final<<<1, 32, 0, st>>>(scratch, scratch + kConsQ * kConsBlocks);
}

void launch_forces(const Buffers& b, int cur, const Geometry& g, const Phys& ph, ForceMode mode, int acc_dt,
                   cudaStream_t st) {
    if (ph.general) {
        launch_forces_models(b, cur, g, ph, mode, acc_dt, st);
        return;
    }
    const bool skin = b.pos_ref != nullptr;
    if (ph.visc == SPH_VISC_LAMINAR)
        launch_forces_v<SPH_VISC_LAMINAR>(b, cur, g, ph, mode, acc_dt, st, skin);
    else
        launch_forces_v<SPH_VISC_ARTIFICIAL>(b, cur, g, ph, mode, acc_dt, st, skin);
}

const char* forces_variant_name(int v) {
    static const char* names[kForcesVariants] = {"64 threads, <=64 regs", "128 threads, <=64 regs",
                                                 "256 threads, <=64 regs", "128 threads, <=85 regs",
                                                 "128 threads, <=128 regs"};
    return v >= 0 && v < kForcesVariants ? names[v] : "?";
}

void launch_dt(const Buffers& b, const Geometry& g, const Phys& ph, int advance_time, cudaStream_t st,
               int with_build) {
    k_dt<<<1, 256, 0, st>>>(b.scenes, b.dyn, b.status, g.n_scenes, ph.h_d, ph.cfl, ph.dt_fixed, advance_time,
                            ph.rebuild_every, ph.skin_trig2, with_build ? 1u : 0u);
}

// blocks of the persistent step kernel: all resident (a cooperative launch refuses more)
template <int VISC>
int persistent_grid() {
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_step_persistent<VISC>, kPipeBlock, 0) != cudaSuccess)
        return 0;
    return sms * per_sm;
}

cudaError_t launch_step_persistent(const Buffers& b, int cur, const Geometry& g, const Phys& ph, uint32_t nsteps,
                                   cudaStream_t st) {
    const bool lam = ph.visc == SPH_VISC_LAMINAR;
    const int grid = lam ? persistent_grid<SPH_VISC_LAMINAR>() : persistent_grid<SPH_VISC_ARTIFICIAL>();
    if (grid <= 0) return cudaErrorLaunchFailure;
    Buffers bb = b;
    Geometry gg = g;
    Phys pp = ph;
    int c0 = cur;
    uint32_t ns = nsteps;
    void* args[] = {&bb, &gg, &pp, &c0, &ns};
    const void* fn = lam ? (const void*)k_step_persistent<SPH_VISC_LAMINAR>
                         : (const void*)k_step_persistent<SPH_VISC_ARTIFICIAL>;
    return cudaLaunchCooperativeKernel(fn, dim3((unsigned)grid), dim3(kPipeBlock), args, 0, st);
}

void launch_build_predict(const Buffers& b, int cur, const Geometry& g, const Phys& ph, cudaStream_t st) {
    const unsigned grid = g.cap ? (g.cap + kPipeBlock - 1) / kPipeBlock : 1;
    if (ph.visc == SPH_VISC_LAMINAR)
        k_build_predict<SPH_VISC_LAMINAR><<<grid, kPipeBlock, 0, st>>>(b, cur, ph);
    else
        k_build_predict<SPH_VISC_ARTIFICIAL><<<grid, kPipeBlock, 0, st>>>(b, cur, ph);
}

void launch_dt_peek(const Buffers& b, const Phys& ph, cudaStream_t st) {
    k_dt_peek<<<1, 32, 0, st>>>(b.scenes, b.dyn, b.status, ph.h_d, ph.cfl, ph.dt_fixed);
}

void launch_predict_from_forces(const Buffers& b, int cur, const Geometry& g, const Phys& ph, cudaStream_t st) {
    const unsigned grid = g.cap ? (g.cap + 255) / 256 : 1;
    k_predict_from_forces<<<grid, 256, 0, st>>>(b.pos[cur], b.vel[cur], b.force, b.pinfo[cur], b.scenes, b.dyn,
                                                b.status, ph, b.pos_s, b.vel_s, b.phat_s);
}

}  // namespace sphg
