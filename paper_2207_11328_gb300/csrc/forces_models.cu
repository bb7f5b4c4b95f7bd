// Interaction kernels for the model options of Table 1 beyond the default
// (Wendland C2, formulation 1, artificial or Morris/harmonic viscosity, no
// density diffusion, which forces.cu runs with tuned launch shapes):
//
//   kernels (kernel-templates listing, Section 4), F = aF f(q):
//     Wendland (q-2)^3; cubic spline -3 + 9/4 q (q<1), -3/4 (2-q)^2/q (q<2);
//     quadratic (q-2)/q; Gaussian -exp(-q^2) cut at the influence radius
//   formulation 2 (Section 2.1, readings C1/C2):
//     drho_i = sum_j (rho_i/rho_j) m_j u_ij.x_ij F,  pressure (P_i+P_j)/(rho_i rho_j)
//     = phat_i rho_i/rho_j + phat_j rho_j/rho_i with phat = P/rho^2
//   laminar viscous models (Section 3), omega = m_j/(rho_i rho_j), mubar the
//   average (harmonic, arithmetic, geometric) of rho nu:
//     Morris            omega 2 mubar F u_ij
//     Monaghan          5 omega 2 mubar F (u.x/r^2) x_ij
//     Espanol-Revenga   omega F ((5/3 mubar - zetabar) u_ij + 5 (mubar/3 + zetabar)(u.x/r^2) x_ij)
//     all written as (lam_u u_ij + lam_x (u.x/r^2) x_ij) m_j f avg(r_i, r_j)/(r_i r_j)
//     with r = rho/rho0 = 1 + delta and lam_* carrying nu, zeta and 1/rho0
//   density diffusion, Molteni & Colagrossi (reading D1, fluid pairs):
//     drho_i += 2 xi h c0 sum_j (rho_i - rho_j) F m_j/rho_j = dd_coef (delta_i - delta_j) m_j F / r_j
//
// Same structure as the tuned kernels: one thread per particle, split
// neighbour list read four entries (two chunks) ahead, aF applied once per particle, the
// predictor/corrector epilogue of forces_common.cuh.  The kernel and the
// viscous model are template parameters; formulation, averaging, diffusion
// and the skin list are uniform run-time switches.
#include "forces_common.cuh"

namespace sphg {

namespace {

constexpr int kModelBlock = 128;

// f(q) of F = aF f(q) for a listed pair (r below the list radius)
template <int KT>
__device__ __forceinline__ float kernel_shape(float r2, float rinv, const Phys& ph) {
    const float q = r2 * rinv * ph.inv_h;
    if (KT == SPH_KERNEL_WENDLAND) {
        const float t = fminf(q - 2.0f, 0.0f);
        return t * t * t;
    }
    if (KT == SPH_KERNEL_CUBIC_SPLINE) {
        if (q < 1.0f) return fmaf(2.25f, q, -3.0f);
        const float t = fmaxf(2.0f - q, 0.0f);
        return -0.75f * t * t * (ph.h * rinv);  // 1/q = h/r
    }
    if (KT == SPH_KERNEL_QUADRATIC) return fminf(q - 2.0f, 0.0f) * (ph.h * rinv);
    return -expf(-(q * q));  // Gaussian
}

// avg(r_i, r_j)/(r_i r_j) for the laminar viscosity
__device__ __forceinline__ float visc_weight(int op, float ri, float rj) {
    if (op == SPH_AVG_ARITHMETIC) return __fdividef(0.5f * (ri + rj), ri * rj);
    if (op == SPH_AVG_GEOMETRIC) return rsqrtf(ri * rj);
    return __fdividef(2.0f, ri + rj);
}

// one neighbour of a fluid particle (BND: boundary neighbour, negated mass, u_j = 0)
// (filter: skin list, skip pairs beyond the cutoff and count the rest; returns
// whether the pair is within it)
template <int KT, int VISC, bool BND>
__device__ __forceinline__ bool model_pair(uint32_t e, const Central& ci, const float4& vi, float phat_i, float ri,
                                           const float4* __restrict__ pos, const float4* __restrict__ vel,
                                           const float* __restrict__ phat, float pi_coef, float dd_coef,
                                           const Phys& ph, bool filter, Acc& acc, uint32_t& npairs) {
    const uint32_t j = e >> kCodeBits;
    const float4 pj = pos[j];
    const float4 vj = vel[j];
    const float phat_j = phat[j];
    const float rx = pick(e, ci.xm, ci.x0, ci.xp) - pj.x;
    const float ry = pick(e >> 2, ci.ym, ci.y0, ci.yp) - pj.y;
    const float rz = pick(e >> 4, ci.zm, ci.z0, ci.zp) - pj.z;
    const float r2 = fmaxf(fmaf(rx, rx, fmaf(ry, ry, rz * rz)), 1e-30f);
    if (filter) {
        if (!(r2 < ph.R2)) return false;
        ++npairs;
    }
    const float rinv = rsqrtf(r2);
    const float mF = (BND ? -pj.w : pj.w) * kernel_shape<KT>(r2, rinv, ph);  // m_j F / aF
    const float rj = 1.0f + vj.w;
    const float ux = BND ? vi.x : vi.x - vj.x;
    const float uy = BND ? vi.y : vi.y - vj.y;
    const float uz = BND ? vi.z : vi.z - vj.z;
    const float udx = fmaf(ux, rx, fmaf(uy, ry, uz * rz));
    const bool form2 = ph.form == SPH_FORM_2;
    const float rij = form2 ? __fdividef(ri, rj) : 1.0f;  // rho_i/rho_j
    acc.drho = fmaf(mF * rij, udx, acc.drho);
    if (!BND && ph.ddiff == SPH_DDIFF_MOLTENI)
        acc.drho = fmaf(dd_coef * (vi.w - vj.w), __fdividef(mF, rj), acc.drho);
    float bracket = form2 ? fmaf(phat_i, rij, __fdividef(phat_j, rij)) : phat_i + phat_j;
    if (VISC == SPH_VISC_ARTIFICIAL) {
        // approaching pairs only (u.x < 0), without a branch: receding pairs add -pi*0
        const float den = (r2 + ph.eps_h2) * fmaf(0.5f, vi.w + vj.w, 1.0f);
        bracket = fmaf(-pi_coef, __fdividef(fminf(udx, 0.f), den), bracket);
    }
    const float coef = mF * bracket;
    acc.ax = fmaf(-coef, rx, acc.ax);
    acc.ay = fmaf(-coef, ry, acc.ay);
    acc.az = fmaf(-coef, rz, acc.az);
    if (VISC != SPH_VISC_ARTIFICIAL) {
        const float w = mF * visc_weight(ph.visc_avg, ri, rj);
        if (VISC == SPH_VISC_MORRIS || VISC == SPH_VISC_ESPANOL_REVENGA) {
            const float lu = ph.lam_u * w;
            acc.ax = fmaf(lu, ux, acc.ax);
            acc.ay = fmaf(lu, uy, acc.ay);
            acc.az = fmaf(lu, uz, acc.az);
        }
        if (VISC == SPH_VISC_MONAGHAN || VISC == SPH_VISC_ESPANOL_REVENGA) {
            const float lx = ph.lam_x * w * udx * (rinv * rinv);
            acc.ax = fmaf(lx, rx, acc.ax);
            acc.ay = fmaf(lx, ry, acc.ay);
            acc.az = fmaf(lx, rz, acc.az);
        }
    }
    return true;
}

template <int KT, int VISC, int MODE>
__global__ void __launch_bounds__(kModelBlock, 4) k_forces_m(
    const float4* __restrict__ pos, const float4* __restrict__ vel, const float* __restrict__ phat,
    float4* io_pos, float4* io_vel, float* io_phat, float4* __restrict__ force_out,
    const uint32_t* __restrict__ pinfo, const uint32_t* __restrict__ nlist, const uint32_t* __restrict__ ncount,
    const SceneDev* __restrict__ scenes, SceneDyn* __restrict__ dyn, DevStatus* __restrict__ st, const Phys ph,
    int acc_dt, int skin, const float4* __restrict__ pos_ref, uint32_t* __restrict__ nlist_x,
    uint32_t* __restrict__ ncount_x, const uint32_t* __restrict__ pid) {
    // skin list: the predictor (and sph_forces) filter by the cutoff; the predictor keeps the
    // pairs within it (the step's exact list) for the corrector, which reads that list as is
    const bool filter = skin && MODE != kCorrect;
    const bool compact = skin && MODE == kPredict;
    const bool chunked = skin && MODE == kCorrect;  // nlist/ncount: that exact list, in chunks of four
    const uint32_t n = st->n_active;
    uint32_t npairs = 0;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const uint32_t s = pinfo[i];
        const SceneDev& sc = scenes[s];
        const float4 pi = pos[i];
        const float4 vi = vel[i];
        const uint32_t cnt = ncount[i];
        uint32_t nf = cnt & 0xffffu, nb = cnt >> 16;
        SPH_GUARD(nf + nb <= ph.max_neibs, st, nf = nb = 0)
        const bool fluid_i = pi.w > 0.f;
        const Central ci = central_of(pi, sc.cell_f[0], sc.cell_f[1], sc.cell_f[2]);
        const float ri = 1.0f + vi.w;
        const size_t S = ph.stride;
        Acc acc{0.f, 0.f, 0.f, 0.f};
        const uint32_t kxb = exact_bnd_chunk(ph.max_neibs);
        ChunkWriter xf{make_uint4(0u, 0u, 0u, 0u), 0u, reinterpret_cast<uint4*>(nlist_x), S, i};
        ChunkWriter xb{make_uint4(0u, 0u, 0u, 0u), 0u, reinterpret_cast<uint4*>(nlist_x) + (size_t)kxb * S, S, i};
        // entry k of the fluid / boundary part: the list of the build (two-entry
        // chunks, boundary part from the back) or, in the skin-list corrector, the
        // step's exact list (four-entry chunks, boundary part from chunk kxb)
        auto fluid_entry = [&](uint32_t k) -> uint32_t {
            return chunked ? __ldg(nlist + ((size_t)(k >> 2) * S + i) * 4 + (k & 3u))
                           : __ldg(nlist + list_fluid_word(k, i, S));
        };
        auto bnd_entry = [&](uint32_t k) -> uint32_t {
            return chunked ? __ldg(nlist + ((size_t)(kxb + (k >> 2)) * S + i) * 4 + (k & 3u))
                           : __ldg(nlist + list_bnd_word(k, i, S, ph.max_neibs));
        };
        if (fluid_i) {
            const float phat_i = phat[i];
            const float pic = sc.pi_coef, ddc = sc.dd_coef;
            uint32_t k = 0;
#define SPH_KEEP_F(e) if (compact) xf.put(e);
#define SPH_KEEP_B(e) if (compact) xb.put(e);
            for (; k + 4 <= nf; k += 4) {
                uint32_t e0, e1, e2, e3;
                if (chunked) {
                    const uint4 q = __ldg(reinterpret_cast<const uint4*>(nlist) + (size_t)(k >> 2) * S + i);
                    e0 = q.x;
                    e1 = q.y;
                    e2 = q.z;
                    e3 = q.w;
                } else {
                    const uint2* lp = reinterpret_cast<const uint2*>(nlist) + (size_t)(k >> 1) * S + i;
                    const uint2 a = __ldg(lp), b = __ldg(lp + S);
                    e0 = a.x;
                    e1 = a.y;
                    e2 = b.x;
                    e3 = b.y;
                }
                SPH_GUARD((max(max(e0, e1), max(e2, e3)) >> kCodeBits) < n, st, break)
                if (model_pair<KT, VISC, false>(e0, ci, vi, phat_i, ri, pos, vel, phat, pic, ddc, ph, filter, acc, npairs)) SPH_KEEP_F(e0)
                if (model_pair<KT, VISC, false>(e1, ci, vi, phat_i, ri, pos, vel, phat, pic, ddc, ph, filter, acc, npairs)) SPH_KEEP_F(e1)
                if (model_pair<KT, VISC, false>(e2, ci, vi, phat_i, ri, pos, vel, phat, pic, ddc, ph, filter, acc, npairs)) SPH_KEEP_F(e2)
                if (model_pair<KT, VISC, false>(e3, ci, vi, phat_i, ri, pos, vel, phat, pic, ddc, ph, filter, acc, npairs)) SPH_KEEP_F(e3)
            }
            for (; k < nf; ++k) {
                const uint32_t e = fluid_entry(k);
                SPH_GUARD((e >> kCodeBits) < n, st, continue)
                if (model_pair<KT, VISC, false>(e, ci, vi, phat_i, ri, pos, vel, phat, pic, ddc, ph, filter, acc, npairs)) SPH_KEEP_F(e)
            }
            for (k = 0; k < nb; ++k) {
                const uint32_t e = bnd_entry(k);
                SPH_GUARD((e >> kCodeBits) < n, st, continue)
                if (model_pair<KT, VISC, true>(e, ci, vi, phat_i, ri, pos, vel, phat, pic, ddc, ph, filter, acc, npairs)) SPH_KEEP_B(e)
            }
            acc.ax = fmaf(ph.aF, acc.ax, ph.g[0]);
            acc.ay = fmaf(ph.aF, acc.ay, ph.g[1]);
            acc.az = fmaf(ph.aF, acc.az, ph.g[2]);
            acc.drho *= ph.aF;
        } else {
            // boundary particle: continuity over its fluid neighbours, u_i = 0
            const bool form2 = ph.form == SPH_FORM_2;
#pragma unroll 2
            for (uint32_t k = 0; k < nf; ++k) {
                const uint32_t e = fluid_entry(k);
                const uint32_t j = e >> kCodeBits;
                SPH_GUARD(j < n, st, continue)
                const float4 pj = pos[j];
                const float4 vj = vel[j];
                const float rx = pick(e, ci.xm, ci.x0, ci.xp) - pj.x;
                const float ry = pick(e >> 2, ci.ym, ci.y0, ci.yp) - pj.y;
                const float rz = pick(e >> 4, ci.zm, ci.z0, ci.zp) - pj.z;
                const float r2 = fmaxf(fmaf(rx, rx, fmaf(ry, ry, rz * rz)), 1e-30f);
                if (filter) {
                    if (!(r2 < ph.R2)) continue;
                    ++npairs;
                }
                SPH_KEEP_F(e)
                float mF = pj.w * kernel_shape<KT>(r2, rsqrtf(r2), ph);
                if (form2) mF *= __fdividef(ri, 1.0f + vj.w);
                const float udx = -fmaf(vj.x, rx, fmaf(vj.y, ry, vj.z * rz));
                acc.drho = fmaf(mF, udx, acc.drho);
            }
            acc.drho *= ph.aF;
        }
#undef SPH_KEEP_F
#undef SPH_KEEP_B
        if (compact) {
            xf.flush();
            xb.flush();
            ncount_x[i] = xf.n | (xb.n << 16);
        }
        finish_particle<MODE>(i, s, sc, pi, vi, fluid_i, acc, io_pos, io_vel, io_phat, force_out, dyn, st, ph,
                              acc_dt, pos_ref, pid);
    }
    if (compact) {
        const uint32_t w = __reduce_add_sync(0xffffffffu, npairs);
        if ((threadIdx.x & 31) == 0 && w) atomicAdd(&st->interactions, (unsigned long long)w);
    }
}

template <int KT, int VISC>
void launch_m(const Buffers& b, int cur, const Geometry& g, const Phys& ph, ForceMode mode, int acc_dt,
              cudaStream_t st) {
    const unsigned grid = g.cap ? (g.cap + kModelBlock - 1) / kModelBlock : 1;
    const int skin = b.pos_ref != nullptr;
    switch (mode) {
        case kForcesOnly:
            k_forces_m<KT, VISC, kForcesOnly><<<grid, kModelBlock, 0, st>>>(
                b.pos[cur], b.vel[cur], b.phat[cur], nullptr, nullptr, nullptr, b.force, b.pinfo[cur], b.nlist,
                b.ncount, b.scenes, b.dyn, b.status, ph, acc_dt, skin, nullptr, nullptr, nullptr, b.pid[cur]);
            break;
        case kPredict:
            k_forces_m<KT, VISC, kPredict><<<grid, kModelBlock, 0, st>>>(
                b.pos[cur], b.vel[cur], b.phat[cur], b.pos_s, b.vel_s, b.phat_s, nullptr, b.pinfo[cur], b.nlist,
                b.ncount, b.scenes, b.dyn, b.status, ph, 0, skin, nullptr, b.nlist_x, b.ncount_x, b.pid[cur]);
            break;
        case kCorrect:
            k_forces_m<KT, VISC, kCorrect><<<grid, kModelBlock, 0, st>>>(  // a skin list: the predictor's exact list
                b.pos_s, b.vel_s, b.phat_s, b.pos[cur], b.vel[cur], b.phat[cur], nullptr, b.pinfo[cur],
                skin ? b.nlist_x : b.nlist, skin ? b.ncount_x : b.ncount, b.scenes, b.dyn, b.status, ph, 0, skin,
                b.pos_ref, nullptr, nullptr, b.pid[cur]);
            break;
    }
}

template <int KT>
void launch_k(const Buffers& b, int cur, const Geometry& g, const Phys& ph, ForceMode mode, int acc_dt,
              cudaStream_t st) {
    switch (ph.visc) {
        case SPH_VISC_MORRIS: launch_m<KT, SPH_VISC_MORRIS>(b, cur, g, ph, mode, acc_dt, st); break;
        case SPH_VISC_MONAGHAN: launch_m<KT, SPH_VISC_MONAGHAN>(b, cur, g, ph, mode, acc_dt, st); break;
        case SPH_VISC_ESPANOL_REVENGA: launch_m<KT, SPH_VISC_ESPANOL_REVENGA>(b, cur, g, ph, mode, acc_dt, st); break;
        default: launch_m<KT, SPH_VISC_ARTIFICIAL>(b, cur, g, ph, mode, acc_dt, st); break;
    }
}

}  // namespace

void launch_forces_models(const Buffers& b, int cur, const Geometry& g, const Phys& ph, ForceMode mode, int acc_dt,
                          cudaStream_t st) {
    switch (ph.kernel_type) {
        case SPH_KERNEL_CUBIC_SPLINE: launch_k<SPH_KERNEL_CUBIC_SPLINE>(b, cur, g, ph, mode, acc_dt, st); break;
        case SPH_KERNEL_QUADRATIC: launch_k<SPH_KERNEL_QUADRATIC>(b, cur, g, ph, mode, acc_dt, st); break;
        case SPH_KERNEL_GAUSSIAN: launch_k<SPH_KERNEL_GAUSSIAN>(b, cur, g, ph, mode, acc_dt, st); break;
        default: launch_k<SPH_KERNEL_WENDLAND>(b, cur, g, ph, mode, acc_dt, st); break;
    }
}

}  // namespace sphg
