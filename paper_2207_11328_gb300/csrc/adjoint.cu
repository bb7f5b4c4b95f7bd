// Hand-written adjoint of one predictor-corrector step (reverse mode).
//
// Forward step (reading C6), neighbour list L_n fixed within the step:
//   (a, drho)   = f(x, u, delta)                      forces at n
//   u* = u + h a,  delta* = delta + h drho/rho0,  x* = x + h u     (h = dt/2)
//   (a*, drho*) = f(x*, u*, delta*)                   forces at *
//   u' = u + dt a*,  delta' = delta + dt drho*/rho0,  x' = x + (dt/2)(u + u')
// Boundary particles integrate delta only; their x and u are constants.
//
// The vector-Jacobian product of f is a gather over each particle's own
// neighbour list: particle k adds the derivatives of its own pair terms
// T_kj (seeded with its own adjoints) and of its neighbours' terms T_jk
// (seeded with the neighbours' adjoints), which the symmetric list makes
// available without atomics, so the adjoint is deterministic.  The viscosity
// switch u_ij.x_ij < 0 is taken on the primal value, as the forward does.
//
// Adjoint layout per particle, sorted order of the step:
//   xb4 = (xbar, deltabar), ub4 = (ubar, alphabar partial), seed4 = (abar, drhobar).
#include "sph_internal.cuh"

namespace sphg {

namespace {

constexpr int kBlock = 128;

__device__ __forceinline__ float cell_delta(uint32_t bits2, float cell) {
    return bits2 == 0u ? -cell : (bits2 == 2u ? cell : 0.0f);
}

// d(P/rho^2)/d delta = phat_coef * [gamma (1+d)^(gamma-3) - 2 ((1+d)^gamma - 1)/(1+d)^3]
__device__ __forceinline__ float eos_dphat(float d, const Phys& ph, float phat_coef) {
    const float opd = 1.0f + d;
    float pw = 1.0f;  // (1+d)^gamma
    for (int k = 0; k < ph.gamma_i; ++k) pw *= opd;
    const float inv = 1.0f / opd;
    const float g = (float)ph.gamma_i;
    return phat_coef * (g * pw * inv * inv * inv - 2.0f * (pw - 1.0f) * inv * inv * inv);
}

// user layout (n*3, n floats; NULL = zero) <-> id-space float4 adjoints
__global__ void k_adj_load(uint32_t n, const float* __restrict__ xbar, const float* __restrict__ ubar,
                           const float* __restrict__ dbar, float4* __restrict__ xb_id, float4* __restrict__ ub_id) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        xb_id[i] = xbar ? make_float4(xbar[3 * (size_t)i], xbar[3 * (size_t)i + 1], xbar[3 * (size_t)i + 2], 0.f)
                        : make_float4(0.f, 0.f, 0.f, 0.f);
        if (dbar) xb_id[i].w = dbar[i];
        ub_id[i] = ubar ? make_float4(ubar[3 * (size_t)i], ubar[3 * (size_t)i + 1], ubar[3 * (size_t)i + 2], 0.f)
                        : make_float4(0.f, 0.f, 0.f, 0.f);
    }
}

__global__ void k_adj_store(uint32_t n, const float4* __restrict__ xb_id, const float4* __restrict__ ub_id,
                            float* __restrict__ xbar, float* __restrict__ ubar, float* __restrict__ dbar) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float4 x = xb_id[i], u = ub_id[i];
        if (xbar) {
            xbar[3 * (size_t)i] = x.x;
            xbar[3 * (size_t)i + 1] = x.y;
            xbar[3 * (size_t)i + 2] = x.z;
        }
        if (ubar) {
            ubar[3 * (size_t)i] = u.x;
            ubar[3 * (size_t)i + 1] = u.y;
            ubar[3 * (size_t)i + 2] = u.z;
        }
        if (dbar) dbar[i] = x.w;
    }
}

// Start of one reversed step, per particle (sorted order of the step):
//   d(P/rho^2)/d delta at n and at *; the adjoint of state n+1 gathered from id
//   space; reverse of the corrector: the seeds of the VJP at * and the partial
//   adjoint of state n.
//   x' = x + dt/2 (u + u'), u' = u + dt a*, delta' = delta + dt drho*/rho0:
//   u'bar_tot = u'bar + dt/2 x'bar;  ubar_n = u'bar_tot + dt/2 x'bar;
//   seeds at *: abar = dt u'bar_tot, drhobar = dt/rho0 delta'bar.
__global__ void k_adj_pre(const float4* __restrict__ pos, const float4* __restrict__ vel,
                          const float4* __restrict__ vel_s, const uint32_t* __restrict__ pinfo,
                          const uint32_t* __restrict__ pid, const SceneDev* __restrict__ scenes,
                          const DevStatus* __restrict__ st, const Phys ph, float dt,
                          const float4* __restrict__ xb_id, const float4* __restrict__ ub_id,
                          float* __restrict__ dphat, float* __restrict__ dphat_s, float4* __restrict__ xb,
                          float4* __restrict__ ub, float4* __restrict__ seed) {
    const uint32_t n = st->n_active;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float c = scenes[pinfo[i]].phat_coef;
        dphat[i] = eos_dphat(vel[i].w, ph, c);
        dphat_s[i] = eos_dphat(vel_s[i].w, ph, c);
        const uint32_t id = pid[i];
        const bool fluid = pos[i].w > 0.f;
        float4 x = xb_id[id], u = ub_id[id];
        const float dbar = x.w;
        float4 sd = make_float4(0.f, 0.f, 0.f, dt * ph.inv_rho0 * dbar);
        if (fluid) {
            const float hx = 0.5f * dt * x.x, hy = 0.5f * dt * x.y, hz = 0.5f * dt * x.z;
            const float tx = u.x + hx, ty = u.y + hy, tz = u.z + hz;
            sd.x = dt * tx;
            sd.y = dt * ty;
            sd.z = dt * tz;
            u.x = tx + hx;
            u.y = ty + hy;
            u.z = tz + hz;
        } else {
            x.x = x.y = x.z = 0.f;
            u.x = u.y = u.z = 0.f;
        }
        xb[i] = x;  // xbar_n = x'bar, deltabar_n = delta'bar
        ub[i] = u;
        seed[i] = sd;
    }
}

// Tape copies: n elements of each of `count` arrays (16- or 4-byte elements)
// between the particle buffers and a flat tape block, one launch per copy.
struct TapeCopy {
    const void* src[kTapeArrays];
    void* dst[kTapeArrays];
    uint32_t wide;  // bit k: array k has 16-byte elements
    int count;
};

__global__ void k_tape_copy(const TapeCopy tc, uint32_t n) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
#pragma unroll
        for (int k = 0; k < kTapeArrays; ++k) {
            if (k >= tc.count) break;
            if ((tc.wide >> k) & 1u)
                static_cast<float4*>(tc.dst[k])[i] = static_cast<const float4*>(tc.src[k])[i];
            else
                static_cast<uint32_t*>(tc.dst[k])[i] = static_cast<const uint32_t*>(tc.src[k])[i];
        }
    }
}

// Both terms of pair (k, j) that the VJP of particle k needs, evaluated together:
// its own term T_kj seeded with k's adjoints (abar_k, drhobar_k) and the
// neighbour's term T_jk seeded with j's.  Everything that depends on the pair
// alone (r, F, F'/r, u.x, the viscosity switch and its derivatives) is
// symmetric and computed once: x_jk = -x_kj and u_jk = -u_kj leave u.x, r and
// Pi unchanged and flip the odd derivatives.  Returns the derivative of
// S_kj + S_jk w.r.t. x_k, u_k and delta_k, and of S_kj w.r.t. alpha (T_jk's
// alpha derivative belongs to particle j).  Same sums as two calls of
// pair_grad (own term plus the neighbour's term, transposed).
struct PairIn2 {
    float rx, ry, rz, r2;   // x_kj
    float ux, uy, uz;       // u_kj
    float dk, dj;           // delta_k, delta_j
    float phk, phj, dphk;   // P/rho^2 of k and j, d(P/rho^2)/d delta of k
    float mj, mk;
    float3 Ak, Aj;          // abar of k and j
    float rbk, rbj;         // drhobar of k and j
};

struct PairGrad2 {
    float gx, gy, gz, gux, guy, guz, gd, ga;
};

template <int VISC>
__device__ __forceinline__ PairGrad2 pair_grad2(const PairIn2& p, const Phys& ph, float pic, float pic_unit) {
    PairGrad2 g;
    const float r2 = fmaxf(p.r2, 1e-30f);
    const float r = r2 * rsqrtf(r2);
    const float t = fminf(fmaf(r, ph.inv_h, -2.0f), 0.0f);
    const float F = ph.aF * t * t * t;
    const float Fr = 3.0f * ph.aF * t * t * ph.inv_h / r;  // (dF/dr)/r
    const float w = fmaf(p.ux, p.rx, fmaf(p.uy, p.ry, p.uz * p.rz));
    const float sa = fmaf(p.Ak.x, p.rx, fmaf(p.Ak.y, p.ry, p.Ak.z * p.rz));      // abar_k . x_kj
    const float sb = -fmaf(p.Aj.x, p.rx, fmaf(p.Aj.y, p.ry, p.Aj.z * p.rz));     // abar_j . x_jk
    float Pi = 0.f, dPx = 0.f, dPy = 0.f, dPz = 0.f, dPux = 0.f, dPuy = 0.f, dPuz = 0.f, dPd = 0.f, dPa = 0.f;
    if (VISC == SPH_VISC_ARTIFICIAL && w < 0.f) {
        const float E = fmaf(0.5f, p.dk + p.dj, 1.0f);
        const float D = r2 + ph.eps_h2;
        const float inv = 1.0f / (D * E);
        Pi = -pic * w * inv;
        const float k = -pic * inv;             // dPi/du_kj = k x ; dPi/dx_kj = k (u - 2 w x / D)
        const float c2 = 2.0f * w / D;
        dPx = k * (p.ux - c2 * p.rx);
        dPy = k * (p.uy - c2 * p.ry);
        dPz = k * (p.uz - c2 * p.rz);
        dPux = k * p.rx;
        dPuy = k * p.ry;
        dPuz = k * p.rz;
        dPd = -0.5f * Pi / E;                    // dPi/d delta_k = dPi/d delta_j
        dPa = -pic_unit * w * inv;               // dPi/d alpha
    }
    const float S = p.phk + p.phj + Pi;
    const float Bca = -p.mj * S, Bcb = -p.mk * S;
    const float mFa = p.mj * F, mFb = p.mk * F;
    const float sFma = -sa * mFa, sFmb = -sb * mFb;
    const float C1 = (sa * Bca + p.rbk * p.mj * w) * Fr + (sb * Bcb + p.rbj * p.mk * w) * Fr;
    const float C2 = p.rbk * mFa + p.rbj * mFb;
    const float C3 = sFma + sFmb;
    g.gx = F * (Bca * p.Ak.x - Bcb * p.Aj.x) + C1 * p.rx + C2 * p.ux + C3 * dPx;
    g.gy = F * (Bca * p.Ak.y - Bcb * p.Aj.y) + C1 * p.ry + C2 * p.uy + C3 * dPy;
    g.gz = F * (Bca * p.Ak.z - Bcb * p.Aj.z) + C1 * p.rz + C2 * p.uz + C3 * dPz;
    g.gux = C3 * dPux + C2 * p.rx;
    g.guy = C3 * dPuy + C2 * p.ry;
    g.guz = C3 * dPuz + C2 * p.rz;
    g.gd = C3 * (p.dphk + dPd);
    g.ga = sFma * dPa;
    if (VISC == SPH_VISC_LAMINAR) {
        // a_kj += lam m_j F u_kj / (2 + d_k + d_j), lam = 4 nu / rho0 (and a_jk likewise with m_k)
        const float inv2 = 1.0f / (2.0f + p.dk + p.dj);
        const float lam = ph.nu4 * ph.inv_rho0 * inv2;
        const float Aua = fmaf(p.Ak.x, p.ux, fmaf(p.Ak.y, p.uy, p.Ak.z * p.uz));
        const float Aub = -fmaf(p.Aj.x, p.ux, fmaf(p.Aj.y, p.uy, p.Aj.z * p.uz));
        const float cx = lam * (p.mj * Aua + p.mk * Aub) * Fr;
        g.gx += cx * p.rx;
        g.gy += cx * p.ry;
        g.gz += cx * p.rz;
        g.gux += lam * (mFa * p.Ak.x - mFb * p.Aj.x);
        g.guy += lam * (mFa * p.Ak.y - mFb * p.Aj.y);
        g.guz += lam * (mFa * p.Ak.z - mFb * p.Aj.z);
        g.gd += -lam * inv2 * (mFa * Aua + mFb * Aub);
    }
    return g;
}

// VJP of f on one state: for every particle k, the derivative of
// sum_i (abar_i . a_i + drhobar_i drho_i) w.r.t. x_k, u_k, delta_k, alpha,
// followed by the particle's next reverse stage (no separate launch):
//   STAR (the VJP at the predicted state): reverse of the predictor,
//     x* = x + h u, u* = u + h a, delta* = delta + h drho/rho0 (h = dt/2):
//     xbar_n += x*bar, ubar_n += h x*bar + u*bar, deltabar_n += delta*bar,
//     seeds at n: abar = h u*bar, drhobar = h/rho0 delta*bar  -> (xb, ub, seed_n);
//   otherwise (the VJP at n): adds to (xb, ub) and writes the step's result to
//     id space (x and u of boundary particles are constants: dropped).
// LANES consecutive lanes share one particle: lane l of the group takes the list
// entries q = l (mod LANES), and the partial sums are combined by a fixed xor
// tree of shuffles, so the result is deterministic (for a given LANES).  More
// lanes per particle keep small states (the differentiable run's 32^3 box) from
// leaving most of the GPU idle.  Seven resident blocks per SM (<= 72 registers, no
// spills) hold the 4096 warps of that box's four-lane launch in one wave on 152
// SMs; at the 90 registers the kernel takes uncapped, five blocks fit and a second,
// one-third-full wave followed (backward 11.5 -> 9.9 ms, measured).
template <int VISC, bool STAR, int LANES>
__global__ void __launch_bounds__(kBlock, 7) k_adj_vjp(
    const float4* __restrict__ pos, const float4* __restrict__ vel, const float* __restrict__ phat,
    const float* __restrict__ dphat, const float4* __restrict__ seed, const uint32_t* __restrict__ pinfo,
    const uint32_t* __restrict__ nlist, const uint32_t* __restrict__ ncount, const SceneDev* __restrict__ scenes,
    const DevStatus* __restrict__ st, const Phys ph, float dt, const uint32_t* __restrict__ pid,
    float4* __restrict__ xb, float4* __restrict__ ub, float4* __restrict__ seed_n, float4* __restrict__ xb_id,
    float4* __restrict__ ub_id) {
    static_assert(LANES == 1 || LANES == 2 || LANES == 4 || LANES == 8, "a power of two within a warp");
    const uint32_t n = st->n_active;
    const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t sub = tid % LANES;
    const unsigned gmask = LANES == 1 ? 0xffffffffu
                                      : ((1u << LANES) - 1u) << ((threadIdx.x & 31u) & ~(uint32_t)(LANES - 1));
    for (uint32_t k = tid / LANES; k < n; k += (gridDim.x * blockDim.x) / LANES) {
        const SceneDev& sc = scenes[pinfo[k]];
        const float4 pk = pos[k];
        const float4 vk = vel[k];
        const float4 sk = seed[k];
        const float phk = phat[k], dphk = dphat[k];
        const float mk = fabsf(pk.w);
        const uint32_t cnt = ncount[k];
        const uint32_t nf = cnt & 0xffffu, nb = cnt >> 16;
        float gx = 0.f, gy = 0.f, gz = 0.f, gux = 0.f, guy = 0.f, guz = 0.f, gd = 0.f, ga = 0.f;
        for (uint32_t q = sub; q < nf + nb; q += LANES) {
            const uint32_t e = nlist[q < nf ? list_fluid_word(q, k, ph.stride)
                                            : list_bnd_word(q - nf, k, ph.stride, ph.max_neibs)];
            const uint32_t j = e >> kCodeBits;
            SPH_GUARD(j < st->n_active, st, continue)
            const float4 pj = pos[j];
            const float4 vj = vel[j];
            const float4 sj = seed[j];
            PairIn2 in;
            in.rx = pk.x - pj.x - cell_delta(e & 3u, sc.cell_f[0]);
            in.ry = pk.y - pj.y - cell_delta((e >> 2) & 3u, sc.cell_f[1]);
            in.rz = pk.z - pj.z - cell_delta((e >> 4) & 3u, sc.cell_f[2]);
            in.r2 = fmaf(in.rx, in.rx, fmaf(in.ry, in.ry, in.rz * in.rz));
            in.ux = vk.x - vj.x;
            in.uy = vk.y - vj.y;
            in.uz = vk.z - vj.z;
            in.dk = vk.w;
            in.dj = vj.w;
            in.phk = phk;
            in.phj = phat[j];
            in.dphk = dphk;
            in.mj = fabsf(pj.w);
            in.mk = mk;
            in.Ak = make_float3(sk.x, sk.y, sk.z);
            in.rbk = sk.w;
            in.Aj = make_float3(sj.x, sj.y, sj.z);
            in.rbj = sj.w;
            const PairGrad2 g = pair_grad2<VISC>(in, ph, sc.pi_coef, sc.pi_unit);
            gx += g.gx;
            gy += g.gy;
            gz += g.gz;
            gux += g.gux;
            guy += g.guy;
            guz += g.guz;
            gd += g.gd;
            ga += g.ga;
        }
        if (LANES > 1) {
#pragma unroll
            for (int o = LANES / 2; o >= 1; o >>= 1) {
                gx += __shfl_xor_sync(gmask, gx, o);
                gy += __shfl_xor_sync(gmask, gy, o);
                gz += __shfl_xor_sync(gmask, gz, o);
                gux += __shfl_xor_sync(gmask, gux, o);
                guy += __shfl_xor_sync(gmask, guy, o);
                guz += __shfl_xor_sync(gmask, guz, o);
                gd += __shfl_xor_sync(gmask, gd, o);
                ga += __shfl_xor_sync(gmask, ga, o);
            }
            if (sub != 0) continue;
        }
        const bool fluid = pk.w > 0.f;
        if (STAR) {
            float4 xs = make_float4(0.f, 0.f, 0.f, 0.f), us = make_float4(0.f, 0.f, 0.f, 0.f);
            xs.x += gx;
            xs.y += gy;
            xs.z += gz;
            xs.w += gd;
            us.x += gux;
            us.y += guy;
            us.z += guz;
            us.w += ga;
            const float h = 0.5f * dt;
            float4 x = xb[k], u = ub[k];
            float4 sd = make_float4(0.f, 0.f, 0.f, h * ph.inv_rho0 * xs.w);
            x.w += xs.w;
            u.w += us.w;  // alphabar partial of the star VJP
            if (fluid) {
                x.x += xs.x;
                x.y += xs.y;
                x.z += xs.z;
                u.x += h * xs.x + us.x;
                u.y += h * xs.y + us.y;
                u.z += h * xs.z + us.z;
                sd.x = h * us.x;
                sd.y = h * us.y;
                sd.z = h * us.z;
            }
            xb[k] = x;
            ub[k] = u;
            seed_n[k] = sd;
        } else {
            float4 x = xb[k], u = ub[k];
            x.x += gx;
            x.y += gy;
            x.z += gz;
            x.w += gd;
            u.x += gux;
            u.y += guy;
            u.z += guz;
            u.w += ga;
            if (!fluid) {
                x.x = x.y = x.z = 0.f;
                u.x = u.y = u.z = 0.f;
            }
            const uint32_t id = pid[k];
            xb_id[id] = x;
            ub_id[id] = u;
        }
    }
}

inline unsigned grid_for(uint32_t n, int block) {
    uint32_t g = (n + block - 1) / block;
    return g ? g : 1;
}

// one block: fixed-order sum of the alphabar partials in id space (deterministic)
__global__ void k_adj_sum_alpha(const float4* __restrict__ ub_id, uint32_t n, double* __restrict__ out) {
    __shared__ double part[256];
    double s = 0.0;
    for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) s += (double)ub_id[i].w;
    part[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) part[threadIdx.x] += part[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = part[0];
}

}  // namespace

void launch_tape_copy(const void* const* src, void* const* dst, const bool* wide, int count, uint32_t n,
                      cudaStream_t st) {
    TapeCopy tc{};
    tc.count = count;
    for (int k = 0; k < count && k < kTapeArrays; ++k) {
        tc.src[k] = src[k];
        tc.dst[k] = dst[k];
        tc.wide |= wide[k] ? (1u << k) : 0u;
    }
    k_tape_copy<<<grid_for(n ? n : 1, 256), 256, 0, st>>>(tc, n);
}

void launch_adj_load(const AdjBuffers& a, uint32_t n, const float* xbar, const float* ubar, const float* dbar,
                     cudaStream_t st) {
    k_adj_load<<<grid_for(n, 256), 256, 0, st>>>(n, xbar, ubar, dbar, a.xb_id, a.ub_id);
}

void launch_adj_store(const AdjBuffers& a, uint32_t n, float* xbar, float* ubar, float* dbar, cudaStream_t st) {
    k_adj_store<<<grid_for(n, 256), 256, 0, st>>>(n, a.xb_id, a.ub_id, xbar, ubar, dbar);
}

template <int VISC, int LANES>
void launch_adj_vjps(const AdjBuffers& a, const Buffers& b, int cur, const Geometry& g, const Phys& ph, float dt,
                     cudaStream_t st) {
    const unsigned grid = grid_for(g.cap * LANES, kBlock);
    // VJP at the predicted state (+ reverse of the predictor), then at n (+ to id space)
    k_adj_vjp<VISC, true, LANES><<<grid, kBlock, 0, st>>>(b.pos_s, b.vel_s, b.phat_s, a.dphat_s, a.seed, b.pinfo[cur],
                                                          b.nlist, b.ncount, b.scenes, b.status, ph, dt, b.pid[cur],
                                                          a.xb, a.ub, a.seed_n, nullptr, nullptr);
    k_adj_vjp<VISC, false, LANES><<<grid, kBlock, 0, st>>>(b.pos[cur], b.vel[cur], b.phat[cur], a.dphat, a.seed_n,
                                                           b.pinfo[cur], b.nlist, b.ncount, b.scenes, b.status, ph,
                                                           dt, b.pid[cur], a.xb, a.ub, nullptr, a.xb_id, a.ub_id);
}

template <int VISC>
void launch_adj_vjps_v(const AdjBuffers& a, const Buffers& b, int cur, const Geometry& g, const Phys& ph, float dt,
                       cudaStream_t st) {
    // lanes per particle: enough threads to fill the GPU (~150k resident) on small states
    if (g.cap <= (1u << 16))
        launch_adj_vjps<VISC, 4>(a, b, cur, g, ph, dt, st);
    else if (g.cap <= (1u << 18))
        launch_adj_vjps<VISC, 2>(a, b, cur, g, ph, dt, st);
    else
        launch_adj_vjps<VISC, 1>(a, b, cur, g, ph, dt, st);
}

void launch_adj_step(const AdjBuffers& a, const Buffers& b, int cur, const Geometry& g, const Phys& ph, float dt,
                     cudaStream_t st) {
    k_adj_pre<<<grid_for(g.cap, 256), 256, 0, st>>>(b.pos[cur], b.vel[cur], b.vel_s, b.pinfo[cur], b.pid[cur], b.scenes,
                                                    b.status, ph, dt, a.xb_id, a.ub_id, a.dphat, a.dphat_s, a.xb, a.ub,
                                                    a.seed);
    if (ph.visc == SPH_VISC_LAMINAR)
        launch_adj_vjps_v<SPH_VISC_LAMINAR>(a, b, cur, g, ph, dt, st);
    else
        launch_adj_vjps_v<SPH_VISC_ARTIFICIAL>(a, b, cur, g, ph, dt, st);
}

void launch_adj_sum_alpha(const AdjBuffers& a, uint32_t n, double* out, cudaStream_t st) {
    k_adj_sum_alpha<<<1, 256, 0, st>>>(a.ub_id, n, out);
}

}  // namespace sphg
