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

__global__ void k_adj_dphat(const float4* __restrict__ vel, const float4* __restrict__ vel_s,
                            const uint32_t* __restrict__ pinfo, const SceneDev* __restrict__ scenes,
                            const DevStatus* __restrict__ st, float* __restrict__ dphat, float* __restrict__ dphat_s,
                            const Phys ph) {
    const uint32_t n = st->n_active;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float c = scenes[pinfo[i]].phat_coef;
        dphat[i] = eos_dphat(vel[i].w, ph, c);
        dphat_s[i] = eos_dphat(vel_s[i].w, ph, c);
    }
}

// id space <-> sorted order of the step
__global__ void k_adj_gather(const uint32_t* __restrict__ pid, const DevStatus* __restrict__ st,
                             const float4* __restrict__ xb_id, const float4* __restrict__ ub_id,
                             float4* __restrict__ xb, float4* __restrict__ ub) {
    const uint32_t n = st->n_active;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const uint32_t id = pid[i];
        xb[i] = xb_id[id];
        ub[i] = ub_id[id];
    }
}

// (x, u of boundary particles are constants: their adjoints are dropped here)
__global__ void k_adj_scatter(const uint32_t* __restrict__ pid, const float4* __restrict__ pos,
                              const DevStatus* __restrict__ st, const float4* __restrict__ xb,
                              const float4* __restrict__ ub, float4* __restrict__ xb_id, float4* __restrict__ ub_id) {
    const uint32_t n = st->n_active;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const uint32_t id = pid[i];
        float4 x = xb[i], u = ub[i];
        if (!(pos[i].w > 0.f)) {
            x.x = x.y = x.z = 0.f;
            u.x = u.y = u.z = 0.f;
        }
        xb_id[id] = x;
        ub_id[id] = u;
    }
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

// reverse of the corrector: adjoint of state n+1 (in xb, ub) -> seeds at *
// and the partial adjoint of state n (in place)
__global__ void k_adj_corrector(const float4* __restrict__ pos, const DevStatus* __restrict__ st, float dt,
                                float inv_rho0, float4* __restrict__ xb, float4* __restrict__ ub,
                                float4* __restrict__ seed) {
    const uint32_t n = st->n_active;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const bool fluid = pos[i].w > 0.f;
        float4 x = xb[i], u = ub[i];
        const float dbar = x.w;
        float4 sd = make_float4(0.f, 0.f, 0.f, dt * inv_rho0 * dbar);
        if (fluid) {
            // x' = x + dt/2 (u + u'):  u'bar_tot = u'bar + dt/2 x'bar;  ubar_n = u'bar_tot + dt/2 x'bar
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

// reverse of the predictor: star adjoint (xbs, ubs) -> partial adjoint of n
// (+=) and seeds at n
__global__ void k_adj_predictor(const float4* __restrict__ pos, const DevStatus* __restrict__ st, float dt,
                                float inv_rho0, const float4* __restrict__ xbs, const float4* __restrict__ ubs,
                                float4* __restrict__ xb, float4* __restrict__ ub, float4* __restrict__ seed) {
    const uint32_t n = st->n_active;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const bool fluid = pos[i].w > 0.f;
        const float h = 0.5f * dt;
        const float4 xs = xbs[i], us = ubs[i];
        float4 x = xb[i], u = ub[i];
        float4 sd = make_float4(0.f, 0.f, 0.f, h * inv_rho0 * xs.w);
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
        xb[i] = x;
        ub[i] = u;
        seed[i] = sd;
    }
}

struct PairIn {
    float rx, ry, rz, r2;   // x_ij
    float ux, uy, uz;       // u_ij
    float di, dj;           // delta_i, delta_j
    float phi, phj;         // P/rho^2
    float dphi, dphj;       // d(P/rho^2)/d delta
    float m;                // m_j
    float Ax, Ay, Az, rb;   // adjoint seeds of particle i's a and drho
};

struct PairGrad {
    float gx, gy, gz;       // d S / d x_ij
    float gux, guy, guz;    // d S / d u_ij
    float gdi, gdj, ga;     // d S / d delta_i, d delta_j, d alpha
};

// S = A . a_ij + rb * drho_ij for one pair term of particle i (see forces.cu).
template <int VISC>
__device__ __forceinline__ PairGrad pair_grad(const PairIn& p, const Phys& ph, float pic, float pic_unit) {
    PairGrad g;
    const float r2 = fmaxf(p.r2, 1e-30f);
    const float r = r2 * rsqrtf(r2);
    const float t = fminf(fmaf(r, ph.inv_h, -2.0f), 0.0f);
    const float F = ph.aF * t * t * t;
    const float Fr = 3.0f * ph.aF * t * t * ph.inv_h / r;  // (dF/dr)/r
    const float w = fmaf(p.ux, p.rx, fmaf(p.uy, p.ry, p.uz * p.rz));
    const float s = fmaf(p.Ax, p.rx, fmaf(p.Ay, p.ry, p.Az * p.rz));
    float Pi = 0.f, dPx = 0.f, dPy = 0.f, dPz = 0.f, dPux = 0.f, dPuy = 0.f, dPuz = 0.f, dPd = 0.f, dPa = 0.f;
    if (VISC == SPH_VISC_ARTIFICIAL && w < 0.f) {
        const float E = fmaf(0.5f, p.di + p.dj, 1.0f);
        const float D = r2 + ph.eps_h2;
        const float inv = 1.0f / (D * E);
        Pi = -pic * w * inv;
        const float k = -pic * inv;             // dPi/du = k x ; dPi/dx = k (u - 2 w x / D)
        const float c2 = 2.0f * w / D;
        dPx = k * (p.ux - c2 * p.rx);
        dPy = k * (p.uy - c2 * p.ry);
        dPz = k * (p.uz - c2 * p.rz);
        dPux = k * p.rx;
        dPuy = k * p.ry;
        dPuz = k * p.rz;
        dPd = -0.5f * Pi / E;                    // dPi/d delta_i = dPi/d delta_j
        dPa = -pic_unit * w * inv;               // dPi/d alpha
    }
    const float Bc = -p.m * (p.phi + p.phj + Pi);
    const float mF = p.m * F;
    const float cFr = (s * Bc + p.rb * p.m * w) * Fr;
    const float sFm = -s * mF;                   // s F (-m)
    g.gx = Bc * F * p.Ax + cFr * p.rx + p.rb * mF * p.ux + sFm * dPx;
    g.gy = Bc * F * p.Ay + cFr * p.ry + p.rb * mF * p.uy + sFm * dPy;
    g.gz = Bc * F * p.Az + cFr * p.rz + p.rb * mF * p.uz + sFm * dPz;
    g.gux = sFm * dPux + p.rb * mF * p.rx;
    g.guy = sFm * dPuy + p.rb * mF * p.ry;
    g.guz = sFm * dPuz + p.rb * mF * p.rz;
    g.gdi = sFm * (p.dphi + dPd);
    g.gdj = sFm * (p.dphj + dPd);
    g.ga = sFm * dPa;
    if (VISC == SPH_VISC_LAMINAR) {
        // a_ij += lam m F u / (2 + di + dj), lam = 4 nu / rho0
        const float inv2 = 1.0f / (2.0f + p.di + p.dj);
        const float lam = ph.nu4 * ph.inv_rho0 * inv2;
        const float Au = fmaf(p.Ax, p.ux, fmaf(p.Ay, p.uy, p.Az * p.uz));
        const float cx = lam * p.m * Au * Fr;
        g.gx += cx * p.rx;
        g.gy += cx * p.ry;
        g.gz += cx * p.rz;
        g.gux += lam * mF * p.Ax;
        g.guy += lam * mF * p.Ay;
        g.guz += lam * mF * p.Az;
        const float dd = -lam * mF * Au * inv2;
        g.gdi += dd;
        g.gdj += dd;
    }
    return g;
}

// VJP of f on one state: for every particle k, the derivative of
// sum_i (abar_i . a_i + drhobar_i drho_i) w.r.t. x_k, u_k, delta_k, alpha.
// ACCUM: add to (xb, ub) instead of assigning.
template <int VISC, bool ACCUM>
__global__ void __launch_bounds__(kBlock, 2) k_adj_vjp(
    const float4* __restrict__ pos, const float4* __restrict__ vel, const float* __restrict__ phat,
    const float* __restrict__ dphat, const float4* __restrict__ seed, const uint32_t* __restrict__ pinfo,
    const uint32_t* __restrict__ nlist, const uint32_t* __restrict__ ncount, const SceneDev* __restrict__ scenes,
    const DevStatus* __restrict__ st, const Phys ph, float4* __restrict__ xb, float4* __restrict__ ub) {
    const uint32_t n = st->n_active;
    for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const SceneDev& sc = scenes[pinfo[k]];
        const float4 pk = pos[k];
        const float4 vk = vel[k];
        const float4 sk = seed[k];
        const float phk = phat[k], dphk = dphat[k];
        const float mk = fabsf(pk.w);
        const uint32_t cnt = ncount[k];
        const uint32_t nf = cnt & 0xffffu, nb = cnt >> 16;
        float gx = 0.f, gy = 0.f, gz = 0.f, gux = 0.f, guy = 0.f, guz = 0.f, gd = 0.f, ga = 0.f;
        for (uint32_t q = 0; q < nf + nb; ++q) {
            const uint32_t e = nlist[q < nf ? list_fluid_word(q, k, ph.stride)
                                            : list_bnd_word(q - nf, k, ph.stride, ph.max_neibs)];
            const uint32_t j = e >> kCodeBits;
            SPH_GUARD(j < st->n_active, st, continue)
            const float4 pj = pos[j];
            const float4 vj = vel[j];
            const float4 sj = seed[j];
            PairIn in;
            in.rx = pk.x - pj.x - cell_delta(e & 3u, sc.cell_f[0]);
            in.ry = pk.y - pj.y - cell_delta((e >> 2) & 3u, sc.cell_f[1]);
            in.rz = pk.z - pj.z - cell_delta((e >> 4) & 3u, sc.cell_f[2]);
            in.r2 = fmaf(in.rx, in.rx, fmaf(in.ry, in.ry, in.rz * in.rz));
            in.ux = vk.x - vj.x;
            in.uy = vk.y - vj.y;
            in.uz = vk.z - vj.z;
            // own term T_kj, seeded with k's adjoints
            in.di = vk.w;
            in.dj = vj.w;
            in.phi = phk;
            in.phj = phat[j];
            in.dphi = dphk;
            in.dphj = dphat[j];
            in.m = fabsf(pj.w);
            in.Ax = sk.x;
            in.Ay = sk.y;
            in.Az = sk.z;
            in.rb = sk.w;
            const PairGrad a = pair_grad<VISC>(in, ph, sc.pi_coef, sc.pi_unit);
            gx += a.gx;
            gy += a.gy;
            gz += a.gz;
            gux += a.gux;
            guy += a.guy;
            guz += a.guz;
            gd += a.gdi;
            ga += a.ga;
            // neighbour's term T_jk (x_jk = -x_kj, u_jk = -u_kj), seeded with j's adjoints
            PairIn rv = in;
            rv.rx = -in.rx;
            rv.ry = -in.ry;
            rv.rz = -in.rz;
            rv.ux = -in.ux;
            rv.uy = -in.uy;
            rv.uz = -in.uz;
            rv.di = in.dj;
            rv.dj = in.di;
            rv.phi = in.phj;
            rv.phj = in.phi;
            rv.dphi = in.dphj;
            rv.dphj = in.dphi;
            rv.m = mk;
            rv.Ax = sj.x;
            rv.Ay = sj.y;
            rv.Az = sj.z;
            rv.rb = sj.w;
            const PairGrad b = pair_grad<VISC>(rv, ph, sc.pi_coef, sc.pi_unit);
            gx -= b.gx;
            gy -= b.gy;
            gz -= b.gz;
            gux -= b.gux;
            guy -= b.guy;
            guz -= b.guz;
            gd += b.gdj;
        }
        float4 x = ACCUM ? xb[k] : make_float4(0.f, 0.f, 0.f, 0.f);
        float4 u = ACCUM ? ub[k] : make_float4(0.f, 0.f, 0.f, 0.f);
        x.x += gx;
        x.y += gy;
        x.z += gz;
        x.w += gd;
        u.x += gux;
        u.y += guy;
        u.z += guz;
        u.w += ga;
        xb[k] = x;
        ub[k] = u;
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

void launch_adj_dphat(const AdjBuffers& a, const Buffers& b, int cur, const Geometry& g, const Phys& ph,
                      cudaStream_t st) {
    k_adj_dphat<<<grid_for(g.cap, 256), 256, 0, st>>>(b.vel[cur], b.vel_s, b.pinfo[cur], b.scenes, b.status, a.dphat,
                                                       a.dphat_s, ph);
}

void launch_adj_gather(const AdjBuffers& a, const Buffers& b, int cur, const Geometry& g, cudaStream_t st) {
    k_adj_gather<<<grid_for(g.cap, 256), 256, 0, st>>>(b.pid[cur], b.status, a.xb_id, a.ub_id, a.xb, a.ub);
}

void launch_adj_scatter(const AdjBuffers& a, const Buffers& b, int cur, const Geometry& g, cudaStream_t st) {
    k_adj_scatter<<<grid_for(g.cap, 256), 256, 0, st>>>(b.pid[cur], b.pos[cur], b.status, a.xb, a.ub, a.xb_id,
                                                         a.ub_id);
}

void launch_adj_load(const AdjBuffers& a, uint32_t n, const float* xbar, const float* ubar, const float* dbar,
                     cudaStream_t st) {
    k_adj_load<<<grid_for(n, 256), 256, 0, st>>>(n, xbar, ubar, dbar, a.xb_id, a.ub_id);
}

void launch_adj_store(const AdjBuffers& a, uint32_t n, float* xbar, float* ubar, float* dbar, cudaStream_t st) {
    k_adj_store<<<grid_for(n, 256), 256, 0, st>>>(n, a.xb_id, a.ub_id, xbar, ubar, dbar);
}

void launch_adj_step(const AdjBuffers& a, const Buffers& b, int cur, const Geometry& g, const Phys& ph, float dt,
                     cudaStream_t st) {
    const unsigned grid = grid_for(g.cap, kBlock);
    k_adj_corrector<<<grid_for(g.cap, 256), 256, 0, st>>>(b.pos[cur], b.status, dt, ph.inv_rho0, a.xb, a.ub, a.seed);
    if (ph.visc == SPH_VISC_LAMINAR) {
        k_adj_vjp<SPH_VISC_LAMINAR, false><<<grid, kBlock, 0, st>>>(b.pos_s, b.vel_s, b.phat_s, a.dphat_s, a.seed,
                                                                     b.pinfo[cur], b.nlist, b.ncount, b.scenes,
                                                                     b.status, ph, a.xbs, a.ubs);
    } else {
        k_adj_vjp<SPH_VISC_ARTIFICIAL, false><<<grid, kBlock, 0, st>>>(b.pos_s, b.vel_s, b.phat_s, a.dphat_s, a.seed,
                                                                        b.pinfo[cur], b.nlist, b.ncount, b.scenes,
                                                                        b.status, ph, a.xbs, a.ubs);
    }
    k_adj_predictor<<<grid_for(g.cap, 256), 256, 0, st>>>(b.pos[cur], b.status, dt, ph.inv_rho0, a.xbs, a.ubs, a.xb,
                                                          a.ub, a.seed);
    if (ph.visc == SPH_VISC_LAMINAR) {
        k_adj_vjp<SPH_VISC_LAMINAR, true><<<grid, kBlock, 0, st>>>(b.pos[cur], b.vel[cur], b.phat[cur], a.dphat, a.seed,
                                                                    b.pinfo[cur], b.nlist, b.ncount, b.scenes,
                                                                    b.status, ph, a.xb, a.ub);
    } else {
        k_adj_vjp<SPH_VISC_ARTIFICIAL, true><<<grid, kBlock, 0, st>>>(b.pos[cur], b.vel[cur], b.phat[cur], a.dphat,
                                                                       a.seed, b.pinfo[cur], b.nlist, b.ncount,
                                                                       b.scenes, b.status, ph, a.xb, a.ub);
    }
}

void launch_adj_sum_alpha(const AdjBuffers& a, uint32_t n, double* out, cudaStream_t st) {
    k_adj_sum_alpha<<<1, 256, 0, st>>>(a.ub_id, n, out);
}

}  // namespace sphg
