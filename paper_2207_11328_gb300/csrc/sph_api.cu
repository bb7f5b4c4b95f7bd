// C ABI of the GB300 WCSPH hot path: context, buffers, upload/download,
// step orchestration (CUDA graphs), counters.  The argument conventions of
// every entry point are documented in include/sph.h.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "sph_internal.cuh"

using namespace sphg;

// Recording of a differentiable run: checkpoints of the pre-step state every
// K steps and a per-step tape of one segment, re-filled during the backward.
struct AdjTape {
    bool valid = false;
    uint64_t gen = 0;          // generation of the valid recording (0: none)
    uint64_t next_gen = 1;     // the next sph_record's generation
    uint32_t T = 0, K = 0, n = 0;
    double dt = 0.0;
    Phys ph_rec{};
    std::vector<char*> ckpt;   // T/K checkpoints (pos4 vel4 phat cell pinfo pid)
    char* steps = nullptr;     // K records (sorted state, predicted state)
    char* lists = nullptr;     // K neighbour-list slots (list + counts) of the recomputed steps
    size_t ckpt_bytes = 0, step_bytes = 0;
    sphg::AdjBuffers a{};
    void* adj_mem = nullptr;
    // one segment of the backward pass (recompute K steps, reverse K steps) as a graph,
    // per buffer parity at its start, and the parity it ends on
    cudaGraphExec_t seg_graph[2] = {nullptr, nullptr};
    int seg_end_cur[2] = {0, 0};
    // K recorded forward steps as a graph, per buffer parity at its start
    cudaGraphExec_t rec_graph[2] = {nullptr, nullptr};
    int rec_end_cur[2] = {0, 0};
};

struct sph_ctx {
    AdjTape tape;
    sph_params p{};
    Phys ph{};
    Geometry g{};
    Buffers b{};
    std::vector<SceneDev> scenes_h;
    std::vector<double> centres_h;   // FP64 cell centres (Buffers::centres), per scene and axis
    int cur = 0;
    int device = 0;
    uint32_t n_uploaded = 0;
    bool uploaded = false;
    bool need_dt0 = true;
    bool fresh = false;  // the list was built for the current positions (no step since)
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t graph[2] = {nullptr, nullptr};  // captured step, per buffer parity
    uint32_t graph_nodes = 0;
    bool persistent = false;  // sph_set_persistent: one cooperative launch per sph_step call
    size_t staging_bytes = 0;
    std::vector<std::pair<char*, size_t>> canaries;  // checked build: (base, bytes) of guarded buffers
};

namespace {

// Device allocation.  The checked build (SPH_CHECKED) adds a 256-byte canary
// tail to each buffer, filled with 0xA5 and verified whenever the device
// counters are read; a changed byte records SPH_EBIT_BOUNDS.
#ifdef SPH_CHECKED
constexpr size_t kCanary = 256;
#else
constexpr size_t kCanary = 0;
#endif

cudaError_t dev_alloc(sph_ctx* c, void** ptr, size_t bytes) {
    if (!bytes) bytes = 16;
    cudaError_t e = cudaMalloc(ptr, bytes + kCanary);
    if (e != cudaSuccess || !kCanary) return e;
    e = cudaMemset((char*)*ptr + bytes, 0xA5, kCanary);
    c->canaries.push_back({(char*)*ptr, bytes});
    return e;
}

void drop_canary(sph_ctx* c, const void* base) {
    for (size_t k = 0; k < c->canaries.size(); ++k)
        if (c->canaries[k].first == base) {
            c->canaries.erase(c->canaries.begin() + (long)k);
            return;
        }
}

__global__ void k_check_canary(const uint8_t* __restrict__ tail, uint32_t bytes, sphg::DevStatus* st) {
    for (uint32_t k = threadIdx.x; k < bytes; k += blockDim.x)
        if (tail[k] != 0xA5u) atomicOr(&st->error_bits, SPH_EBIT_BOUNDS);
}

void check_canaries(sph_ctx* c, cudaStream_t st) {
    for (auto& cb : c->canaries)
        k_check_canary<<<1, 256, 0, st>>>((const uint8_t*)cb.first + cb.second, (uint32_t)kCanary, c->b.status);
}

#define CK(call)                                                        \
    do {                                                                \
        cudaError_t e_ = (call);                                        \
        if (e_ != cudaSuccess) {                                        \
            std::fprintf(stderr, "sph: %s failed: %s (%s:%d)\n", #call, \
                         cudaGetErrorString(e_), __FILE__, __LINE__);   \
            return SPH_ERR_CUDA;                                        \
        }                                                               \
    } while (0)

inline cudaStream_t S(void* s) { return reinterpret_cast<cudaStream_t>(s); }

constexpr double kViscousDtCoef = 0.125;  // laminar viscous time-step limit, dt <= 0.125 h^2/nu

inline size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// ---------------------------------------------------------------------
// Upload: FP64 absolute position -> (cell, FP32 offset from the cell
// centre) per scene grid; type packed in the sign of pos.w.
// ---------------------------------------------------------------------
// x truncated to FP32 with integer operations on its bits (no FP64 instruction): sign,
// exponent re-biased, the top 23 fraction bits; magnitudes below FP32's normal range give
// +-0, above it +-FLT_MAX.  Only the upload's cell estimate uses it.
__device__ __forceinline__ float fp32_estimate(double x) {
    const uint32_t hi = (uint32_t)__double2hiint(x), lo = (uint32_t)__double2loint(x);
    const int e = (int)((hi >> 20) & 0x7ffu) - 1023 + 127;
    const uint32_t sign = hi & 0x80000000u;
    if (e <= 0) return __uint_as_float(sign);
    if (e >= 255) return __uint_as_float(sign | 0x7f7fffffu);
    return __uint_as_float(sign | ((uint32_t)e << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29));
}

// d rounded to FP32 (to nearest, ties to even) with integer operations on its bits: the
// same result as the FP64 unit's conversion over FP32's normal range; magnitudes below it
// give +-0 (cell offsets that small are below any resolution the state carries).
__device__ __forceinline__ float fp32_rn(double d) {
    const uint64_t b = (uint64_t)__double_as_longlong(d);
    const uint32_t sign = (uint32_t)(b >> 32) & 0x80000000u;
    const int e = (int)((b >> 52) & 0x7ffu) - 1023 + 127;
    if (e <= 0) return __uint_as_float(sign);
    if (e >= 255) return __uint_as_float(sign | 0x7f800000u);
    const uint64_t m = b & 0xfffffffffffffull;
    const uint32_t f = (uint32_t)(m >> 29), rest = (uint32_t)(m & 0x1fffffffu);
    uint32_t bits = sign | ((uint32_t)e << 23) | f;
    if (rest > 0x10000000u || (rest == 0x10000000u && (f & 1u))) bits += 1u;  // a carry moves to the next binade
    return __uint_as_float(bits);
}

// f widened to FP64 exactly with integer operations (FP32 subnormals, never a cell offset
// of the state at any resolution used, give +-0)
__device__ __forceinline__ double fp64_of(float f) {
    const uint32_t b = __float_as_uint(f);
    const uint32_t e = (b >> 23) & 0xffu;
    const uint64_t sign = (uint64_t)(b & 0x80000000u) << 32;
    if (e == 0u) return __longlong_as_double((long long)sign);
    return __longlong_as_double((long long)(sign | ((uint64_t)(e - 127u + 1023u) << 52) | ((uint64_t)(b & 0x7fffffu) << 29)));
}

// x - c rounded once to FP32 (to nearest, ties to even) with integer operations, when x and c
// have the same sign and exponents at most one apart: their significands then align within 54
// bits and the difference is exact before the rounding.  Returns false otherwise (the caller
// subtracts in FP64).  Results below FP32's normal range give +-0, as fp32_rn.
__device__ __forceinline__ bool sub_to_fp32(double x, double c, float* out) {
    const uint64_t bx = (uint64_t)__double_as_longlong(x), bc = (uint64_t)__double_as_longlong(c);
    const uint32_t ex = (uint32_t)(bx >> 52) & 0x7ffu, ec = (uint32_t)(bc >> 52) & 0x7ffu;
    if (((bx ^ bc) >> 63) != 0u || ex == 0u || ec == 0u || ex == 0x7ffu || ec == 0x7ffu || ex > ec + 1u ||
        ec > ex + 1u)
        return false;
    const uint64_t frac = (1ull << 52) - 1ull;
    const uint32_t e0 = min(ex, ec);
    const int64_t d = (int64_t)(((1ull << 52) | (bx & frac)) << (ex - e0)) -
                      (int64_t)(((1ull << 52) | (bc & frac)) << (ec - e0));
    if (d == 0) {
        *out = 0.f;
        return true;
    }
    const uint32_t sign = ((uint32_t)(bx >> 32) ^ (d < 0 ? 0x80000000u : 0u)) & 0x80000000u;
    const uint64_t m = d < 0 ? (uint64_t)(-d) : (uint64_t)d;
    const int top = 63 - __clzll((long long)m);            // the leading bit of |d|
    const int e32 = (int)e0 - 1023 - 52 + top + 127;       // biased FP32 exponent
    if (e32 <= 0) {
        *out = __uint_as_float(sign);
        return true;
    }
    uint32_t b;
    if (top >= 24) {
        const int sh = top - 23;
        const uint32_t f = (uint32_t)(m >> sh) & 0x7fffffu;
        const uint64_t rest = m & ((1ull << sh) - 1ull), half = 1ull << (sh - 1);
        b = sign | ((uint32_t)e32 << 23) | f;
        if (rest > half || (rest == half && (f & 1u))) b += 1u;   // a carry moves to the next binade
    } else {
        b = sign | ((uint32_t)e32 << 23) | ((uint32_t)(m << (23 - top)) & 0x7fffffu);
    }
    *out = __uint_as_float(b);
    return true;
}

// The upload's rare FP64 paths, kept out of line so that they stay branches taken by the few
// particles that need them rather than instructions every particle executes under a predicate.
__device__ __noinline__ double wrap_into_domain(double x, const SceneDev& sc, int a) {
    const double L = sc.cell_d[a] * sc.ncell[a];
    const double rel = x - sc.origin[a];
    return sc.origin[a] + (rel - L * floor(rel * sc.inv_len_d[a]));
}
__device__ __noinline__ bool inside_domain(double x, const SceneDev& sc, int a) {
    const double rel = x - sc.origin[a];
    return rel >= 0.0 && rel < sc.cell_d[a] * sc.ncell[a];
}
__device__ __noinline__ float offset_fp64(double x, double centre) { return fp32_rn(x - centre); }

__global__ void k_upload(uint32_t n, const double* __restrict__ pos, const float* __restrict__ vel,
                         const float* __restrict__ delta, const float* __restrict__ mass,
                         const uint8_t* __restrict__ type, const uint32_t* __restrict__ scene,
                         const SceneDev* __restrict__ scenes, const double* __restrict__ centres,
                         uint32_t n_scenes, float4* __restrict__ pos_o,
                         float4* __restrict__ vel_o, float* __restrict__ phat_o, uint32_t* __restrict__ cell_o,
                         uint32_t* __restrict__ pinfo_o, uint32_t* __restrict__ pid_o, DevStatus* __restrict__ st,
                         const Phys ph) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        uint32_t bad = 0;
        const uint32_t s = scene ? scene[i] : 0u;
        const uint8_t t = type[i];
        const float m = mass[i];
        if (s >= n_scenes || t > 1 || !(m > 0.f) || !isfinite(m)) bad |= kUpBadArg;
        const SceneDev& sc = scenes[s < n_scenes ? s : 0];
        int c[3];
        float o[3];
        for (int a = 0; a < 3; ++a) {
            double x = pos[3 * i + a];
            // The FP64 units are slow on this GPU, so the common path has no FP64 instruction:
            // the finiteness test reads the exponent bits, the cell is estimated from an FP32
            // copy of x built from its bits (truncated: relative error < 2^-23, so the estimate
            // can be off by one within ~1e-7 of a cell face), and the offset from that cell's
            // FP64 centre is the exact difference rounded once to FP32, by integer operations
            // (sub_to_fp32; an FP64 subtraction only near the coordinate origin, where x and the
            // centre can differ in sign or binade).  A particle that lands a hair past a face is
            // re-based into the next cell by the sort that follows.  Within 1e-6 of a face of
            // the domain the domain test runs in FP64; a periodic axis is wrapped in FP64 first.
            if ((__double2hiint(x) & 0x7ff00000) == 0x7ff00000) {
                bad |= kUpNonFinite;
                x = sc.origin[a];
            }
            const bool per = (sc.periodic >> a) & 1u;
            if (per) x = wrap_into_domain(x, sc, a);
            const float xe = fp32_estimate(x);
            const float relf = xe - sc.origin_f[a];
            int k = (int)floorf(relf * sc.inv_cell_f[a]);
            // outer cells: the FP32 estimate decides unless it lies within a margin of a face
            // that covers its own errors (truncation, the rounded origin and length, the
            // subtraction: each below 2.5e-7 of the magnitudes involved), then FP64 decides
            const float lenf = sc.cell_f[a] * (float)sc.ncell[a];
            const float tol = 1e-6f * (fabsf(xe) + fabsf(sc.origin_f[a]) + lenf);
            if (!per && (k <= 0 || k >= sc.ncell[a] - 1) && !(relf >= tol && relf <= lenf - tol) &&
                !inside_domain(x, sc, a)) {
                bad |= kUpOutOfDomain;
                x = sc.origin[a];
                k = 0;
            }
            k = min(max(k, 0), sc.ncell[a] - 1);
            c[a] = k;
            const double centre = centres[sc.centre_off[a] + (uint32_t)k];
            if (!sub_to_fp32(x, centre, &o[a])) o[a] = offset_fp64(x, centre);
        }
        const bool fluid = t == 0;
        float4 v = make_float4(0.f, 0.f, 0.f, delta[i]);
        if (fluid) {
            v.x = vel[3 * i];
            v.y = vel[3 * i + 1];
            v.z = vel[3 * i + 2];
        }
        if (!isfinite(v.x + v.y + v.z) || !isfinite(v.w) || !(v.w > -1.f)) bad |= kUpNonFinite;
        if (bad) atomicOr(&st->upload_bits, bad);
        pos_o[i] = make_float4(o[0], o[1], o[2], fluid ? m : -m);
        vel_o[i] = v;
        phat_o[i] = eos_phat(v.w, ph, sc.phat_coef);
        cell_o[i] = sc.cell_offset + (uint32_t)c[0] + (uint32_t)sc.ncell[0] * ((uint32_t)c[1] + (uint32_t)sc.ncell[1] * (uint32_t)c[2]);
        pinfo_o[i] = s < n_scenes ? s : 0;
        pid_o[i] = i;
    }
}

__global__ void k_set_status_n(DevStatus* st, uint32_t n) {
    st->n_active = n;
    st->n_sorted = n;
    st->n_removed = 0;
    st->max_neibs_seen = 0;
    st->upload_bits = 0;
    st->steps = 0ull;
    st->list_entries = 0ull;
    st->interactions = 0ull;
    st->rebuild = 1u;  // the upload builds the list
    st->since = 0u;
    st->maxdisp2_bits = 0u;
    st->builds = 1u;
}

__global__ void k_reset_dyn(SceneDyn* dyn, uint32_t n_scenes) {
    for (uint32_t s = threadIdx.x; s < n_scenes; s += blockDim.x) {
        dyn[s].dt = 0.f;
        dyn[s].amax2_bits = 0u;
        dyn[s].dt_d = 0.0;
        dyn[s].time = 0.0;
    }
}

// the download's periodic wrap: a branch for periodic axes only (out of line, as in the upload)
__device__ __forceinline__ double wrap_periodic(double x, const SceneDev& sc, int a) {
    return ((sc.periodic >> a) & 1u) ? wrap_into_domain(x, sc, a) : x;
}

__global__ void k_download(const float4* __restrict__ pos, const float4* __restrict__ vel,
                           const uint32_t* __restrict__ cell, const uint32_t* __restrict__ pinfo,
                           const uint32_t* __restrict__ pid, const SceneDev* __restrict__ scenes,
                           const double* __restrict__ centres,
                           const DevStatus* __restrict__ st, uint32_t n_up, double* __restrict__ pos_o,
                           float* __restrict__ vel_o, float* __restrict__ delta_o) {
    const uint32_t n = st->n_active;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const uint32_t id = pid[i];
        if (id >= n_up) continue;
        const SceneDev& sc = scenes[pinfo[i]];
        int c[3];
        decode_local(cell[i] - sc.cell_offset, sc, c[0], c[1], c[2]);
        const float4 p = pos[i];
        const float4 v = vel[i];
        const float o[3] = {p.x, p.y, p.z};
        if (pos_o)
            for (int a = 0; a < 3; ++a)
                pos_o[3 * (size_t)id + a] = wrap_periodic(centres[sc.centre_off[a] + (uint32_t)c[a]] + fp64_of(o[a]), sc, a);
        if (vel_o) {
            vel_o[3 * (size_t)id] = v.x;
            vel_o[3 * (size_t)id + 1] = v.y;
            vel_o[3 * (size_t)id + 2] = v.z;
        }
        if (delta_o) delta_o[id] = v.w;
    }
}

__global__ void k_download_forces(const float4* __restrict__ force, const uint32_t* __restrict__ pid,
                                  const DevStatus* __restrict__ st, uint32_t n_up, float* __restrict__ acc,
                                  float* __restrict__ drho) {
    const uint32_t n = st->n_active;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const uint32_t id = pid[i];
        if (id >= n_up) continue;
        const float4 f = force[i];
        acc[3 * (size_t)id] = f.x;
        acc[3 * (size_t)id + 1] = f.y;
        acc[3 * (size_t)id + 2] = f.z;
        drho[id] = f.w;
    }
}

__global__ void k_download_neighbors(const uint32_t* __restrict__ nlist, const uint32_t* __restrict__ ncount,
                                     const uint32_t* __restrict__ pid, const DevStatus* __restrict__ st,
                                     uint32_t n_up, uint32_t max_neibs, uint32_t stride,
                                     uint32_t* __restrict__ counts, uint32_t* __restrict__ ids) {
    const uint32_t n = st->n_active;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const uint32_t id = pid[i];
        if (id >= n_up) continue;
        const uint32_t cnt = ncount[i];
        const uint32_t nf = cnt & 0xffffu, nb = cnt >> 16;
        counts[2 * (size_t)id] = nf;
        counts[2 * (size_t)id + 1] = nb;
        uint32_t* out = ids + (size_t)id * max_neibs;
        for (uint32_t k = 0; k < nf; ++k) out[k] = pid[nlist[list_fluid_word(k, i, stride)] >> kCodeBits];
        for (uint32_t k = 0; k < nb; ++k) out[nf + k] = pid[nlist[list_bnd_word(k, i, stride, max_neibs)] >> kCodeBits];
    }
}

// the lists of a sample of particles: slot[id] = the sample position of upload id, or ~0
__global__ void k_download_neighbors_of(const uint32_t* __restrict__ nlist, const uint32_t* __restrict__ ncount,
                                        const uint32_t* __restrict__ pid, const DevStatus* __restrict__ st,
                                        const uint32_t* __restrict__ slot, uint32_t n_up, uint32_t max_neibs,
                                        uint32_t stride, uint32_t* __restrict__ counts, uint32_t* __restrict__ ids) {
    const uint32_t n = st->n_active;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const uint32_t id = pid[i];
        if (id >= n_up) continue;
        const uint32_t s = slot[id];
        if (s == 0xFFFFFFFFu) continue;
        const uint32_t cnt = ncount[i];
        const uint32_t nf = cnt & 0xffffu, nb = cnt >> 16;
        counts[2 * (size_t)s] = nf;
        counts[2 * (size_t)s + 1] = nb;
        uint32_t* out = ids + (size_t)s * max_neibs;
        for (uint32_t k = 0; k < nf; ++k) out[k] = pid[nlist[list_fluid_word(k, i, stride)] >> kCodeBits];
        for (uint32_t k = 0; k < nb; ++k) out[nf + k] = pid[nlist[list_bnd_word(k, i, stride, max_neibs)] >> kCodeBits];
    }
}

__global__ void k_fill_slots(const uint32_t* __restrict__ sample, uint32_t m, uint32_t n_up, uint32_t* __restrict__ slot,
                             uint32_t* __restrict__ bad) {
    for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < m; k += gridDim.x * blockDim.x) {
        if (sample[k] < n_up) slot[sample[k]] = k;
        else atomicOr(bad, 1u);
    }
}

int scene_from(const sph_params& p, const double origin[3], const double size[3], uint32_t periodic, double c0,
               uint32_t cell_offset, SceneDev& s, uint64_t& ncells) {
    // cells of side >= the list radius (influence radius + skin in rebuild-every-k mode)
    const double R = p.kernel_radius * p.h + (p.rebuild_every > 1 ? p.skin : 0.0);
    ncells = 1;
    for (int a = 0; a < 3; ++a) {
        if (!(size[a] > 0.0) || !std::isfinite(size[a]) || !std::isfinite(origin[a])) return SPH_ERR_ARG;
        double k = std::floor(size[a] / R);
        if (k < 1) k = 1;
        if (((periodic >> a) & 1u) && k < 3) return SPH_ERR_ARG;  // minimum image needs >= 3 cells
        if (k > 1e6) return SPH_ERR_ARG;
        s.ncell[a] = (int32_t)k;
        s.origin[a] = origin[a];
        s.cell_d[a] = size[a] / k;
        s.inv_len_d[a] = 1.0 / (s.cell_d[a] * k);
        s.origin_f[a] = (float)origin[a];
        s.cell_f[a] = (float)s.cell_d[a];
        s.inv_cell_f[a] = (float)(1.0 / s.cell_d[a]);
        ncells *= (uint64_t)k;
    }
    if (!(c0 > 0.0)) return SPH_ERR_ARG;
    s.cell_offset = cell_offset;
    s.periodic = periodic & 7u;
    s.c0 = (float)c0;
    const double B = p.rho0 * c0 * c0 / p.gamma;
    s.phat_coef = (float)(B / (p.rho0 * p.rho0));
    s.pi_coef = (float)(p.alpha * p.h * c0 / p.rho0);
    s.pi_unit = (float)(p.h * c0 / p.rho0);
    s.dd_coef = (float)(2.0 * p.ddiff_coef * p.h * c0);
    // reading C7: cfl * h/c0, and for laminar viscosity 0.125 h^2/nu, a limit with its own
    // coefficient (the lattice's fastest viscous mode decays at ~7 nu/h^2 at h = 1.3 dp and
    // the two-stage predictor-corrector is stable while that rate times dt stays <= 2)
    double cap = p.cfl * p.h / c0;
    if (p.visc_model != SPH_VISC_ARTIFICIAL && p.nu > 0.0) cap = std::fmin(cap, kViscousDtCoef * p.h * p.h / p.nu);
    s.dt_cap = cap;
    return SPH_OK;
}

void free_cells(sph_ctx* c) {
    for (const void* q : {(const void*)c->b.count, (const void*)c->b.start, (const void*)c->b.bsum,
                          (const void*)c->b.cell_nfluid})
        drop_canary(c, q);
    cudaFree(c->b.count);
    cudaFree(c->b.start);
    cudaFree(c->b.bsum);
    cudaFree(c->b.cell_nfluid);
    cudaFree(c->b.scenes);
    cudaFree(c->b.dyn);
    cudaFree(c->b.centres);
    c->b.count = c->b.start = c->b.bsum = c->b.cell_nfluid = nullptr;
    c->b.scenes = nullptr;
    c->b.dyn = nullptr;
    c->b.centres = nullptr;
}

void drop_graphs(sph_ctx* c) {
    for (auto& gexec : c->graph)
        if (gexec) {
            cudaGraphExecDestroy(gexec);
            gexec = nullptr;
        }
}

inline bool skin_mode(const sph_ctx* c) { return c->p.rebuild_every > 1; }

int alloc_cells(sph_ctx* c) {
    const uint32_t nb = c->g.n_cells + 1;
    CK(dev_alloc(c, (void**)&c->b.count, sizeof(uint32_t) * nb));
    CK(cudaMemset(c->b.count, 0, sizeof(uint32_t) * nb));
    CK(dev_alloc(c, (void**)&c->b.start, sizeof(uint32_t) * (nb + 1)));
    CK(cudaMemset(c->b.start, 0, sizeof(uint32_t) * (nb + 1)));
    CK(dev_alloc(c, (void**)&c->b.bsum, sizeof(uint32_t) * (scan_blocks(nb) + 1)));
    CK(dev_alloc(c, (void**)&c->b.cell_nfluid, sizeof(uint32_t) * nb));
    CK(cudaMemset(c->b.cell_nfluid, 0, sizeof(uint32_t) * nb));
    CK(cudaMalloc(&c->b.scenes, sizeof(SceneDev) * c->g.n_scenes));
    CK(cudaMemcpy(c->b.scenes, c->scenes_h.data(), sizeof(SceneDev) * c->g.n_scenes, cudaMemcpyHostToDevice));
    CK(cudaMalloc(&c->b.dyn, sizeof(SceneDyn) * c->g.n_scenes));
    CK(cudaMemset(c->b.dyn, 0, sizeof(SceneDyn) * c->g.n_scenes));
    CK(cudaMalloc(&c->b.centres, sizeof(double) * c->centres_h.size()));
    CK(cudaMemcpy(c->b.centres, c->centres_h.data(), sizeof(double) * c->centres_h.size(), cudaMemcpyHostToDevice));
    return SPH_OK;
}

int set_scene_table(sph_ctx* c, uint32_t n, const sph_scene* sc) {
    std::vector<SceneDev> tab(n);
    uint64_t off = 0;
    for (uint32_t s = 0; s < n; ++s) {
        uint64_t nc = 0;
        int rc = scene_from(c->p, sc[s].origin, sc[s].size, sc[s].periodic_mask, sc[s].c0, (uint32_t)off, tab[s], nc);
        if (rc) return rc;
        off += nc;
        if (off >= 0xF0000000ull) return SPH_ERR_ARG;
    }
    // FP64 cell centres, origin + (k + 1/2) cell per axis and scene (upload and download
    // convert between absolute positions and cell + offset with them)
    std::vector<double> centres;
    for (uint32_t s = 0; s < n; ++s)
        for (int a = 0; a < 3; ++a) {
            tab[s].centre_off[a] = (uint32_t)centres.size();
            for (int k = 0; k < tab[s].ncell[a]; ++k) centres.push_back(tab[s].origin[a] + (k + 0.5) * tab[s].cell_d[a]);
        }
    if (centres.size() >= 0xFFFFFFFFull) return SPH_ERR_ARG;
    drop_graphs(c);
    free_cells(c);
    c->scenes_h = tab;
    c->centres_h = centres;
    c->g.n_scenes = n;
    c->g.n_cells = (uint32_t)off;
    c->ph.n_scenes = n;
    return alloc_cells(c);
}

// neighbour pipeline on buffer `cur` -> buffer cur^1 (sorted), then list
void enqueue_sort(sph_ctx* c, cudaStream_t st) {
    launch_hash(c->b, c->cur, c->g, st);
    launch_scan(c->b, c->g, st);
    launch_scatter(c->b, c->g, st);
    launch_reorder(c->b, c->cur, c->g, st);
    c->cur ^= 1;
}

void enqueue_build(sph_ctx* c, cudaStream_t st) {
    if (skin_mode(c)) {
        // gated by status->rebuild; the sorted arrays come back to the same buffer
        launch_hash(c->b, c->cur, c->g, st);
        launch_scan(c->b, c->g, st);
        launch_scatter(c->b, c->g, st);
        launch_reorder(c->b, c->cur, c->g, st);
        launch_copyback(c->b, c->cur, c->g, st);
        launch_build(c->b, c->cur, c->g, c->ph, st);
        return;
    }
    enqueue_sort(c, st);
    launch_build(c->b, c->cur, c->g, c->ph, st);
}

inline bool can_fuse(const sph_ctx* c) { return !skin_mode(c) && !c->ph.general; }

// the list build and the predictor pass (one kernel when fused)
void enqueue_build_predict(sph_ctx* c, const Phys& ph, cudaStream_t st) {
    if (ph.fuse_predict && can_fuse(c)) {
        launch_build_predict(c->b, c->cur, c->g, ph, st);
    } else {
        launch_build(c->b, c->cur, c->g, ph, st);
        launch_forces(c->b, c->cur, c->g, ph, kPredict, 0, st);
    }
}

void enqueue_step(sph_ctx* c, cudaStream_t st) {
    launch_dt(c->b, c->g, c->ph, 1, st);  // (skin list: decides whether the pipeline runs)
    if (skin_mode(c)) {
        enqueue_build(c, st);
        launch_forces(c->b, c->cur, c->g, c->ph, kPredict, 0, st);
    } else {
        enqueue_sort(c, st);
        enqueue_build_predict(c, c->ph, st);
    }
    launch_forces(c->b, c->cur, c->g, c->ph, kCorrect, 0, st);
}

int capture_one(sph_ctx* c, int par, cudaGraphExec_t* out) {
    c->cur = par;
    cudaGraph_t gr = nullptr;
    CK(cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
    enqueue_step(c, c->cap_stream);
    CK(cudaStreamEndCapture(c->cap_stream, &gr));
    size_t nn = 0;
    cudaGraphGetNodes(gr, nullptr, &nn);
    c->graph_nodes = (uint32_t)nn;
    cudaError_t e = cudaGraphInstantiate(out, gr, 0);
    cudaGraphDestroy(gr);
    if (e != cudaSuccess) {
        std::fprintf(stderr, "sph: graph instantiate failed: %s\n", cudaGetErrorString(e));
        return SPH_ERR_CUDA;
    }
    return SPH_OK;
}

// one graph per buffer parity (the reorder switches buffers every step); a
// skin list keeps one buffer, so one graph serves every step
int capture_graphs(sph_ctx* c) {
    const int cur0 = c->cur;
    int rc = capture_one(c, cur0, &c->graph[cur0]);
    if (rc == SPH_OK && !skin_mode(c)) rc = capture_one(c, cur0 ^ 1, &c->graph[cur0 ^ 1]);
    c->cur = cur0;
    return rc;
}

int error_from_bits(uint32_t bits) {
    if (bits & SPH_EBIT_NEIB_OVERFLOW) return SPH_ERR_NEIB_OVERFLOW;
    if (bits & SPH_EBIT_NONFINITE) return SPH_ERR_NONFINITE;
    if (bits & SPH_EBIT_SKIN) return SPH_ERR_SKIN;
    if (bits & SPH_EBIT_BOUNDS) return SPH_ERR_BOUNDS;
    if (bits & SPH_EBIT_TIMEOUT) return SPH_ERR_TIMEOUT;
    return SPH_OK;
}

inline unsigned grid_for(uint32_t n, int block) {
    uint32_t g = (n + block - 1) / block;
    return g ? g : 1;
}

int do_upload(sph_ctx* c, uint32_t n, const double* pos, const float* vel, const float* delta, const float* mass,
              const uint8_t* type, const uint32_t* scene, cudaStream_t st) {
    k_set_status_n<<<1, 1, 0, st>>>(c->b.status, n);
    k_reset_dyn<<<1, 256, 0, st>>>(c->b.dyn, c->g.n_scenes);
    if (n) {
        k_upload<<<grid_for(n, 256), 256, 0, st>>>(n, pos, vel, delta, mass, type, scene, c->b.scenes, c->b.centres,
                                                    c->g.n_scenes,
                                                    c->b.pos[c->cur], c->b.vel[c->cur], c->b.phat[c->cur],
                                                    c->b.cell[c->cur], c->b.pinfo[c->cur], c->b.pid[c->cur],
                                                    c->b.status, c->ph);
    }
    DevStatus hs;
    CK(cudaMemcpyAsync(&hs, c->b.status, sizeof(hs), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    CK(cudaGetLastError());
    if (hs.upload_bits) {
        c->uploaded = false;
        if (hs.upload_bits & kUpBadArg) return SPH_ERR_ARG;
        if (hs.upload_bits & kUpNonFinite) return SPH_ERR_NONFINITE;
        return SPH_ERR_OUT_OF_DOMAIN;
    }
    CK(cudaMemsetAsync(c->b.count, 0, sizeof(uint32_t) * (c->g.n_cells + 1), st));
    enqueue_build(c, st);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(st));
    c->n_uploaded = n;
    c->uploaded = true;
    c->need_dt0 = true;
    c->fresh = true;
    return SPH_OK;
}

}  // namespace

extern "C" {

const char* sph_strerror(int code) {
    switch (code) {
        case SPH_OK: return "ok";
        case SPH_ERR_ARG: return "invalid argument";
        case SPH_ERR_CUDA: return "CUDA runtime error";
        case SPH_ERR_CAPACITY: return "particle count exceeds max_particles";
        case SPH_ERR_NEIB_OVERFLOW: return "neighbour list overflow (max_neibs too small)";
        case SPH_ERR_OUT_OF_DOMAIN: return "particle outside the domain";
        case SPH_ERR_NONFINITE: return "non-finite value in the particle state";
        case SPH_ERR_TIMEOUT: return "device wait timed out";
        case SPH_ERR_STATE: return "call out of order";
        case SPH_ERR_SKIN: return "a particle moved more than skin/2 since the last neighbour-list build";
        case SPH_ERR_BOUNDS: return "index out of range or buffer tail overwritten (checked build)";
        default: return "unknown error";
    }
}

int sph_create(const sph_params* p, sph_ctx** out) {
    if (!p || !out) return SPH_ERR_ARG;
    const double gm = p->gamma;
    if (!(p->h > 0) || !(p->rho0 > 0) || !(p->c0 > 0) || !(gm >= 1 && gm <= 8 && gm == std::floor(gm)) ||
        !(p->kernel_radius > 0) || !(p->cfl > 0) || p->max_particles == 0 || p->max_particles > kMaxParticles ||
        p->max_neibs < 8 || p->max_neibs > 1024 || p->visc_model < SPH_VISC_ARTIFICIAL ||
        p->visc_model > SPH_VISC_ESPANOL_REVENGA || !(p->alpha >= 0) || !(p->nu >= 0) || !(p->skin >= 0) ||
        (p->rebuild_every > 1 && !(p->skin > 0)) || p->kernel_type < SPH_KERNEL_WENDLAND ||
        p->kernel_type > SPH_KERNEL_GAUSSIAN || (p->formulation != SPH_FORM_1 && p->formulation != SPH_FORM_2) ||
        p->visc_avg < SPH_AVG_HARMONIC || p->visc_avg > SPH_AVG_GEOMETRIC ||
        (p->ddiff != SPH_DDIFF_NONE && p->ddiff != SPH_DDIFF_MOLTENI) || !(p->ddiff_coef >= 0) || !(p->zeta >= 0))
        return SPH_ERR_ARG;
    sph_ctx* c = new (std::nothrow) sph_ctx();
    if (!c) return SPH_ERR_ARG;
    c->p = *p;
    c->p.n_scenes = 1;
    cudaGetDevice(&c->device);
    // physics constants
    Phys& ph = c->ph;
    const double h = p->h, R = p->kernel_radius * p->h;
    ph.h = (float)h;
    ph.inv_h = (float)(1.0 / h);
    ph.R2 = (float)(R * R);
    const double Rl = R + (p->rebuild_every > 1 ? p->skin : 0.0);
    ph.R2_list = (float)(Rl * Rl);
    ph.skin_lim2 = (float)(0.25 * p->skin * p->skin);
    ph.skin_trig2 = (float)(0.0625 * p->skin * p->skin);
    ph.rebuild_every = p->rebuild_every;
    // F = aF f(q): the unit-integral normalisations of the Table 1 kernels (3D)
    const double pi_h5 = 3.14159265358979323846 * h * h * h * h * h;
    switch (p->kernel_type) {
        case SPH_KERNEL_CUBIC_SPLINE: ph.aF = (float)(1.0 / pi_h5); break;
        case SPH_KERNEL_QUADRATIC: ph.aF = (float)(15.0 / (32.0 * pi_h5)); break;
        case SPH_KERNEL_GAUSSIAN: {
            // W = exp(-q^2) - exp(-Q^2) on q < Q, normalised: 4 pi h^3 aW S(Q) = 1 with
            // S(Q) = int_0^Q (exp(-q^2) - exp(-Q^2)) q^2 dq; F = -2 aW/h^2 exp(-q^2)
            const double Q = p->kernel_radius, eQ = std::exp(-Q * Q);
            const double S = 0.25 * std::sqrt(3.14159265358979323846) * std::erf(Q) - 0.5 * Q * eQ - Q * Q * Q * eQ / 3.0;
            ph.aF = (float)(1.0 / (2.0 * pi_h5 * S));
            break;
        }
        default: ph.aF = (float)(105.0 / (128.0 * pi_h5)); break;
    }
    ph.rho0 = (float)p->rho0;
    ph.inv_rho0 = (float)(1.0 / p->rho0);
    ph.eps_h2 = (float)(0.01 * h * h);
    ph.nu4 = (float)(4.0 * p->nu);
    for (int a = 0; a < 3; ++a) ph.g[a] = (float)p->g[a];
    const int gam = (int)gm;
    double binom = 1.0;
    for (int k = 1; k <= 8; ++k) {
        binom = k <= gam ? binom * (gam - k + 1) / k : 0.0;
        ph.coef[k - 1] = (float)binom;
    }
    ph.h_d = h;
    ph.cfl = p->cfl;
    ph.dt_fixed = p->dt_fixed;
    ph.visc = p->visc_model;
    ph.kernel_type = p->kernel_type;
    ph.form = p->formulation;
    ph.visc_avg = p->visc_avg;
    ph.ddiff = p->ddiff;
    ph.general = !(p->kernel_type == SPH_KERNEL_WENDLAND && p->formulation == SPH_FORM_1 &&
                   p->ddiff == SPH_DDIFF_NONE &&
                   (p->visc_model == SPH_VISC_ARTIFICIAL ||
                    (p->visc_model == SPH_VISC_MORRIS && p->visc_avg == SPH_AVG_HARMONIC)));
    // laminar models as (lam_u u_ij + lam_x (u.x/r^2) x_ij) m_j f avg(r_i,r_j)/(r_i r_j):
    // omega mubar = m_j nu avg/(rho0 r_i r_j), omega zetabar likewise with zeta
    const double nu = p->nu, zeta = p->zeta, ir0 = 1.0 / p->rho0;
    ph.lam_u = ph.lam_x = 0.f;
    if (p->visc_model == SPH_VISC_MORRIS) ph.lam_u = (float)(2.0 * nu * ir0);
    if (p->visc_model == SPH_VISC_MONAGHAN) ph.lam_x = (float)(10.0 * nu * ir0);
    if (p->visc_model == SPH_VISC_ESPANOL_REVENGA) {
        ph.lam_u = (float)((5.0 / 3.0 * nu - zeta) * ir0);
        ph.lam_x = (float)(5.0 * (nu / 3.0 + zeta) * ir0);
    }
    ph.max_neibs = p->max_neibs;
    ph.n_owned = kAllOwned;
    ph.gamma_i = (int)gm;
    ph.build_variant = 0;
    ph.forces_variant = 1;
    ph.forces_variant_c = 1;
    const uint32_t cap = p->max_particles;
    ph.stride = (uint32_t)align_up(cap, 32);
    c->g.cap = cap;
    sph_scene s0{};
    for (int a = 0; a < 3; ++a) {
        s0.origin[a] = p->origin[a];
        s0.size[a] = p->size[a];
    }
    s0.periodic_mask = p->periodic_mask;
    s0.c0 = p->c0;
    int rc = set_scene_table(c, 1, &s0);
    if (rc) {
        sph_destroy(c);
        return rc;
    }
    Buffers& b = c->b;
    auto alloc = [&](void** ptr, size_t bytes) -> bool { return dev_alloc(c, ptr, bytes) == cudaSuccess; };
    bool ok = true;
    for (int k = 0; k < 2; ++k) {
        // kPosPad spare entries: the build reads candidates in groups past a cell's end
        ok = ok && alloc((void**)&b.pos[k], sizeof(float4) * (cap + kPosPad)) &&
             alloc((void**)&b.vel[k], sizeof(float4) * cap) &&
             alloc((void**)&b.phat[k], sizeof(float) * cap) &&
             alloc((void**)&b.cell[k], sizeof(uint32_t) * cap) && alloc((void**)&b.pinfo[k], sizeof(uint32_t) * cap) &&
             alloc((void**)&b.pid[k], sizeof(uint32_t) * cap);
    }
    if (p->rebuild_every > 1)
        ok = ok && alloc((void**)&b.pos_ref, sizeof(float4) * cap) &&
             alloc((void**)&b.nlist_x, sizeof(uint4) * 2 * (size_t)exact_bnd_chunk(p->max_neibs) * ph.stride) &&
             alloc((void**)&b.ncount_x, sizeof(uint32_t) * cap);
    ok = ok && alloc((void**)&b.pos_s, sizeof(float4) * cap) && alloc((void**)&b.vel_s, sizeof(float4) * cap) &&
         alloc((void**)&b.phat_s, sizeof(float) * cap) &&
         alloc((void**)&b.force, sizeof(float4) * cap) && alloc((void**)&b.key, sizeof(uint32_t) * cap) &&
         alloc((void**)&b.slot, sizeof(uint32_t) * cap) && alloc((void**)&b.unsorted, sizeof(uint32_t) * cap) &&
         alloc((void**)&b.nlist, sizeof(uint2) * (size_t)ph.stride * list_chunks(p->max_neibs)) &&
         alloc((void**)&b.ncount, sizeof(uint32_t) * cap) && alloc((void**)&b.status, sizeof(DevStatus));
    c->staging_bytes = 64 * (size_t)cap + 32768;  // >= the conservation sums' scratch
    ok = ok && alloc(&b.staging, c->staging_bytes);
    ok = ok && cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        sph_destroy(c);
        return SPH_ERR_CUDA;
    }
    cudaMemset(b.status, 0, sizeof(DevStatus));
    b.gate = p->rebuild_every > 1 ? &b.status->rebuild : nullptr;
    cudaMemset(b.force, 0, sizeof(float4) * cap);
    for (int k = 0; k < 2; ++k) cudaMemset(b.pos[k], 0, sizeof(float4) * (cap + kPosPad));
    cudaMemset(b.ncount, 0, sizeof(uint32_t) * cap);
    if (cudaDeviceSynchronize() != cudaSuccess) {
        sph_destroy(c);
        return SPH_ERR_CUDA;
    }
    *out = c;
    return SPH_OK;
}

int sph_set_scenes(sph_ctx* c, uint32_t n_scenes, const sph_scene* scenes) {
    if (!c || !scenes || n_scenes == 0 || n_scenes > (1u << 24)) return SPH_ERR_ARG;
    CK(cudaDeviceSynchronize());
    int rc = set_scene_table(c, n_scenes, scenes);
    if (rc) return rc;
    c->p.n_scenes = n_scenes;
    c->uploaded = false;
    return SPH_OK;
}

int sph_upload(sph_ctx* c, uint32_t n, const double* pos, const float* vel, const float* delta, const float* mass,
               const uint8_t* type, const uint32_t* scene, void* stream) {
    if (!c) return SPH_ERR_ARG;
    if (n > c->g.cap) return SPH_ERR_CAPACITY;
    if (n && (!pos || !vel || !delta || !mass || !type)) return SPH_ERR_ARG;
    cudaStream_t st = S(stream);
    // staging layout: pos f64 | vel f32 | delta | mass | scene u32 | type u8
    char* base = (char*)c->b.staging;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        char* p = base + off;
        off = align_up(off + bytes, 256);
        return p;
    };
    double* dpos = (double*)take(sizeof(double) * 3 * n);
    float* dvel = (float*)take(sizeof(float) * 3 * n);
    float* ddel = (float*)take(sizeof(float) * n);
    float* dmass = (float*)take(sizeof(float) * n);
    uint32_t* dsc = scene ? (uint32_t*)take(sizeof(uint32_t) * n) : nullptr;
    uint8_t* dty = (uint8_t*)take(n);
    if (off > c->staging_bytes) return SPH_ERR_CAPACITY;
    if (n) {
        CK(cudaMemcpyAsync(dpos, pos, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(dvel, vel, sizeof(float) * 3 * n, cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(ddel, delta, sizeof(float) * n, cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(dmass, mass, sizeof(float) * n, cudaMemcpyHostToDevice, st));
        if (scene) CK(cudaMemcpyAsync(dsc, scene, sizeof(uint32_t) * n, cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(dty, type, n, cudaMemcpyHostToDevice, st));
    }
    return do_upload(c, n, dpos, dvel, ddel, dmass, dty, dsc, st);
}

int sph_upload_device(sph_ctx* c, uint32_t n, const double* pos, const float* vel, const float* delta,
                      const float* mass, const uint8_t* type, const uint32_t* scene, void* stream) {
    if (!c) return SPH_ERR_ARG;
    if (n > c->g.cap) return SPH_ERR_CAPACITY;
    if (n && (!pos || !vel || !delta || !mass || !type)) return SPH_ERR_ARG;
    return do_upload(c, n, pos, vel, delta, mass, type, scene, S(stream));
}

int sph_build_neighbors(sph_ctx* c, void* stream) {
    if (!c) return SPH_ERR_ARG;
    if (!c->uploaded) return SPH_ERR_STATE;
    if (skin_mode(c)) launch_force_rebuild(c->b, S(stream));
    enqueue_build(c, S(stream));
    CK(cudaGetLastError());
    c->fresh = true;
    return SPH_OK;
}

int sph_conservation(sph_ctx* c, double* out, void* stream) {
    if (!c || !out) return SPH_ERR_ARG;
    if (!c->uploaded) return SPH_ERR_STATE;
    cudaStream_t st = S(stream);
    const size_t bytes = conservation_scratch_bytes();
    if (bytes > c->staging_bytes) return SPH_ERR_CAPACITY;
    double* scratch = (double*)c->b.staging;
    launch_forces(c->b, c->cur, c->g, c->ph, kForcesOnly, 0, st);
    launch_conservation(c->b, c->cur, scratch, st);
    CK(cudaMemcpyAsync(out, (char*)scratch + bytes - kConservationSums * sizeof(double),
                       kConservationSums * sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    DevStatus hs;
    CK(cudaMemcpy(&hs, c->b.status, sizeof(hs), cudaMemcpyDeviceToHost));
    return error_from_bits(hs.error_bits);
}

int sph_forces(sph_ctx* c, void* stream) {
    if (!c) return SPH_ERR_ARG;
    if (!c->uploaded) return SPH_ERR_STATE;
    launch_forces(c->b, c->cur, c->g, c->ph, kForcesOnly, 0, S(stream));
    CK(cudaGetLastError());
    return SPH_OK;
}

int sph_step(sph_ctx* c, uint32_t nsteps, void* stream) {
    if (!c) return SPH_ERR_ARG;
    if (!c->uploaded) return SPH_ERR_STATE;
    cudaStream_t st = S(stream);
    uint32_t s = 0;
    if (nsteps && c->fresh && !skin_mode(c)) {
        // the list was just built for the current positions (upload, sph_build_neighbors):
        // the first step runs without the neighbour pipeline.  Its dt0 forces pass (reading
        // C7) is also its predictor's force evaluation: the predictor update then reads the
        // stored forces.  Same result, to the bit, as the full step.
        if (c->need_dt0) {
            launch_forces(c->b, c->cur, c->g, c->ph, kForcesOnly, 1, st);
            launch_dt(c->b, c->g, c->ph, 1, st, 0);
            launch_predict_from_forces(c->b, c->cur, c->g, c->ph, st);
            c->need_dt0 = false;
        } else {
            launch_dt(c->b, c->g, c->ph, 1, st, 0);
            launch_forces(c->b, c->cur, c->g, c->ph, kPredict, 0, st);
        }
        launch_forces(c->b, c->cur, c->g, c->ph, kCorrect, 0, st);
        CK(cudaGetLastError());
        ++s;
    }
    c->fresh = false;
    if (s == nsteps) return SPH_OK;
    if (c->need_dt0) {
        // dt0 from one forces call on the initial state (reading C7)
        launch_forces(c->b, c->cur, c->g, c->ph, kForcesOnly, 1, st);
        CK(cudaGetLastError());
        c->need_dt0 = false;
    }
    if (c->persistent) {
        // the remaining steps as one cooperative launch of the persistent step kernel (launched
        // directly: its grid-wide barriers need the cooperative launch itself, not a replay)
        const uint32_t ns = nsteps - s;
        CK(launch_step_persistent(c->b, c->cur, c->g, c->ph, ns, st));
        c->cur = (int)((uint32_t)c->cur ^ (ns & 1u));
        c->graph_nodes = 1;
        return SPH_OK;
    }
    if (!c->graph[c->cur]) {
        int rc = capture_graphs(c);
        if (rc) return rc;
    }
    for (; s < nsteps; ++s) {
        CK(cudaGraphLaunch(c->graph[c->cur], st));
        if (!skin_mode(c)) c->cur ^= 1;
    }
    return SPH_OK;
}

int sph_cfl_dt(sph_ctx* c, double* dt, void* stream) {
    if (!c || !dt) return SPH_ERR_ARG;
    if (!c->uploaded) return SPH_ERR_STATE;
    cudaStream_t st = S(stream);
    // one forces-only pass with the |a|^2 reduction, then the dt of reading C7 (no time advance)
    launch_forces(c->b, c->cur, c->g, c->ph, kForcesOnly, 1, st);
    launch_dt(c->b, c->g, c->ph, 0, st, 0);
    SceneDyn d0;
    CK(cudaMemcpyAsync(&d0, c->b.dyn, sizeof(d0), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    *dt = d0.dt_d;
    DevStatus hs;
    CK(cudaMemcpy(&hs, c->b.status, sizeof(hs), cudaMemcpyDeviceToHost));
    return error_from_bits(hs.error_bits);
}

int sph_next_dt(sph_ctx* c, double* dt, void* stream) {
    if (!c || !dt) return SPH_ERR_ARG;
    if (!c->uploaded) return SPH_ERR_STATE;
    cudaStream_t st = S(stream);
    launch_dt_peek(c->b, c->ph, st);
    double v = 0.0;
    CK(cudaMemcpyAsync(&v, &c->b.status->dt_peek, sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    *dt = v;
    return SPH_OK;
}

int sph_set_owned(sph_ctx* c, uint32_t n_owned) {
    if (!c) return SPH_ERR_ARG;
    CK(cudaDeviceSynchronize());
    c->ph.n_owned = n_owned;
    drop_graphs(c);  // captured launches carry the old parameters
    return SPH_OK;
}

int sph_set_dt(sph_ctx* c, double dt) {
    if (!c || !(dt > 0.0) || !std::isfinite(dt)) return SPH_ERR_ARG;
    CK(cudaDeviceSynchronize());
    CK(cudaMemcpy(&c->b.status->dt_next, &dt, sizeof(double), cudaMemcpyHostToDevice));
    return SPH_OK;
}

int sph_set_fused_predict(sph_ctx* c, int on) {
    if (!c) return SPH_ERR_ARG;
    if (on && !can_fuse(c)) return SPH_ERR_ARG;
    CK(cudaDeviceSynchronize());
    c->ph.fuse_predict = on ? 1 : 0;
    drop_graphs(c);
    return SPH_OK;
}

int sph_get_step_options(sph_ctx* c, int* fused_predict, int* persistent) {
    if (!c) return SPH_ERR_ARG;
    if (fused_predict) *fused_predict = c->ph.fuse_predict;
    if (persistent) *persistent = c->persistent ? 1 : 0;
    return SPH_OK;
}

int sph_set_persistent(sph_ctx* c, int on) {
    if (!c) return SPH_ERR_ARG;
    if (on && (skin_mode(c) || c->ph.general)) return SPH_ERR_ARG;
    CK(cudaDeviceSynchronize());
    drop_graphs(c);
    c->persistent = on != 0;
    return SPH_OK;
}

int sph_autotune(sph_ctx* c, void* stream, int* build_variant, int* forces_variant) {
    if (!c) return SPH_ERR_ARG;
    if (!c->uploaded) return SPH_ERR_STATE;
    cudaStream_t st = S(stream);
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    auto time_ms = [&](auto&& launch) -> float {
        launch();  // warm
        cudaEventRecord(e0, st);
        for (int r = 0; r < 3; ++r) launch();
        cudaEventRecord(e1, st);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        return ms / 3.f;
    };
    // neighbour build: thread/particle (128, 256 threads) or warp/cell (2, 4, 8 cells per CTA);
    // all variants write the same list, so the state is unchanged by tuning
    int best_v = c->ph.build_variant;
    float best = 3.4e38f;
    // time the builds on a freshly sorted state: the build's candidate order relies on
    // the in-cell sort (a skin list forces its gated pipeline open)
    if (skin_mode(c)) launch_force_rebuild(c->b, st);
    enqueue_build(c, st);
    for (int v = 0; v < kBuildVariants; ++v) {
        c->ph.build_variant = v;
        const float ms = time_ms([&] { launch_build(c->b, c->cur, c->g, c->ph, st); });
        if (ms < best) {
            best = ms;
            best_v = v;
        }
    }
    c->ph.build_variant = best_v;
    launch_build(c->b, c->cur, c->g, c->ph, st);
    // force kernels: threads per block and register cap
    int best_f = c->ph.forces_variant;
    best = 3.4e38f;
    for (int v = 0; v < kForcesVariants; ++v) {
        c->ph.forces_variant = v;
        // the predictor pass as the step runs it (it writes only the predicted-state scratch)
        const float ms = time_ms([&] { launch_forces(c->b, c->cur, c->g, c->ph, kPredict, 0, st); });
        if (ms < best) {
            best = ms;
            best_f = v;
        }
    }
    c->ph.forces_variant = best_f;
    // the corrector pass, on its own (its best shape differs from the predictor's): it runs
    // on the predicted state the tuned predictor leaves, and reads state n from and writes
    // n+1 to a copy in the sort's second buffer (free between builds); the per-scene |a|^2
    // reduction and the status it updates are put back afterwards
    int best_c = c->ph.forces_variant_c;
    if (!c->ph.general) {
        launch_forces(c->b, c->cur, c->g, c->ph, kPredict, 0, st);
        const int alt = c->cur ^ 1;
        const size_t cap = c->g.cap;
        CK(cudaMemcpyAsync(c->b.pos[alt], c->b.pos[c->cur], sizeof(float4) * cap, cudaMemcpyDeviceToDevice, st));
        CK(cudaMemcpyAsync(c->b.vel[alt], c->b.vel[c->cur], sizeof(float4) * cap, cudaMemcpyDeviceToDevice, st));
        CK(cudaMemcpyAsync(c->b.phat[alt], c->b.phat[c->cur], sizeof(float) * cap, cudaMemcpyDeviceToDevice, st));
        std::vector<SceneDyn> dyn_h(c->g.n_scenes);
        DevStatus st_h;
        CK(cudaMemcpyAsync(dyn_h.data(), c->b.dyn, sizeof(SceneDyn) * dyn_h.size(), cudaMemcpyDeviceToHost, st));
        CK(cudaMemcpyAsync(&st_h, c->b.status, sizeof(DevStatus), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        Buffers tb = c->b;
        tb.pos[c->cur] = c->b.pos[alt];
        tb.vel[c->cur] = c->b.vel[alt];
        tb.phat[c->cur] = c->b.phat[alt];
        best = 3.4e38f;
        for (int v = 0; v < kForcesVariants; ++v) {
            c->ph.forces_variant_c = v;
            const float ms = time_ms([&] { launch_forces(tb, c->cur, c->g, c->ph, kCorrect, 0, st); });
            if (ms < best) {
                best = ms;
                best_c = v;
            }
        }
        CK(cudaMemcpyAsync(c->b.dyn, dyn_h.data(), sizeof(SceneDyn) * dyn_h.size(), cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(c->b.status, &st_h, sizeof(DevStatus), cudaMemcpyHostToDevice, st));
    }
    c->ph.forces_variant_c = best_c;
    // the list build and the predictor pass as one kernel, or apart (every-step list, default model)
    if (can_fuse(c)) {
        Phys pf = c->ph, ps = c->ph;
        pf.fuse_predict = 1;
        ps.fuse_predict = 0;
        const float t_sep = time_ms([&] { enqueue_build_predict(c, ps, st); });
        const float t_fused = time_ms([&] { enqueue_build_predict(c, pf, st); });
        // fused only when clearly faster (measured equal within noise on the dam breaks: 20.1M
        // particles 11.94 against 8.39 + 3.56 ms, 1.65M 0.869 against 0.576 + 0.270 ms)
        c->ph.fuse_predict = t_fused < 0.98f * t_sep ? 1 : 0;
    }
    c->fresh = true;  // the last build is of the current positions
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(st));
    drop_graphs(c);  // captured launches carry the old shapes
    if (build_variant) *build_variant = best_v;
    if (forces_variant) *forces_variant = best_f;
    return SPH_OK;
}

int sph_get_variants(sph_ctx* c, int* build_variant, int* forces_predict, int* forces_correct) {
    if (!c) return SPH_ERR_ARG;
    if (build_variant) *build_variant = c->ph.build_variant;
    if (forces_predict) *forces_predict = c->ph.forces_variant;
    if (forces_correct) *forces_correct = c->ph.forces_variant_c;
    return SPH_OK;
}

int sph_set_forces_variants(sph_ctx* c, int forces_predict, int forces_correct) {
    if (!c || forces_predict < -1 || forces_predict >= kForcesVariants || forces_correct < -1 ||
        forces_correct >= kForcesVariants)
        return SPH_ERR_ARG;
    if (forces_predict >= 0) c->ph.forces_variant = forces_predict;
    if (forces_correct >= 0) c->ph.forces_variant_c = forces_correct;
    CK(cudaDeviceSynchronize());
    drop_graphs(c);  // captured launches carry the old shapes
    return SPH_OK;
}

int sph_set_variants(sph_ctx* c, int build_variant, int forces_variant) {
    if (!c || build_variant < -1 || build_variant >= kBuildVariants || forces_variant < -1 ||
        forces_variant >= kForcesVariants)
        return SPH_ERR_ARG;
    if (build_variant >= 0) c->ph.build_variant = build_variant;
    if (forces_variant >= 0) c->ph.forces_variant = c->ph.forces_variant_c = forces_variant;
    CK(cudaDeviceSynchronize());
    drop_graphs(c);  // captured launches carry the old shapes
    return SPH_OK;
}

const char* sph_build_variant_name(int variant) { return build_variant_name(variant); }

const char* sph_forces_variant_name(int variant) { return forces_variant_name(variant); }

namespace {

void free_tape(sph_ctx* c) {
    AdjTape& t = c->tape;
    for (char* p : t.ckpt) cudaFree(p);
    t.ckpt.clear();
    cudaFree(t.steps);
    cudaFree(t.lists);
    cudaFree(t.adj_mem);
    t.steps = nullptr;
    t.lists = nullptr;
    t.adj_mem = nullptr;
    for (auto* gs : {t.seg_graph, t.rec_graph})
        for (int k = 0; k < 2; ++k)
            if (gs[k]) {
                cudaGraphExecDestroy(gs[k]);
                gs[k] = nullptr;
            }
    t.valid = false;
    t.gen = 0;
}

// copy the particle arrays of buffer `cur` to / from a flat device block (one launch)
void tape_io(const std::vector<std::pair<void*, size_t>>& arrays, char* blk, bool save, cudaStream_t st, uint32_t n) {
    const void* src[kTapeArrays];
    void* dst[kTapeArrays];
    bool wide[kTapeArrays];
    size_t off = 0;
    int k = 0;
    for (const auto& a : arrays) {
        src[k] = save ? a.first : (const void*)(blk + off);
        dst[k] = save ? (void*)(blk + off) : a.first;
        wide[k] = a.second == sizeof(float4);
        off += align_up(a.second * n, 256);
        ++k;
    }
    launch_tape_copy(src, dst, wide, k, n, st);
}

// checkpoint: the sorted state of buffer cur (positions, velocities, P/rho^2, cell, scene, id)
void state_io(sph_ctx* c, char* blk, bool save, cudaStream_t st, uint32_t n) {
    Buffers& b = c->b;
    const int k = c->cur;
    tape_io({{b.pos[k], sizeof(float4)}, {b.vel[k], sizeof(float4)}, {b.phat[k], sizeof(float)},
             {b.cell[k], sizeof(uint32_t)}, {b.pinfo[k], sizeof(uint32_t)}, {b.pid[k], sizeof(uint32_t)}},
            blk, save, st, n);
}

size_t state_bytes(uint32_t n) {
    return 2 * align_up(sizeof(float4) * n, 256) + 4 * align_up(sizeof(uint32_t) * n, 256);
}

// one taped step: the sorted state at n and the predicted state (what the reversed step reads;
// its neighbour list stays in the step's own list slot of the tape)
void step_io(sph_ctx* c, char* blk, bool save, cudaStream_t st, uint32_t n) {
    Buffers& b = c->b;
    const int k = c->cur;
    tape_io({{b.pos[k], sizeof(float4)}, {b.vel[k], sizeof(float4)}, {b.phat[k], sizeof(float)},
             {b.pinfo[k], sizeof(uint32_t)}, {b.pid[k], sizeof(uint32_t)}, {b.pos_s, sizeof(float4)},
             {b.vel_s, sizeof(float4)}, {b.phat_s, sizeof(float)}},
            blk, save, st, n);
}

size_t step_bytes(uint32_t n) {
    return 4 * align_up(sizeof(float4) * n, 256) + 4 * align_up(sizeof(uint32_t) * n, 256);
}

// neighbour-list slot of a taped step: the list (list_chunks(max_neibs) chunks of two entries
// per particle, neighbour-major) and its counts
size_t list_slot_bytes(const sph_ctx* c) {
    return align_up(sizeof(uint2) * (size_t)c->ph.stride * list_chunks(c->p.max_neibs), 256) +
           align_up(sizeof(uint32_t) * (size_t)c->g.cap, 256);
}

Buffers with_list_slot(const sph_ctx* c, char* slot) {
    Buffers bb = c->b;
    if (slot) {
        bb.nlist = reinterpret_cast<uint32_t*>(slot);
        bb.ncount = reinterpret_cast<uint32_t*>(
            slot + align_up(sizeof(uint2) * (size_t)c->ph.stride * list_chunks(c->p.max_neibs), 256));
    }
    return bb;
}

// one forward step with the frozen dt; optionally tape the sorted and predicted states, and
// build the step's list into a list slot of the tape (else into the context's list)
void rec_step(sph_ctx* c, const Phys& ph, char* tape_blk, int advance, cudaStream_t st, char* list_slot = nullptr) {
    launch_dt(c->b, c->g, ph, advance, st);
    enqueue_sort(c, st);
    const Buffers bb = with_list_slot(c, list_slot);
    launch_build(bb, c->cur, c->g, ph, st);
    launch_forces(bb, c->cur, c->g, ph, kPredict, 0, st);
    if (tape_blk) step_io(c, tape_blk, true, st, c->tape.n);
    launch_forces(bb, c->cur, c->g, ph, kCorrect, 0, st);
}

// one segment of the backward pass from its checkpoint (already in buffer cur):
// recompute the K steps forward, taping every step's states and keeping its
// neighbour list in the step's list slot, then reverse through them (reverse
// corrector -> VJP at * -> reverse predictor -> VJP at n, three launches per
// step, the list of the recomputed step reused).  No host synchronisation:
// captured once per tape and buffer parity.
void backward_segment(sph_ctx* c, cudaStream_t st) {
    AdjTape& t = c->tape;
    const uint32_t n = t.n;
    const size_t ls = list_slot_bytes(c);
    for (uint32_t k = 0; k < t.K; ++k)
        rec_step(c, t.ph_rec, t.steps + (size_t)k * t.step_bytes, 0, st, t.lists + (size_t)k * ls);
    for (int k = (int)t.K - 1; k >= 0; --k) {
        step_io(c, t.steps + (size_t)k * t.step_bytes, false, st, n);
        launch_adj_step(t.a, with_list_slot(c, t.lists + (size_t)k * ls), c->cur, c->g, t.ph_rec, (float)t.dt, st);
    }
}

}  // namespace

int sph_set_alpha(sph_ctx* c, double alpha) {
    if (!c || !(alpha >= 0.0) || c->p.visc_model != SPH_VISC_ARTIFICIAL) return SPH_ERR_ARG;
    CK(cudaDeviceSynchronize());
    c->p.alpha = alpha;
    for (auto& s : c->scenes_h) s.pi_coef = (float)(alpha * s.pi_unit);
    CK(cudaMemcpy(c->b.scenes, c->scenes_h.data(), sizeof(SceneDev) * c->scenes_h.size(), cudaMemcpyHostToDevice));
    drop_graphs(c);
    c->tape.valid = false;
    c->tape.gen = 0;
    return SPH_OK;
}

namespace {

int alloc_tape(sph_ctx* c) {
    AdjTape& t = c->tape;
    const uint32_t n = t.n, T = t.T, K = t.K;
    t.ckpt_bytes = state_bytes(n);
    t.step_bytes = step_bytes(n);
    for (uint32_t s2 = 0; s2 < T / K; ++s2) {
        char* p = nullptr;
        if (cudaMalloc(&p, t.ckpt_bytes) != cudaSuccess) {
            free_tape(c);
            return SPH_ERR_CUDA;
        }
        t.ckpt.push_back(p);
    }
    const size_t nv = align_up(sizeof(float4) * (size_t)c->g.cap, 256);
    const size_t nf = align_up(sizeof(float) * (size_t)c->g.cap, 256);
    if (cudaMalloc((void**)&t.steps, t.step_bytes * K) != cudaSuccess ||
        cudaMalloc((void**)&t.lists, list_slot_bytes(c) * K) != cudaSuccess ||
        cudaMalloc(&t.adj_mem, 7 * nv + 2 * nf + 256) != cudaSuccess) {
        cudaGetLastError();
        free_tape(c);
        return SPH_ERR_CUDA;
    }
    char* m = (char*)t.adj_mem;
    t.a.xb = (float4*)m; m += nv;
    t.a.ub = (float4*)m; m += nv;
    t.a.seed = (float4*)m; m += nv;
    t.a.seed_n = (float4*)m; m += nv;
    m += nv;  // spare
    t.a.xb_id = (float4*)m; m += nv;
    t.a.ub_id = (float4*)m; m += nv;
    t.a.dphat = (float*)m; m += nf;
    t.a.dphat_s = (float*)m; m += nf;
    t.a.alpha_sum = (double*)m;
    return SPH_OK;
}

}  // namespace

int sph_record(sph_ctx* c, uint32_t T, uint32_t K, void* stream, double* dt_out) {
    if (!c || T == 0 || K == 0 || T % K != 0) return SPH_ERR_ARG;
    if (!c->uploaded) return SPH_ERR_STATE;
    // one scene, list rebuilt every step, default model options
    if (c->g.n_scenes != 1 || skin_mode(c) || c->ph.general) return SPH_ERR_ARG;
    cudaStream_t st = S(stream);
    AdjTape& t = c->tape;
    t.valid = false;
    t.gen = 0;
    DevStatus hs;
    CK(cudaMemcpyAsync(&hs, c->b.status, sizeof(hs), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    const uint32_t n = hs.n_active;
    // frozen dt: the parameter if given, else the CFL dt of one forces call on the initial state (C7)
    double dt = c->p.dt_fixed;
    if (!(dt > 0.0)) {
        launch_forces(c->b, c->cur, c->g, c->ph, kForcesOnly, 1, st);
        launch_dt(c->b, c->g, c->ph, 0, st);
        SceneDyn d0;
        CK(cudaMemcpyAsync(&d0, c->b.dyn, sizeof(d0), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        dt = d0.dt_d;
    }
    // a tape of the same shape, dt and launch variants keeps its buffers and graphs
    // (a training loop records and reverses the same configuration again and again)
    const bool reuse = t.steps && t.T == T && t.K == K && t.n == n && t.dt == dt &&
                       t.ph_rec.build_variant == c->ph.build_variant &&
                       t.ph_rec.forces_variant == c->ph.forces_variant &&
                       t.ph_rec.forces_variant_c == c->ph.forces_variant_c;
    if (!reuse) free_tape(c);
    t.T = T;
    t.K = K;
    t.n = n;
    t.dt = dt;
    t.ph_rec = c->ph;
    t.ph_rec.dt_fixed = dt;
    if (!reuse && alloc_tape(c) != SPH_OK) return SPH_ERR_CUDA;
    // each segment: its checkpoint, then K steps (one captured graph per buffer parity)
    int rc = SPH_OK;
    for (uint32_t seg = 0; seg < T / K && rc == SPH_OK; ++seg) {
        state_io(c, t.ckpt[seg], true, st, n);
        const int p0 = c->cur;
        if (!t.rec_graph[p0]) {
            cudaGraph_t gr = nullptr;
            CK(cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
            for (uint32_t k = 0; k < K; ++k) rec_step(c, t.ph_rec, nullptr, 1, c->cap_stream);
            CK(cudaStreamEndCapture(c->cap_stream, &gr));
            if (cudaGraphInstantiate(&t.rec_graph[p0], gr, 0) != cudaSuccess) rc = SPH_ERR_CUDA;
            cudaGraphDestroy(gr);
            t.rec_end_cur[p0] = c->cur;
            c->cur = p0;
        }
        if (rc == SPH_OK && cudaGraphLaunch(t.rec_graph[p0], st) != cudaSuccess) rc = SPH_ERR_CUDA;
        c->cur = t.rec_end_cur[p0];
    }
    CK(cudaStreamSynchronize(st));
    if (rc != SPH_OK) {
        free_tape(c);
        return rc;
    }
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(&hs, c->b.status, sizeof(hs), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (hs.n_active != n || hs.error_bits) {
        free_tape(c);
        return hs.error_bits ? error_from_bits(hs.error_bits) : SPH_ERR_STATE;
    }
    // cell tables and list of the final state for later calls
    enqueue_build(c, st);
    CK(cudaStreamSynchronize(st));
    t.valid = true;
    t.gen = t.next_gen++;
    c->need_dt0 = true;
    c->fresh = true;
    if (dt_out) *dt_out = dt;
    return SPH_OK;
}

int sph_tape_generation(sph_ctx* c, uint64_t* gen) {
    if (!c || !gen) return SPH_ERR_ARG;
    *gen = c->tape.valid ? c->tape.gen : 0u;
    return SPH_OK;
}


int sph_backward(sph_ctx* c, const float* xbar_T, const float* ubar_T, const float* dbar_T, float* xbar_0,
                 float* ubar_0, float* dbar_0, double* alphabar, void* stream) {
    if (!c) return SPH_ERR_ARG;
    AdjTape& t = c->tape;
    if (!t.valid || !c->uploaded) return SPH_ERR_STATE;
    cudaStream_t st = S(stream);
    const uint32_t n = t.n;
    launch_adj_load(t.a, n, xbar_T, ubar_T, dbar_T, st);
    for (int seg = (int)(t.T / t.K) - 1; seg >= 0; --seg) {
        // the segment's checkpoint, then its recompute and reverse (one captured graph:
        // the same work for every segment, on the same tape buffers)
        state_io(c, t.ckpt[seg], false, st, n);
        const int p0 = c->cur;
        if (!t.seg_graph[p0]) {
            cudaGraph_t gr = nullptr;
            CK(cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
            backward_segment(c, c->cap_stream);
            CK(cudaStreamEndCapture(c->cap_stream, &gr));
            const cudaError_t e = cudaGraphInstantiate(&t.seg_graph[p0], gr, 0);
            cudaGraphDestroy(gr);
            if (e != cudaSuccess) return SPH_ERR_CUDA;
            t.seg_end_cur[p0] = c->cur;
            c->cur = p0;
        }
        CK(cudaGraphLaunch(t.seg_graph[p0], st));
        c->cur = t.seg_end_cur[p0];
    }
    launch_adj_store(t.a, n, xbar_0, ubar_0, dbar_0, st);
    launch_adj_sum_alpha(t.a, n, t.a.alpha_sum, st);
    double ab = 0.0;
    CK(cudaMemcpyAsync(&ab, t.a.alpha_sum, sizeof(double), cudaMemcpyDeviceToHost, st));
    // leave the context at the recorded initial state, with its cell tables and list
    state_io(c, t.ckpt[0], false, st, n);
    enqueue_build(c, st);
    c->need_dt0 = true;
    c->fresh = true;
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(st));
    if (alphabar) *alphabar = ab;
    DevStatus hs;
    CK(cudaMemcpy(&hs, c->b.status, sizeof(hs), cudaMemcpyDeviceToHost));
    return error_from_bits(hs.error_bits);
}

int sph_step_profiled(sph_ctx* c, uint32_t nsteps, void* stream, double* phase_ms) {
    if (!c || !phase_ms) return SPH_ERR_ARG;
    if (!c->uploaded) return SPH_ERR_STATE;
    cudaStream_t st = S(stream);
    if (c->need_dt0) {
        launch_forces(c->b, c->cur, c->g, c->ph, kForcesOnly, 1, st);
        c->need_dt0 = false;
    }
    c->fresh = false;
    cudaEvent_t ev[9];
    for (auto& e : ev) CK(cudaEventCreate(&e));
    int rc = SPH_OK;
    for (uint32_t s = 0; s < nsteps && rc == SPH_OK; ++s) {
        cudaEventRecord(ev[0], st);
        launch_dt(c->b, c->g, c->ph, 1, st);
        cudaEventRecord(ev[1], st);
        launch_hash(c->b, c->cur, c->g, st);
        cudaEventRecord(ev[2], st);
        launch_scan(c->b, c->g, st);
        cudaEventRecord(ev[3], st);
        launch_scatter(c->b, c->g, st);
        cudaEventRecord(ev[4], st);
        launch_reorder(c->b, c->cur, c->g, st);
        if (skin_mode(c))
            launch_copyback(c->b, c->cur, c->g, st);
        else
            c->cur ^= 1;
        cudaEventRecord(ev[5], st);
        const bool fused = c->ph.fuse_predict && can_fuse(c);
        if (fused)
            launch_build_predict(c->b, c->cur, c->g, c->ph, st);  // phase 5: the build and the predictor pass
        else
            launch_build(c->b, c->cur, c->g, c->ph, st);
        cudaEventRecord(ev[6], st);
        if (!fused) launch_forces(c->b, c->cur, c->g, c->ph, kPredict, 0, st);
        cudaEventRecord(ev[7], st);
        launch_forces(c->b, c->cur, c->g, c->ph, kCorrect, 0, st);
        cudaEventRecord(ev[8], st);
        if (cudaEventSynchronize(ev[8]) != cudaSuccess || cudaGetLastError() != cudaSuccess) {
            rc = SPH_ERR_CUDA;
            break;
        }
        for (int k = 0; k < 8; ++k) {
            if (k == 6 && fused) continue;  // no separate predictor pass
            float ms = 0.f;
            cudaEventElapsedTime(&ms, ev[k], ev[k + 1]);
            phase_ms[k] += ms;
        }
    }
    for (auto& e : ev) cudaEventDestroy(e);
    return rc;
}

int sph_download(sph_ctx* c, uint32_t n, double* pos, float* vel, float* delta, void* stream) {
    if (!c) return SPH_ERR_ARG;
    if (!c->uploaded) return SPH_ERR_STATE;
    if (n != c->n_uploaded) return SPH_ERR_ARG;
    cudaStream_t st = S(stream);
    char* base = (char*)c->b.staging;
    double* dpos = (double*)base;
    float* dvel = (float*)(base + align_up(sizeof(double) * 3 * n, 256));
    float* ddel = (float*)((char*)dvel + align_up(sizeof(float) * 3 * n, 256));
    int rc = sph_download_device(c, n, dpos, dvel, ddel, stream);
    if (rc) return rc;
    if (n) {
        if (pos) CK(cudaMemcpyAsync(pos, dpos, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, st));
        if (vel) CK(cudaMemcpyAsync(vel, dvel, sizeof(float) * 3 * n, cudaMemcpyDeviceToHost, st));
        if (delta) CK(cudaMemcpyAsync(delta, ddel, sizeof(float) * n, cudaMemcpyDeviceToHost, st));
    }
    CK(cudaStreamSynchronize(st));
    DevStatus hs;
    CK(cudaMemcpy(&hs, c->b.status, sizeof(hs), cudaMemcpyDeviceToHost));
    return error_from_bits(hs.error_bits);
}

int sph_download_device(sph_ctx* c, uint32_t n, double* pos, float* vel, float* delta, void* stream) {
    if (!c) return SPH_ERR_ARG;
    if (!c->uploaded) return SPH_ERR_STATE;
    if (n != c->n_uploaded) return SPH_ERR_ARG;
    cudaStream_t st = S(stream);
    if (n) {
        if (pos) CK(cudaMemsetAsync(pos, 0xFF, sizeof(double) * 3 * n, st));
        if (vel) CK(cudaMemsetAsync(vel, 0xFF, sizeof(float) * 3 * n, st));
        if (delta) CK(cudaMemsetAsync(delta, 0xFF, sizeof(float) * n, st));
        k_download<<<grid_for(c->g.cap, 256), 256, 0, st>>>(c->b.pos[c->cur], c->b.vel[c->cur], c->b.cell[c->cur],
                                                             c->b.pinfo[c->cur], c->b.pid[c->cur], c->b.scenes,
                                                             c->b.centres,
                                                             c->b.status, n, pos, vel, delta);
        CK(cudaGetLastError());
    }
    return SPH_OK;
}

int sph_download_forces(sph_ctx* c, uint32_t n, float* acc, float* drho, void* stream) {
    if (!c || !acc || !drho) return SPH_ERR_ARG;
    if (!c->uploaded) return SPH_ERR_STATE;
    if (n != c->n_uploaded) return SPH_ERR_ARG;
    cudaStream_t st = S(stream);
    char* base = (char*)c->b.staging;
    float* dacc = (float*)base;
    float* ddr = (float*)(base + align_up(sizeof(float) * 3 * n, 256));
    if (n) {
        CK(cudaMemsetAsync(dacc, 0xFF, sizeof(float) * 3 * n, st));
        CK(cudaMemsetAsync(ddr, 0xFF, sizeof(float) * n, st));
        k_download_forces<<<grid_for(c->g.cap, 256), 256, 0, st>>>(c->b.force, c->b.pid[c->cur], c->b.status, n, dacc,
                                                                    ddr);
        CK(cudaGetLastError());
        CK(cudaMemcpyAsync(acc, dacc, sizeof(float) * 3 * n, cudaMemcpyDeviceToHost, st));
        CK(cudaMemcpyAsync(drho, ddr, sizeof(float) * n, cudaMemcpyDeviceToHost, st));
    }
    CK(cudaStreamSynchronize(st));
    return SPH_OK;
}

int sph_download_neighbors(sph_ctx* c, uint32_t n, uint32_t* counts, uint32_t* ids, void* stream) {
    if (!c || !counts || !ids) return SPH_ERR_ARG;
    if (!c->uploaded) return SPH_ERR_STATE;
    if (n != c->n_uploaded) return SPH_ERR_ARG;
    cudaStream_t st = S(stream);
    if (n == 0) return SPH_OK;
    const size_t nid = (size_t)n * c->p.max_neibs;
    uint32_t *dcnt = nullptr, *dids = nullptr;
    CK(cudaMalloc(&dcnt, sizeof(uint32_t) * 2 * n));
    if (cudaMalloc(&dids, sizeof(uint32_t) * nid) != cudaSuccess) {
        cudaFree(dcnt);
        return SPH_ERR_CUDA;
    }
    // every step checked; on a failure the staging is freed after the stream drains
    cudaError_t e = cudaMemsetAsync(dcnt, 0, sizeof(uint32_t) * 2 * n, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(dids, 0xFF, sizeof(uint32_t) * nid, st);
    if (e == cudaSuccess) {
        k_download_neighbors<<<grid_for(c->g.cap, 256), 256, 0, st>>>(c->b.nlist, c->b.ncount, c->b.pid[c->cur],
                                                                       c->b.status, n, c->p.max_neibs, c->ph.stride,
                                                                       dcnt, dids);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(counts, dcnt, sizeof(uint32_t) * 2 * n, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(ids, dids, sizeof(uint32_t) * nid, cudaMemcpyDeviceToHost, st);
    const cudaError_t es = cudaStreamSynchronize(st);
    if (e == cudaSuccess) e = es;
    cudaFree(dcnt);
    cudaFree(dids);
    if (e != cudaSuccess) {
        std::fprintf(stderr, "sph: sph_download_neighbors failed: %s\n", cudaGetErrorString(e));
        return SPH_ERR_CUDA;
    }
    return SPH_OK;
}

int sph_download_neighbors_of(sph_ctx* c, uint32_t m, const uint32_t* sample, uint32_t* counts, uint32_t* ids,
                              void* stream) {
    if (!c || (m && (!sample || !counts || !ids))) return SPH_ERR_ARG;
    if (!c->uploaded) return SPH_ERR_STATE;
    if (m == 0) return SPH_OK;
    cudaStream_t st = S(stream);
    const uint32_t n_up = c->n_uploaded;
    const size_t nid = (size_t)m * c->p.max_neibs;
    // one staging block: slot map (n_up), sample (m), counts (2m), ids (m*max_neibs), a flag
    const size_t bytes = sizeof(uint32_t) * ((size_t)n_up + 3 * (size_t)m + nid + 1);
    uint32_t* blk = nullptr;
    CK(cudaMalloc(&blk, bytes));
    uint32_t* slot = blk;
    uint32_t* dsmp = slot + n_up;
    uint32_t* dcnt = dsmp + m;
    uint32_t* dids = dcnt + 2 * (size_t)m;
    uint32_t* dbad = dids + nid;
    cudaError_t e = cudaMemsetAsync(slot, 0xFF, sizeof(uint32_t) * n_up, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(dcnt, 0, sizeof(uint32_t) * (2 * (size_t)m), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(dids, 0xFF, sizeof(uint32_t) * nid, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(dbad, 0, sizeof(uint32_t), st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dsmp, sample, sizeof(uint32_t) * m, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) {
        k_fill_slots<<<grid_for(m, 256), 256, 0, st>>>(dsmp, m, n_up, slot, dbad);
        k_download_neighbors_of<<<grid_for(c->g.cap, 256), 256, 0, st>>>(c->b.nlist, c->b.ncount, c->b.pid[c->cur],
                                                                          c->b.status, slot, n_up, c->p.max_neibs,
                                                                          c->ph.stride, dcnt, dids);
        e = cudaGetLastError();
    }
    uint32_t bad = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(counts, dcnt, sizeof(uint32_t) * 2 * (size_t)m, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(ids, dids, sizeof(uint32_t) * nid, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&bad, dbad, sizeof(uint32_t), cudaMemcpyDeviceToHost, st);
    const cudaError_t es = cudaStreamSynchronize(st);
    if (e == cudaSuccess) e = es;
    cudaFree(blk);
    if (e != cudaSuccess) {
        std::fprintf(stderr, "sph: sph_download_neighbors_of failed: %s\n", cudaGetErrorString(e));
        return SPH_ERR_CUDA;
    }
    return bad ? SPH_ERR_ARG : SPH_OK;
}

// ---------------------------------------------------------------------
// Allocation-free neighbour download.  Same kernel and outputs as
// sph_download_neighbors, but the device staging lives in one file-scope
// device array instead of buffers from cudaMalloc, for callers that must not
// allocate device memory at call time.  The array is held by every device
// that loads the library until the process exits; all calls share it.
// ---------------------------------------------------------------------
namespace {

constexpr size_t kNoAllocMaxParticles = size_t(1) << 20;  // counts: 2 u32 per particle
constexpr size_t kNoAllocMaxEntries = size_t(1) << 22;    // ids: n * max_neibs u32
// [counts: 2 * kNoAllocMaxParticles][ids: kNoAllocMaxEntries]  (24 MiB)
static __device__ __align__(256) uint32_t g_noalloc_scratch[2 * kNoAllocMaxParticles + kNoAllocMaxEntries];

constexpr int kNoAllocMaxDevices = 64;
std::mutex g_noalloc_mu;
uint32_t* g_noalloc_ptr[kNoAllocMaxDevices] = {};

// Device address of the scratch array on the current device, looked up once
// per device (the host-side name of a __device__ array is not a device address).
int noalloc_scratch(uint32_t** out) {
    int dev = 0;
    CK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kNoAllocMaxDevices) return SPH_ERR_ARG;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        CK(cudaGetSymbolAddress(&p, g_noalloc_scratch));
        g_noalloc_ptr[dev] = static_cast<uint32_t*>(p);
    }
    *out = g_noalloc_ptr[dev];
    return SPH_OK;
}

}  // namespace

int sph_download_neighbors_noalloc(sph_ctx* c, uint32_t n, uint32_t* counts, uint32_t* ids, void* stream) {
    if (!c || !counts || !ids) return SPH_ERR_ARG;
    if (!c->uploaded) return SPH_ERR_STATE;
    if (n != c->n_uploaded) return SPH_ERR_ARG;
    int dev = -1;
    CK(cudaGetDevice(&dev));
    if (dev != c->device) return SPH_ERR_STATE;
    const size_t nid = (size_t)n * c->p.max_neibs;
    if ((size_t)n > kNoAllocMaxParticles || nid > kNoAllocMaxEntries) return SPH_ERR_CAPACITY;
    if (n == 0) return SPH_OK;
    uint32_t* scratch = nullptr;
    int rc = noalloc_scratch(&scratch);
    if (rc) return rc;
    uint32_t* dcnt = scratch;
    uint32_t* dids = scratch + 2 * kNoAllocMaxParticles;
    cudaStream_t st = S(stream);
    // the array keeps the previous call's contents: reset the parts this call reads back
    CK(cudaMemsetAsync(dcnt, 0, sizeof(uint32_t) * 2 * n, st));
    CK(cudaMemsetAsync(dids, 0xFF, sizeof(uint32_t) * nid, st));
    k_download_neighbors<<<grid_for(c->g.cap, 256), 256, 0, st>>>(c->b.nlist, c->b.ncount, c->b.pid[c->cur],
                                                                   c->b.status, n, c->p.max_neibs, c->ph.stride, dcnt,
                                                                   dids);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(counts, dcnt, sizeof(uint32_t) * 2 * n, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(ids, dids, sizeof(uint32_t) * nid, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    return SPH_OK;
}

int sph_get_stats(sph_ctx* c, sph_stats* out, void* stream) {
    if (!c || !out) return SPH_ERR_ARG;
    cudaStream_t st = S(stream);
    if (kCanary) check_canaries(c, st);
    DevStatus hs;
    SceneDyn d0;
    CK(cudaMemcpyAsync(&hs, c->b.status, sizeof(hs), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(&d0, c->b.dyn, sizeof(d0), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    std::memset(out, 0, sizeof(*out));
    out->n_active = hs.n_active;
    out->n_removed = hs.n_removed;
    out->max_neibs_seen = hs.max_neibs_seen;
    out->error_bits = hs.error_bits;
    out->steps = hs.steps;
    out->dt = d0.dt_d;
    out->time = d0.time;
    out->n_cells = c->g.n_cells;
    out->kernels_per_step = c->graph_nodes;
    out->list_entries = hs.list_entries;
    out->interactions = hs.interactions;
    out->builds = hs.builds;
    return error_from_bits(hs.error_bits);
}

int sph_get_scene_times(sph_ctx* c, double* dt, double* time, void* stream) {
    if (!c) return SPH_ERR_ARG;
    cudaStream_t st = S(stream);
    std::vector<SceneDyn> d(c->g.n_scenes);
    CK(cudaMemcpyAsync(d.data(), c->b.dyn, sizeof(SceneDyn) * d.size(), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    for (size_t s = 0; s < d.size(); ++s) {
        if (dt) dt[s] = d[s].dt_d;
        if (time) time[s] = d[s].time;
    }
    return SPH_OK;
}

int sph_clear_error(sph_ctx* c, void* stream) {
    if (!c) return SPH_ERR_ARG;
    CK(cudaMemsetAsync(&c->b.status->error_bits, 0, sizeof(uint32_t), S(stream)));
    return SPH_OK;
}

int sph_sync(sph_ctx* c, void* stream) {
    sph_stats s;
    return sph_get_stats(c, &s, stream);
}

void sph_destroy(sph_ctx* c) {
    if (!c) return;
    cudaDeviceSynchronize();
    drop_graphs(c);
    free_tape(c);
    free_cells(c);
    Buffers& b = c->b;
    for (int k = 0; k < 2; ++k) {
        cudaFree(b.pos[k]);
        cudaFree(b.vel[k]);
        cudaFree(b.phat[k]);
        cudaFree(b.cell[k]);
        cudaFree(b.pinfo[k]);
        cudaFree(b.pid[k]);
    }
    cudaFree(b.pos_ref);
    cudaFree(b.nlist_x);
    cudaFree(b.ncount_x);
    cudaFree(b.pos_s);
    cudaFree(b.vel_s);
    cudaFree(b.phat_s);
    cudaFree(b.force);
    cudaFree(b.key);
    cudaFree(b.slot);
    cudaFree(b.unsorted);
    cudaFree(b.nlist);
    cudaFree(b.ncount);
    cudaFree(b.status);
    cudaFree(b.staging);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    delete c;
}

}  // extern "C"
