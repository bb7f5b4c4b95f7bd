// Internal definitions shared by the library's translation units.
//
// Data layout in HBM (all arrays sorted by (cell, type, id) after each
// neighbour pipeline, capacity `cap` particles):
//   pos4[i]  float4 (ox, oy, oz, +-m): offset from the centre of the
//            particle's cell (cell-relative positions, paper Section 2.3:
//            uniform FP32 accuracy without extended precision); w holds the
//            mass, negated for boundary particles (type in the sign bit).
//   vel4[i]  float4 (ux, uy, uz, delta): velocity and relative density
//            delta = rho/rho0 - 1 (FP32 near rest keeps ~1e-7 relative
//            accuracy in P, which absolute rho ~ 1000 would not).
//   cell[i]  u32 global cell key (scene cell offset + linear cell index).
//   pinfo[i] u32 scene index.   pid[i] u32 upload id.
//   nlist    uint2[list_chunks(max_neibs) * stride], neighbour-major in
//            chunks of two entries (chunk c of particle i at c*stride + i:
//            the paper's Section 4 "interleaved" layout, two slots wide);
//            fluid neighbours from chunk 0 up, boundary neighbours from the
//            last chunk down (see list_chunks).  Entry = j << 6 | code,
//            code = 2 bits per axis of the cell delta (d+1), so the
//            separation is x_ij = o_i - o_j - d * cell (periodic images too).
//   ncount[i] u32 nf | nb << 16.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "sph.h"

namespace sphg {

constexpr uint32_t kMarker = 0xFFFFFFFFu;
// skin list: first chunk (of four entries) of the boundary part of the step's exact list
__host__ __device__ constexpr uint32_t exact_bnd_chunk(uint32_t max_neibs) { return (max_neibs + 3u) / 4u; }
constexpr int kCodeBits = 6;
constexpr uint32_t kMaxParticles = 1u << (32 - kCodeBits);

// ---- neighbour list layout ------------------------------------------------
// Two entries per chunk (uint2): a particle's entries leave the build in
// 8-byte stores and a warp of consecutive particles reads 256 contiguous
// bytes per chunk.  Fluid entries fill chunks 0, 1, 2, ..., boundary entries
// chunks C-1, C-2, ... with C = list_chunks(max_neibs) chunks per particle:
// every split nf + nb <= max_neibs fits, as ceil(nf/2) + ceil(nb/2) <=
// (nf + nb)/2 + 1.  The unused half of an odd last chunk holds kMarker.
__host__ __device__ constexpr uint32_t list_chunks(uint32_t max_neibs) { return (max_neibs + 1u) / 2u + 1u; }

// u32 index of entry k of the fluid / boundary part of particle i's list
__host__ __device__ inline size_t list_fluid_word(uint32_t k, uint32_t i, size_t stride) {
    return 2 * ((size_t)(k >> 1) * stride + i) + (k & 1u);
}
__host__ __device__ inline size_t list_bnd_word(uint32_t k, uint32_t i, size_t stride, uint32_t max_neibs) {
    return 2 * ((size_t)(list_chunks(max_neibs) - 1u - (k >> 1)) * stride + i) + (k & 1u);
}

// One part (fluid or boundary) of one particle's list, written entry by entry
// by the thread that owns the particle: a chunk is stored once it is full.
struct ListWriter {
    uint2 buf;       // .y the newest entry
    uint32_t n;      // entries written
    uint2* p;        // the chunk being filled
    ptrdiff_t step;  // +stride (fluid part) or -stride (boundary part), in chunks
    __device__ __forceinline__ void put(uint32_t e) {
        buf.x = buf.y;
        buf.y = e;
        if ((++n & 1u) == 0u) {
            *p = buf;
            p += step;
        }
    }
    // with n even: a whole chunk (a, b), or a as the open entry of the next one
    __device__ __forceinline__ void put2(uint32_t a, uint32_t b) {
        *p = make_uint2(a, b);
        p += step;
        n += 2u;
    }
    __device__ __forceinline__ void open(uint32_t a) {
        buf.y = a;
        ++n;
    }
    __device__ __forceinline__ void flush() {
        if (n & 1u) *p = make_uint2(buf.y, kMarker);
    }
};
__device__ __forceinline__ ListWriter list_fluid_writer(uint32_t* nlist, uint32_t i, size_t stride) {
    return ListWriter{make_uint2(0u, 0u), 0u, reinterpret_cast<uint2*>(nlist) + i, (ptrdiff_t)stride};
}
__device__ __forceinline__ ListWriter list_bnd_writer(uint32_t* nlist, uint32_t i, size_t stride,
                                                      uint32_t max_neibs) {
    return ListWriter{make_uint2(0u, 0u), 0u,
                      reinterpret_cast<uint2*>(nlist) + (size_t)(list_chunks(max_neibs) - 1u) * stride + i,
                      -(ptrdiff_t)stride};
}

struct SceneDev {
    double origin[3];
    double cell_d[3];        // cell side in FP64 (upload/download conversion)
    double inv_len_d[3];     // 1 / (cell_d * ncell): the periodic wrap by a product
    uint32_t centre_off[3];  // this scene's cell centres per axis in Buffers::centres
    float origin_f[3];       // origin in FP32 (the upload's cell estimate)
    float cell_f[3];         // cell side in FP32 (device geometry)
    float inv_cell_f[3];
    int32_t ncell[3];
    uint32_t cell_offset;    // first global cell key of this scene
    uint32_t periodic;       // bit mask
    float c0;
    float phat_coef;         // B / rho0^2: P/rho^2 = phat_coef * delta*poly(delta)/(1+delta)^2
    float pi_coef;           // alpha*h*c0/rho0: Pi = -pi_coef * (u.x)/((r^2+0.01h^2)(1+(d_i+d_j)/2))
    float pi_unit;           // h*c0/rho0 (d pi_coef / d alpha)
    float dd_coef;           // 2 xi h c0: Molteni-Colagrossi density diffusion (per-scene c0)
    double dt_cap;           // cfl * min(h/c0, h^2/nu)
};

struct SceneDyn {
    float dt;                // time step used by this step's integration (FP32)
    uint32_t amax2_bits;     // float bits of max |a|^2 over fluid particles (atomicMax)
    double dt_d;             // the same dt in FP64 (reported)
    double time;             // simulated time
};

struct DevStatus {
    uint32_t n_active;       // particles in the sorted arrays
    uint32_t n_sorted;       // in-domain count found by the last scan
    uint32_t n_removed;      // cumulative removed (left the domain)
    uint32_t max_neibs_seen; // largest count of the last build
    uint32_t error_bits;     // SPH_EBIT_*
    uint32_t upload_bits;    // validation of the last upload
    uint32_t rebuild;        // skin list: run the neighbour pipeline this step (gate of its kernels)
    uint32_t since;          // skin list: steps taken with the current list
    unsigned long long steps;
    unsigned long long list_entries;  // cumulative neighbour-list entries written
    unsigned long long interactions;  // pairs within the influence radius (counted passes)
    uint32_t maxdisp2_bits;  // skin list: max displacement^2 since the build (float bits)
    uint32_t builds;         // neighbour-list builds since upload (the upload's included)
    double dt_next;          // > 0: the time step of the next step, set by the host (sph_set_dt), then cleared
    double dt_peek;          // sph_next_dt: the CFL dt of scene 0 from the last |a| reduction
};

// upload validation bits
constexpr uint32_t kUpBadArg = 1u, kUpOutOfDomain = 2u, kUpNonFinite = 4u;

// Kernel-uniform physics, passed by value (lands in the constant bank).
struct Phys {
    float h, inv_h, R2;      // R2 = (kernel_radius*h)^2: interactions
    float R2_list;           // (kernel_radius*h + skin)^2: neighbour list
    float skin_lim2;         // (skin/2)^2: largest displacement^2 the list tolerates
    float skin_trig2;        // (skin/4)^2: displacement^2 that triggers a rebuild
    uint32_t rebuild_every;  // > 1: skin list, rebuilt at least every rebuild_every steps
    float aF;                // F(q) = aF (q-2)^3, aF = 105/(128 pi h^5)
    float rho0, inv_rho0;
    float eps_h2;            // 0.01 h^2
    float nu4;               // 4 nu
    float g[3];
    float coef[8];           // C(gamma,k), k = 1..8, zero-padded
    double h_d, cfl, dt_fixed;
    int visc;
    uint32_t max_neibs;
    uint32_t stride;         // neighbour-major stride (>= cap, multiple of 32)
    uint32_t n_scenes;
    int gamma_i;             // EOS exponent (integer)
    int build_variant;       // neighbour-build kernel variant (autotuned), see build_variant_name
    int forces_variant;      // launch shape of the forces-only and predictor passes (autotuned), see
                             //   forces_variant_name
    int forces_variant_c;    // launch shape of the corrector pass (autotuned on its own)
    int fuse_predict;        // the list build and the predictor pass as one kernel (autotuned)
    // model options (Table 1); general != 0 selects the kernels of forces_models.cu
    int general;
    int kernel_type;         // SPH_KERNEL_*: F = aF f(q)
    int form;                // SPH_FORM_*
    int visc_avg;            // SPH_AVG_*
    int ddiff;               // SPH_DDIFF_*
    float lam_u, lam_x;      // laminar models: a += (lam_u u_ij + lam_x (u.x/r^2) x_ij) m_j f avg/(r_i r_j)
    uint32_t n_owned;        // particles with upload id >= n_owned are halo copies (sph_set_owned):
                             //   left out of the CFL reduction; kAllOwned: none
};
constexpr uint32_t kAllOwned = 0xFFFFFFFFu;

// whether particle i takes part in the CFL reduction (a halo copy's forces are incomplete)
__device__ __forceinline__ bool cfl_counts(const Phys& ph, const uint32_t* __restrict__ pid, uint32_t i) {
    return ph.n_owned == kAllOwned || pid[i] < ph.n_owned;
}

constexpr int kBuildVariants = 5;
constexpr uint32_t kPosPad = 8;  // spare float4 entries after pos[k][cap - 1] (read, never used)
const char* build_variant_name(int v);
constexpr int kForcesVariants = 5;
const char* forces_variant_name(int v);

// P/rho^2 of Cole's EOS from delta = rho/rho0 - 1 (binomial form, no
// cancellation near rest): phat_coef * delta * sum_k C(gamma,k) delta^(k-1) / (1+delta)^2.
// Stored per particle by every kernel that writes delta, and recomputed from a
// neighbour's delta by the tuned force kernels (one function, so both agree
// bit for bit).  The quotient is __fdividef (reciprocal and product, within
// 2 ulp for (1+delta)^2 in (2^-126, 2^126)): no slow-path call in the pair loop.
__device__ __forceinline__ float eos_phat(float d, const Phys& ph, float phat_coef) {
    float poly = ph.coef[7];
#pragma unroll
    for (int k = 6; k >= 0; --k) poly = fmaf(poly, d, ph.coef[k]);
    const float opd = 1.0f + d;
    return __fdividef(phat_coef * d * poly, opd * opd);
}

// ---- checked build ----------------------------------------------------
// Compiled with SPH_CHECKED, the kernels test the list and cell indices they
// follow; a bad one records SPH_EBIT_BOUNDS and the access is skipped (no trap).
// The ordinary build compiles the checks away.
#ifdef SPH_CHECKED
#define SPH_GUARD(cond, st, action)                                                   \
    if (!(cond)) {                                                                    \
        atomicOr(&const_cast<DevStatus*>(static_cast<const DevStatus*>(st))->error_bits, \
                 SPH_EBIT_BOUNDS);                                                    \
        action;                                                                       \
    }
#else
#define SPH_GUARD(cond, st, action)
#endif

// ---- cell helpers ------------------------------------------------------
__device__ __forceinline__ int cell_shift(float o, float cell, float inv_cell, float* rebased = nullptr) {
    // number of cells the offset o has moved past the cell centre: the integer s
    // with o - s*cell in [-cell/2, cell/2) exactly.  The estimate from o/cell can be
    // off by one at a cell face; the exact fix-up makes re-basing idempotent (a
    // second sort of an unchanged state moves no particle).  |s| <= 1 between sorts,
    // where o - s*cell is exact (Sterbenz).
    int s = (int)floorf(fmaf(o, inv_cell, 0.5f));
    float r = o - (float)s * cell;
    const float half = 0.5f * cell;
    const bool up = r >= half, dn = r < -half;  // branch-free: the reorder is latency-bound
    r = up ? r - cell : (dn ? r + cell : r);
    s += (int)up - (int)dn;
    if (rebased) *rebased = r;
    return s;
}

__device__ __forceinline__ void decode_local(uint32_t local, const SceneDev& s, int& cx, int& cy, int& cz) {
    const uint32_t nx = (uint32_t)s.ncell[0], ny = (uint32_t)s.ncell[1];
    cx = (int)(local % nx);
    const uint32_t r = local / nx;
    cy = (int)(r % ny);
    cz = (int)(r / ny);
}

__device__ __forceinline__ uint32_t encode_entry(uint32_t j, int dx, int dy, int dz) {
    return (j << kCodeBits) | (uint32_t)(dx + 1) | ((uint32_t)(dy + 1) << 2) | ((uint32_t)(dz + 1) << 4);
}

// ---- launch wrappers (host side) --------------------------------------
struct Buffers {
    float4* pos[2];
    float4* vel[2];
    uint32_t* cell[2];
    uint32_t* pinfo[2];
    uint32_t* pid[2];
    float* phat[2];          // P/rho^2 per particle, same order as pos/vel
    float4* pos_ref;         // offsets at the last list build (rebuild_every > 1), else null
    uint32_t* nlist_x;       // skin list: the step's exact list (pairs within R at x^n), written by
    uint32_t* ncount_x;      //   the predictor pass, read by the corrector pass; else null
    const uint32_t* gate;    // &status->rebuild for a skin list (pipeline kernels skip when 0), else null
    float4* pos_s;           // predicted state
    float4* vel_s;
    float* phat_s;
    float4* force;           // (ax, ay, az, drho) of sph_forces
    uint32_t* key;           // new cell key per particle (hash)
    uint32_t* slot;          // rank within the new cell at hash time (unordered)
    uint32_t* count;         // per bucket counts (n_cells + 1 buckets)
    uint32_t* start;         // exclusive scan (n_cells + 2 entries)
    uint32_t* cell_nfluid;   // fluid particles per cell (they come first in the cell)
    uint32_t* bsum;          // scan block sums
    uint32_t* unsorted;      // particle index per sorted slot before the in-cell sort
    uint32_t* nlist;
    uint32_t* ncount;
    SceneDev* scenes;
    SceneDyn* dyn;
    double* centres;         // FP64 cell centres origin + (k + 1/2) cell, per scene and axis
    DevStatus* status;
    void* staging;           // upload/download staging (64 B per particle)
};

struct Geometry {
    uint32_t cap;
    uint32_t n_cells;        // over all scenes (the sentinel bucket is n_cells)
    uint32_t n_scenes;
};

// neighbours.cu
void launch_hash(const Buffers& b, int cur, const Geometry& g, cudaStream_t st);
void launch_scan(const Buffers& b, const Geometry& g, cudaStream_t st);
void launch_scatter(const Buffers& b, const Geometry& g, cudaStream_t st);
void launch_reorder(const Buffers& b, int cur, const Geometry& g, cudaStream_t st);
void launch_build(const Buffers& b, int cur, const Geometry& g, const Phys& ph, cudaStream_t st);
uint32_t scan_blocks(uint32_t n_buckets);

// adjoint.cu
struct AdjBuffers {
    float* dphat;            // d(P/rho^2)/d delta at n and at the predicted state
    float* dphat_s;
    float4* xb;              // (xbar, deltabar) of state n, sorted order of the step
    float4* ub;              // (ubar, alphabar partial)
    float4* seed;            // (abar, drhobar) seeds of the VJP at the predicted state
    float4* seed_n;          // seeds of the VJP at n
    float4* xb_id;           // adjoints between steps, indexed by upload id
    float4* ub_id;
    double* alpha_sum;
};
// one reversed step: reverse corrector, VJP at *, reverse predictor, VJP at n (three launches)
void launch_adj_step(const AdjBuffers& a, const Buffers& b, int cur, const Geometry& g, const Phys& ph, float dt,
                     cudaStream_t st);
void launch_adj_sum_alpha(const AdjBuffers& a, uint32_t n, double* out, cudaStream_t st);
void launch_adj_load(const AdjBuffers& a, uint32_t n, const float* xbar, const float* ubar, const float* dbar,
                     cudaStream_t st);
void launch_adj_store(const AdjBuffers& a, uint32_t n, float* xbar, float* ubar, float* dbar, cudaStream_t st);
// copies of n elements of `count` arrays (16-byte elements where wide[k], else 4-byte), one launch
constexpr int kTapeArrays = 8;
void launch_tape_copy(const void* const* src, void* const* dst, const bool* wide, int count, uint32_t n,
                      cudaStream_t st);

// forces.cu
enum ForceMode { kForcesOnly = 0, kPredict = 1, kCorrect = 2 };
// With a skin list (pos_ref allocated) the predictor pass also writes the
// pairs within R at x^n to nlist_x/ncount_x, and the corrector reads those.
// With a skin list (pos_ref allocated) the kernels skip pairs beyond the
// cutoff, the first pass counts the pairs within it (DevStatus.interactions)
// and the corrector checks the displacement since the build.
void launch_forces(const Buffers& b, int cur, const Geometry& g, const Phys& ph, ForceMode mode,
                   int acc_dt, cudaStream_t st);
// forces_models.cu: the same passes for the other model options of Table 1
void launch_forces_models(const Buffers& b, int cur, const Geometry& g, const Phys& ph, ForceMode mode,
                          int acc_dt, cudaStream_t st);
void launch_copyback(const Buffers& b, int cur, const Geometry& g, cudaStream_t st);
// conservation sums of the state in buffer cur and the forces in b.force
// (kConservationSums doubles at the end of the scratch, after the block partials)
constexpr int kConservationSums = 9;
size_t conservation_scratch_bytes();
void launch_conservation(const Buffers& b, int cur, double* scratch, cudaStream_t st);
void launch_force_rebuild(const Buffers& b, cudaStream_t st);
// with_build: the step runs the neighbour pipeline (counted in DevStatus.builds; a
// skin list counts its own rebuilds)
void launch_dt(const Buffers& b, const Geometry& g, const Phys& ph, int advance_time, cudaStream_t st,
               int with_build = 1);
// nsteps steps of the every-step pipeline (default model, no skin list) as one cooperative
// launch of the persistent step kernel; buffer parity cur at the start, cur ^ (nsteps & 1) after
cudaError_t launch_step_persistent(const Buffers& b, int cur, const Geometry& g, const Phys& ph, uint32_t nsteps,
                                   cudaStream_t st);
// the list build and the predictor pass as one kernel (every-step list, default model)
void launch_build_predict(const Buffers& b, int cur, const Geometry& g, const Phys& ph, cudaStream_t st);
// DevStatus.dt_peek = the CFL dt the next step of scene 0 would take (no state change)
void launch_dt_peek(const Buffers& b, const Phys& ph, cudaStream_t st);
// the predictor update from b.force (a forces-only pass at the same state, reading C6)
void launch_predict_from_forces(const Buffers& b, int cur, const Geometry& g, const Phys& ph, cudaStream_t st);

}  // namespace sphg
