// Neighbour pipeline (paper Section 2.3 and Section 4):
//   cell hash -> counting sort by cell (histogram, exclusive scan, scatter)
//   -> in-cell order by (type, id) + reorder of the particle arrays
//   -> cell start/end table (the scan itself) -> split neighbour list.
//
// Deterministic: the histogram counts are order-free, the in-cell rank is a
// comparison count on the unique key (type, id), so the sorted arrays are
// bit-identical from run to run whatever order the atomics took.
#include "sph_internal.cuh"

namespace sphg {

namespace {

constexpr int kBlock = 256;
constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;                       // per thread
constexpr int kScanTile = kScanThreads * kScanItems;  // buckets per block

// ---------------------------------------------------------------------
// a1: cell hash.  New cell = old cell + floor(offset/cell + 1/2) per axis
// (cell-relative positions never leave FP32 range); periodic axes wrap;
// on other axes a particle outside the grid goes to the sentinel bucket
// (removed during the sort, paper "The GPU in GPUSPH").
// ---------------------------------------------------------------------
__global__ void __launch_bounds__(kBlock) k_hash(const float4* __restrict__ pos, const uint32_t* __restrict__ cell,
                                                 const uint32_t* __restrict__ pinfo,
                                                 const SceneDev* __restrict__ scenes,
                                                 const DevStatus* __restrict__ st, uint32_t* __restrict__ key,
                                                 uint32_t* __restrict__ slot, uint32_t* __restrict__ count,
                                                 uint32_t sentinel, const uint32_t* __restrict__ gate) {
    if (gate && *gate == 0u) return;  // skin list: no rebuild this step
    const uint32_t n = st->n_active;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const SceneDev& sc = scenes[pinfo[i]];
        const float4 p = pos[i];
        const uint32_t c = cell[i];
        const int sx = cell_shift(p.x, sc.cell_f[0], sc.inv_cell_f[0]);
        const int sy = cell_shift(p.y, sc.cell_f[1], sc.inv_cell_f[1]);
        const int sz = cell_shift(p.z, sc.cell_f[2], sc.inv_cell_f[2]);
        uint32_t k = c;
        if ((sx | sy | sz) != 0) {
            int cx, cy, cz;
            decode_local(c - sc.cell_offset, sc, cx, cy, cz);
            int nc[3] = {cx + sx, cy + sy, cz + sz};
            bool out = false;
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                const int n_a = sc.ncell[a];
                if ((sc.periodic >> a) & 1u) {
                    nc[a] %= n_a;
                    if (nc[a] < 0) nc[a] += n_a;
                } else if (nc[a] < 0 || nc[a] >= n_a) {
                    out = true;
                }
            }
            k = out ? sentinel
                    : sc.cell_offset + (uint32_t)nc[0] +
                          (uint32_t)sc.ncell[0] * ((uint32_t)nc[1] + (uint32_t)sc.ncell[1] * (uint32_t)nc[2]);
        }
        key[i] = k;
        // one atomic per distinct cell of the warp (consecutive particles mostly share
        // one): the leader reserves the slots of its peers, each takes base + its rank.
        // The order within a cell is the reorder's to fix, so any slot order will do.
        const unsigned act = __activemask();
        const unsigned peers = __match_any_sync(act, k);
        const int lane = threadIdx.x & 31;
        const int leader = __ffs(peers) - 1;
        uint32_t base = 0;
        if (lane == leader) base = atomicAdd(&count[k], (uint32_t)__popc(peers));
        base = __shfl_sync(peers, base, leader);
        slot[i] = base + (uint32_t)__popc(peers & ((1u << lane) - 1u));
    }
}

// ---------------------------------------------------------------------
// a2/a4: exclusive scan of the bucket counts -> cell start table.
// Three passes: block sums, scan of block sums, down-sweep.  The down-sweep
// zeroes the counts for the next hash and publishes the in-domain count.
// ---------------------------------------------------------------------
__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

// block-wide exclusive scan of one value per thread; returns the block total in *total
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t* total) {
    __shared__ uint32_t wsum[32];
    __shared__ uint32_t wtotal;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const uint32_t inc = warp_incl_scan(v);
    if (lane == 31) wsum[w] = inc;
    __syncthreads();
    if (w == 0) {
        const int nw = blockDim.x >> 5;
        const uint32_t s = lane < nw ? wsum[lane] : 0u;
        const uint32_t si = warp_incl_scan(s);
        if (lane < nw) wsum[lane] = si - s;
        if (lane == nw - 1) wtotal = si;
    }
    __syncthreads();
    const uint32_t res = wsum[w] + inc - v;
    *total = wtotal;
    __syncthreads();
    return res;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_reduce(const uint32_t* __restrict__ count, uint32_t nb,
                                                              uint32_t* __restrict__ bsum,
                                                              const uint32_t* __restrict__ gate) {
    if (gate && *gate == 0u) return;  // skin list: no rebuild this step

    const uint32_t base = blockIdx.x * kScanTile + threadIdx.x * kScanItems;
    uint32_t s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k)
        if (base + k < nb) s += count[base + k];
    uint32_t total;
    block_excl_scan(s, &total);
    if (threadIdx.x == 0) bsum[blockIdx.x] = total;
}

__global__ void __launch_bounds__(1024) k_scan_bsums(uint32_t* __restrict__ bsum, uint32_t nblocks,
                                                     const uint32_t* __restrict__ gate) {
    if (gate && *gate == 0u) return;  // skin list: no rebuild this step

    uint32_t carry = 0;
    for (uint32_t base = 0; base < nblocks; base += blockDim.x) {
        const uint32_t i = base + threadIdx.x;
        const uint32_t v = i < nblocks ? bsum[i] : 0u;
        uint32_t total;
        const uint32_t ex = block_excl_scan(v, &total);
        if (i < nblocks) bsum[i] = carry + ex;
        carry += total;
    }
}

__global__ void __launch_bounds__(kScanThreads) k_scan_down(uint32_t* __restrict__ count, uint32_t nb,
                                                            const uint32_t* __restrict__ bsum,
                                                            uint32_t* __restrict__ start,
                                                            DevStatus* __restrict__ st,
                                                            const uint32_t* __restrict__ gate) {
    if (gate && *gate == 0u) return;  // skin list: no rebuild this step

    const uint32_t base = blockIdx.x * kScanTile + threadIdx.x * kScanItems;
    uint32_t v[kScanItems];
    uint32_t s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        v[k] = base + k < nb ? count[base + k] : 0u;
        s += v[k];
    }
    uint32_t total;
    uint32_t run = block_excl_scan(s, &total) + bsum[blockIdx.x];
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        const uint32_t b = base + k;
        if (b < nb) {
            start[b] = run;
            count[b] = 0u;
            if (b == nb - 1) {
                // bucket nb-1 is the sentinel of removed particles
                start[nb] = run + v[k];
                st->n_sorted = run;
                st->n_removed += v[k];
            }
        }
        run += v[k];
    }
}

// ---------------------------------------------------------------------
// a2: scatter particle indices to their bucket slots (order within a
// bucket is the atomics' order; the reorder fixes it).
// ---------------------------------------------------------------------
__global__ void __launch_bounds__(kBlock) k_scatter(const uint32_t* __restrict__ key, const uint32_t* __restrict__ slot,
                                                    const uint32_t* __restrict__ start,
                                                    const DevStatus* __restrict__ st, uint32_t* __restrict__ unsorted,
                                                    uint32_t nkeys, const uint32_t* __restrict__ gate) {
    if (gate && *gate == 0u) return;  // skin list: no rebuild this step
    const uint32_t n = st->n_active;
    (void)nkeys;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        SPH_GUARD(key[i] < nkeys && start[key[i]] + slot[i] < start[key[i] + 1], st, continue)
        unsorted[start[key[i]] + slot[i]] = i;
    }
}

// ---------------------------------------------------------------------
// a3: one warp per cell (a warp takes kReorderCells consecutive cells in turn).
// Rank each particle of the cell by its unique key (type, id) -> final slot; gather its data from the old arrays, re-base
// the offset to the new cell (exact: Sterbenz), write the new arrays.
// ---------------------------------------------------------------------
// (type, id) in 32 bits (ids < kMaxParticles = 2^26): one shuffle per comparison of the rank
static_assert(kMaxParticles <= (1u << 31), "the id fits below the type bit");
__device__ __forceinline__ uint32_t sort_key(const float4* pos, const uint32_t* pid, uint32_t idx) {
    const uint32_t bnd = __float_as_uint(pos[idx].w) >> 31;  // sign bit = boundary
    return (bnd << 31) | pid[idx];
}

// cells per warp: 4 measured fastest (1.65M dam break, most cells empty: 78 -> 61 us;
// 2.1M box, no empty cell: unchanged at 56 us; 8 and 16 cells per warp leave too few warps)
constexpr int kReorderCells = 4;
static_assert(kReorderCells >= 1 && kReorderCells <= 32, "one lane per cell");

__global__ void __launch_bounds__(kBlock) k_reorder(
    const float4* __restrict__ pos, const float4* __restrict__ vel, const float* __restrict__ phat,
    const uint32_t* __restrict__ pinfo,
    const uint32_t* __restrict__ pid, const uint32_t* __restrict__ start, const uint32_t* __restrict__ unsorted,
    const SceneDev* __restrict__ scenes, uint32_t n_cells, DevStatus* __restrict__ st, uint32_t* __restrict__ cell_nfluid,
    float4* __restrict__ pos_o,
    float4* __restrict__ vel_o, float* __restrict__ phat_o, uint32_t* __restrict__ cell_o,
    uint32_t* __restrict__ pinfo_o, uint32_t* __restrict__ pid_o, const uint32_t* __restrict__ gate) {
    if (gate && *gate == 0u) return;  // skin list: no rebuild this step

    const int lane = threadIdx.x & 31;
    const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        st->n_active = st->n_sorted;
        st->max_neibs_seen = 0u;
    }
    // kReorderCells consecutive cells per warp: their ranges in one load, empty cells
    // (most of a tank's cells) skipped without a round trip each
    for (uint32_t c0 = warp * kReorderCells; c0 < n_cells; c0 += nwarps * kReorderCells) {
        const uint32_t cl = c0 + (uint32_t)lane;
        const bool own = lane < kReorderCells && cl < n_cells;
        const uint32_t b_l = own ? start[cl] : 0u, e_l = own ? start[cl + 1] : 0u;
        if (own && e_l == b_l) cell_nfluid[cl] = 0u;
        unsigned todo = __ballot_sync(0xffffffffu, e_l > b_l);
        while (todo) {
            const int kc = __ffs(todo) - 1;
            todo &= todo - 1u;
            const uint32_t c = c0 + (uint32_t)kc;
            const uint32_t beg = __shfl_sync(0xffffffffu, b_l, kc), end = __shfl_sync(0xffffffffu, e_l, kc);
            const uint32_t n = end - beg;
            uint32_t nfluid = 0;
            for (uint32_t base = 0; base < n; base += 32) {
                const uint32_t l = base + lane;
                uint32_t idx = 0;
                uint32_t mine = ~0u;  // above every key
                if (l < n) {
                    idx = unsorted[beg + l];
                    mine = sort_key(pos, pid, idx);
                }
                nfluid += __popc(__ballot_sync(0xffffffffu, l < n && (mine >> 31) == 0u));
                uint32_t rank = 0;
                if (n <= 32) {
                    for (uint32_t k = 0; k < n; ++k) {
                        const uint32_t o = __shfl_sync(0xffffffffu, mine, (int)k);
                        rank += o < mine;
                    }
                } else {
                    for (uint32_t k = 0; k < n; ++k) {
                        const uint32_t o = sort_key(pos, pid, unsorted[beg + k]);
                        rank += o < mine;
                    }
                }
                if (l < n) {
                    const uint32_t s = pinfo[idx];
                    const SceneDev& sc = scenes[s];
                    float4 p = pos[idx];
                    cell_shift(p.x, sc.cell_f[0], sc.inv_cell_f[0], &p.x);
                    cell_shift(p.y, sc.cell_f[1], sc.inv_cell_f[1], &p.y);
                    cell_shift(p.z, sc.cell_f[2], sc.inv_cell_f[2], &p.z);
                    const uint32_t d = beg + rank;
                    SPH_GUARD(d < end, st, continue)
                    pos_o[d] = p;
                    vel_o[d] = vel[idx];
                    phat_o[d] = phat[idx];
                    cell_o[d] = c;
                    pinfo_o[d] = s;
                    pid_o[d] = pid[idx];
                }
            }
            if (lane == 0) cell_nfluid[c] = nfluid;
        }
    }
}

// ---------------------------------------------------------------------
// a5: split neighbour list (paper Section 4), one warp per cell (the paper's
// warp-per-cell build, Section 7).  The warp first stages every candidate of
// the 27-cell neighbourhood into shared memory: its position already shifted
// into the frame of the central cell (o_j + d*cell) and its list entry
// (j << 6 | cell-delta code).  Lanes hold the cell's particles (32 at a time)
// and each lane tests the whole flat candidate array (shared-memory
// broadcast, no per-cell control flow in the inner loop).  Within a cell
// particles are sorted fluid-first; boundary particles keep only fluid
// neighbours (boundary-boundary pairs carry no interaction), and a warp of
// boundary particles only stages fluid candidates.
// ---------------------------------------------------------------------
constexpr int kStage = 256;  // staged candidates per warp and window (multiple of 32)

template <int kBuildWarps>
__global__ void __launch_bounds__(kBuildWarps * 32, 24 / kBuildWarps) k_build_cell(
    const float4* __restrict__ pos, const uint32_t* __restrict__ pinfo, const uint32_t* __restrict__ start,
    const uint32_t* __restrict__ cell_nfluid, const SceneDev* __restrict__ scenes, uint32_t n_cells,
    DevStatus* __restrict__ st, uint32_t* __restrict__ nlist, uint32_t* __restrict__ ncount, float R2,
    uint32_t max_neibs, uint32_t stride, const uint32_t* __restrict__ gate) {
    if (gate && *gate == 0u) return;  // skin list: no rebuild this step
    __shared__ float4 sq[kBuildWarps][kStage];
    __shared__ uint32_t se[kBuildWarps][kStage];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    float4* const q_s = sq[wib];
    uint32_t* const e_s = se[wib];
    const uint32_t nwarps = gridDim.x * kBuildWarps;
    for (uint32_t c = blockIdx.x * kBuildWarps + wib; c < n_cells; c += nwarps) {
        const uint32_t b0 = start[c], e0 = start[c + 1];
        if (b0 == e0) continue;
        const SceneDev& sc = scenes[pinfo[b0]];
        // a cell of boundary particles only needs the fluid candidates (first in each cell)
        const bool all_bnd = cell_nfluid[c] == 0;
        int cx, cy, cz;
        decode_local(c - sc.cell_offset, sc, cx, cy, cz);
        // lane k < 27: neighbour cell k = (dx, dy, dz), its candidate range and exclusive offset
        uint32_t kb = 0, kn = 0;
        {
            const int dx = lane % 3 - 1, dy = (lane / 3) % 3 - 1, dz = lane / 9 - 1;
            int nc[3] = {cx + dx, cy + dy, cz + dz};
            bool ok = lane < 27;
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                if (nc[a] < 0 || nc[a] >= sc.ncell[a]) {
                    if ((sc.periodic >> a) & 1u)
                        nc[a] = nc[a] < 0 ? nc[a] + sc.ncell[a] : nc[a] - sc.ncell[a];
                    else
                        ok = false;
                }
            }
            if (ok) {
                const uint32_t cc = sc.cell_offset + (uint32_t)nc[0] +
                                    (uint32_t)sc.ncell[0] * ((uint32_t)nc[1] + (uint32_t)sc.ncell[1] * (uint32_t)nc[2]);
                kb = start[cc];
                kn = all_bnd ? cell_nfluid[cc] : start[cc + 1] - kb;
            }
        }
        uint32_t koff = kn;  // inclusive scan over lanes -> exclusive offsets
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(0xffffffffu, koff, o);
            if (lane >= o) koff += t;
        }
        const uint32_t total = __shfl_sync(0xffffffffu, koff, 31);
        koff -= kn;
        if (total == 0) {
            for (uint32_t base = b0; base < e0; base += 32) {
                const uint32_t i = base + lane;
                if (i < e0) ncount[i] = 0u;
            }
            continue;
        }
        for (uint32_t base = b0; base < e0; base += 32) {
            const uint32_t i = base + lane;
            const bool active = i < e0;
            const float4 pi = active ? pos[i] : make_float4(0.f, 0.f, 0.f, -1.f);
            const bool fluid_i = active && pi.w > 0.f;
            // parked lanes sit far away on one side, padding candidates on the other
            const float px = active ? pi.x : 3.0e18f, py = pi.y, pz = pi.z;
            uint32_t nfound = 0;
            ListWriter wf = list_fluid_writer(nlist, i, stride);
            ListWriter wb = list_bnd_writer(nlist, i, stride, max_neibs);
            for (uint32_t w0 = 0; w0 < total; w0 += kStage) {
                const uint32_t w1 = min(total, w0 + (uint32_t)kStage);
                __syncwarp();
                for (int k = 0; k < 27; ++k) {
                    const uint32_t b = __shfl_sync(0xffffffffu, kb, k);
                    const uint32_t n = __shfl_sync(0xffffffffu, kn, k);
                    const uint32_t off = __shfl_sync(0xffffffffu, koff, k);
                    if (off >= w1 || off + n <= w0) continue;
                    const int dx = k % 3 - 1, dy = (k / 3) % 3 - 1, dz = k / 9 - 1;
                    const float shx = (float)dx * sc.cell_f[0], shy = (float)dy * sc.cell_f[1],
                                shz = (float)dz * sc.cell_f[2];
                    const uint32_t code = (uint32_t)(dx + 1) | ((uint32_t)(dy + 1) << 2) | ((uint32_t)(dz + 1) << 4);
                    const uint32_t t0 = off < w0 ? w0 - off : 0u;
                    const uint32_t t1 = min(n, w1 - off);
                    for (uint32_t t = t0 + lane; t < t1; t += 32) {
                        const uint32_t j = b + t;
                        SPH_GUARD(j < st->n_active, st, continue)
                        float4 q = pos[j];
                        q.x += shx;
                        q.y += shy;
                        q.z += shz;
                        q_s[off + t - w0] = q;
                        e_s[off + t - w0] = (j << kCodeBits) | code;
                    }
                }
                const uint32_t cnt = w1 - w0;
                const uint32_t padded = (cnt + 31u) & ~31u;
                if (cnt + lane < padded) q_s[cnt + lane] = make_float4(-3.0e18f, 0.f, 0.f, 1.f);
                __syncwarp();
                for (uint32_t kb32 = 0; kb32 < padded; kb32 += 32) {
                    // fluid candidates of this block (uniform), then branch-free distance tests
                    const uint32_t fmask = __ballot_sync(0xffffffffu, q_s[kb32 + lane].w > 0.f);
                    uint32_t hits = 0;
#pragma unroll
                    for (int u = 0; u < 32; ++u) {
                        const float4 q = q_s[kb32 + u];
                        const float rx = px - q.x, ry = py - q.y, rz = pz - q.z;
                        const float r2 = fmaf(rx, rx, fmaf(ry, ry, rz * rz));
                        hits |= (uint32_t)(r2 < R2 && r2 > 0.f) << u;
                    }
                    uint32_t hf = hits & fmask;
                    uint32_t hb = fluid_i ? hits & ~fmask : 0u;
                    const uint32_t cf = __popc(hf), cb = __popc(hb);
                    nfound += cf + cb;
                    if (wf.n + wb.n + cf + cb <= max_neibs) {
                        while (hf) {
                            const int u = __ffs(hf) - 1;
                            hf &= hf - 1u;
                            wf.put(e_s[kb32 + u]);
                        }
                        while (hb) {
                            const int u = __ffs(hb) - 1;
                            hb &= hb - 1u;
                            wb.put(e_s[kb32 + u]);
                        }
                    } else {
                        // list full: keep the first hits in candidate order, count the rest
                        uint32_t h = hf | hb;
                        while (h) {
                            const int u = __ffs(h) - 1;
                            h &= h - 1u;
                            if (wf.n + wb.n >= max_neibs) break;
                            if ((fmask >> u) & 1u)
                                wf.put(e_s[kb32 + u]);
                            else
                                wb.put(e_s[kb32 + u]);
                        }
                    }
                }
            }
            if (active) {
                wf.flush();
                wb.flush();
                ncount[i] = wf.n | (wb.n << 16);
                if (nfound > max_neibs) atomicOr(&st->error_bits, SPH_EBIT_NEIB_OVERFLOW);
            }
            const uint32_t m = __reduce_max_sync(0xffffffffu, active ? nfound : 0u);
            const uint32_t wsum = __reduce_add_sync(0xffffffffu, active ? wf.n + wb.n : 0u);
            if (lane == 0) {
                atomicMax(&st->max_neibs_seen, m);
                atomicAdd(&st->list_entries, (unsigned long long)wsum);
            }
        }
    }
}

// ---------------------------------------------------------------------
// a5, second variant: one thread per particle (the paper's baseline
// build, Section 7).  Lanes of a warp are consecutive particles of ~2 cells
// and read the same candidates (L1 broadcast).  Candidates are fluid-first
// in each cell (cell_nfluid), so a boundary particle walks only the fluid
// part of each neighbour cell and types need no per-candidate test.
// ---------------------------------------------------------------------

// The list of particle i; returns its entry count, *nfound = pairs found
// (more than max_neibs: overflow, the list keeps the first ones).
__device__ __forceinline__ uint32_t build_particle(uint32_t i, const float4* __restrict__ pos,
                                                   const uint32_t* __restrict__ cell, const uint32_t* __restrict__ pinfo,
                                                   const uint32_t* __restrict__ start,
                                                   const uint32_t* __restrict__ cell_nfluid,
                                                   const SceneDev* __restrict__ scenes, uint32_t* __restrict__ nlist,
                                                   uint32_t* __restrict__ ncount, uint32_t r2lim, uint32_t max_neibs,
                                                   uint32_t stride, uint32_t* nfound_out, DevStatus* st, uint32_t n) {
    constexpr int kGroup = 6;
    static_assert(kPosPad >= kGroup - 1, "a group reads up to kGroup - 1 entries past the last particle");
    const SceneDev& sc = scenes[pinfo[i]];
    const float4 pi = pos[i];
    const bool fluid_i = pi.w > 0.f;
    int cx, cy, cz;
    decode_local(cell[i] - sc.cell_offset, sc, cx, cy, cz);
    uint32_t nfound = 0;
    ListWriter wf = list_fluid_writer(nlist, i, stride);
    ListWriter wb = list_bnd_writer(nlist, i, stride, max_neibs);
    // candidates [b, e) of one neighbour cell and one type, appended to w in candidate order:
    // groups of kGroup candidates (independent loads in flight), hits gathered in a bit mask.
    // A group may read up to kGroup - 1 entries past the range (the next cell's, or the
    // kPosPad spare entries at the end): masked off.  With room for the whole group the hits
    // are appended by predicated puts (no loop whose trip count differs between lanes).
    auto scan_part = [&](uint32_t b, uint32_t e, ListWriter& w, float bx, float by, float bz, uint32_t code) {
        for (uint32_t j = b; j < e; j += kGroup) {
            uint32_t hits = 0;
            const float4* pg = pos + j;
#pragma unroll
            for (int u = 0; u < kGroup; ++u) {
                const float4 pj = pg[u];
                const float rx = bx - pj.x, ry = by - pj.y, rz = bz - pj.z;
                const float r2 = fmaf(rx, rx, fmaf(ry, ry, rz * rz));
                // 0 < r2 < R2 as one unsigned compare on the bits (r2 >= +0)
                hits |= (uint32_t)(__float_as_uint(r2) - 1u < r2lim) << u;
            }
            const uint32_t rem = e - j;
            if (rem < (uint32_t)kGroup) hits &= (1u << rem) - 1u;
            if (!hits) continue;
            nfound += __popc(hits);
            const uint32_t e0 = (j << kCodeBits) | code;
            if (wf.n + wb.n + kGroup <= max_neibs) {
#pragma unroll
                for (int u = 0; u < kGroup; ++u)
                    if ((hits >> u) & 1u) w.put(e0 + ((uint32_t)u << kCodeBits));
            } else {
                while (hits) {
                    const int u = __ffs(hits) - 1;
                    hits &= hits - 1u;
                    if (wf.n + wb.n < max_neibs) w.put(e0 + ((uint32_t)u << kCodeBits));
                }
            }
        }
    };
    for (int dz = -1; dz <= 1; ++dz) {
        int z = cz + dz;
        if (z < 0 || z >= sc.ncell[2]) {
            if (!((sc.periodic >> 2) & 1u)) continue;
            z = z < 0 ? z + sc.ncell[2] : z - sc.ncell[2];
        }
        for (int dy = -1; dy <= 1; ++dy) {
            int y = cy + dy;
            if (y < 0 || y >= sc.ncell[1]) {
                if (!((sc.periodic >> 1) & 1u)) continue;
                y = y < 0 ? y + sc.ncell[1] : y - sc.ncell[1];
            }
            const uint32_t row = sc.cell_offset + (uint32_t)sc.ncell[0] * ((uint32_t)y + (uint32_t)sc.ncell[1] * (uint32_t)z);
            const float by = pi.y - (float)dy * sc.cell_f[1];
            const float bz = pi.z - (float)dz * sc.cell_f[2];
            // the row's three cell ranges, loaded together (one round trip per row)
            uint32_t rb[3], ref[3], re[3];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                int x = cx + k - 1;
                bool ok = true;
                if (x < 0 || x >= sc.ncell[0]) {
                    if (sc.periodic & 1u) x = x < 0 ? x + sc.ncell[0] : x - sc.ncell[0];
                    else ok = false;
                }
                rb[k] = ref[k] = re[k] = 0u;
                if (ok) {
                    const uint32_t cc = row + (uint32_t)x;
                    rb[k] = start[cc];
                    ref[k] = rb[k] + cell_nfluid[cc];  // end of the fluid part
                    re[k] = fluid_i ? start[cc + 1] : ref[k];
                    SPH_GUARD(rb[k] <= ref[k] && ref[k] <= start[cc + 1] && start[cc + 1] <= n, st,
                              rb[k] = ref[k] = re[k] = 0u)
                }
            }
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const int dx = k - 1;
                const float bx = pi.x - (float)dx * sc.cell_f[0];
                const uint32_t code = (uint32_t)(dx + 1) | ((uint32_t)(dy + 1) << 2) | ((uint32_t)(dz + 1) << 4);
                // the cell's fluid candidates (to the fluid part), then its boundary candidates
                // (to the boundary part; fluid i only): each group's hits go to one part
                scan_part(rb[k], ref[k], wf, bx, by, bz, code);
                scan_part(ref[k], re[k], wb, bx, by, bz, code);
            }
        }
    }
    wf.flush();
    wb.flush();
    ncount[i] = wf.n | (wb.n << 16);
    *nfound_out = nfound;
    return wf.n + wb.n;
}

// warp-level list statistics: overflow flag, largest count, entries written
__device__ __forceinline__ void build_stats(DevStatus* st, uint32_t nfound, uint32_t nent, uint32_t max_neibs,
                                            unsigned mask) {
    if (nfound > max_neibs) atomicOr(&st->error_bits, SPH_EBIT_NEIB_OVERFLOW);
    const uint32_t m = __reduce_max_sync(mask, nfound);
    const uint32_t wsum = __reduce_add_sync(mask, nent);
    if ((threadIdx.x & 31) == (uint32_t)(__ffs(mask) - 1)) {
        atomicMax(&st->max_neibs_seen, m);
        atomicAdd(&st->list_entries, (unsigned long long)wsum);
    }
}

// 1024 resident threads per SM (64 registers, a 12-byte spill): faster than 768 threads at
// 80 registers without a spill (sort + build 0.713 -> 0.669 ms on the 1.65M dam break,
// 1.346 -> 1.283 ms on the 2.1M box), the issue slots of the extra warps outweigh the spill
template <int kBlockT>
__global__ void __launch_bounds__(kBlockT, 1024 / kBlockT) k_build_tpp(
    const float4* __restrict__ pos, const uint32_t* __restrict__ cell, const uint32_t* __restrict__ pinfo,
    const uint32_t* __restrict__ start, const uint32_t* __restrict__ cell_nfluid, const SceneDev* __restrict__ scenes,
    DevStatus* __restrict__ st, uint32_t* __restrict__ nlist, uint32_t* __restrict__ ncount, float R2,
    uint32_t max_neibs, uint32_t stride, const uint32_t* __restrict__ gate) {
    if (gate && *gate == 0u) return;  // skin list: no rebuild this step
    const uint32_t r2lim = __float_as_uint(R2) - 1u;
    const uint32_t n = st->n_active;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        uint32_t nfound;
        const uint32_t nent = build_particle(i, pos, cell, pinfo, start, cell_nfluid, scenes, nlist, ncount, r2lim,
                                             max_neibs, stride, &nfound, st, n);
        build_stats(st, nfound, nent, max_neibs, __activemask());
    }
}

inline unsigned grid_for(uint32_t n, int block) {
    uint32_t g = (n + block - 1) / block;
    return g ? g : 1;
}

}  // namespace

uint32_t scan_blocks(uint32_t n_buckets) { return (n_buckets + kScanTile - 1) / kScanTile; }

void launch_hash(const Buffers& b, int cur, const Geometry& g, cudaStream_t st) {
    k_hash<<<grid_for(g.cap, kBlock), kBlock, 0, st>>>(b.pos[cur], b.cell[cur], b.pinfo[cur], b.scenes, b.status,
                                                        b.key, b.slot, b.count, g.n_cells, b.gate);
}

void launch_scan(const Buffers& b, const Geometry& g, cudaStream_t st) {
    const uint32_t nb = g.n_cells + 1;
    const uint32_t blocks = scan_blocks(nb);
    k_scan_reduce<<<blocks, kScanThreads, 0, st>>>(b.count, nb, b.bsum, b.gate);
    k_scan_bsums<<<1, 1024, 0, st>>>(b.bsum, blocks, b.gate);
    k_scan_down<<<blocks, kScanThreads, 0, st>>>(b.count, nb, b.bsum, b.start, b.status, b.gate);
}

void launch_scatter(const Buffers& b, const Geometry& g, cudaStream_t st) {
    k_scatter<<<grid_for(g.cap, kBlock), kBlock, 0, st>>>(b.key, b.slot, b.start, b.status, b.unsorted,
                                                           g.n_cells + 1, b.gate);
}

void launch_reorder(const Buffers& b, int cur, const Geometry& g, cudaStream_t st) {
    const int nxt = cur ^ 1;
    const uint32_t warps_per_block = kBlock / 32;
    const uint32_t warps = (g.n_cells + kReorderCells - 1) / kReorderCells;
    uint32_t blocks = (warps + warps_per_block - 1) / warps_per_block;
    if (blocks == 0) blocks = 1;
    k_reorder<<<blocks, kBlock, 0, st>>>(b.pos[cur], b.vel[cur], b.phat[cur], b.pinfo[cur], b.pid[cur], b.start,
                                          b.unsorted, b.scenes, g.n_cells, b.status, b.cell_nfluid,
                                          b.pos[nxt], b.vel[nxt],
                                          b.phat[nxt], b.cell[nxt], b.pinfo[nxt], b.pid[nxt], b.gate);
}

template <int W>
void launch_build_cell(const Buffers& b, int cur, const Geometry& g, const Phys& ph, cudaStream_t st) {
    uint32_t blocks = (g.n_cells + W - 1) / W;
    if (blocks == 0) blocks = 1;
    k_build_cell<W><<<blocks, W * 32, 0, st>>>(b.pos[cur], b.pinfo[cur], b.start, b.cell_nfluid, b.scenes, g.n_cells,
                                                b.status, b.nlist, b.ncount, ph.R2_list, ph.max_neibs, ph.stride,
                                                b.gate);
}

template <int B>
void launch_build_tpp(const Buffers& b, int cur, const Geometry& g, const Phys& ph, cudaStream_t st) {
    k_build_tpp<B><<<grid_for(g.cap, B), B, 0, st>>>(b.pos[cur], b.cell[cur], b.pinfo[cur], b.start, b.cell_nfluid,
                                                     b.scenes, b.status, b.nlist, b.ncount, ph.R2_list, ph.max_neibs,
                                                     ph.stride, b.gate);
}

const char* build_variant_name(int v) {
    static const char* names[kBuildVariants] = {"thread/particle x128", "thread/particle x256", "warp/cell x2 cells/CTA",
                                                "warp/cell x4 cells/CTA", "warp/cell x8 cells/CTA"};
    return v >= 0 && v < kBuildVariants ? names[v] : "?";
}

// skin list: the reorder wrote the sorted arrays to the other buffer; copy
// them back (the step graph keeps one buffer) and record the offsets at the
// build for the displacement check.
__global__ void k_copyback(const float4* __restrict__ pos, const float4* __restrict__ vel,
                           const float* __restrict__ phat, const uint32_t* __restrict__ cell,
                           const uint32_t* __restrict__ pinfo, const uint32_t* __restrict__ pid,
                           const DevStatus* __restrict__ st, float4* __restrict__ pos_o, float4* __restrict__ vel_o,
                           float* __restrict__ phat_o, uint32_t* __restrict__ cell_o, uint32_t* __restrict__ pinfo_o,
                           uint32_t* __restrict__ pid_o, float4* __restrict__ pos_ref,
                           const uint32_t* __restrict__ gate) {
    if (gate && *gate == 0u) return;
    const uint32_t n = st->n_active;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float4 p = pos[i];
        pos_o[i] = p;
        pos_ref[i] = p;
        vel_o[i] = vel[i];
        phat_o[i] = phat[i];
        cell_o[i] = cell[i];
        pinfo_o[i] = pinfo[i];
        pid_o[i] = pid[i];
    }
}

__global__ void k_force_rebuild(DevStatus* st) {
    st->rebuild = 1u;
    st->since = 0u;  // steps taken with the list built now
    st->maxdisp2_bits = 0u;
    st->builds += 1u;
}

void launch_copyback(const Buffers& b, int cur, const Geometry& g, cudaStream_t st) {
    const int alt = cur ^ 1;
    k_copyback<<<grid_for(g.cap, kBlock), kBlock, 0, st>>>(b.pos[alt], b.vel[alt], b.phat[alt], b.cell[alt],
                                                            b.pinfo[alt], b.pid[alt], b.status, b.pos[cur],
                                                            b.vel[cur], b.phat[cur], b.cell[cur], b.pinfo[cur],
                                                            b.pid[cur], b.pos_ref, b.gate);
}

void launch_force_rebuild(const Buffers& b, cudaStream_t st) { k_force_rebuild<<<1, 1, 0, st>>>(b.status); }

void launch_build(const Buffers& b, int cur, const Geometry& g, const Phys& ph, cudaStream_t st) {
    switch (ph.build_variant) {
        case 0: launch_build_tpp<128>(b, cur, g, ph, st); break;
        case 1: launch_build_tpp<256>(b, cur, g, ph, st); break;
        case 2: launch_build_cell<2>(b, cur, g, ph, st); break;
        case 3: launch_build_cell<4>(b, cur, g, ph, st); break;
        default: launch_build_cell<8>(b, cur, g, ph, st); break;
    }
}

}  // namespace sphg
