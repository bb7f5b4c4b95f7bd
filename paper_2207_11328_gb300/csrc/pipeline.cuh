// Bodies of the neighbour-pipeline kernels (paper Section 2.3 and Section 4):
// cell hash, counting sort (histogram, scan, scatter), in-cell order and
// reorder, thread-per-particle list build.  Each body is a device function of
// the threads of one launch; neighbors.cu wraps each in its own kernel, and the
// persistent step kernel (forces.cu) runs them one after the other with grid-wide
// barriers between them.  Grid-stride loops: any grid size computes the same.
#pragma once
#include "sph_internal.cuh"

namespace sphg {

namespace {

constexpr int kPipeBlock = 256;   // threads per block of the pipeline kernels
constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;                       // per thread
constexpr int kScanTile = kScanThreads * kScanItems;  // buckets per block

// ---------------------------------------------------------------------
// a1: cell hash.  New cell = old cell + floor(offset/cell + 1/2) per axis
// (cell-relative positions never leave FP32 range); periodic axes wrap;
// on other axes a particle outside the grid goes to the sentinel bucket
// (removed during the sort, paper "The GPU in GPUSPH").
// ---------------------------------------------------------------------
__device__ __forceinline__ void hash_body(const float4* __restrict__ pos, const uint32_t* __restrict__ cell,
                                          const uint32_t* __restrict__ pinfo, const SceneDev* __restrict__ scenes,
                                          const DevStatus* __restrict__ st, uint32_t* __restrict__ key,
                                          uint32_t* __restrict__ slot, uint32_t* __restrict__ count, uint32_t sentinel) {
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

__device__ __forceinline__ void scan_reduce_tile(const uint32_t* __restrict__ count, uint32_t nb,
                                                 uint32_t* __restrict__ bsum, uint32_t tile) {
    const uint32_t base = tile * kScanTile + threadIdx.x * kScanItems;
    uint32_t s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k)
        if (base + k < nb) s += count[base + k];
    uint32_t total;
    block_excl_scan(s, &total);
    if (threadIdx.x == 0) bsum[tile] = total;
}

__device__ __forceinline__ void scan_bsums_body(uint32_t* __restrict__ bsum, uint32_t nblocks) {

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

__device__ __forceinline__ void scan_down_tile(uint32_t* __restrict__ count, uint32_t nb,
                                               const uint32_t* __restrict__ bsum, uint32_t* __restrict__ start,
                                               DevStatus* __restrict__ st, uint32_t tile) {
    const uint32_t base = tile * kScanTile + threadIdx.x * kScanItems;
    uint32_t v[kScanItems];
    uint32_t s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        v[k] = base + k < nb ? count[base + k] : 0u;
        s += v[k];
    }
    uint32_t total;
    uint32_t run = block_excl_scan(s, &total) + bsum[tile];
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
__device__ __forceinline__ void scatter_body(const uint32_t* __restrict__ key, const uint32_t* __restrict__ slot,
                                             const uint32_t* __restrict__ start, const DevStatus* __restrict__ st,
                                             uint32_t* __restrict__ unsorted, uint32_t nkeys) {
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

__device__ __forceinline__ void reorder_body(
    const float4* __restrict__ pos, const float4* __restrict__ vel, const float* __restrict__ phat,
    const uint32_t* __restrict__ pinfo,
    const uint32_t* __restrict__ pid, const uint32_t* __restrict__ start, const uint32_t* __restrict__ unsorted,
    const SceneDev* __restrict__ scenes, uint32_t n_cells, DevStatus* __restrict__ st, uint32_t* __restrict__ cell_nfluid,
    float4* __restrict__ pos_o,
    float4* __restrict__ vel_o, float* __restrict__ phat_o, uint32_t* __restrict__ cell_o,
    uint32_t* __restrict__ pinfo_o, uint32_t* __restrict__ pid_o) {
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
// a5, second variant: one thread per particle (the paper's baseline
// build, Section 7).  Lanes of a warp are consecutive particles of ~2 cells
// and read the same candidates (L1 broadcast).  Candidates are fluid-first
// in each cell (cell_nfluid), so a boundary particle walks only the fluid
// part of each neighbour cell and types need no per-candidate test.
// ---------------------------------------------------------------------

// m with all but its k lowest set bits cleared
__device__ __forceinline__ uint32_t lowest_set_bits(uint32_t m, uint32_t k) {
    uint32_t out = 0u;
    for (uint32_t c = 0; c < k && m; ++c) {
        const uint32_t b = m & (0u - m);
        out |= b;
        m ^= b;
    }
    return out;
}

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
    constexpr int kWindow = 5 * kGroup;  // candidates per hit mask (bits 0..29)
    static_assert(kPosPad >= kGroup - 1, "a group reads up to kGroup - 1 entries past the last particle");
    const SceneDev& sc = scenes[pinfo[i]];
    const float4 pi = pos[i];
    const bool fluid_i = pi.w > 0.f;
    int cx, cy, cz;
    decode_local(cell[i] - sc.cell_offset, sc, cx, cy, cz);
    uint32_t nfound = 0;
    ListWriter wf = list_fluid_writer(nlist, i, stride);
    ListWriter wb = list_bnd_writer(nlist, i, stride, max_neibs);
    // candidates [b, e) of one neighbour cell and one type, appended to w in candidate order.
    // The distance tests run in groups of kGroup candidates (independent loads in flight); the
    // hits of up to kWindow candidates are gathered in one bit mask, which a loop over its set
    // bits then appends: a lane spends append work on its own hits only, where an append
    // predicated per candidate slot costs the whole warp every slot of a group as soon as one
    // lane hits in it.  A group may read up to kGroup - 1 entries past the range (the next
    // cell's, or the kPosPad spare entries at the end): masked off.  Past max_neibs entries the
    // list keeps the first ones in candidate order (the window's mask is cut to the room left).
    auto scan_part = [&](uint32_t b, uint32_t e, ListWriter& w, float bx, float by, float bz, uint32_t code) {
        for (uint32_t j0 = b; j0 < e; j0 += kWindow) {
            uint32_t mask = 0;
#pragma unroll
            for (int g = 0; g < kWindow; g += kGroup) {
                const uint32_t j = j0 + (uint32_t)g;
                if (j >= e) break;
                const float4* pg = pos + j;
                uint32_t hits = 0;
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
                mask |= hits << g;
            }
            if (!mask) continue;
            const uint32_t found = (uint32_t)__popc(mask);
            nfound += found;
            const uint32_t room = max_neibs - (wf.n + wb.n);
            if (found > room) mask = lowest_set_bits(mask, room);
            const uint32_t e0 = (j0 << kCodeBits) | code;
            // the first hit completes a chunk left open by the previous range; then two hits
            // per chunk store, an odd last hit left open
            if (mask && (w.n & 1u)) {
                const uint32_t u = (uint32_t)__ffs(mask) - 1u;
                mask &= mask - 1u;
                w.put(e0 + (u << kCodeBits));
            }
            while (mask) {
                const uint32_t u0 = (uint32_t)__ffs(mask) - 1u;
                mask &= mask - 1u;
                const uint32_t a = e0 + (u0 << kCodeBits);
                if (!mask) {
                    w.open(a);
                    break;
                }
                const uint32_t u1 = (uint32_t)__ffs(mask) - 1u;
                mask &= mask - 1u;
                w.put2(a, e0 + (u1 << kCodeBits));
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

__device__ __forceinline__ void build_tpp_body(
    const float4* __restrict__ pos, const uint32_t* __restrict__ cell, const uint32_t* __restrict__ pinfo,
    const uint32_t* __restrict__ start, const uint32_t* __restrict__ cell_nfluid, const SceneDev* __restrict__ scenes,
    DevStatus* __restrict__ st, uint32_t* __restrict__ nlist, uint32_t* __restrict__ ncount, float R2,
    uint32_t max_neibs, uint32_t stride) {
    const uint32_t r2lim = __float_as_uint(R2) - 1u;
    const uint32_t n = st->n_active;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        uint32_t nfound;
        const uint32_t nent = build_particle(i, pos, cell, pinfo, start, cell_nfluid, scenes, nlist, ncount, r2lim,
                                             max_neibs, stride, &nfound, st, n);
        build_stats(st, nfound, nent, max_neibs, __activemask());
    }
}

}  // namespace

}  // namespace sphg
