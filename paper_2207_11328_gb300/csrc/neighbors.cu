// Neighbour pipeline (paper Section 2.3 and Section 4):
//   cell hash -> counting sort by cell (histogram, exclusive scan, scatter)
//   -> in-cell order by (type, id) + reorder of the particle arrays
//   -> cell start/end table (the scan itself) -> split neighbour list.
//
// Deterministic: the histogram counts are order-free, the in-cell rank is a
// comparison count on the unique key (type, id), so the sorted arrays are
// bit-identical from run to run whatever order the atomics took.
#include "pipeline.cuh"

namespace sphg {

namespace {

// kernels of the pipeline bodies (pipeline.cuh); a skin list gates them with
// status->rebuild (no rebuild this step: every kernel exits at once)
__global__ void __launch_bounds__(kPipeBlock) k_hash(const float4* __restrict__ pos, const uint32_t* __restrict__ cell,
                                                     const uint32_t* __restrict__ pinfo,
                                                     const SceneDev* __restrict__ scenes,
                                                     const DevStatus* __restrict__ st, uint32_t* __restrict__ key,
                                                     uint32_t* __restrict__ slot, uint32_t* __restrict__ count,
                                                     uint32_t sentinel, const uint32_t* __restrict__ gate) {
    if (gate && *gate == 0u) return;
    hash_body(pos, cell, pinfo, scenes, st, key, slot, count, sentinel);
}

__global__ void __launch_bounds__(kScanThreads) k_scan_reduce(const uint32_t* __restrict__ count, uint32_t nb,
                                                              uint32_t* __restrict__ bsum,
                                                              const uint32_t* __restrict__ gate) {
    if (gate && *gate == 0u) return;
    scan_reduce_tile(count, nb, bsum, blockIdx.x);
}

__global__ void __launch_bounds__(1024) k_scan_bsums(uint32_t* __restrict__ bsum, uint32_t nblocks,
                                                     const uint32_t* __restrict__ gate) {
    if (gate && *gate == 0u) return;
    scan_bsums_body(bsum, nblocks);
}

__global__ void __launch_bounds__(kScanThreads) k_scan_down(uint32_t* __restrict__ count, uint32_t nb,
                                                            const uint32_t* __restrict__ bsum,
                                                            uint32_t* __restrict__ start,
                                                            DevStatus* __restrict__ st,
                                                            const uint32_t* __restrict__ gate) {
    if (gate && *gate == 0u) return;
    scan_down_tile(count, nb, bsum, start, st, blockIdx.x);
}

__global__ void __launch_bounds__(kPipeBlock) k_scatter(const uint32_t* __restrict__ key,
                                                        const uint32_t* __restrict__ slot,
                                                        const uint32_t* __restrict__ start,
                                                        const DevStatus* __restrict__ st,
                                                        uint32_t* __restrict__ unsorted, uint32_t nkeys,
                                                        const uint32_t* __restrict__ gate) {
    if (gate && *gate == 0u) return;
    scatter_body(key, slot, start, st, unsorted, nkeys);
}

__global__ void __launch_bounds__(kPipeBlock) k_reorder(
    const float4* __restrict__ pos, const float4* __restrict__ vel, const float* __restrict__ phat,
    const uint32_t* __restrict__ pinfo, const uint32_t* __restrict__ pid, const uint32_t* __restrict__ start,
    const uint32_t* __restrict__ unsorted, const SceneDev* __restrict__ scenes, uint32_t n_cells,
    DevStatus* __restrict__ st, uint32_t* __restrict__ cell_nfluid, float4* __restrict__ pos_o,
    float4* __restrict__ vel_o, float* __restrict__ phat_o, uint32_t* __restrict__ cell_o,
    uint32_t* __restrict__ pinfo_o, uint32_t* __restrict__ pid_o, const uint32_t* __restrict__ gate) {
    if (gate && *gate == 0u) return;
    reorder_body(pos, vel, phat, pinfo, pid, start, unsorted, scenes, n_cells, st, cell_nfluid, pos_o, vel_o, phat_o,
                 cell_o, pinfo_o, pid_o);
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

// the entries e[u] of the set bits u of `mask` appended to w in bit order: the first completes
// a chunk left open, then two entries per 8-byte chunk store, an odd last one left open
__device__ __forceinline__ void append_hits(ListWriter& w, uint32_t mask, const uint32_t* e) {
    if (mask && (w.n & 1u)) {
        const int u = __ffs(mask) - 1;
        mask &= mask - 1u;
        w.put(e[u]);
    }
    while (mask) {
        const int u0 = __ffs(mask) - 1;
        mask &= mask - 1u;
        if (!mask) {
            w.open(e[u0]);
            break;
        }
        const int u1 = __ffs(mask) - 1;
        mask &= mask - 1u;
        w.put2(e[u0], e[u1]);
    }
}

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
                        append_hits(wf, hf, e_s + kb32);
                        append_hits(wb, hb, e_s + kb32);
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

// 1024 resident threads per SM (64 registers, a 12-byte spill): faster than 768 threads at
// 80 registers without a spill (sort + build 0.713 -> 0.669 ms on the 1.65M dam break,
// 1.346 -> 1.283 ms on the 2.1M box), the issue slots of the extra warps outweigh the spill
template <int kBlockT>
__global__ void __launch_bounds__(kBlockT, 1024 / kBlockT) k_build_tpp(
    const float4* __restrict__ pos, const uint32_t* __restrict__ cell, const uint32_t* __restrict__ pinfo,
    const uint32_t* __restrict__ start, const uint32_t* __restrict__ cell_nfluid, const SceneDev* __restrict__ scenes,
    DevStatus* __restrict__ st, uint32_t* __restrict__ nlist, uint32_t* __restrict__ ncount, float R2,
    uint32_t max_neibs, uint32_t stride, const uint32_t* __restrict__ gate) {
    if (gate && *gate == 0u) return;
    build_tpp_body(pos, cell, pinfo, start, cell_nfluid, scenes, st, nlist, ncount, R2, max_neibs, stride);
}

inline unsigned grid_for(uint32_t n, int block) {
    uint32_t g = (n + block - 1) / block;
    return g ? g : 1;
}

}  // namespace

uint32_t scan_blocks(uint32_t n_buckets) { return (n_buckets + kScanTile - 1) / kScanTile; }

void launch_hash(const Buffers& b, int cur, const Geometry& g, cudaStream_t st) {
    k_hash<<<grid_for(g.cap, kPipeBlock), kPipeBlock, 0, st>>>(b.pos[cur], b.cell[cur], b.pinfo[cur], b.scenes, b.status,
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
    k_scatter<<<grid_for(g.cap, kPipeBlock), kPipeBlock, 0, st>>>(b.key, b.slot, b.start, b.status, b.unsorted,
                                                           g.n_cells + 1, b.gate);
}

void launch_reorder(const Buffers& b, int cur, const Geometry& g, cudaStream_t st) {
    const int nxt = cur ^ 1;
    const uint32_t warps_per_block = kPipeBlock / 32;
    const uint32_t warps = (g.n_cells + kReorderCells - 1) / kReorderCells;
    uint32_t blocks = (warps + warps_per_block - 1) / warps_per_block;
    if (blocks == 0) blocks = 1;
    k_reorder<<<blocks, kPipeBlock, 0, st>>>(b.pos[cur], b.vel[cur], b.phat[cur], b.pinfo[cur], b.pid[cur], b.start,
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
    k_copyback<<<grid_for(g.cap, kPipeBlock), kPipeBlock, 0, st>>>(b.pos[alt], b.vel[alt], b.phat[alt], b.cell[alt],
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
