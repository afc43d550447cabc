// hm_binned.cu -- the screen-tile binned rasterizer (arXiv 2607.04230,
// Sec. 3.1.2: atomicMin visibility), an alternative to the direct
// rasterizer that the autotuner can select (hm_tuning.raster_bin_w != 0).
//
// The direct rasterizer issues one global 64-bit atomicMin per covered
// (pixel, layer), each on its own 32-byte L2 sector.  Here the atomics go to
// shared memory instead:
//   1. count: the strand segments are generated and projected as in the
//      direct rasterizer; each set-up segment is stored (48 B) and counted
//      into the screen tiles its conservative pixel box overlaps;
//   2. scan: per-tile offsets into one pair list, and per-tile chunk counts
//      (chunks of at most 2^KL segments);
//   3. fill: each segment's index is appended to the lists of its tiles;
//   4. tile pass: a persistent grid takes (tile, chunk) units from a ticket,
//      rasterizes the chunk's segments clipped to the tile with shared-memory
//      atomicMin into a TW x TH key tile, then flushes the tile's non-empty
//      keys with coalesced global atomicMin (four keys per 32-byte sector);
//      several chunks of one tile meet there, so the order never matters.
// Every (pixel, layer) key is computed by the same raster_item as in the
// direct rasterizer, so the two layers are bit-identical to it.
//
// The caller's clear (or pre-fill) runs first, as for the direct rasterizer.
#include <cstdint>
#include <cuda_runtime.h>

#include "hm_device.cuh"
#include "hm_kernels.h"
#include "hm_raster.cuh"

namespace hm {

namespace {

// A set-up segment as the tile pass reads it back (the fields of SegRec that
// cannot be derived from the others).
struct __align__(16) BinSeg {
    int32_t uA, vA, du, dv;
    float zA, dz, fden, slope;
    int32_t hc, flags;
    uint32_t id_lo, id_hi;
};
static_assert(sizeof(BinSeg) == 48, "BinSeg is read as three 16-byte words");

constexpr uint32_t kNoBox = 0xFFFFFFFFu;
constexpr uint32_t kPairsPerSlot = 8;     // pair-list capacity per segment slot
enum BinCtl : int { kCtlUnitTicket = 0, kCtlPairs = 1, kCtlUnits = 2, kCtlWords = 4 };

// Views into the caller's workspace (binned_workspace_bytes).
struct BinLayout {
    BinSeg *segs;          // [slots] set-up segment of batch slot b * 32 + lane (lane < 31)
    uint2 *tbox;           // [slots] tile box (tx0 | ty0 << 16, tx1 | ty1 << 16); x = kNoBox: none
    uint32_t *tile_cnt;    // [ntiles] pairs per tile (count), then fill cursors
    uint32_t *tile_off;    // [ntiles + 1] exclusive prefix of the pair counts
    uint32_t *chunk_off;   // [ntiles + 1] exclusive prefix of the chunk counts
    uint32_t *list;        // [pair_cap] segment slots, grouped by tile
    uint32_t *ctl;         // [kCtlWords]
    uint32_t slots, pair_cap;
    int32_t ntx, ntiles;
};

size_t align16(size_t b) { return (b + 15) & ~(size_t)15; }

BinLayout bin_layout(void *ws, uint64_t slots, int W, int H, int tw, int th) {
    BinLayout l;
    const int ntx = (W + tw - 1) / tw, nty = (H + th - 1) / th;
    l.ntx = ntx;
    l.ntiles = ntx * nty;
    l.slots = (uint32_t)slots;
    l.pair_cap = (uint32_t)(slots * kPairsPerSlot);
    char *p = static_cast<char *>(ws);
    l.segs = reinterpret_cast<BinSeg *>(p);
    p += align16(slots * sizeof(BinSeg));
    l.tbox = reinterpret_cast<uint2 *>(p);
    p += align16(slots * sizeof(uint2));
    l.tile_cnt = reinterpret_cast<uint32_t *>(p);
    p += align16((size_t)l.ntiles * 4);
    l.tile_off = reinterpret_cast<uint32_t *>(p);
    p += align16(((size_t)l.ntiles + 1) * 4);
    l.chunk_off = reinterpret_cast<uint32_t *>(p);
    p += align16(((size_t)l.ntiles + 1) * 4);
    l.ctl = reinterpret_cast<uint32_t *>(p);
    p += align16(kCtlWords * 4);
    l.list = reinterpret_cast<uint32_t *>(p);
    return l;
}

// Tiles of a lane's box as a count nt (row-major over a tw-wide box).
__device__ __forceinline__ int box_tiles(uint2 box, int &tx0, int &ty0, int &tw) {
    if (box.x == kNoBox) return 0;
    tx0 = (int)(box.x & 0xFFFF);
    ty0 = (int)(box.x >> 16);
    tw = (int)(box.y & 0xFFFF) - tx0 + 1;
    return tw * ((int)(box.y >> 16) - ty0 + 1);
}

// 1. count.  Persistent, one warp per work-list batch from the ticket (as
// the direct rasterizer: a control point per lane, segments closed by the
// next lane's point).  Per tile, the lanes of a warp that hit
// it add their count with one atomic.
template <int TWL, int THL>
__global__ void __launch_bounds__(kRasterThreads, 4) bin_count_kernel(CallTable tab, CamDev cam, BinLayout bl) {
    __shared__ uint32_t s_goff[HM_MAX_GROOMS_PER_CALL + 1];
    groom_batch_offsets(tab, s_goff);
    const uint32_t total = s_goff[tab.n];
    const int lane = threadIdx.x & 31;
    uint32_t *ticket = tab.g[0].counters + kCtrTicket;
    const int W = cam.W, H = cam.H;
    for (;;) {
        uint32_t b = 0;
        if (lane == 0) b = atomicAdd(ticket, 1u);
        b = __shfl_sync(kFull, b, 0);
        // the host sizes the workspace for every batch the grooms can have
        if (b >= total || b >= bl.slots / kBatchLanes) break;
        const int gi = batch_groom(s_goff, tab.n, b);
        const GroomDev &g = tab.g[gi];
        const uint32_t lb = b - s_goff[gi];
        const uint32_t slot = b * kBatchLanes + lane;
        uint2 box = make_uint2(kNoBox, 0u);
        const BatchPoint bp = batch_lane_point(g, lb, lane);
        const float3 cp[2] = {bp.p, next_lane(bp.p)};
        if (bp.seg_ok && g.segpts) store_segment_points(g.segpts, bp.seg, cp);
        Proj A, B;
        if (batch_lane_segment(cam, bp, A, B)) {
            SegRec r;
            segment_frame(cam, g.width_m, A, B, r);
            const bool xm = r.flags & 1;
            int ilo, ihi, mlo, mhi;
            if (segment_pixel_box(r, xm ? W : H, xm ? H : W, ilo, ihi, mlo, mhi)) {
                const uint64_t id = ((g.base + (uint64_t)bp.s) << 7) | (uint64_t)bp.j;
                BinSeg q;
                q.uA = r.uA;
                q.vA = r.vA;
                q.du = r.du;
                q.dv = r.dv;
                q.zA = r.zA;
                q.dz = r.dz;
                q.fden = r.fden;
                q.slope = r.slope;
                q.hc = r.hc;
                q.flags = r.flags;
                q.id_lo = (uint32_t)id;
                q.id_hi = (uint32_t)(id >> 32);
                bl.segs[slot] = q;
                const int x0 = xm ? ilo : mlo, x1 = xm ? ihi : mhi;
                const int y0 = xm ? mlo : ilo, y1 = xm ? mhi : ihi;
                box = make_uint2((uint32_t)(x0 >> TWL) | ((uint32_t)(y0 >> THL) << 16),
                                 (uint32_t)(x1 >> TWL) | ((uint32_t)(y1 >> THL) << 16));
            }
        }
        bl.tbox[slot] = box;
        int tx0 = 0, ty0 = 0, tw = 1;
        const int nt = box_tiles(box, tx0, ty0, tw);
        const int maxnt = (int)__reduce_max_sync(kFull, (unsigned)nt);
        for (int k = 0; k < maxnt; ++k) {
            const bool has = k < nt;
            const uint32_t t = has ? (uint32_t)((ty0 + k / tw) * bl.ntx + tx0 + k % tw) : kNoBox;
            const unsigned peers = __match_any_sync(kFull, t);
            if (has && lane == __ffs(peers) - 1) atomicAdd(&bl.tile_cnt[t], (uint32_t)__popc(peers));
        }
    }
}

// 2. scan (one CTA of 1024 threads): pair offsets (and the fill cursors),
// chunk offsets; a pair count above the list's capacity sets the device
// status bit and the tile pass then reads only the pairs that fit.
template <int KL>
__global__ void __launch_bounds__(1024) bin_scan_kernel(BinLayout bl, uint32_t *status) {
    __shared__ uint32_t s_w[32];
    __shared__ uint32_t s_carry;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    for (int pass = 0; pass < 2; ++pass) {
        if (tid == 0) s_carry = 0;
        __syncthreads();
        for (int base = 0; base < bl.ntiles; base += 1024) {
            const int t = base + tid;
            uint32_t c = 0;
            if (t < bl.ntiles)
                c = pass == 0 ? bl.tile_cnt[t] : (bl.tile_off[t + 1] - bl.tile_off[t] + (1u << KL) - 1) >> KL;
            uint32_t incl = c;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(kFull, incl, o);
                if (lane >= o) incl += y;
            }
            if (lane == 31) s_w[w] = incl;
            __syncthreads();
            if (w == 0) {
                uint32_t v = s_w[lane];
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const uint32_t y = __shfl_up_sync(kFull, v, o);
                    if (lane >= o) v += y;
                }
                s_w[lane] = v;
            }
            __syncthreads();
            const uint32_t excl = s_carry + (w ? s_w[w - 1] : 0u) + incl - c;
            if (t < bl.ntiles) {
                if (pass == 0) {
                    bl.tile_off[t] = excl;
                    bl.tile_cnt[t] = excl;
                } else {
                    bl.chunk_off[t] = excl;
                }
            }
            __syncthreads();
            if (tid == 1023) s_carry = excl + c;
            __syncthreads();
        }
        if (tid == 0) {
            if (pass == 0) {
                bl.tile_off[bl.ntiles] = s_carry;
                bl.ctl[kCtlPairs] = s_carry;
                if (s_carry > bl.pair_cap) atomicOr(status, kStatusBinOverflow);
            } else {
                bl.chunk_off[bl.ntiles] = s_carry;
                bl.ctl[kCtlUnits] = s_carry;
                bl.ctl[kCtlUnitTicket] = 0;
            }
        }
        __syncthreads();
    }
}

// 3. fill: every segment slot appends itself to its tiles' lists; the lanes
// of a warp that share a tile reserve their places with one atomic.
__global__ void __launch_bounds__(256) bin_fill_kernel(CallTable tab, BinLayout bl) {
    __shared__ uint32_t s_goff[HM_MAX_GROOMS_PER_CALL + 1];
    groom_batch_offsets(tab, s_goff);
    const uint32_t nslots = min(s_goff[tab.n] * (uint32_t)kBatchLanes, bl.slots);
    const int lane = threadIdx.x & 31;
    const uint32_t stride = gridDim.x * blockDim.x;
    // warp-uniform loop: base is the warp's first slot
    for (uint32_t base = blockIdx.x * blockDim.x + (threadIdx.x & ~31u); base < nslots; base += stride) {
        const uint32_t slot = base + lane;
        const uint2 box = slot < nslots ? bl.tbox[slot] : make_uint2(kNoBox, 0u);
        int tx0 = 0, ty0 = 0, tw = 1;
        const int nt = box_tiles(box, tx0, ty0, tw);
        const int maxnt = (int)__reduce_max_sync(kFull, (unsigned)nt);
        for (int k = 0; k < maxnt; ++k) {
            const bool has = k < nt;
            const uint32_t t = has ? (uint32_t)((ty0 + k / tw) * bl.ntx + tx0 + k % tw) : kNoBox;
            const unsigned peers = __match_any_sync(kFull, t);
            const int leader = __ffs(peers) - 1;
            uint32_t pos = 0;
            if (has && lane == leader) pos = atomicAdd(&bl.tile_cnt[t], (uint32_t)__popc(peers));
            pos = __shfl_sync(kFull, pos, leader) + (uint32_t)__popc(peers & ((1u << lane) - 1u));
            if (has && pos < bl.pair_cap) bl.list[pos] = slot;
        }
    }
}

// Sink of the tile pass: shared-memory atomicMin into the tile's two layers.
template <int TWL>
struct TileKeys {
    unsigned long long *s_c, *s_a;
    int x0, y0;
    __device__ __forceinline__ uint32_t index(int px, int py) const {
        return ((uint32_t)(py - y0) << TWL) | (uint32_t)(px - x0);
    }
    __device__ __forceinline__ uint32_t step(bool x_major, bool) const { return x_major ? (1u << TWL) : 1u; }
    __device__ __forceinline__ void operator()(uint32_t loc, uint64_t key, bool cen) const {
        atomicMin(&s_a[loc], (unsigned long long)key);
        if (cen) atomicMin(&s_c[loc], (unsigned long long)key);
    }
};

// 4. tile pass.  Unit u is chunk c of tile t, chunk_off[t] <= u <
// chunk_off[t + 1]; its segments are list[tile_off[t] + c 2^KL ..].
template <int TWL, int THL, int KL>
__global__ void __launch_bounds__(kRasterThreads, 4) bin_tile_kernel(CamDev cam, BinLayout bl, uint64_t *vis_c,
                                                                      uint64_t *vis_a, hm_frame_stats *stats) {
    constexpr int TW = 1 << TWL, TH = 1 << THL, NPX = TW * TH;
    __shared__ unsigned long long s_c[NPX], s_a[NPX];
    __shared__ SegRec s_rec[kRasterWarps][32];
    __shared__ uint32_t s_unit, s_next;
    const int W = cam.W, H = cam.H;
    const int lane = threadIdx.x & 31;
    SegRec *rec = s_rec[threadIdx.x >> 5];
    uint32_t n_cons = 0, n_cen = 0;
    const uint32_t npairs = min(bl.ctl[kCtlPairs], bl.pair_cap);
    const uint32_t nunits = bl.ctl[kCtlUnits];
    for (;;) {
        if (threadIdx.x == 0) {
            s_unit = atomicAdd(&bl.ctl[kCtlUnitTicket], 1u);
            s_next = 0;
        }
        for (int k = threadIdx.x; k < NPX; k += kRasterThreads) {
            s_c[k] = kEmptyKey;
            s_a[k] = kEmptyKey;
        }
        __syncthreads();
        const uint32_t u = s_unit;
        if (u >= nunits) break;
        // tile of unit u: the last t with chunk_off[t] <= u (it has chunks)
        int t = 0, hi = bl.ntiles;
        while (hi - t > 1) {
            const int mid = (t + hi) >> 1;
            if (bl.chunk_off[mid] <= u) t = mid; else hi = mid;
        }
        const uint32_t first = bl.tile_off[t] + ((u - bl.chunk_off[t]) << KL);
        const uint32_t lo = min(first, npairs);
        const uint32_t end = min(min(first + (1u << KL), bl.tile_off[t + 1]), npairs);
        const uint32_t n = end > lo ? end - lo : 0u;
        const int x0 = (t % bl.ntx) << TWL, y0 = (t / bl.ntx) << THL;
        const int x1 = min(x0 + TW, W) - 1, y1 = min(y0 + TH, H) - 1;
        const TileKeys<TWL> sink{s_c, s_a, x0, y0};
        for (;;) {
            uint32_t chunk = 0;
            if (lane == 0) chunk = atomicAdd(&s_next, 32u);
            chunk = __shfl_sync(kFull, chunk, 0);
            if (chunk >= n) break;
            SegRec r;
            int nmaj = 0;
            if (chunk + lane < n) {
                const BinSeg q = bl.segs[bl.list[lo + chunk + lane]];
                r.uA = q.uA;
                r.vA = q.vA;
                r.du = q.du;
                r.dv = q.dv;
                r.umin = min(q.uA, q.uA + q.du);
                r.umax = max(q.uA, q.uA + q.du);
                r.vmin = min(q.vA, q.vA + q.dv);
                r.vmax = max(q.vA, q.vA + q.dv);
                r.zA = q.zA;
                r.dz = q.dz;
                r.fden = q.fden;
                r.rden = __frcp_rn(q.fden);
                r.slope = q.slope;
                r.hc = q.hc;
                r.flags = q.flags;
                r.id_lo = q.id_lo;
                r.id_hi = q.id_hi;
                // major pixels of the segment's conservative box inside the tile
                const bool xm = q.flags & 1;
                r.ilo = max(((r.umin + 255) >> 8) - 1, xm ? x0 : y0);
                const int ihi = min(r.umax >> 8, xm ? x1 : y1);
                nmaj = ihi >= r.ilo ? ihi - r.ilo + 1 : 0;
            }
            for_each_item(rec, r, nmaj, [&](const SegRec &q, int i) {
                const bool xm = q.flags & 1;
                if (q.flags & 2)
                    raster_item<int32_t, false>(q, i, xm ? y0 : x0, xm ? y1 : x1, sink, n_cons, n_cen);
                else
                    raster_item<int64_t, false>(q, i, xm ? y0 : x0, xm ? y1 : x1, sink, n_cons, n_cen);
            });
        }
        __syncthreads();
        // flush: consecutive threads on consecutive keys of a tile row
        for (int k = threadIdx.x; k < NPX; k += kRasterThreads) {
            const int px = x0 + (k & (TW - 1)), py = y0 + (k >> TWL);
            if (px > x1 || py > y1) continue;
            const uint32_t p = key_index(cam, px, py);
            const unsigned long long a = s_a[k], c = s_c[k];
            if (a != kEmptyKey) atomicMin(reinterpret_cast<unsigned long long *>(vis_a + p), a);
            if (c != kEmptyKey) atomicMin(reinterpret_cast<unsigned long long *>(vis_c + p), c);
        }
        __syncthreads();
    }
    if (stats) {
        unsigned long long v[2] = {n_cons, n_cen};
        unsigned long long *const dst[2] = {(unsigned long long *)&stats->covered_cons,
                                            (unsigned long long *)&stats->covered_center};
        block_add_counters<kRasterThreads, 2>(v, dst);
    }
}

template <typename K>
int fit_per_sm(PerDevice<int> &cache, K kernel, int threads) {
    const int v = cache.get([&](int) {
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, 0);
        return per_sm;
    });
    return v < 1 ? 1 : v;
}

template <int TWL, int THL, int KL>
cudaError_t launch_binned_t(const CallTable &tab, const CamDev &cam, uint64_t *vis_c, uint64_t *vis_a,
                            const BinLayout &bl, uint32_t *status, hm_frame_stats *stats, cudaStream_t st) {
    static PerDevice<int> fit_count, fit_tile;
    cudaError_t e = cudaMemsetAsync(bl.tile_cnt, 0, (size_t)bl.ntiles * 4, st);
    if (e != cudaSuccess) return e;
    const int sms = num_sms();
    bin_count_kernel<TWL, THL>
        <<<fit_per_sm(fit_count, bin_count_kernel<TWL, THL>, kRasterThreads) * sms, kRasterThreads, 0, st>>>(tab, cam,
                                                                                                             bl);
    bin_scan_kernel<KL><<<1, 1024, 0, st>>>(bl, status);
    bin_fill_kernel<<<sms * 8, 256, 0, st>>>(tab, bl);
    bin_tile_kernel<TWL, THL, KL>
        <<<fit_per_sm(fit_tile, bin_tile_kernel<TWL, THL, KL>, kRasterThreads) * sms, kRasterThreads, 0, st>>>(
            cam, bl, vis_c, vis_a, stats);
    return cudaGetLastError();
}

template <int TWL, int THL>
cudaError_t launch_binned_k(int chunk, const CallTable &tab, const CamDev &cam, uint64_t *vis_c, uint64_t *vis_a,
                            const BinLayout &bl, uint32_t *status, hm_frame_stats *stats, cudaStream_t st) {
    return chunk == 1024 ? launch_binned_t<TWL, THL, 10>(tab, cam, vis_c, vis_a, bl, status, stats, st)
                         : launch_binned_t<TWL, THL, 8>(tab, cam, vis_c, vis_a, bl, status, stats, st);
}

}  // namespace

size_t binned_workspace_bytes(uint64_t slots, int W, int H, int tile_w, int tile_h) {
    if (slots == 0 || W < 1 || H < 1 || tile_w < 1 || tile_h < 1) return 0;
    if (slots * kPairsPerSlot >= (1ull << 32)) return 0;     // pair indices are 32-bit
    const size_t ntiles = (size_t)((W + tile_w - 1) / tile_w) * (size_t)((H + tile_h - 1) / tile_h);
    return align16(slots * sizeof(BinSeg)) + align16(slots * sizeof(uint2)) + align16(ntiles * 4) +
           2 * align16((ntiles + 1) * 4) + align16(kCtlWords * 4) + slots * kPairsPerSlot * 4;
}

cudaError_t launch_raster_binned(const CallTable &tab, const CamDev &cam, uint64_t *vis_c, uint64_t *vis_a, void *ws,
                                 uint64_t slots, int tile_w, int tile_h, int chunk, uint32_t *status,
                                 hm_frame_stats *stats, cudaStream_t st) {
    const BinLayout bl = bin_layout(ws, slots, cam.W, cam.H, tile_w, tile_h);
    if (tile_w == 16)
        return tile_h == 16 ? launch_binned_k<4, 4>(chunk, tab, cam, vis_c, vis_a, bl, status, stats, st)
                            : launch_binned_k<4, 5>(chunk, tab, cam, vis_c, vis_a, bl, status, stats, st);
    return tile_h == 16 ? launch_binned_k<5, 4>(chunk, tab, cam, vis_c, vis_a, bl, status, stats, st)
                        : launch_binned_k<5, 5>(chunk, tab, cam, vis_c, vis_a, bl, status, stats, st);
}

}  // namespace hm
