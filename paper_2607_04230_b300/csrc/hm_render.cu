// hm_render.cu -- visibility pass of the deferred hair rasterizer
// (arXiv 2607.04230, Sec. 3.1-3.2): clear, LOD pre-pass with the device work
// list, and the strand-generation + 64-bit atomicMin rasterizer.
#include <cstdint>
#include <type_traits>
#include <cstdlib>
#include <cuda_runtime.h>

#include "hm_device.cuh"
#include "hm_kernels.h"
#include "hm_raster.cuh"

namespace hm {

// ---------------------------------------------------------------------------
// clear: both layers to EMPTY or to the scene-depth pre-fill; zero the stats
// ---------------------------------------------------------------------------
constexpr int kClearCtasPerSm = 2;

// Pre-fill key of key slot k of a key layer in layout (W, H, layout, Wb):
// the scene depth of its pixel, or EMPTY for the padding of the blocked
// layout.  scene_d24 is row-major [H][W].
__device__ __forceinline__ uint64_t prefill_key(const uint32_t *scene_d24, const CamDev &c, int64_t k) {
    int64_t p = k;
    if (c.layout != HM_KEYS_ROW_MAJOR) {
        const int64_t b = k >> 2;
        const int x = (int)(b % c.Wb) * 2 + (int)(k & 1), y = (int)(b / c.Wb) * 2 + (int)((k >> 1) & 1);
        if (x >= c.W || y >= c.H) return kEmptyKey;
        p = (int64_t)y * c.W + x;
    }
    return ((uint64_t)(scene_d24[p] & 0xFFFFFFu) << 40) | kPayloadMask;
}

// nkeys keys per layer (npairs = nkeys / 2 whole 16-byte pairs); cam gives
// the pre-fill's pixel of each key.
__global__ void __launch_bounds__(256) clear_kernel(ulonglong2 *vis_c, ulonglong2 *vis_a, int64_t npairs,
                                                    const uint32_t *scene_d24, int64_t nkeys, CamDev cam,
                                                    int do_clear, hm_frame_stats *stats) {
    // the LOD selection may start beside the clear (it touches neither the
    // keys nor, until it waits for the clear, the stats)
    pdl_launch_dependents();
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0 && stats) {
        stats->strands = 0;
        stats->segments = 0;
        stats->bundles_culled = 0;
        stats->covered_center = 0;
        stats->covered_cons = 0;
    }
    if (!do_clear) return;
    // an odd last key is written alone
    if (i == 0 && (nkeys & 1)) {
        const int64_t k = nkeys - 1;
        const uint64_t v = scene_d24 ? prefill_key(scene_d24, cam, k) : kEmptyKey;
        reinterpret_cast<uint64_t *>(vis_c)[k] = v;
        reinterpret_cast<uint64_t *>(vis_a)[k] = v;
    }
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (; i < npairs; i += stride) {
        ulonglong2 v;
        if (scene_d24) {
            v.x = prefill_key(scene_d24, cam, 2 * i);
            v.y = prefill_key(scene_d24, cam, 2 * i + 1);
        } else {
            v.x = kEmptyKey;
            v.y = kEmptyKey;
        }
        vis_c[i] = v;
        if (vis_a != vis_c) vis_a[i] = v;
    }
}

// ---------------------------------------------------------------------------
// LOD pre-pass (Sec. 3.2, Eqs. 1-5): one thread per bundle, one CTA per groom
// ---------------------------------------------------------------------------
__device__ __forceinline__ void lod_counts(float Lf, int nfull, float delta, int L, int cmax, int &n_out,
                                           int &c_out) {
    int n = 0;
    if (nfull > 0) {
        float v = ceilf(fmul(Lf, fadd(__int2float_rn(nfull), delta)));
        n = (int)v;
        if (n < 1) n = 1;
        if (n > nfull) n = nfull;
    }
    int craw = (int)floorf(fmul(__fsqrt_rn(Lf), __int2float_rn(cmax)));
    if (craw < L) craw = L;
    int c = (1 << (31 - __clz(craw - 1))) + 1;
    if (c > cmax) c = cmax;
    int lo = L < cmax ? L : cmax;
    if (c < lo) c = lo;
    n_out = n;
    c_out = c;
}

// Screen AABB over every layer's triangle (Eq. 3), frustum cull, L (Eq. 2).
// A bundle wholly behind the near plane is culled; one straddling it is
// drawn at L = 1.  Returns false when culled.
__device__ __forceinline__ bool lod_select(const GroomDev &g, const CamDev &cam, int f, float &Lf) {
    int4 tri = __ldg(&g.faces[f]);
    float xmin = __int_as_float(0x7f800000), xmax = -__int_as_float(0x7f800000);
    float ymin = xmin, ymax = xmax;
    bool behind = false, front = false;
    // the next layer's three vertices are loaded while this layer's are
    // projected (the AABB is a min/max, independent of the order)
    float4 nv[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) nv[c] = __ldg(&g.lv[c == 0 ? tri.x : (c == 1 ? tri.y : tri.z)]);
    for (int k = 0; k < g.L; ++k) {
        float4 cv[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) cv[c] = nv[c];
        if (k + 1 < g.L) {
            const float4 *next = g.lv + (int64_t)(k + 1) * g.V;
#pragma unroll
            for (int c = 0; c < 3; ++c) nv[c] = __ldg(&next[c == 0 ? tri.x : (c == 1 ? tri.y : tri.z)]);
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float4 v = cv[c];
            Proj p = project(cam, make_float3(v.x, v.y, v.z));
            if (!p.valid) { behind = true; continue; }
            front = true;
            if (p.xs < xmin) xmin = p.xs;
            if (p.xs > xmax) xmax = p.xs;
            if (p.ys < ymin) ymin = p.ys;
            if (p.ys > ymax) ymax = p.ys;
        }
    }
    if (!front) return false;
    if (behind) { Lf = 1.0f; return true; }
    if (xmax < 0.0f || xmin > __int2float_rn(cam.W) || ymax < 0.0f || ymin > __int2float_rn(cam.H)) return false;
    float dx = fsub(xmax, xmin), dy = fsub(ymax, ymin);
    float diag = __fsqrt_rn(fadd(fmul(dx, dx), fmul(dy, dy)));
    Lf = fclamp(fmul(fdiv(diag, __int2float_rn(cam.H)), g.lod_lambda), 0.0f, 1.0f);
    return true;
}

template <int NT>
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t &total, uint32_t *sm) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(kFull, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sm[w] = x;
    __syncthreads();
    if (w == 0) {
        uint32_t s = lane < NT / 32 ? sm[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(kFull, s, o);
            if (lane >= o) s += y;
        }
        if (lane < NT / 32) sm[lane] = s;
    }
    __syncthreads();
    uint32_t off = w > 0 ? sm[w - 1] : 0;
    total = sm[NT / 32 - 1];
    __syncthreads();
    return off + x - v;
}

// The LOD decision of every bundle, all grooms at once (one thread per
// bundle): lod[f] = (N_LOD, C, -, -); the scan fills in the offsets.
constexpr int kLodSelThreads = 256;

__global__ void __launch_bounds__(kLodSelThreads) lod_select_kernel(CallTable tab, CamDev cam,
                                                                    hm_frame_stats *stats) {
    const GroomDev &g = tab.g[blockIdx.y];
    const int f = blockIdx.x * kLodSelThreads + (int)threadIdx.x;
    unsigned long long strands = 0, segs = 0, culled = 0;
    if (f < g.F) {
        const int nfull = __ldg(&g.faces[f + 1]).w - __ldg(&g.faces[f]).w;
        int n = nfull, c = g.cmax;
        if (g.lod_enabled) {
            float Lf = 0.0f;
            if (lod_select(g, cam, f, Lf)) {
                lod_counts(Lf, nfull, __ldg(&g.delta[f]), g.L, g.cmax, n, c);
            } else {
                n = 0;
                culled = 1;
            }
        }
        const uint32_t nseg = (uint32_t)n * (uint32_t)(c - 1);
        g.lod[f] = make_uint4((uint32_t)n, (uint32_t)c, 0u, 0u);
        strands = (unsigned long long)n;
        segs = nseg;
    }
    // launched as a programmatic dependent of the clear: the stats it zeroes
    // are added to only after it has completed
    pdl_wait();
    if (stats) {
        unsigned long long v[3] = {strands, segs, culled};
        unsigned long long *const dst[3] = {(unsigned long long *)&stats->strands,
                                            (unsigned long long *)&stats->segments,
                                            (unsigned long long *)&stats->bundles_culled};
        block_add_counters<kLodSelThreads, 3>(v, dst);
    }
}

// The bundles' first drawn segment and first drawn control point
// (exclusive scans of N_LOD (C - 1) and N_LOD C), and the work list the
// rasterizers pull from: batch b holds the groom's drawn control points
// kBatchStride b .. kBatchStride b + 31 in bundle order (one batch may span
// several bundles, so lanes stay busy when LOD leaves bundles a few points),
// listed with the bundle holding its first point.  grid.y = groom, grid.x =
// slices of kLodFillPerCta batches: every CTA of a groom repeats the (short)
// scans over its bundles, the first one publishes them, and each fills its
// slice one batch per thread by a binary search over the point scan (a
// bundle without points shares its first point with the next one, so the
// search lands on the bundle that holds the point).
constexpr int kLodScanThreads = 1024, kLodScanCache = 12000, kLodFillPerCta = 8192;

__global__ void __launch_bounds__(kLodScanThreads) lod_scan_kernel(CallTable tab) {
    __shared__ uint32_t sm[kLodScanThreads / 32];
    __shared__ uint32_t s_first[kLodScanCache + 1];
    const GroomDev &g = tab.g[blockIdx.y];
    const bool cache = g.F <= kLodScanCache;
    const bool lead = blockIdx.x == 0;
    if (!cache && !lead) return;                  // large meshes: the first CTA fills serially
    if (!lead && blockIdx.x * (uint32_t)kLodFillPerCta >= g.max_batches) return;   // beyond this groom's list
    uint32_t segs = 0, pts = 0;
    for (int base = 0; base < g.F; base += kLodScanThreads) {
        const int f = base + (int)threadIdx.x;
        uint32_t n = 0, c = 0;
        if (f < g.F) {
            const uint4 lo = g.lod[f];
            n = lo.x;
            c = lo.y;
        }
        uint32_t tot_s, tot_p;
        const uint32_t first_s = segs + block_excl_scan<kLodScanThreads>(n * (c - 1), tot_s, sm);
        const uint32_t first_p = pts + block_excl_scan<kLodScanThreads>(n * c, tot_p, sm);
        if (f < g.F) {
            if (lead) {
                g.lod[f].z = first_s;
                g.lod[f].w = first_p;
            }
            if (cache) {
                s_first[f] = first_p;
            } else if (n > 0) {
                for (uint32_t b = (first_p + kBatchStride - 1) / kBatchStride; b * kBatchStride < first_p + n * c; ++b)
                    g.batch_map[b] = (uint32_t)f;
            }
        }
        segs += tot_s;
        pts += tot_p;
    }
    // every segment (q, q + 1) with q < pts - 1 lies in batch q / kBatchStride
    const uint32_t nbatch = pts > 1 ? (pts - 2) / kBatchStride + 1 : 0;
    if (cache) {
        if (threadIdx.x == 0) s_first[g.F] = pts;
        __syncthreads();
        const uint32_t b0 = blockIdx.x * (uint32_t)kLodFillPerCta;
        const uint32_t b1 = min(b0 + (uint32_t)kLodFillPerCta, nbatch);
        for (uint32_t b = b0 + threadIdx.x; b < b1; b += kLodScanThreads) {
            const uint32_t x = b * kBatchStride;    // first point of the batch
            int lo = 0, hi = g.F;                   // s_first[lo] <= x < s_first[hi]
            while (hi - lo > 1) {
                const int mid = (lo + hi) >> 1;
                if (s_first[mid] <= x) lo = mid; else hi = mid;
            }
            g.batch_map[b] = (uint32_t)lo;
        }
    }
    if (lead && threadIdx.x == 0) {
        g.counters[kCtrBatches] = nbatch;
        g.counters[kCtrSegs] = segs;
        g.counters[kCtrCps] = pts;
        if (blockIdx.y == 0) g.counters[kCtrTicket] = 0;
    }
}

// ---------------------------------------------------------------------------
// rasterizer (Sec. 3.1.1 strand assembly, Sec. 3.1.2 atomicMin visibility,
// Sec. 3.3 two layers)
//
// Persistent grid; each warp pulls work-list batches from a ticket.  A lane
// generates one control point and projects and snaps it; the next lane's
// point, taken by shuffle, closes the lane's segment (so each point is
// generated and projected once, not once per segment that ends in it).  The
// warp then enumerates the batch's candidate pixels together: work items are
// (segment, pixel step along the major axis), load-balanced across the warp
// by a prefix sum, and each item tests its 2-4 minor-axis pixels with the
// exact predicate and issues the 64-bit atomicMin for each layer.
// ---------------------------------------------------------------------------
// kMode: 0 one view, 1 several views (strands assembled once), 2 one view
// with the compressed payload.  kBlocked: the views' key layers are in 2 x 2
// blocks (HM_KEYS_BLOCK_2X2), else row-major.
template <bool kPrecheck, int kMinBlocks, int kMode, bool kBlocked>
__global__ void __launch_bounds__(kRasterThreads, kMinBlocks) raster_kernel(CallTable tab, ViewSet views,
                                                                            hm_frame_stats *stats) {
    constexpr bool kMulti = kMode == 1, kCgb = kMode == 2;
    __shared__ uint32_t s_goff[HM_MAX_GROOMS_PER_CALL + 1];
    __shared__ SegRec s_rec[kRasterWarps][32];
    groom_batch_offsets(tab, s_goff);
    const uint32_t total = s_goff[tab.n];
    const int lane = threadIdx.x & 31;
    SegRec *rec = s_rec[threadIdx.x >> 5];
    uint32_t *ticket = tab.g[0].counters + kCtrTicket;
    const int W = views.cam[0].W, H = views.cam[0].H;
    uint32_t n_cons = 0, n_cen = 0;

    for (;;) {
        uint32_t b = 0;
        if (lane == 0) b = atomicAdd(ticket, 1u);
        b = __shfl_sync(kFull, b, 0);
        if (b >= total) break;
        const int gi = batch_groom(s_goff, tab.n, b);
        const GroomDev &g = tab.g[gi];
        const uint32_t lb = b - s_goff[gi];
        // this lane's control point, and its segment to lane + 1's point
        const BatchPoint bp = batch_lane_point(g, lb, lane);
        const bool active = bp.seg_ok;
        const float3 cp[2] = {bp.p, next_lane(bp.p)};
        if (active && g.segpts) store_segment_points(g.segpts, bp.seg, cp);
        uint32_t cgb_hi = 0;
        float aoA = 1.0f, aoB = 1.0f;
        if (kCgb) {
            Root rt;
            if (bp.has) {
                rt = make_root(g, bp.s, bp.f);
                aoA = control_ao_exact(g, rt, bp.C, bp.j);
            }
            aoB = __shfl_down_sync(kFull, aoA, 1);
            if (active) cgb_hi = (oct_encode(v3unit(v3sub(cp[1], cp[0]))) << 12) | root_uv_codes(g, rt);
        }
        const int n_views = kMulti ? views.n : 1;
        for (int view = 0; view < n_views; ++view) {
        const CamDev &cam = views.cam[view];
        Proj A, B;
        const bool drawn = batch_lane_segment(cam, bp, A, B);
        SegRec r;
        int nmaj = 0;
        if (drawn) {
            segment_frame(cam, g.width_m, A, B, r);
            if (kCgb) {
                r.id_lo = (uint32_t)bp.j;
                r.id_hi = (uint32_t)(bp.C - 1);
                r.cgb_hi = cgb_hi;
                r.aoA = aoA;
                r.dao = fsub(aoB, aoA);
            } else {
                const uint64_t id = ((g.base + (uint64_t)bp.s) << 7) | (uint64_t)bp.j;
                r.id_lo = (uint32_t)id;
                r.id_hi = (uint32_t)(id >> 32);
            }
            const bool xm = r.flags & 1;
            int ihi, mlo, mhi;
            if (segment_pixel_box(r, xm ? W : H, xm ? H : W, r.ilo, ihi, mlo, mhi)) nmaj = ihi - r.ilo + 1;
        }
        const GlobalKeys<kPrecheck, kBlocked> sink{views.vis_c[view], views.vis_a[view], (uint32_t)W,
                                                   (uint32_t)cam.Wb};
        for_each_item(rec, r, nmaj, [&](const SegRec &q, int i) {
            const int mmax = (q.flags & 1) ? H - 1 : W - 1;
            if (q.flags & 2)
                raster_item<int32_t, kCgb>(q, i, 0, mmax, sink, n_cons, n_cen);
            else
                raster_item<int64_t, kCgb>(q, i, 0, mmax, sink, n_cons, n_cen);
        });
        }   // views
    }
    if (stats) {
        unsigned long long v[2] = {n_cons, n_cen};
        unsigned long long *const dst[2] = {(unsigned long long *)&stats->covered_cons,
                                            (unsigned long long *)&stats->covered_center};
        block_add_counters<kRasterThreads, 2>(v, dst);
    }
}

// ---------------------------------------------------------------------------
// multisample rasterizer (Sec. 3.3: samples recorded into multiple uint64
// layers, the paper's MSAA reference)
//
// Sample k of pixel (i, m) sits at offset (ox_k, oy_k) from the pixel centre
// and is covered iff the closed box of the segment's centre half-width h_c
// around the sample point meets the segment (the centre-sample predicate at
// the sample); its key's depth uses the sample's projection parameter.
// Sample boxes reach at most 7/16 + 1/2 px from the pixel centre, so the
// candidate pixels of a segment are taken one pixel wider on each side.
// ---------------------------------------------------------------------------
template <typename I, int N>
__device__ __forceinline__ void raster_item_msaa(const SegRec &q_shared, int i, int W, int H,
                                                 uint64_t *__restrict__ vis_s, int64_t npx, uint32_t &n_hits) {
    const SegRec q = q_shared;
    const bool xm = q.flags & 1;
    const int32_t cu = 256 * i + 128;
    const int dimv = xm ? H : W;
    // float error of a minor-axis value on the line is below |dV| 2^-21 + 1
    // unit; with |vA| <= 2^28 (guard band) and |slope| <= 1 every term fits 32 bits
    const int32_t slack = 8 + (abs(q.dv) >> 20);
    // I: 32-bit for short segments (|dU|, |dV| < 2^14), whose cross products
    // and numerators at the candidate samples stay below 2^30
    const I du = q.du, dv = q.dv;
    const I k_cen = (I)q.hc * ((I)abs(q.du) + (I)abs(q.dv));
    const uint64_t id = ((uint64_t)q.id_hi << 32) | q.id_lo;
    const bool degenerate = (q.du == 0 && q.dv == 0);
    typedef typename std::make_unsigned<I>::type U;
#pragma unroll
    for (int k = 0; k < N; ++k) {
        int ox, oy;
        sample_offset<N>(k, ox, oy);
        const int32_t ou = xm ? ox : oy, ov = xm ? oy : ox;
        const int32_t su = cu + ou;
        // a covered sample's box [su +- hc] x [sv +- hc] holds a segment point
        // (u*, v*): u* in [su - hc, su + hc] clipped to the segment, v* on the
        // line there (within the float range [vlo, vhi]), |v* - sv| <= hc; so
        // the sample's row m has vlo - hc <= 256 m + 128 + ov <= vhi + hc
        const int32_t ua = max(su - q.hc, q.umin), ub = min(su + q.hc, q.umax);
        if (ua > ub) continue;
        const float va = (float)(ua - q.uA) * q.slope, vb = (float)(ub - q.uA) * q.slope;
        const int32_t vlo = q.vA + (int32_t)floorf(fminf(va, vb)) - slack;
        const int32_t vhi = q.vA + (int32_t)ceilf(fmaxf(va, vb)) + slack;
        const int mlo = max((vlo - q.hc - 128 - ov + 255) >> 8, 0);
        const int mhi = min((vhi + q.hc - 128 - ov) >> 8, dimv - 1);
        const I ru = (I)(su - q.uA);
        for (int m = mlo; m <= mhi; ++m) {
            const int32_t sv = 256 * m + 128 + ov;
            // closed box of half-width hc around the sample: boxes overlap and
            // |cross product| <= hc (|dU| + |dV|) (one unsigned compare)
            if (q.vmin > sv + q.hc || q.vmax < sv - q.hc) continue;
            const I rv = (I)(sv - q.vA);
            if ((U)(du * rv - dv * ru + k_cen) > (U)(2 * k_cen)) continue;
            float t = 0.0f;
            if (!degenerate) {
                const I nk = ru * du + rv * dv;
                const float fn = sizeof(I) == 4 ? __int2float_rn((int32_t)nk) : __ll2float_rn((int64_t)nk);
                t = fclamp(quotient_rn(fn, q.fden, q.rden), 0.0f, 1.0f);
            }
            const uint32_t d24 = depth_d24(q, t);
            const int px = xm ? i : m, py = xm ? m : i;
            const int64_t p = (int64_t)((uint32_t)py * (uint32_t)W + (uint32_t)px);
            atomicMin(reinterpret_cast<unsigned long long *>(vis_s + (int64_t)k * npx + p),
                      (unsigned long long)(((uint64_t)d24 << 40) | id));
            n_hits += 1;
        }
    }
}

template <int N>
__global__ void __launch_bounds__(kRasterThreads, 4) raster_msaa_kernel(CallTable tab, CamDev cam,
                                                                        uint64_t *__restrict__ vis_s,
                                                                        hm_frame_stats *stats) {
    __shared__ uint32_t s_goff[HM_MAX_GROOMS_PER_CALL + 1];
    __shared__ SegRec s_rec[kRasterWarps][32];
    groom_batch_offsets(tab, s_goff);
    const uint32_t total = s_goff[tab.n];
    const int lane = threadIdx.x & 31;
    SegRec *rec = s_rec[threadIdx.x >> 5];
    uint32_t *ticket = tab.g[0].counters + kCtrTicket;
    const int W = cam.W, H = cam.H;
    const int64_t npx = (int64_t)W * H;
    uint32_t n_hits = 0;
    for (;;) {
        uint32_t b = 0;
        if (lane == 0) b = atomicAdd(ticket, 1u);
        b = __shfl_sync(kFull, b, 0);
        if (b >= total) break;
        const int gi = batch_groom(s_goff, tab.n, b);
        const GroomDev &g = tab.g[gi];
        const uint32_t lb = b - s_goff[gi];
        const BatchPoint bp = batch_lane_point(g, lb, lane);
        const float3 cp[2] = {bp.p, next_lane(bp.p)};
        if (bp.seg_ok && g.segpts) store_segment_points(g.segpts, bp.seg, cp);
        Proj A, B;
        const bool drawn = batch_lane_segment(cam, bp, A, B);
        SegRec r;
        int nmaj = 0;
        if (drawn) {
            segment_frame(cam, g.width_m, A, B, r);
            const uint64_t id = ((g.base + (uint64_t)bp.s) << 7) | (uint64_t)bp.j;
            r.id_lo = (uint32_t)id;
            r.id_hi = (uint32_t)(id >> 32);
            const bool xm = r.flags & 1;
            const int du = xm ? W : H, dv = xm ? H : W;
            // columns i whose sample boxes (centre 256 i + 128, sample
            // offsets up to kOff, half-width hc) can reach [umin, umax]
            constexpr int32_t kOff = N == 1 ? 0 : (N == 2 ? 64 : (N == 4 ? 96 : 112));
            const int32_t reach = kOff + r.hc;
            int ilo = (r.umin - reach - 128 + 255) >> 8, ihi = (r.umax + reach - 128) >> 8;
            ilo = max(ilo, 0);
            ihi = min(ihi, du - 1);
            const bool vin = r.vmax >= -256 && r.vmin <= 256 * dv + 256;
            r.ilo = ilo;
            nmaj = (vin && ihi >= ilo) ? ihi - ilo + 1 : 0;
        }
        for_each_item(rec, r, nmaj, [&](const SegRec &q, int i) {
            if (q.flags & 2)
                raster_item_msaa<int32_t, N>(q, i, W, H, vis_s, npx, n_hits);
            else
                raster_item_msaa<int64_t, N>(q, i, W, H, vis_s, npx, n_hits);
        });
    }
    if (stats) {
        unsigned long long v[1] = {n_hits};
        unsigned long long *const dst[1] = {(unsigned long long *)&stats->covered_center};
        block_add_counters<kRasterThreads, 1>(v, dst);
    }
}

cudaError_t launch_raster_msaa(const CallTable &tab, const CamDev &cam, int samples, uint64_t *vis_s,
                               hm_frame_stats *stats, cudaStream_t st) {
    int per_sm = 0;
    switch (samples) {
        case 1:
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, raster_msaa_kernel<1>, kRasterThreads, 0);
            raster_msaa_kernel<1><<<(per_sm > 0 ? per_sm : 1) * num_sms(), kRasterThreads, 0, st>>>(tab, cam, vis_s, stats);
            break;
        case 2:
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, raster_msaa_kernel<2>, kRasterThreads, 0);
            raster_msaa_kernel<2><<<(per_sm > 0 ? per_sm : 1) * num_sms(), kRasterThreads, 0, st>>>(tab, cam, vis_s, stats);
            break;
        case 4:
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, raster_msaa_kernel<4>, kRasterThreads, 0);
            raster_msaa_kernel<4><<<(per_sm > 0 ? per_sm : 1) * num_sms(), kRasterThreads, 0, st>>>(tab, cam, vis_s, stats);
            break;
        default:
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, raster_msaa_kernel<8>, kRasterThreads, 0);
            raster_msaa_kernel<8><<<(per_sm > 0 ? per_sm : 1) * num_sms(), kRasterThreads, 0, st>>>(tab, cam, vis_s, stats);
            break;
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// roofline probe: 64-bit atomicMin throughput on a frame-sized buffer
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) probe_atomic_min_kernel(unsigned long long *buf, int64_t n, int rounds,
                                                               int pattern) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int r = 0; r < rounds; ++r) {
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
            // 0: consecutive lanes on consecutive elements; 1: multiplicatively
            // hashed element per lane; 2: one hashed element per warp (32-way contended)
            const uint64_t h = pattern == 2 ? (uint64_t)(i >> 5) : (uint64_t)i;
            int64_t a = pattern ? (int64_t)((h * 0x9E3779B97F4A7C15ull) % (uint64_t)n) : i;
            atomicMin(buf + a, (unsigned long long)((int64_t)rounds - r) << 40 | (unsigned long long)i);
        }
    }
}

cudaError_t launch_probe_atomic_min(uint64_t *buf, int64_t n, int rounds, int pattern, cudaStream_t st) {
    int grid = num_sms() * 8;
    probe_atomic_min_kernel<<<grid, 256, 0, st>>>(reinterpret_cast<unsigned long long *>(buf), n, rounds, pattern);
    return cudaGetLastError();
}

// The rasterizers' depth-parameter quotient over arrays (hm_probe_quotient):
// the per-segment reciprocal, then quotient_rn.
__global__ void __launch_bounds__(256) probe_quotient_kernel(const float *__restrict__ num,
                                                             const float *__restrict__ den,
                                                             float *__restrict__ out, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float b = __ldg(&den[i]);
        out[i] = quotient_rn(__ldg(&num[i]), b, __frcp_rn(b));
    }
}

cudaError_t launch_probe_quotient(const float *num, const float *den, float *out, int64_t n, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    const int64_t want = (n + 255) / 256, cap = (int64_t)num_sms() * 8;
    probe_quotient_kernel<<<(unsigned)(want < cap ? want : cap), 256, 0, st>>>(num, den, out, n);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
cudaError_t launch_clear(uint64_t *vis_c, uint64_t *vis_a, int64_t nkeys, const uint32_t *scene_d24, const CamDev &cam,
                         int do_clear, hm_frame_stats *stats, cudaStream_t st) {
    int64_t npairs = nkeys / 2;
    // a grid-stride store stream on a few CTAs per SM, leaving room for the
    // LOD selection that runs beside it
    const int64_t cap = (int64_t)num_sms() * kClearCtasPerSm;
    int64_t want = (npairs + 255) / 256;
    int grid = (int)(want < cap ? (want > 0 ? want : 1) : cap);
    clear_kernel<<<grid, 256, 0, st>>>(reinterpret_cast<ulonglong2 *>(vis_c), reinterpret_cast<ulonglong2 *>(vis_a),
                                       npairs, scene_d24, nkeys, cam, do_clear, stats);
    return cudaGetLastError();
}

cudaError_t launch_lod(const CallTable &tab, const CamDev &cam, hm_frame_stats *stats, cudaStream_t st) {
    int fmax = 1;
    for (int i = 0; i < tab.n; ++i) fmax = tab.g[i].F > fmax ? tab.g[i].F : fmax;
    // a programmatic dependent of the clear that precedes it on the stream:
    // it may start while the clear runs and waits for it before the stats
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)((fmax + kLodSelThreads - 1) / kLodSelThreads), (unsigned)tab.n);
    cfg.blockDim = dim3(kLodSelThreads);
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaError_t e = cudaLaunchKernelEx(&cfg, lod_select_kernel, tab, cam, stats);
    if (e != cudaSuccess) return e;
    uint32_t bmax = 1;
    for (int i = 0; i < tab.n; ++i) bmax = tab.g[i].max_batches > bmax ? tab.g[i].max_batches : bmax;
    const dim3 sgrid((unsigned)((bmax + kLodFillPerCta - 1) / kLodFillPerCta), (unsigned)tab.n);
    lod_scan_kernel<<<sgrid, kLodScanThreads, 0, st>>>(tab);
    return cudaGetLastError();
}

// Raster variants: read-before-atomic on/off, and the register budget
// (min resident CTAs per SM of 256 threads: 3 -> up to 80 registers,
// 4 -> 64).  The persistent grid is ctas_per_sm CTAs per SM, capped at what
// fits (0 = as many as fit).
template <bool P, int M, int V, bool B>
static int raster_fit_per_sm() {
    static PerDevice<int> fit;
    const int v = fit.get([](int) {
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, raster_kernel<P, M, V, B>, kRasterThreads, 0);
        return per_sm;
    });
    return v < 1 ? 1 : v;
}

template <bool P, int M, int V, bool B>
static cudaError_t launch_raster_v(const CallTable &tab, const ViewSet &views, int ctas_per_sm, hm_frame_stats *stats,
                                   cudaStream_t st) {
    const int fit = raster_fit_per_sm<P, M, V, B>();
    const int per_sm = (ctas_per_sm > 0 && ctas_per_sm < fit) ? ctas_per_sm : fit;
    raster_kernel<P, M, V, B><<<per_sm * num_sms(), kRasterThreads, 0, st>>>(tab, views, stats);
    return cudaGetLastError();
}

template <int V, bool B>
static cudaError_t launch_raster_layout(const CallTable &tab, const ViewSet &views, bool precheck, int min_blocks,
                                        int ctas_per_sm, hm_frame_stats *stats, cudaStream_t st) {
    const bool m3 = min_blocks == 3;
    if (precheck)
        return m3 ? launch_raster_v<true, 3, V, B>(tab, views, ctas_per_sm, stats, st)
                  : launch_raster_v<true, 4, V, B>(tab, views, ctas_per_sm, stats, st);
    return m3 ? launch_raster_v<false, 3, V, B>(tab, views, ctas_per_sm, stats, st)
              : launch_raster_v<false, 4, V, B>(tab, views, ctas_per_sm, stats, st);
}

template <int V>
static cudaError_t launch_raster_views(const CallTable &tab, const ViewSet &views, bool precheck, int min_blocks,
                                       int ctas_per_sm, hm_frame_stats *stats, cudaStream_t st) {
    // every view of a launch shares the key layout (checked by the caller)
    if (views.cam[0].layout == HM_KEYS_BLOCK_2X2)
        return launch_raster_layout<V, true>(tab, views, precheck, min_blocks, ctas_per_sm, stats, st);
    return launch_raster_layout<V, false>(tab, views, precheck, min_blocks, ctas_per_sm, stats, st);
}

cudaError_t launch_raster(const CallTable &tab, const ViewSet &views, bool precheck, int min_blocks, int ctas_per_sm,
                          hm_frame_stats *stats, cudaStream_t st, bool compressed) {
    if (compressed) return launch_raster_views<2>(tab, views, precheck, min_blocks, ctas_per_sm, stats, st);
    if (views.n > 1) return launch_raster_views<1>(tab, views, precheck, min_blocks, ctas_per_sm, stats, st);
    return launch_raster_views<0>(tab, views, precheck, min_blocks, ctas_per_sm, stats, st);
}

}  // namespace hm

namespace hm {

// xyz from a packed [n][3] array; w (ambient occlusion of layer vertices)
// is kept.
__global__ void pack_float3_kernel(const float *__restrict__ src, float4 *__restrict__ dst, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = make_float4(src[3 * i], src[3 * i + 1], src[3 * i + 2], dst[i].w);
}

cudaError_t launch_pack_float3(const float *src, float4 *dst, int64_t n, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    pack_float3_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(src, dst, n);
    return cudaGetLastError();
}

}  // namespace hm
