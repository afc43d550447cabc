// hm_raster.cuh -- pieces shared by the rasterizers (arXiv 2607.04230,
// Sec. 3.1.2 atomicMin visibility, Sec. 3.3 two layers): the batch work list,
// the screen-space set-up of a segment and the exact per-pixel coverage and
// depth of one work item, written once so that the direct rasterizer and the
// screen-tile binned one produce the same key for every (pixel, layer).
#pragma once

#include <cstdint>
#include <type_traits>
#include <cuda_runtime.h>

#include "hm_device.cuh"

namespace hm {

constexpr unsigned kFull = 0xFFFFFFFFu;

// Adds the block's per-thread counters v[0..K) to dst[0..K) with one atomic
// per counter per block (warp shuffles, then shared memory), so the frame's
// thousands of warps do not queue on the same few addresses at the end of a
// pass.  Block-wide (every thread calls it); NT = blockDim.x.
template <int NT, int K>
__device__ __forceinline__ void block_add_counters(unsigned long long (&v)[K], unsigned long long *const (&dst)[K]) {
    __shared__ unsigned long long s_red[NT / 32][K];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < K; ++k) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(kFull, v[k], o);
        if (lane == 0) s_red[w][k] = v[k];
    }
    __syncthreads();
    if ((int)threadIdx.x < K) {
        unsigned long long t = 0;
#pragma unroll
        for (int i = 0; i < NT / 32; ++i) t += s_red[i][threadIdx.x];
        if (t) atomicAdd(dst[threadIdx.x], t);
    }
}

// s_goff[0..n] = the exclusive prefix of the call's per-groom batch counts
// (written by the LOD pass): one thread loads each count (independent
// global loads, instead of one thread chaining n of them), then one thread
// sums them in shared memory.  Block-wide; blockDim >= HM_MAX_GROOMS_PER_CALL.
__device__ __forceinline__ void groom_batch_offsets(const CallTable &tab, uint32_t *s_goff) {
    if ((int)threadIdx.x < tab.n) s_goff[threadIdx.x + 1] = tab.g[threadIdx.x].counters[kCtrBatches];
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t acc = 0;
        s_goff[0] = 0;
        for (int i = 1; i <= tab.n; ++i) {
            acc += s_goff[i];
            s_goff[i] = acc;
        }
    }
    __syncthreads();
}

// Groom of work batch b: the last groom whose first batch is <= b (goff
// holds the n + 1 prefix batch counts, so grooms without batches are passed
// over); a binary search, as a crowd call holds up to 64 grooms.
__device__ __forceinline__ int batch_groom(const uint32_t *goff, int n, uint32_t b) {
    int lo = 0, hi = n;          // goff[lo] <= b < goff[n]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (goff[mid] <= b) lo = mid; else hi = mid;
    }
    return lo;
}

// Drawn control point q of a groom, found from the bundle f0 that holds
// its batch's first point: its bundle f, strand s, index j along the strand,
// the strand's point count C, and the drawn segment it starts (seg, when
// j < C - 1).  Bundles that draw nothing share their first point with the
// next bundle and are passed over.
__device__ __forceinline__ void batch_point(const GroomDev &g, uint32_t f0, uint32_t q, uint32_t &f, int64_t &s,
                                            int &j, int &C, uint32_t &seg) {
    f = f0;
    while (f + 1 < (uint32_t)g.F && g.lod[f + 1].w <= q) ++f;
    const uint4 lo = g.lod[f];
    C = (int)lo.y;
    const uint32_t local = q - lo.w;
    const uint32_t sl = local / (uint32_t)C;
    j = (int)(local - sl * (uint32_t)C);
    s = (int64_t)__ldg(&g.faces[f]).w + sl;
    seg = lo.z + sl * (uint32_t)(C - 1) + (uint32_t)j;
}

// The lane's work-list point: lane l of batch b (local to groom g) holds
// drawn control point kBatchStride b + l, generated here (bit-identical to
// generating it within its segment); `seg_ok` when it starts a segment whose
// other end, the strand's next point, is lane l + 1's.  Warp-uniform call.
struct BatchPoint {
    float3 p;
    int64_t s;
    int j, C;
    uint32_t f, seg;
    bool has, seg_ok;
};

__device__ __forceinline__ BatchPoint batch_lane_point(const GroomDev &g, uint32_t lb, int lane) {
    BatchPoint r;
    const uint32_t q = lb * (uint32_t)kBatchStride + (uint32_t)lane;
    r.has = q < g.counters[kCtrCps];
    r.p = make_float3(0.0f, 0.0f, 0.0f);
    r.s = 0;
    r.j = 0;
    r.C = 2;
    r.f = 0;
    r.seg = 0;
    if (r.has) {
        batch_point(g, __ldg(&g.batch_map[lb]), q, r.f, r.s, r.j, r.C, r.seg);
        float3 one[1];
        control_pts<1>(g, make_root(g, r.s, r.f), r.C, r.j, one);
        r.p = one[0];
    }
    r.seg_ok = r.has && lane < kBatchStride && r.j < r.C - 1;
    return r;
}

// Lane l + 1's value (lane 31 gets its own back; it never starts a segment).
__device__ __forceinline__ float3 next_lane(float3 v) {
    return make_float3(__shfl_down_sync(kFull, v.x, 1), __shfl_down_sync(kFull, v.y, 1),
                       __shfl_down_sync(kFull, v.z, 1));
}

// Lane l + 1's projection: the fields the segment set-up reads (X, Y, w, z,
// valid).
__device__ __forceinline__ Proj next_lane(const Proj &p) {
    Proj r;
    r.X = __shfl_down_sync(kFull, p.X, 1);
    r.Y = __shfl_down_sync(kFull, p.Y, 1);
    r.w = __shfl_down_sync(kFull, p.w, 1);
    r.z = __shfl_down_sync(kFull, p.z, 1);
    r.xs = r.ys = 0.0f;
    r.valid = __shfl_down_sync(kFull, (int)p.valid, 1) != 0;
    return r;
}

// The lane's segment seen by one camera: each lane projects its own point
// and takes the far end from lane + 1.  False when the lane starts no
// segment or an end lies in front of the near plane.  Warp-uniform call.
__device__ __forceinline__ bool batch_lane_segment(const CamDev &cam, const BatchPoint &bp, Proj &A, Proj &B) {
    A.X = A.Y = 0;
    A.w = A.z = A.xs = A.ys = 0.0f;
    A.valid = false;
    if (bp.has) A = project(cam, bp.p);
    B = next_lane(A);
    return bp.seg_ok && A.valid && B.valid;
}

// A projected segment in the frame of its major screen axis u (x when
// |dX| >= |dY|) and minor axis v, in 1/256 px.
struct __align__(16) SegRec {
    int32_t uA, vA;              // start point in the major (u) / minor (v) frame, 1/256 px
    int32_t du, dv;              // B - A in that frame
    int32_t umin, umax, vmin, vmax;
    float zA, dz;                // linear depth at A and zB - zA, both x 2^24
    float fden;                  // float(|B - A|^2), the depth parameter's denominator
    float slope;                 // dv / du (0 for a point)
    int32_t hc;                  // centre-sample half-width, 1/256 px
    int32_t ilo;                 // first major pixel index
    int32_t start;               // first work item of this segment
    int32_t flags;               // bit0: u is x; bit1: short (32-bit arithmetic)
    uint32_t id_lo, id_hi;       // payload strand << 7 | segment; compressed: j, C - 1
    uint32_t cgb_hi;             // compressed: payload bits 39..12 (tangent, u, v) >> 12
    float aoA, dao;              // compressed: AO at A, AO(B) - AO(A)
    float rden;                  // RN(1 / fden), for quotient_rn
    uint32_t pad_[2];            // 96 bytes: read back with 16-byte loads
};
static_assert(sizeof(SegRec) == 96, "SegRec is read as six 16-byte words");

constexpr int kRasterThreads = 256;
static_assert(kRasterThreads >= HM_MAX_GROOMS_PER_CALL, "one thread per groom in the prologue");
constexpr int kRasterWarps = kRasterThreads / 32;

// Screen-space set-up of the segment between the projected control points A
// and B (both valid): its major-axis frame, extents, endpoint depths, the
// centre-sample half-width and the depth parameter's denominator.  Fills
// every field but the payload (id_lo, id_hi, cgb_hi, aoA, dao), ilo and
// start.  The operation order is fixed: the keys depend on it bit for bit.
__device__ __forceinline__ void segment_frame(const CamDev &cam, float width_m, const Proj &A, const Proj &B,
                                              SegRec &r) {
    const bool xm = abs(B.X - A.X) >= abs(B.Y - A.Y);
    const int32_t uA = xm ? A.X : A.Y, vA = xm ? A.Y : A.X;
    const int32_t uB = xm ? B.X : B.Y, vB = xm ? B.Y : B.X;
    r.uA = uA;
    r.vA = vA;
    r.du = uB - uA;
    r.dv = vB - vA;
    r.umin = min(uA, uB);
    r.umax = max(uA, uB);
    r.vmin = min(vA, vB);
    r.vmax = max(vA, vB);
    // depth pre-scaled to d24 units: a power-of-two scale is exact and
    // commutes with every rounding of depth_d24 (which floors the result)
    r.zA = fmul(A.z, 16777216.0f);
    r.dz = fmul(fsub(B.z, A.z), 16777216.0f);
    r.hc = centre_halfwidth(cam, width_m, A.w, B.w);
    const int64_t dX = (int64_t)B.X - A.X, dY = (int64_t)B.Y - A.Y;
    r.fden = __ll2float_rn(dX * dX + dY * dY);
    r.rden = __frcp_rn(r.fden);
    r.slope = r.du == 0 ? 0.0f : (float)r.dv / (float)r.du;
    const bool shrt = abs(r.du) < (1 << 14) && abs(r.dv) < (1 << 14);
    r.flags = (xm ? 1 : 0) | (shrt ? 2 : 0);
}

// Pixel ranges a segment's conservative boxes can meet: major pixels
// [ilo, ihi] and minor pixels [mlo, mhi] (pixel m's box spans [256 m,
// 256 m + 256]), clipped to a dim_u x dim_v frame; false if empty.
__device__ __forceinline__ bool segment_pixel_box(const SegRec &r, int dim_u, int dim_v, int &ilo, int &ihi, int &mlo,
                                                  int &mhi) {
    ilo = max(((r.umin + 255) >> 8) - 1, 0);
    ihi = min(r.umax >> 8, dim_u - 1);
    mlo = max((r.vmin - 1) >> 8, 0);
    mhi = min(r.vmax >> 8, dim_v - 1);
    return ilo <= ihi && r.vmax >= 0 && r.vmin <= 256 * dim_v;
}

// Correctly rounded binary32 quotient a / b given y = RN(1 / b): Markstein's
// FMA division (P. Markstein, IBM J. Res. Dev. 34(1), 1990).  q0 = RN(a y)
// lies within 1.5 ulp of a / b; one correction q1 = RN(q0 + RN(a - b q0) y)
// brings it within one ulp; Markstein's theorem (y within half an ulp of
// 1 / b, q1 within one ulp of a / b, radix 2) makes the residual a - b q1
// exact and q2 = RN(q1 + (a - b q1) y) equal to RN(a / b).  Valid while the
// quotient and the residuals stay normal or zero: here a is an integer-valued
// depth numerator (|a| < 2^63) and b = |B - A|^2 >= 1, so they do.
__device__ __forceinline__ float quotient_rn(float a, float b, float y) {
    const float q0 = __fmul_rn(a, y);
    const float q1 = __fmaf_rn(__fmaf_rn(-q0, b, a), y, q0);
    return __fmaf_rn(__fmaf_rn(-q1, b, a), y, q1);
}

// 24-bit depth of a candidate at depth parameter t (Sec. 3.1.2): z = clamp(zA
// + dz t, 0, 1), d24 = min(floor(z 2^24), 2^24 - 1).  zA and dz carry the 2^24
// scale, so z 2^24 is computed directly and d24 equals the unscaled
// formula's bit for bit.  t = clamp(fn / |B - A|^2, 0, 1) comes from
// quotient_rn (0 for a point segment).
__device__ __forceinline__ uint32_t depth_d24(const SegRec &q, float t) {
    const float zs = fclamp(fadd(q.zA, fmul(q.dz, t)), 0.0f, 16777216.0f);
    const uint32_t d24 = (uint32_t)floorf(zs);
    return d24 > 16777215u ? 16777215u : d24;
}

// Low 40 bits of a compressed key at projection parameter t.
__device__ __forceinline__ uint64_t compressed_payload(const SegRec &q, float t) {
    const float w = fdiv(fadd(__uint2float_rn(q.id_lo), t), __uint2float_rn(q.id_hi));
    const uint32_t cw = quantize(w, 63.0f, 63u);
    const uint32_t ca = quantize(fadd(q.aoA, fmul(q.dao, t)), 62.0f, 62u);
    return ((uint64_t)q.cgb_hi << 12) | (uint64_t)((cw << 6) | ca);
}

// Candidate pixels of one work item: the minor-axis pixels of major-axis
// pixel i whose conservative box can meet the segment.  The exact
// predicate (bounding boxes overlap and the box's corners are not all
// strictly on one side of the line) is evaluated in incremental form: the
// corner cross products are e0 + h (sy dU - sx dV) for sx, sy = +-1, with e0 =
// dU (cv - vA) - dV (cu - uA) the cross product at the box centre (the x/y one
// up to sign), so "min <= 0 <= max" is |e0| <= h (|dU| + |dV|); e0 and the
// depth numerator num = (cu - uA) dU + (cv - vA) dV change by constants from
// one pixel to the next along the minor axis.  For short segments (|dU|,
// |dV| < 2^14) every quantity fits in 32 bits; long ones use 64 bits.
//
// The minor range is clipped to [mclip_lo, mclip_hi] (the frame, or one
// screen tile of the binned rasterizer).  The incremental terms are exact
// integers, so a pixel's key does not depend on where its range starts.
// Each covered (pixel, layer) goes to sink(index, key, centre_covered),
// index = sink.index(px, py) advanced per minor step by
// sink.step(x_major, minor coordinate odd).
template <typename I, bool kCgb, typename Sink>
__device__ __forceinline__ void raster_item(const SegRec &q_shared, int i, int mclip_lo, int mclip_hi,
                                            const Sink &sink, uint32_t &n_cons, uint32_t &n_cen) {
    const SegRec q = q_shared;
    const bool xm = q.flags & 1;
    const int32_t ua = max(256 * i, q.umin), ub = min(256 * i + 256, q.umax);
    const float va = (float)(ua - q.uA) * q.slope, vb = (float)(ub - q.uA) * q.slope;
    const float flo = floorf(fminf(va, vb)), fhi = ceilf(fmaxf(va, vb));
    // float error of the minor range is below |dV| 2^-21 + 1 unit; with
    // |vA| <= 2^28 (guard band) and |slope| <= 1 every term fits 32 bits
    const int32_t slack = 8 + (abs(q.dv) >> 20);
    const int32_t vlo = q.vA + (int32_t)flo - slack;
    const int32_t vhi = q.vA + (int32_t)fhi + slack;
    // rows whose conservative box can meet the line, and whose box overlaps
    // the segment's minor extent: vmin <= 256 m + 256 and vmax >= 256 m
    const int mlo = max(max(((vlo + 255) >> 8) - 1, (q.vmin - 1) >> 8), mclip_lo);
    const int mhi = min(min(vhi >> 8, q.vmax >> 8), mclip_hi);
    if (mlo > mhi) return;
    const int32_t cu = 256 * i + 128;
    const I ru = (I)(cu - q.uA), rv = (I)(256 * mlo + 128 - q.vA);
    const I du = q.du, dv = q.dv;
    I e0 = du * rv - dv * ru;
    I num = ru * du + rv * dv;
    const I de = du * 256, dn = dv * 256;
    const I span = (I)abs(q.du) + (I)abs(q.dv);
    const I k_cons = span * 128, k_cen = span * (I)q.hc;
    // minor pixels m whose centre box (half-width hc) overlaps the segment's
    // bounding box: vmin <= 256 m + 128 + hc and vmax >= 256 m + 128 - hc,
    // i.e. cm_lo <= m <= cm_hi (an empty range when the major extent misses)
    const bool ucen = (q.umin <= cu + q.hc) && (q.umax >= cu - q.hc);
    const int cm_lo = ucen ? (q.vmin - 128 - q.hc + 255) >> 8 : 1;
    const int cm_hi = ucen ? (q.vmax - 128 + q.hc) >> 8 : 0;
    const uint64_t id = ((uint64_t)q.id_hi << 32) | q.id_lo;
    const bool degenerate = (q.du == 0 && q.dv == 0);
    typedef typename std::make_unsigned<I>::type U;
    // the sink's index of pixel (i, mlo) in the major / minor frame, and its
    // step to the next minor pixel from an even or an odd minor coordinate
    uint32_t at = xm ? sink.index(i, mlo) : sink.index(mlo, i);
    const uint32_t step_even = sink.step(xm, false), step_odd = sink.step(xm, true);
    for (int m = mlo; m <= mhi; at += (m & 1) ? step_odd : step_even, ++m, e0 += de, num += dn) {
        // conservative line test |e0| <= k_cons (the overlaps hold by the row range)
        if ((U)(e0 + k_cons) > (U)(2 * k_cons)) continue;
        const bool cen = m >= cm_lo && m <= cm_hi && (U)(e0 + k_cen) <= (U)(2 * k_cen);
        float t = 0.0f;
        if (!degenerate) {
            const float fn = sizeof(I) == 4 ? __int2float_rn((int32_t)num) : __ll2float_rn((int64_t)num);
            t = fclamp(quotient_rn(fn, q.fden, q.rden), 0.0f, 1.0f);
        }
        const uint32_t d24 = depth_d24(q, t);
        const uint64_t key = ((uint64_t)d24 << 40) | (kCgb ? compressed_payload(q, t) : id);
        n_cons += 1;
        n_cen += cen;
        sink(at, key, cen);
    }
}

// Runs fn(q, i) for every work item of a warp's set-up segments (lane l
// holds segment r with nmaj items, major pixels r.ilo ..): the items are
// dealt to the lanes 32 at a time through a prefix sum over the lanes'
// counts and a binary search in it, so long and short segments share the
// warp evenly.  Stores the segments in rec (the warp's 32 shared records).
// Warp-wide.
template <typename F>
__device__ __forceinline__ void for_each_item(SegRec *rec, SegRec &r, int nmaj, const F &fn) {
    const int lane = threadIdx.x & 31;
    int incl = nmaj;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += y;
    }
    r.start = incl - nmaj;
    rec[lane] = r;
    __syncwarp();
    const int items = __shfl_sync(kFull, incl, 31);
    for (int base = 0; base < items; base += 32) {
        const int item = base + lane;
        int src = 0;
#pragma unroll
        for (int step = 16; step > 0; step >>= 1) {
            const int v = __shfl_sync(kFull, incl, src + step - 1);
            if (v <= item) src += step;
        }
        if (item >= items) continue;
        const SegRec &q = rec[src];
        fn(q, q.ilo + (item - q.start));
    }
    __syncwarp();
}

// Sink of the direct rasterizer: 64-bit atomicMin into the two key layers,
// row-major [H][W] or (kBlocked) in 2 x 2 blocks over Wb block columns (the
// index of key_index); with kPrecheck the key is read first and atomics that
// cannot lower it are skipped.
template <bool kPrecheck, bool kBlocked>
struct GlobalKeys {
    uint64_t *vis_c;
    uint64_t *vis_a;
    uint32_t W, Wb;
    __device__ __forceinline__ uint32_t index(int px, int py) const {
        if (!kBlocked) return (uint32_t)py * W + (uint32_t)px;   // < 2^28 pixels
        return ((((uint32_t)py >> 1) * Wb + ((uint32_t)px >> 1)) << 2) | (((uint32_t)py & 1u) << 1) |
               ((uint32_t)px & 1u);
    }
    // x-major items walk down a column, y-major ones along a row; in 2 x 2
    // blocks an even coordinate steps within its block, an odd one to the next
    __device__ __forceinline__ uint32_t step(bool x_major, bool odd) const {
        if (!kBlocked) return x_major ? W : 1u;
        return x_major ? (odd ? 4u * Wb - 2u : 2u) : (odd ? 3u : 1u);
    }
    __device__ __forceinline__ void operator()(uint32_t p, uint64_t key, bool cen) const {
        unsigned long long *a = reinterpret_cast<unsigned long long *>(vis_a + p);
        unsigned long long *c = reinterpret_cast<unsigned long long *>(vis_c + p);
        if (!kPrecheck || key < __ldcg(a)) atomicMin(a, (unsigned long long)key);
        if (cen && (!kPrecheck || key < __ldcg(c))) atomicMin(c, (unsigned long long)key);
    }
};

}  // namespace hm
