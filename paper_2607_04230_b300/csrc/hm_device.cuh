// hm_device.cuh -- device-side data layout and the FP32 "decision layer" of
// the deferred hair rasterizer (arXiv 2607.04230).
//
// Every quantity that decides an integer (covered pixels, packed keys, LOD
// counts, filter masks) is computed here with explicit round-to-nearest
// intrinsics (__fadd_rn, __fmul_rn, __fdiv_rn, __fsqrt_rn, ...), which the
// compiler never contracts into FMA or reorders, so the results are the same
// IEEE binary32 values on every launch.  The continuous part of the resolve
// (shading, filter weights) lives in hm_resolve.cu and may use FMA.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/hm.h"

namespace hm {

constexpr uint64_t kEmptyKey = ~0ull;
constexpr uint64_t kPayloadMask = 0xFFFFFFFFFFull;
constexpr uint64_t kStrandMask = 0x1FFFFFFFFull;   // 33 bits
constexpr float kGuard = 1048576.0f;               // 2^20 px guard band
// The rasterizers' work list: batch b of a groom holds its drawn control
// points kBatchStride b .. kBatchStride b + 31 (bundle order, then strand,
// then index along the strand), one per lane of a warp; lane l's segment
// joins its point to lane l + 1's.  Consecutive batches share one point, so
// every segment lies in exactly one batch.
constexpr int kBatchLanes = 32;
constexpr int kBatchStride = kBatchLanes - 1;

// Per-groom device counters (one block of words per groom): work-list
// batches, the rasterizer's ticket, drawn segments, drawn control points.
enum CounterWord : int { kCtrBatches = 0, kCtrTicket = 1, kCtrSegs = 2, kCtrCps = 3, kCtrWords = 4 };

// Programmatic dependent launch: a kernel launched with programmatic stream
// serialization after `pdl_launch_dependents` has run in every CTA of the
// kernel before it may start while that kernel still runs; `pdl_wait` blocks
// until the preceding kernel has completed and its memory is visible (at
// once when there is no programmatic dependency).
__device__ __forceinline__ void pdl_launch_dependents() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Device status bits (read by hm_get_device_status).
enum StatusBit : uint32_t { kStatusBadKey = 1u, kStatusBadBatch = 2u, kStatusBinOverflow = 4u };

// One groom as the kernels see it.  Arrays are device memory owned by the
// groom handle.
struct GroomDev {
    const float4 *lv;        // [L][V] layer vertices, xyz (w unused)
    const int4 *faces;       // [F + 1] (i0, i1, i2, first strand); faces[F].w = S
    const uint32_t *sface;   // [S] bundle of each strand
    const float2 *bary;      // [S] (b1, b2)
    const float4 *albedo;    // [S] rgb
    const float *delta;      // [F] LOD offset of Eq. 1
    uint4 *lod;              // [F] (N_LOD, C, first drawn segment, first drawn control point)
    uint32_t *batch_map;     // [max_batches] bundle holding the first control point of each batch
    uint32_t *counters;      // [kCtrWords]
    int32_t L, V, F, cmax;
    int64_t S;
    uint64_t base;           // global id of strand 0 in this call
    float width_m, roughness, tilt, lod_lambda;
    int32_t lod_enabled;
    int32_t has_ao;          // layer vertices carry baked ambient occlusion in w
    const float2 *uv;        // [V] scalp texture coordinates, or null (compressed payload)
    uint32_t max_batches;    // work-list batches at full detail (batch_map capacity)
    // [drawn segments][2] control points j and j+1 of every drawn segment,
    // (p_j.xyz, p_j+1.x), (p_j+1.yz, 0, 0), indexed by drawn segment
    // (lod[f].z + strand-in-bundle (C - 1) + j).  The rasterizer writes them
    // when non-null; key decoding reads them instead of regenerating the
    // strand when non-null (the host passes them only while they match the
    // groom's LOD state and layer vertices).
    float4 *segpts;
};

struct CallTable {
    int32_t n;
    int32_t pad_[3];
    GroomDev g[HM_MAX_GROOMS_PER_CALL];
};

struct CamDev {
    float m[16];
    float cam_pos[3];
    float near_m, far_m, tan_half;
    int32_t W, H;
    int32_t layout;    // key layout: HM_KEYS_ROW_MAJOR or HM_KEYS_BLOCK_2X2
    int32_t Wb;        // block columns of the 2 x 2 layout, ceil(W / 2)
};

// Index of pixel (x, y)'s key in one of the camera's key layers: row-major,
// or 2 x 2 blocks of four keys (one 32-byte sector) row-major over Wb block
// columns.  x < W, y < H: below hm_vis_buffer_keys(cam) < 2^30.
__device__ __forceinline__ uint32_t key_index(const CamDev &c, int x, int y) {
    if (c.layout == HM_KEYS_ROW_MAJOR) return (uint32_t)y * (uint32_t)c.W + (uint32_t)x;
    return ((((uint32_t)y >> 1) * (uint32_t)c.Wb + ((uint32_t)x >> 1)) << 2) | (((uint32_t)y & 1u) << 1) |
           ((uint32_t)x & 1u);
}

// The views of one rasterizer launch: the strands are assembled once and
// projected into each view's pair of key layers (all views share W, H).
struct ViewSet {
    int32_t n;
    int32_t pad_[3];
    CamDev cam[HM_MAX_VIEWS];
    uint64_t *vis_c[HM_MAX_VIEWS];
    uint64_t *vis_a[HM_MAX_VIEWS];
};

// ---------------------------------------------------------------------------
// binary32 helpers with a fixed evaluation order
// ---------------------------------------------------------------------------
__device__ __forceinline__ float fadd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float fsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float fmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float fdiv(float a, float b) { return __fdiv_rn(a, b); }
__device__ __forceinline__ float fclamp(float v, float lo, float hi) {
    return v < lo ? lo : (v > hi ? hi : v);
}

__device__ __forceinline__ float3 v3sub(float3 a, float3 b) {
    return make_float3(fsub(a.x, b.x), fsub(a.y, b.y), fsub(a.z, b.z));
}
// ((x x + y y) + z z)
__device__ __forceinline__ float v3len2(float3 v) {
    return fadd(fadd(fmul(v.x, v.x), fmul(v.y, v.y)), fmul(v.z, v.z));
}
// v / sqrt(|v|^2), zero for a zero vector
__device__ __forceinline__ float3 v3unit(float3 v) {
    float n2 = v3len2(v);
    if (n2 == 0.0f) return make_float3(0.0f, 0.0f, 0.0f);
    float n = __fsqrt_rn(n2);
    return make_float3(fdiv(v.x, n), fdiv(v.y, n), fdiv(v.z, n));
}
// Finite-difference tangent of point i of an n-point polyline (Sec. 3.1.1):
// forward at the root, backward at the tip, central elsewhere.
__device__ __forceinline__ float3 fd_tangent(int i, int n, float3 prev, float3 cur, float3 next) {
    if (i == 0) return v3unit(v3sub(next, cur));
    if (i == n - 1) return v3unit(v3sub(cur, prev));
    return v3unit(v3sub(next, prev));
}

// ---------------------------------------------------------------------------
// strand generation from the hair mesh (Sec. 2 Background; Sec. 3.1.1)
// ---------------------------------------------------------------------------
struct Root {
    int32_t i0, i1, i2;
    float b0, b1, b2;
};

__device__ __forceinline__ Root make_root(const GroomDev &g, int64_t s, uint32_t f) {
    int4 t = __ldg(&g.faces[f]);
    float2 b = __ldg(&g.bary[s]);
    Root r;
    r.i0 = t.x; r.i1 = t.y; r.i2 = t.z;
    r.b1 = b.x; r.b2 = b.y;
    r.b0 = fsub(fsub(1.0f, b.x), b.y);
    return r;
}

// Layer point k: the root's barycentric coordinates on layer k's triangle,
// ((b0 V0 + b1 V1) + b2 V2).
__device__ __forceinline__ float3 layer_pt(const GroomDev &g, const Root &r, int k) {
    const float4 *row = g.lv + (int64_t)k * g.V;
    float4 a = __ldg(&row[r.i0]);
    float4 b = __ldg(&row[r.i1]);
    float4 c = __ldg(&row[r.i2]);
    return make_float3(fadd(fadd(fmul(r.b0, a.x), fmul(r.b1, b.x)), fmul(r.b2, c.x)),
                       fadd(fadd(fmul(r.b0, a.y), fmul(r.b1, b.y)), fmul(r.b2, c.y)),
                       fadd(fadd(fmul(r.b0, a.z), fmul(r.b1, b.z)), fmul(r.b2, c.z)));
}

// Control point j of a C-point strand: cubic Hermite through the layer
// points with finite-difference tangents scaled by the interval's chord
// length; interval k = min(j (L-1) / (C-1), L-2), local parameter
// s = (j (L-1) - k (C-1)) / (C-1).  Only the layer points the interval needs
// are evaluated.
__device__ __forceinline__ float3 control_pt(const GroomDev &g, const Root &r, int C, int j) {
    const int L = g.L;
    int x = j * (L - 1);
    int k = x / (C - 1);
    if (k > L - 2) k = L - 2;
    float s = fdiv(__int2float_rn(x - k * (C - 1)), __int2float_rn(C - 1));
    float3 P0 = layer_pt(g, r, k);
    float3 P1 = layer_pt(g, r, k + 1);
    float3 Pm = (k > 0) ? layer_pt(g, r, k - 1) : P0;
    float3 P2 = (k + 2 <= L - 1) ? layer_pt(g, r, k + 2) : P1;
    float3 t0 = fd_tangent(k, L, Pm, P0, P1);
    float3 t1 = fd_tangent(k + 1, L, P0, P1, P2);
    float ell = __fsqrt_rn(v3len2(v3sub(P1, P0)));
    float3 m0 = make_float3(fmul(t0.x, ell), fmul(t0.y, ell), fmul(t0.z, ell));
    float3 m1 = make_float3(fmul(t1.x, ell), fmul(t1.y, ell), fmul(t1.z, ell));
    float s2 = fmul(s, s);
    float s3 = fmul(s2, s);
    float h00 = fadd(fsub(fmul(2.0f, s3), fmul(3.0f, s2)), 1.0f);
    float h10 = fadd(fsub(s3, fmul(2.0f, s2)), s);
    float h01 = fsub(fmul(3.0f, s2), fmul(2.0f, s3));
    float h11 = fsub(s3, s2);
    return make_float3(
        fadd(fadd(fadd(fmul(h00, P0.x), fmul(h10, m0.x)), fmul(h01, P1.x)), fmul(h11, m1.x)),
        fadd(fadd(fadd(fmul(h00, P0.y), fmul(h10, m0.y)), fmul(h01, P1.y)), fmul(h11, m1.y)),
        fadd(fadd(fadd(fmul(h00, P0.z), fmul(h10, m0.z)), fmul(h01, P1.z)), fmul(h11, m1.z)));
}

// Record of drawn segment `seg`: its two control points (bit-identical to
// control_pts<2>; the decode rebuilds X and T from the same values).
__device__ __forceinline__ void store_segment_points(float4 *segpts, uint32_t seg, const float3 (&cp)[2]) {
    float4 *p = segpts + 2 * (size_t)seg;
    p[0] = make_float4(cp[0].x, cp[0].y, cp[0].z, cp[1].x);
    p[1] = make_float4(cp[1].y, cp[1].z, 0.0f, 0.0f);
}

// Control points j0, j0+1, ..., j0+N-1 (each clamped to [0, C-1]); the
// layer points, tangents and chord of an interval are evaluated once and
// reused by consecutive control points in the same interval.  Each result is
// bit-identical to control_pt().
template <int N>
__device__ __forceinline__ void control_pts(const GroomDev &g, const Root &r, int C, int j0, float3 (&out)[N]) {
    const int L = g.L;
    int kcur = -1;
    float3 P0 = make_float3(0.f, 0.f, 0.f), P1 = P0, m0 = P0, m1 = P0, Pm = P0, P2 = P0, t0 = P0, t1 = P0;
#pragma unroll
    for (int c = 0; c < N; ++c) {
        int j = j0 + c;
        j = j < 0 ? 0 : (j > C - 1 ? C - 1 : j);
        const int x = j * (L - 1);
        int k = x / (C - 1);
        if (k > L - 2) k = L - 2;
        if (k != kcur) {
            if (kcur >= 0 && k == kcur + 1) {
                // next interval: its first layer point, the one before it and
                // its first tangent are the previous interval's (the same
                // values from the same operations)
                Pm = P0;
                P0 = P1;
                P1 = P2;
                t0 = t1;
            } else {
                P0 = layer_pt(g, r, k);
                P1 = layer_pt(g, r, k + 1);
                Pm = (k > 0) ? layer_pt(g, r, k - 1) : P0;
                t0 = fd_tangent(k, L, Pm, P0, P1);
            }
            P2 = (k + 2 <= L - 1) ? layer_pt(g, r, k + 2) : P1;
            t1 = fd_tangent(k + 1, L, P0, P1, P2);
            const float ell = __fsqrt_rn(v3len2(v3sub(P1, P0)));
            m0 = make_float3(fmul(t0.x, ell), fmul(t0.y, ell), fmul(t0.z, ell));
            m1 = make_float3(fmul(t1.x, ell), fmul(t1.y, ell), fmul(t1.z, ell));
            kcur = k;
        }
        const float s = fdiv(__int2float_rn(x - k * (C - 1)), __int2float_rn(C - 1));
        const float s2 = fmul(s, s);
        const float s3 = fmul(s2, s);
        const float h00 = fadd(fsub(fmul(2.0f, s3), fmul(3.0f, s2)), 1.0f);
        const float h10 = fadd(fsub(s3, fmul(2.0f, s2)), s);
        const float h01 = fsub(fmul(3.0f, s2), fmul(2.0f, s3));
        const float h11 = fsub(s3, s2);
        out[c] = make_float3(
            fadd(fadd(fadd(fmul(h00, P0.x), fmul(h10, m0.x)), fmul(h01, P1.x)), fmul(h11, m1.x)),
            fadd(fadd(fadd(fmul(h00, P0.y), fmul(h10, m0.y)), fmul(h01, P1.y)), fmul(h11, m1.y)),
            fadd(fadd(fadd(fmul(h00, P0.z), fmul(h10, m0.z)), fmul(h01, P1.z)), fmul(h11, m1.z)));
    }
}

// ---------------------------------------------------------------------------
// projection, 16.8 snap, depth (Sec. 3.1.2)
// ---------------------------------------------------------------------------
__device__ __forceinline__ float clip_row(const CamDev &c, int r, float3 p) {
    const float *m = c.m + 4 * r;
    return fadd(fadd(fadd(fmul(m[0], p.x), fmul(m[1], p.y)), fmul(m[2], p.z)), m[3]);
}

struct Proj {
    int32_t X, Y;      // 1/256 px
    float w, z;        // view depth (m), linear depth in [0, 1] when inside
    float xs, ys;      // unsnapped pixel position
    bool valid;        // w >= near
};

__device__ __forceinline__ Proj project(const CamDev &c, float3 p) {
    Proj r;
    float c0 = clip_row(c, 0, p);
    float c1 = clip_row(c, 1, p);
    float w = clip_row(c, 3, p);
    r.w = w;
    r.valid = (w >= c.near_m);
    r.z = fdiv(fsub(w, c.near_m), fsub(c.far_m, c.near_m));
    r.X = r.Y = 0;
    r.xs = r.ys = 0.0f;
    if (!r.valid) return r;
    float xs = fmul(fmul(fadd(fdiv(c0, w), 1.0f), 0.5f), __int2float_rn(c.W));
    float ys = fmul(fmul(fsub(1.0f, fdiv(c1, w)), 0.5f), __int2float_rn(c.H));
    xs = fclamp(xs, -kGuard, kGuard);
    ys = fclamp(ys, -kGuard, kGuard);
    r.xs = xs;
    r.ys = ys;
    r.X = __float2int_rn(fmul(xs, 256.0f));
    r.Y = __float2int_rn(fmul(ys, 256.0f));
    return r;
}

__device__ __forceinline__ float focal_px(const CamDev &c) {
    return fdiv(fmul(0.5f, __int2float_rn(c.H)), c.tan_half);
}

// Centre-sample half-width in 1/256 px: the projected strand half-width,
// rounded half-even, clamped to [1, 128].
__device__ __forceinline__ int32_t centre_halfwidth(const CamDev &c, float width_m, float wA, float wB) {
    float wm = fmul(fadd(wA, wB), 0.5f);
    float r = fdiv(fmul(fmul(128.0f, width_m), focal_px(c)), wm);
    float q = rintf(r);
    q = q < 1.0f ? 1.0f : (q > 128.0f ? 128.0f : q);
    return (int32_t)q;
}

// Exact separating-axis test of segment AB against the closed box of
// half-width h around (cx, cy): bounding boxes overlap and the box corners
// are not all strictly on one side of AB.
__device__ __forceinline__ bool seg_covers(int32_t XA, int32_t YA, int32_t XB, int32_t YB,
                                           int64_t cx, int64_t cy, int64_t h) {
    int64_t xlo = min(XA, XB), xhi = max(XA, XB);
    int64_t ylo = min(YA, YB), yhi = max(YA, YB);
    if (xhi < cx - h || xlo > cx + h || yhi < cy - h || ylo > cy + h) return false;
    int64_t dX = (int64_t)XB - XA, dY = (int64_t)YB - YA;
    int64_t ax = (cx - h) - XA, bx = (cx + h) - XA;
    int64_t ay = (cy - h) - YA, by = (cy + h) - YA;
    int64_t e0 = dX * ay - dY * ax;
    int64_t e1 = dX * ay - dY * bx;
    int64_t e2 = dX * by - dY * ax;
    int64_t e3 = dX * by - dY * bx;
    int64_t emin = min(min(e0, e1), min(e2, e3));
    int64_t emax = max(max(e0, e1), max(e2, e3));
    return emin <= 0 && emax >= 0;
}

// Pixel-centre projection parameter t = clamp(float(num) / float(den), 0, 1).
__device__ __forceinline__ float seg_t(int32_t XA, int32_t YA, int32_t XB, int32_t YB,
                                       int64_t cx, int64_t cy) {
    int64_t dX = (int64_t)XB - XA, dY = (int64_t)YB - YA;
    int64_t num = (cx - XA) * dX + (cy - YA) * dY;
    int64_t den = dX * dX + dY * dY;
    if (den == 0) return 0.0f;
    return fclamp(fdiv(__ll2float_rn(num), __ll2float_rn(den)), 0.0f, 1.0f);
}

// 24-bit depth: z = zA + (zB - zA) t, clamped, floor(z 2^24), max 2^24 - 1.
__device__ __forceinline__ uint32_t depth24(float zA, float zB, float t) {
    float z = fclamp(fadd(zA, fmul(fsub(zB, zA), t)), 0.0f, 1.0f);
    uint32_t d = (uint32_t)floorf(fmul(z, 16777216.0f));
    return d > 16777215u ? 16777215u : d;
}

__device__ __forceinline__ bool key_empty(uint64_t k) { return (k & kPayloadMask) == kPayloadMask; }

// ---------------------------------------------------------------------------
// resolve-side decode and masks (Sec. 3.1.2 deferred shading; Sec. 3.3)
// ---------------------------------------------------------------------------

// Screen tangent J T / |J T| at X (pixels, y down).  Degenerate -- the strand
// within about 0.6 degrees of the view ray, |J T| w < 0.01 focal -- selects
// the isotropic filter mode.
__device__ __forceinline__ bool screen_tangent(const CamDev &c, float3 X, float3 T, float &tsx, float &tsy) {
    const float *m = c.m;
    float c0 = clip_row(c, 0, X);
    float c1 = clip_row(c, 1, X);
    float w = clip_row(c, 3, X);
    float a0 = fadd(fadd(fmul(m[0], T.x), fmul(m[1], T.y)), fmul(m[2], T.z));
    float a1 = fadd(fadd(fmul(m[4], T.x), fmul(m[5], T.y)), fmul(m[6], T.z));
    float a3 = fadd(fadd(fmul(m[12], T.x), fmul(m[13], T.y)), fmul(m[14], T.z));
    float w2 = fmul(w, w);
    float jx = fmul(fdiv(fsub(fmul(a0, w), fmul(c0, a3)), w2), fmul(0.5f, __int2float_rn(c.W)));
    float jy = -fmul(fdiv(fsub(fmul(a1, w), fmul(c1, a3)), w2), fmul(0.5f, __int2float_rn(c.H)));
    float n = __fsqrt_rn(fadd(fmul(jx, jx), fmul(jy, jy)));
    if (!(fmul(n, w) >= fmul(0.01f, focal_px(c)))) {
        tsx = 0.0f;
        tsy = 0.0f;
        return true;
    }
    tsx = fdiv(jx, n);
    tsy = fdiv(jy, n);
    return false;
}

// Window offset (dx, dy) inside the alpha strip of half-width hw
// (hw2 = hw * hw); the strip of a degenerate tangent is the pixel itself.
__device__ __forceinline__ bool in_strip(bool iso, float tsx, float tsy, int dx, int dy, float hw2,
                                         float &dpar, float &perp2) {
    float fx = __int2float_rn(dx), fy = __int2float_rn(dy);
    if (iso) {
        dpar = 0.0f;
        perp2 = 0.0f;
        return dx == 0 && dy == 0;
    }
    dpar = fadd(fmul(fx, tsx), fmul(fy, tsy));
    float ex = fsub(fx, fmul(dpar, tsx));
    float ey = fsub(fy, fmul(dpar, tsy));
    perp2 = fadd(fmul(ex, ex), fmul(ey, ey));
    return perp2 <= hw2;
}

// Index of the groom owning global strand id sg (ids are numbered groom by
// groom); bases[] holds the n + 1 prefix ids.  -1 if none.
__device__ __forceinline__ int find_groom(const uint64_t *bases, int n, uint64_t sg) {
    int lo = 0, hi = n;          // bases[lo] <= sg < bases[hi]
    if (sg >= bases[n]) return -1;
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (bases[mid] <= sg) lo = mid; else hi = mid;
    }
    return lo;
}

// Baked ambient occlusion of layer point k (w of the layer vertices), with
// the root's barycentric coordinates.
__device__ __forceinline__ float layer_ao(const GroomDev &g, const Root &r, int k) {
    const float4 *row = g.lv + (int64_t)k * g.V;
    return r.b0 * __ldg(&row[r.i0]).w + r.b1 * __ldg(&row[r.i1]).w + r.b2 * __ldg(&row[r.i2]).w;
}

// Ambient occlusion at control point j, interpolated along the strand like
// the position (same interval and local parameter, cubic Hermite) with
// finite-difference slopes of the scalar (one-sided at root and tip).
__device__ __forceinline__ float control_ao(const GroomDev &g, const Root &r, int C, int j) {
    const int L = g.L;
    const int x = j * (L - 1);
    int k = x / (C - 1);
    if (k > L - 2) k = L - 2;
    const float s = (float)(x - k * (C - 1)) / (float)(C - 1);
    const float a0 = layer_ao(g, r, k), a1 = layer_ao(g, r, k + 1);
    const float am = k > 0 ? layer_ao(g, r, k - 1) : a0;
    const float a2 = k + 2 <= L - 1 ? layer_ao(g, r, k + 2) : a1;
    const float m0 = k == 0 ? a1 - a0 : 0.5f * (a1 - am);
    const float m1 = k + 1 == L - 1 ? a1 - a0 : 0.5f * (a2 - a0);
    const float s2 = s * s, s3 = s2 * s;
    return (2.f * s3 - 3.f * s2 + 1.f) * a0 + (s3 - 2.f * s2 + s) * m0 + (3.f * s2 - 2.f * s3) * a1 + (s3 - s2) * m1;
}

// The geometry a key decodes to at pixel (px, py).
struct Decoded {
    float3 X, T;        // FP32 position and unit tangent at the pixel centre
    float t;            // pixel-centre projection parameter
    float tsx, tsy;     // unit screen tangent
    int64_t s;          // local strand index
    int gi;             // groom
    int j, C;           // segment, control points
    bool iso, ok;
};

// Standard multisample positions (1/256 px from the pixel centre, y down)
// for N = 1, 2, 4, 8 samples per pixel.
template <int N>
__device__ __forceinline__ void sample_offset(int k, int &ox, int &oy) {
    if (N == 1) { ox = 0; oy = 0; return; }
    if (N == 2) {
        const int t[2][2] = {{4, 4}, {-4, -4}};
        ox = 16 * t[k][0]; oy = 16 * t[k][1]; return;
    }
    if (N == 4) {
        const int t[4][2] = {{-2, -6}, {6, -2}, {-6, 2}, {2, 6}};
        ox = 16 * t[k][0]; oy = 16 * t[k][1]; return;
    }
    const int t[8][2] = {{1, -3}, {-1, 3}, {5, 1}, {-3, -5}, {-5, 5}, {-7, -1}, {3, 7}, {7, -7}};
    ox = 16 * t[k][0];
    oy = 16 * t[k][1];
}

// Control points j-1 .. j+2 regenerated from the hair mesh (decode without
// the rasterizer's records); kept out of line so the record path's register
// allocation does not carry it.
static __device__ __noinline__ void regenerate_points4(const GroomDev &g, int64_t s, uint32_t f, int C, int j,
                                                float3 (&cp)[4]) {
    control_pts<4>(g, make_root(g, s, f), C, j - 1, cp);
}

// Control points j-1 .. j+2 (clamped to the strand like control_pts) from
// the rasterizer's records of segments j-1, j, j+1 of drawn strand sl of
// bundle f.
__device__ __forceinline__ void recorded_points4(const GroomDev &g, uint32_t f, uint32_t sl, int C, int j,
                                                 float3 (&cp)[4]) {
    const float4 *rp = g.segpts + 2 * ((size_t)g.lod[f].z + (size_t)sl * (uint32_t)(C - 1) + (uint32_t)j);
    const float4 a0 = __ldg(rp), a1 = __ldg(rp + 1);
    cp[1] = make_float3(a0.x, a0.y, a0.z);
    cp[2] = make_float3(a0.w, a1.x, a1.y);
    if (j >= 1) {
        const float4 m0 = __ldg(rp - 2);
        cp[0] = make_float3(m0.x, m0.y, m0.z);
    } else {
        cp[0] = cp[1];
    }
    if (j + 2 <= C - 1) {
        const float4 q0 = __ldg(rp + 2), q1 = __ldg(rp + 3);
        cp[3] = make_float3(q0.w, q1.x, q1.y);
    } else {
        cp[3] = cp[2];
    }
}

struct Decoded;
__device__ __forceinline__ Decoded decode_key_at(const CallTable &tab, const uint64_t *bases, const CamDev &cam,
                                                 uint64_t key, int64_t sx, int64_t sy, uint32_t *status);

__device__ __forceinline__ Decoded decode_key(const CallTable &tab, const uint64_t *bases, const CamDev &cam,
                                              uint64_t key, int px, int py, uint32_t *status) {
    return decode_key_at(tab, bases, cam, key, 256 * (int64_t)px + 128, 256 * (int64_t)py + 128, status);
}

// Decode at an arbitrary sample point (sx, sy) in 1/256 px.
__device__ __forceinline__ Decoded decode_key_at(const CallTable &tab, const uint64_t *bases, const CamDev &cam,
                                                 uint64_t key, int64_t sx, int64_t sy, uint32_t *status) {
    Decoded d;
    d.ok = false;
    d.iso = true;
    d.tsx = d.tsy = 0.0f;
    d.X = d.T = make_float3(0.0f, 0.0f, 0.0f);
    d.t = 0.0f;
    d.s = 0;
    d.gi = 0;
    d.j = 0;
    d.C = 0;
    uint64_t sg = (key >> 7) & kStrandMask;
    int gi = find_groom(bases, tab.n, sg);
    if (gi < 0) { atomicOr(status, kStatusBadKey); return d; }
    const GroomDev &g = tab.g[gi];
    int64_t s = (int64_t)(sg - bases[gi]);
    int j = (int)(key & 127ull);
    uint32_t f = __ldg(&g.sface[s]);
    if (f >= (uint32_t)g.F) { atomicOr(status, kStatusBadKey); return d; }
    int C = (int)g.lod[f].y;
    if (j + 1 >= C) { atomicOr(status, kStatusBadKey); return d; }
    float3 cp[4];
    if (g.segpts) {
        const uint32_t sl = (uint32_t)(s - (int64_t)__ldg(&g.faces[f]).w);
        if (sl >= g.lod[f].x) { atomicOr(status, kStatusBadKey); return d; }   // strand not drawn at this LOD
        recorded_points4(g, f, sl, C, j, cp);
    } else {
        regenerate_points4(g, s, f, C, j, cp);
    }
    const float3 pm = cp[0], p0 = cp[1], p1 = cp[2], pp = cp[3];
    Proj a = project(cam, p0), b = project(cam, p1);
    float t = seg_t(a.X, a.Y, b.X, b.Y, sx, sy);
    d.X = make_float3(fadd(p0.x, fmul(fsub(p1.x, p0.x), t)), fadd(p0.y, fmul(fsub(p1.y, p0.y), t)),
                      fadd(p0.z, fmul(fsub(p1.z, p0.z), t)));
    float3 T0 = fd_tangent(j, C, pm, p0, p1);
    float3 T1 = fd_tangent(j + 1, C, p0, p1, pp);
    d.T = v3unit(make_float3(fadd(T0.x, fmul(fsub(T1.x, T0.x), t)), fadd(T0.y, fmul(fsub(T1.y, T0.y), t)),
                             fadd(T0.z, fmul(fsub(T1.z, T0.z), t))));
    d.iso = screen_tangent(cam, d.X, d.T, d.tsx, d.tsy);
    d.t = t;
    d.s = s;
    d.gi = gi;
    d.j = j;
    d.C = C;
    d.ok = true;
    return d;
}

// ---------------------------------------------------------------------------
// compressed G-buffer payload (Sec. 3.1.2: uvw styling coordinates, an
// octahedral tangent and 8/6-bit quantization beside the 24-bit depth)
//
// Low 40 bits of a compressed key: tangent code x (39..32) and y (31..24),
// the root's scalp coordinates u (23..18) and v (17..12), w = (j + t)/(C-1)
// along the strand (11..6), ambient occlusion 0..62 (5..0; 63 is never used,
// so no payload is all ones).  Every quantization is rint(x scale) clamped;
// the tangent is the segment's chord, octahedral-encoded (Cigolle et al.
// 2014, sign(0) = +1) once per segment; AO is the control points' AO
// interpolated linearly along the segment.  All of it in fixed binary32
// operation order, so the codes are reproducible bit for bit.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t quantize(float x, float scale, uint32_t hi) {
    const float q = rintf(fmul(x, scale));
    if (!(q >= 0.0f)) return 0u;
    if (q >= __uint2float_rn(hi)) return hi;
    return (uint32_t)q;
}

__device__ __forceinline__ float sgn1(float v) { return v >= 0.0f ? 1.0f : -1.0f; }

__device__ __forceinline__ uint32_t oct_encode(float3 T) {
    const float s = fadd(fadd(fabsf(T.x), fabsf(T.y)), fabsf(T.z));
    float ox = 0.0f, oy = 0.0f;
    if (s > 0.0f) {
        ox = fdiv(T.x, s);
        oy = fdiv(T.y, s);
    }
    if (T.z < 0.0f) {
        const float nx = fmul(fsub(1.0f, fabsf(oy)), sgn1(ox));
        const float ny = fmul(fsub(1.0f, fabsf(ox)), sgn1(oy));
        ox = nx;
        oy = ny;
    }
    const uint32_t cx = quantize(fadd(fmul(ox, 0.5f), 0.5f), 255.0f, 255u);
    const uint32_t cy = quantize(fadd(fmul(oy, 0.5f), 0.5f), 255.0f, 255u);
    return (cx << 8) | cy;
}

__device__ __forceinline__ float3 oct_decode(uint32_t code) {
    float ox = fsub(fmul(fdiv(__uint2float_rn(code >> 8), 255.0f), 2.0f), 1.0f);
    float oy = fsub(fmul(fdiv(__uint2float_rn(code & 255u), 255.0f), 2.0f), 1.0f);
    const float z = fsub(fsub(1.0f, fabsf(ox)), fabsf(oy));
    if (z < 0.0f) {
        const float nx = fmul(fsub(1.0f, fabsf(oy)), sgn1(ox));
        const float ny = fmul(fsub(1.0f, fabsf(ox)), sgn1(oy));
        ox = nx;
        oy = ny;
    }
    return v3unit(make_float3(ox, oy, z));
}

// AO of layer point k and of control point j: cubic Hermite over the layer
// values with finite-difference slopes (one-sided at root and tip), in the
// Hermite basis order of the positions.
__device__ __forceinline__ float layer_ao_exact(const GroomDev &g, const Root &r, int k) {
    if (!g.has_ao) return 1.0f;
    const float4 *row = g.lv + (int64_t)k * g.V;
    return fadd(fadd(fmul(r.b0, __ldg(&row[r.i0]).w), fmul(r.b1, __ldg(&row[r.i1]).w)),
                fmul(r.b2, __ldg(&row[r.i2]).w));
}

__device__ __forceinline__ float control_ao_exact(const GroomDev &g, const Root &r, int C, int j) {
    const int L = g.L;
    const int x = j * (L - 1);
    int k = x / (C - 1);
    if (k > L - 2) k = L - 2;
    const float t = fdiv(__int2float_rn(x - k * (C - 1)), __int2float_rn(C - 1));
    const float a0 = layer_ao_exact(g, r, k), a1 = layer_ao_exact(g, r, k + 1);
    const float am = k > 0 ? layer_ao_exact(g, r, k - 1) : a0;
    const float a2 = k + 2 <= L - 1 ? layer_ao_exact(g, r, k + 2) : a1;
    const float m0 = k == 0 ? fsub(a1, a0) : fmul(0.5f, fsub(a1, am));
    const float m1 = k + 1 == L - 1 ? fsub(a1, a0) : fmul(0.5f, fsub(a2, a0));
    const float t2 = fmul(t, t), t3 = fmul(t2, t);
    const float h00 = fadd(fsub(fmul(2.0f, t3), fmul(3.0f, t2)), 1.0f);
    const float h10 = fadd(fsub(t3, fmul(2.0f, t2)), t);
    const float h01 = fsub(fmul(3.0f, t2), fmul(2.0f, t3));
    const float h11 = fsub(t3, t2);
    return fadd(fadd(fadd(fmul(h00, a0), fmul(h10, m0)), fmul(h01, a1)), fmul(h11, m1));
}

// u (bits 11..6) and v (5..0) codes of the root's scalp coordinates.
__device__ __forceinline__ uint32_t root_uv_codes(const GroomDev &g, const Root &r) {
    if (!g.uv) return 0u;
    const float2 a = __ldg(&g.uv[r.i0]), b = __ldg(&g.uv[r.i1]), c = __ldg(&g.uv[r.i2]);
    const float u = fadd(fadd(fmul(r.b0, a.x), fmul(r.b1, b.x)), fmul(r.b2, c.x));
    const float v = fadd(fadd(fmul(r.b0, a.y), fmul(r.b1, b.y)), fmul(r.b2, c.y));
    return (quantize(u, 63.0f, 63u) << 6) | quantize(v, 63.0f, 63u);
}

__device__ __forceinline__ float3 cross3x(float3 a, float3 b) {
    return make_float3(fsub(fmul(a.y, b.z), fmul(a.z, b.y)), fsub(fmul(a.z, b.x), fmul(a.x, b.z)),
                       fsub(fmul(a.x, b.y), fmul(a.y, b.x)));
}

// Position on the ray through pixel position (xs, ys) at view depth w:
// (M0 - xn M3) X = xn M33 - M03, (M1 - yn M3) X = yn M33 - M13,
// M3 X = w - M33, by Cramer's rule.
__device__ __forceinline__ float3 unproject(const CamDev &c, float xs, float ys, float w) {
    const float *m = c.m;
    const float xn = fsub(fdiv(fmul(2.0f, xs), __int2float_rn(c.W)), 1.0f);
    const float yn = fsub(1.0f, fdiv(fmul(2.0f, ys), __int2float_rn(c.H)));
    const float3 ra = make_float3(fsub(m[0], fmul(xn, m[12])), fsub(m[1], fmul(xn, m[13])), fsub(m[2], fmul(xn, m[14])));
    const float3 rb = make_float3(fsub(m[4], fmul(yn, m[12])), fsub(m[5], fmul(yn, m[13])), fsub(m[6], fmul(yn, m[14])));
    const float3 rc = make_float3(m[12], m[13], m[14]);
    const float ka = fsub(fmul(xn, m[15]), m[3]);
    const float kb = fsub(fmul(yn, m[15]), m[7]);
    const float kc = fsub(w, m[15]);
    const float3 bc = cross3x(rb, rc), ca = cross3x(rc, ra), ab = cross3x(ra, rb);
    const float det = fadd(fadd(fmul(ra.x, bc.x), fmul(ra.y, bc.y)), fmul(ra.z, bc.z));
    return make_float3(fdiv(fadd(fadd(fmul(ka, bc.x), fmul(kb, ca.x)), fmul(kc, ab.x)), det),
                       fdiv(fadd(fadd(fmul(ka, bc.y), fmul(kb, ca.y)), fmul(kc, ab.y)), det),
                       fdiv(fadd(fadd(fmul(ka, bc.z), fmul(kb, ca.z)), fmul(kc, ab.z)), det));
}

// Decode of a compressed key at pixel (px, py): position at the middle of
// the depth bin on the pixel-centre ray, tangent from its code, screen
// tangent and isotropic flag as for the id payload.
struct DecodedC {
    float3 X, T;
    float tsx, tsy;
    uint32_t u, v, w, ao;    // payload codes
    bool iso;
};

__device__ __forceinline__ DecodedC decode_compressed(const CamDev &cam, uint64_t key, int px, int py) {
    DecodedC d;
    const float z = fmul(fadd(__uint2float_rn((uint32_t)(key >> 40)), 0.5f), 5.9604644775390625e-8f);
    const float w = fadd(cam.near_m, fmul(z, fsub(cam.far_m, cam.near_m)));
    d.X = unproject(cam, fadd(__int2float_rn(px), 0.5f), fadd(__int2float_rn(py), 0.5f), w);
    d.T = oct_decode((uint32_t)(key >> 24) & 0xFFFFu);
    d.u = (uint32_t)(key >> 18) & 63u;
    d.v = (uint32_t)(key >> 12) & 63u;
    d.w = (uint32_t)(key >> 6) & 63u;
    d.ao = (uint32_t)key & 63u;
    d.iso = screen_tangent(cam, d.X, d.T, d.tsx, d.tsy);
    return d;
}

}  // namespace hm
