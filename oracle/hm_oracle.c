/*
 * hm_oracle.c -- CPU oracle for deferred software rasterization of strand
 * hair generated from hair meshes (arXiv 2607.04230).
 *
 * TEST INFRASTRUCTURE ONLY.  The product path never loads this file: only
 * tests/, the smoke check and the bench's CPU-baseline leg use it.  It shares
 * no source with the CUDA library.
 *
 * This file is the oracle's "FP32 decision layer": every quantity that
 * decides an integer -- a covered pixel, a packed depth|ID key, an LOD count,
 * a filter mask or a hit count -- is computed in IEEE binary32 with one fixed
 * operation order and no contraction (built with -ffp-contract=off on x86-64
 * SSE scalar math, so every float operation rounds once).  Parentheses in the
 * code are the evaluation order.  The continuous colours and gradients are
 * computed in FP64 by value64.py from what this layer decides.
 *
 * Readings of the paper where it is silent are marked "Reading:".
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_EMPTY 0xFFFFFFFFFFFFFFFFull
#define ORC_PAYLOAD_MASK 0xFFFFFFFFFFull
#define ORC_STRAND_MASK 0x1FFFFFFFFull /* 33 bits */
#define ORC_GUARD 1048576.0f           /* 2^20 px guard band */

typedef struct { float x, y, z; } f3;

typedef struct {
    int32_t L, V, F, segs;         /* layers, verts per layer, bundles, full-detail segments */
    int64_t S;                     /* strands */
    const float *layer_verts;      /* [L][V][3] */
    const int32_t *faces;          /* [F][3] */
    const uint32_t *strand_face;   /* [S], ascending */
    const float *strand_bary;      /* [S][2] */
    const int32_t *lod_n;          /* [F] strands drawn per bundle */
    const int32_t *lod_c;          /* [F] control points per strand of the bundle */
    uint64_t strand_base;          /* global strand id of local strand 0 */
    float width_m;                 /* strand width */
    const float *vert_ao;          /* [L][V] baked ambient occlusion, or NULL (= 1) */
    const float *vert_uv;          /* [V][2] scalp texture coordinates, or NULL (= 0) */
} orc_groom;

typedef struct {
    float m[16];                   /* row-major view-projection, clip = M (x,y,z,1) */
    float near, far, tan_half_fovy;
    int32_t width, height;
} orc_camera;

/* ---------------------------------------------------------------------------
 * small vector helpers, fixed evaluation order
 * ------------------------------------------------------------------------- */
static f3 mk(float x, float y, float z) { f3 r; r.x = x; r.y = y; r.z = z; return r; }
static f3 sub3(f3 a, f3 b) { return mk(a.x - b.x, a.y - b.y, a.z - b.z); }
static float len2(f3 v) { return ((v.x * v.x) + (v.y * v.y)) + (v.z * v.z); }

/* normalize(v) = v / sqrt(|v|^2) componentwise, IEEE division and square
 * root.  Reading: a zero vector normalizes to zero (the paper's listing has
 * no guard). */
static f3 normalize3(f3 v) {
    float n2 = len2(v);
    if (n2 == 0.0f) return mk(0.0f, 0.0f, 0.0f);
    float n = sqrtf(n2);
    return mk(v.x / n, v.y / n, v.z / n);
}

/* Finite-difference tangent of point i of an n-point polyline: forward at
 * the root, backward at the tip, central elsewhere (Sec. 3.1.1; Code 1). */
static f3 calc_tangent(int i, int n, f3 prev, f3 cur, f3 next) {
    if (i == 0) return normalize3(sub3(next, cur));
    if (i == n - 1) return normalize3(sub3(cur, prev));
    return normalize3(sub3(next, prev));
}

/* ---------------------------------------------------------------------------
 * strand generation (Sec. 2 Background; Sec. 3.1.1)
 * ------------------------------------------------------------------------- */

/* Layer point k of strand s: the strand root's barycentric coordinates,
 * fixed along the strand, interpolate the bundle's layer-k triangle.
 * Reading (triangle prisms instead of quads): P_k = ((b0 V0 + b1 V1) + b2 V2)
 * with b0 = (1 - b1) - b2. */
static void strand_layer_points(const orc_groom *g, int64_t s, f3 *P) {
    uint32_t f = g->strand_face[s];
    int32_t i0 = g->faces[3 * (int64_t)f + 0];
    int32_t i1 = g->faces[3 * (int64_t)f + 1];
    int32_t i2 = g->faces[3 * (int64_t)f + 2];
    float b1 = g->strand_bary[2 * s + 0];
    float b2 = g->strand_bary[2 * s + 1];
    float b0 = (1.0f - b1) - b2;
    for (int k = 0; k < g->L; ++k) {
        const float *v0 = g->layer_verts + ((int64_t)k * g->V + i0) * 3;
        const float *v1 = g->layer_verts + ((int64_t)k * g->V + i1) * 3;
        const float *v2 = g->layer_verts + ((int64_t)k * g->V + i2) * 3;
        P[k] = mk(((b0 * v0[0]) + (b1 * v1[0])) + (b2 * v2[0]),
                  ((b0 * v0[1]) + (b1 * v1[1])) + (b2 * v2[1]),
                  ((b0 * v0[2]) + (b1 * v1[2])) + (b2 * v2[2]));
    }
}

/* Base-spline tangents at the layer points, by finite differences. */
static void layer_tangents(const f3 *P, int L, f3 *mh) {
    for (int k = 0; k < L; ++k) {
        f3 prev = (k > 0) ? P[k - 1] : P[k];
        f3 next = (k < L - 1) ? P[k + 1] : P[k];
        mh[k] = calc_tangent(k, L, prev, P[k], next);
    }
}

/* Control point j (0..C-1) of a C-point strand: cubic Hermite between the
 * layer points, control points uniform in the strand parameter w (Sec. 2,
 * Sec. 3.1.1).  Reading: tangents scaled by the chord length of the
 * interval; interval k = min(j (L-1) div (C-1), L-2), local parameter
 * s = (j (L-1) - k (C-1)) / (C-1). */
static f3 control_point(const f3 *P, const f3 *mh, int L, int C, int j) {
    int x = j * (L - 1);
    int k = x / (C - 1);
    if (k > L - 2) k = L - 2;
    float s = (float)(x - k * (C - 1)) / (float)(C - 1);
    float ell = sqrtf(len2(sub3(P[k + 1], P[k])));
    f3 m0 = mk(mh[k].x * ell, mh[k].y * ell, mh[k].z * ell);
    f3 m1 = mk(mh[k + 1].x * ell, mh[k + 1].y * ell, mh[k + 1].z * ell);
    float s2 = s * s;
    float s3 = s2 * s;
    float h00 = ((2.0f * s3) - (3.0f * s2)) + 1.0f;
    float h10 = (s3 - (2.0f * s2)) + s;
    float h01 = (3.0f * s2) - (2.0f * s3);
    float h11 = s3 - s2;
    f3 a = P[k], b = P[k + 1];
    return mk((((h00 * a.x) + (h10 * m0.x)) + (h01 * b.x)) + (h11 * m1.x),
              (((h00 * a.y) + (h10 * m0.y)) + (h01 * b.y)) + (h11 * m1.y),
              (((h00 * a.z) + (h10 * m0.z)) + (h01 * b.z)) + (h11 * m1.z));
}

/* ---------------------------------------------------------------------------
 * projection and 16.8 fixed-point snap (Sec. 3.1.2; Eq. 3's viewport map)
 * ------------------------------------------------------------------------- */
typedef struct { int valid; int32_t X, Y; float w, z, xs, ys; } proj_t;

static float clip_row(const float *m, int r, f3 p) {
    return (((m[4 * r + 0] * p.x) + (m[4 * r + 1] * p.y)) + (m[4 * r + 2] * p.z)) + m[4 * r + 3];
}

static float clampf(float v, float lo, float hi) { return v < lo ? lo : (v > hi ? hi : v); }

/* Screen position in pixels (y down), clamped to a 2^20 px guard band,
 * snapped to 1/256 px with round-half-even; linear depth
 * z = (w - near) / (far - near).  valid iff w >= near. */
static proj_t project(const orc_camera *cam, f3 p) {
    proj_t r;
    float c0 = clip_row(cam->m, 0, p);
    float c1 = clip_row(cam->m, 1, p);
    float w = clip_row(cam->m, 3, p);
    r.w = w;
    r.valid = (w >= cam->near);
    r.X = r.Y = 0;
    r.xs = r.ys = 0.0f;
    r.z = (w - cam->near) / (cam->far - cam->near);
    if (!r.valid) return r;
    float xs = (((c0 / w) + 1.0f) * 0.5f) * (float)cam->width;
    float ys = ((1.0f - (c1 / w)) * 0.5f) * (float)cam->height;
    xs = clampf(xs, -ORC_GUARD, ORC_GUARD);
    ys = clampf(ys, -ORC_GUARD, ORC_GUARD);
    r.xs = xs;
    r.ys = ys;
    r.X = (int32_t)rintf(xs * 256.0f);
    r.Y = (int32_t)rintf(ys * 256.0f);
    return r;
}

/* Reading of the paper's "configurable diameter" (Sec. 3.1.2): the centre
 * sample is an axis-aligned box whose half-width is the projected strand
 * half-width in 1/256 px, rounded half-even and clamped to [1, 128]:
 * r = ((128 width) focal) / w_mid, focal = (0.5 H) / tan(fovy/2),
 * w_mid = (wA + wB) 0.5. */
static int32_t center_halfwidth(const orc_camera *cam, float width_m, float wA, float wB) {
    float focal = (0.5f * (float)cam->height) / cam->tan_half_fovy;
    float wm = (wA + wB) * 0.5f;
    float r = ((128.0f * width_m) * focal) / wm;
    float q = rintf(r);
    if (q < 1.0f) q = 1.0f;
    if (q > 128.0f) q = 128.0f;
    return (int32_t)q;
}

/* ---------------------------------------------------------------------------
 * coverage predicate and depth (Sec. 3.1.2, Sec. 3.3)
 * ------------------------------------------------------------------------- */

/* Segment AB (1/256 px units) meets the closed box of half-width h around
 * (cx, cy) iff the bounding boxes overlap and the four box corners are not
 * all strictly on one side of the line AB (exact int64 separating-axis
 * test).  h = 128 is the conservative layer (the whole pixel). */
static int segment_covers(int64_t XA, int64_t YA, int64_t XB, int64_t YB,
                          int64_t cx, int64_t cy, int64_t h) {
    int64_t xmin = XA < XB ? XA : XB, xmax = XA < XB ? XB : XA;
    int64_t ymin = YA < YB ? YA : YB, ymax = YA < YB ? YB : YA;
    if (xmax < cx - h || xmin > cx + h || ymax < cy - h || ymin > cy + h) return 0;
    int64_t dX = XB - XA, dY = YB - YA;
    int64_t e0 = dX * ((cy - h) - YA) - dY * ((cx - h) - XA);
    int64_t e1 = dX * ((cy - h) - YA) - dY * ((cx + h) - XA);
    int64_t e2 = dX * ((cy + h) - YA) - dY * ((cx - h) - XA);
    int64_t e3 = dX * ((cy + h) - YA) - dY * ((cx + h) - XA);
    int64_t emin = e0, emax = e0;
    const int64_t e[3] = {e1, e2, e3};
    for (int i = 0; i < 3; ++i) {
        if (e[i] < emin) emin = e[i];
        if (e[i] > emax) emax = e[i];
    }
    return emin <= 0 && 0 <= emax;
}

/* Parameter of the pixel centre's projection onto AB:
 * t = clamp(float(num) / float(den), 0, 1), num = (Pc - A).(B - A),
 * den = |B - A|^2 in int64, t = 0 for a degenerate segment. */
static float segment_t(int64_t XA, int64_t YA, int64_t XB, int64_t YB,
                       int64_t cx, int64_t cy, int64_t *num_out, int64_t *den_out) {
    int64_t dX = XB - XA, dY = YB - YA;
    int64_t num = (cx - XA) * dX + (cy - YA) * dY;
    int64_t den = dX * dX + dY * dY;
    if (num_out) *num_out = num;
    if (den_out) *den_out = den;
    if (den == 0) return 0.0f;
    float t = (float)num / (float)den;
    return clampf(t, 0.0f, 1.0f);
}

/* 24-bit depth in the key's high bits (Sec. 3.1.2 "Reduced depth
 * precision").  Reading: linear depth interpolated in screen space at the
 * pixel centre, z = zA + (zB - zA) t, quantized d24 = min(floor(z 2^24),
 * 2^24 - 1) after clamping z to [0, 1]. */
static uint32_t depth24(float zA, float zB, float t) {
    float z = zA + ((zB - zA) * t);
    z = clampf(z, 0.0f, 1.0f);
    float q = floorf(z * 16777216.0f);
    uint32_t d = (uint32_t)q;
    return d > 16777215u ? 16777215u : d;
}

/* ---------------------------------------------------------------------------
 * distance/coverage LOD (Sec. 3.2, Eqs. 1-5)
 * ------------------------------------------------------------------------- */
static int floor_log2_u32(uint32_t v) { int r = -1; while (v) { v >>= 1; ++r; } return r; }

/* Eq. 1 (strand count) and Eqs. 4-5 (control points) for one bundle with
 * LOD selection value Lf in [0, 1]. */
static void lod_counts(float Lf, int32_t n_full, float delta, int32_t L, int32_t cmax,
                       int32_t *n_out, int32_t *c_out) {
    int32_t n = 0;
    if (n_full > 0) {
        float v = ceilf(Lf * ((float)n_full + delta));
        n = (int32_t)v;
        if (n < 1) n = 1;
        if (n > n_full) n = n_full;
    }
    int32_t craw = (int32_t)floorf(sqrtf(Lf) * (float)cmax);
    if (craw < L) craw = L;
    int32_t c = (1 << floor_log2_u32((uint32_t)(craw - 1))) + 1;
    if (c > cmax) c = cmax;
    int32_t lo = L < cmax ? L : cmax;
    if (c < lo) c = lo;
    *n_out = n;
    *c_out = c;
}

/* One bundle: screen AABB over every layer's triangle vertices (Eq. 3),
 * frustum cull, L (Eq. 2), N_LOD (Eq. 1), C (Eqs. 4-5).  Reading: C_max =
 * segs + 1; a bundle wholly behind the near plane is culled, one that
 * straddles it gets L = 1 and is not culled; the
 * snap of Eq. 5 is raised back to min(C_layers, C_max), the hard lower
 * bound the text states for Eq. 4. */
static void lod_bundle(const orc_groom *g, const orc_camera *cam, int enabled, float lam,
                       const float *delta, int32_t f, int32_t n_full, int32_t *n_out, int32_t *c_out) {
    int32_t cmax = g->segs + 1;
    if (!enabled) { *n_out = n_full; *c_out = cmax; return; }
    float xmin = INFINITY, xmax = -INFINITY, ymin = INFINITY, ymax = -INFINITY;
    int behind = 0, front = 0;
    for (int k = 0; k < g->L; ++k) {
        for (int c = 0; c < 3; ++c) {
            int32_t vi = g->faces[3 * (int64_t)f + c];
            const float *v = g->layer_verts + ((int64_t)k * g->V + vi) * 3;
            proj_t p = project(cam, mk(v[0], v[1], v[2]));
            if (!p.valid) { behind = 1; continue; }
            front = 1;
            if (p.xs < xmin) xmin = p.xs;
            if (p.xs > xmax) xmax = p.xs;
            if (p.ys < ymin) ymin = p.ys;
            if (p.ys > ymax) ymax = p.ys;
        }
    }
    float Lf;
    if (!front) {                   /* wholly behind the near plane: culled */
        *n_out = 0;
        *c_out = cmax;
        return;
    }
    if (behind) {                   /* straddles the near plane: full detail */
        Lf = 1.0f;
    } else {
        if (xmax < 0.0f || xmin > (float)cam->width || ymax < 0.0f || ymin > (float)cam->height) {
            *n_out = 0;
            *c_out = cmax;
            return;
        }
        float dx = xmax - xmin, dy = ymax - ymin;
        float diag = sqrtf((dx * dx) + (dy * dy));
        Lf = clampf((diag / (float)cam->height) * lam, 0.0f, 1.0f);
    }
    lod_counts(Lf, n_full, delta[f], g->L, cmax, n_out, c_out);
}

static void bundle_offsets(const orc_groom *g, int64_t *off) {
    for (int32_t f = 0; f <= g->F; ++f) off[f] = 0;
    for (int64_t s = 0; s < g->S; ++s) off[g->strand_face[s] + 1]++;
    for (int32_t f = 0; f < g->F; ++f) off[f + 1] += off[f];
}

int orc_lod(const orc_groom *g, const orc_camera *cam, int32_t enabled, float lam,
            const float *delta, int32_t *n_out, int32_t *c_out) {
    int64_t *off = (int64_t *)malloc(sizeof(int64_t) * (g->F + 1));
    if (!off) return 1;
    bundle_offsets(g, off);
    for (int32_t f = 0; f < g->F; ++f)
        lod_bundle(g, cam, enabled, lam, delta, f, (int32_t)(off[f + 1] - off[f]), &n_out[f], &c_out[f]);
    free(off);
    return 0;
}

/* ---------------------------------------------------------------------------
 * rasterization into the two visibility layers (Sec. 3.1.2, Sec. 3.3)
 * ------------------------------------------------------------------------- */
typedef struct {
    int32_t XA, YA, XB, YB;
    float zA, zB;
    int32_t hc;
    int32_t valid;
    uint64_t id;
    /* compressed payload only: bits 39..12 (tangent, u, v), segment index,
     * C - 1 and the AO at both ends */
    uint64_t cgb_hi;
    int32_t j, cm1;
    float aoA, aoB;
} seg_t;

/* ---------------------------------------------------------------------------
 * compressed G-buffer payload (Sec. 3.1.2: uvw styling coordinates instead
 * of shading parameters, an octahedral tangent, every value but depth
 * quantized to 8 or 6 bits, all of it next to the 24-bit depth in 64 bits)
 *
 * Readings (the inset with the bit layout is lost):
 *   bits 39..32 / 31..24  octahedral tangent x / y, 8 bits each;
 *   bits 23..18 / 17..12  the root's scalp texture coordinates u / v, 6 bits;
 *   bits 11..6            w = (j + t) / (C - 1), the position along the strand;
 *   bits 5..0             ambient occlusion, 0..62 (63 is never written, so a
 *                         payload is never all ones, the empty marker).
 * The tangent is the segment's chord p_{j+1} - p_j, encoded once per
 * segment; AO is the control points' AO (Hermite along the strand, as the
 * positions) interpolated linearly in t.  Each quantization is
 * rint(x * scale) clamped, ties to even.  Octahedral encoding after Cigolle
 * et al. 2014 (sign(0) = +1).
 * ------------------------------------------------------------------------- */
static int32_t quantize(float x, float scale, int32_t hi) {
    float q = rintf(x * scale);
    if (!(q >= 0.0f)) return 0;
    if (q >= (float)hi) return hi;
    return (int32_t)q;
}

static float sgn1(float v) { return v >= 0.0f ? 1.0f : -1.0f; }

static uint32_t oct_encode(f3 T) {
    float s = (fabsf(T.x) + fabsf(T.y)) + fabsf(T.z);
    float ox = 0.0f, oy = 0.0f;
    if (s > 0.0f) { ox = T.x / s; oy = T.y / s; }
    if (T.z < 0.0f) {
        float nx = (1.0f - fabsf(oy)) * sgn1(ox);
        float ny = (1.0f - fabsf(ox)) * sgn1(oy);
        ox = nx; oy = ny;
    }
    uint32_t cx = (uint32_t)quantize((ox * 0.5f) + 0.5f, 255.0f, 255);
    uint32_t cy = (uint32_t)quantize((oy * 0.5f) + 0.5f, 255.0f, 255);
    return (cx << 8) | cy;
}

static f3 oct_decode(uint32_t code) {
    float ox = (((float)(code >> 8) / 255.0f) * 2.0f) - 1.0f;
    float oy = (((float)(code & 255u) / 255.0f) * 2.0f) - 1.0f;
    float z = (1.0f - fabsf(ox)) - fabsf(oy);
    if (z < 0.0f) {
        float nx = (1.0f - fabsf(oy)) * sgn1(ox);
        float ny = (1.0f - fabsf(ox)) * sgn1(oy);
        ox = nx; oy = ny;
    }
    return normalize3(mk(ox, oy, z));
}

/* AO of layer point k and of control point j (cubic Hermite over the layer
 * values with finite-difference slopes, one-sided at root and tip). */
static float layer_ao_f32(const orc_groom *g, int64_t s, int k) {
    if (!g->vert_ao) return 1.0f;
    const int32_t *f = &g->faces[3 * g->strand_face[s]];
    float b1 = g->strand_bary[2 * s], b2 = g->strand_bary[2 * s + 1];
    float b0 = (1.0f - b1) - b2;
    const float *row = &g->vert_ao[(int64_t)k * g->V];
    return ((b0 * row[f[0]]) + (b1 * row[f[1]])) + (b2 * row[f[2]]);
}

static float control_ao_f32(const orc_groom *g, int64_t s, int C, int j) {
    int L = g->L;
    int x = j * (L - 1);
    int k = x / (C - 1);
    if (k > L - 2) k = L - 2;
    float t = (float)(x - k * (C - 1)) / (float)(C - 1);
    float a0 = layer_ao_f32(g, s, k), a1 = layer_ao_f32(g, s, k + 1);
    float am = k > 0 ? layer_ao_f32(g, s, k - 1) : a0;
    float a2 = k + 2 <= L - 1 ? layer_ao_f32(g, s, k + 2) : a1;
    float m0 = k == 0 ? a1 - a0 : 0.5f * (a1 - am);
    float m1 = k + 1 == L - 1 ? a1 - a0 : 0.5f * (a2 - a0);
    float t2 = t * t, t3 = t2 * t;
    float h00 = ((2.0f * t3) - (3.0f * t2)) + 1.0f, h10 = (t3 - (2.0f * t2)) + t;
    float h01 = (3.0f * t2) - (2.0f * t3), h11 = t3 - t2;
    return (((h00 * a0) + (h10 * m0)) + (h01 * a1)) + (h11 * m1);
}

static void root_uv(const orc_groom *g, int64_t s, float *u, float *v) {
    *u = *v = 0.0f;
    if (!g->vert_uv) return;
    const int32_t *f = &g->faces[3 * g->strand_face[s]];
    float b1 = g->strand_bary[2 * s], b2 = g->strand_bary[2 * s + 1];
    float b0 = (1.0f - b1) - b2;
    const float *uv = g->vert_uv;
    *u = ((b0 * uv[2 * f[0]]) + (b1 * uv[2 * f[1]])) + (b2 * uv[2 * f[2]]);
    *v = ((b0 * uv[2 * f[0] + 1]) + (b1 * uv[2 * f[1] + 1])) + (b2 * uv[2 * f[2] + 1]);
}

/* Low 40 bits of the compressed key at projection parameter t. */
static uint64_t cgb_payload(const seg_t *q, float t) {
    uint32_t cw = (uint32_t)quantize(((float)q->j + t) / (float)q->cm1, 63.0f, 63);
    uint32_t ca = (uint32_t)quantize(q->aoA + ((q->aoB - q->aoA) * t), 62.0f, 62);
    return q->cgb_hi | ((uint64_t)cw << 6) | (uint64_t)ca;
}

/* Per strand: layer points, base tangents, C control points, projection;
 * segment j joins control points j and j+1 and is dropped when either end
 * is in front of the near plane. */
static void strand_segments(const orc_groom *g, const orc_camera *cam, int64_t s, int C, seg_t *out) {
    f3 P[64], mh[64], cp[128];
    proj_t pr[128];
    float ao[128];
    strand_layer_points(g, s, P);
    layer_tangents(P, g->L, mh);
    for (int j = 0; j < C; ++j) {
        cp[j] = control_point(P, mh, g->L, C, j);
        pr[j] = project(cam, cp[j]);
        ao[j] = control_ao_f32(g, s, C, j);
    }
    uint64_t sg = g->strand_base + (uint64_t)s;
    float u, v;
    root_uv(g, s, &u, &v);
    uint64_t uv_bits = ((uint64_t)quantize(u, 63.0f, 63) << 18) | ((uint64_t)quantize(v, 63.0f, 63) << 12);
    for (int j = 0; j + 1 < C; ++j) {
        seg_t *q = &out[j];
        q->valid = pr[j].valid && pr[j + 1].valid;
        q->XA = pr[j].X; q->YA = pr[j].Y; q->XB = pr[j + 1].X; q->YB = pr[j + 1].Y;
        q->zA = pr[j].z; q->zB = pr[j + 1].z;
        q->hc = q->valid ? center_halfwidth(cam, g->width_m, pr[j].w, pr[j + 1].w) : 0;
        q->id = (sg << 7) | (uint64_t)j;
        q->cgb_hi = ((uint64_t)oct_encode(normalize3(sub3(cp[j + 1], cp[j]))) << 24) | uv_bits;
        q->j = j;
        q->cm1 = C - 1;
        q->aoA = ao[j];
        q->aoB = ao[j + 1];
    }
}

static int64_t floor_div256(int64_t v) { return v >= 0 ? v / 256 : -((-v + 255) / 256); }

/* Rasterize every segment of every drawn strand: for each pixel of the
 * segment's expanded bounding box, test both layers' predicates and keep the
 * minimum key (depth in bits 63..40, strand id in 39..7, segment in 6..0).
 * Rows are split into bands, one band per worker, so each key is written by
 * one thread; min is order independent.  counts[0] += covered (pixel,
 * centre) pairs, counts[1] += covered (pixel, conservative) pairs. */
int orc_raster(const orc_groom *grooms, int32_t n_grooms, const orc_camera *cam,
               uint64_t *vis_c, uint64_t *vis_a, int64_t *counts, int32_t compressed, int32_t nthreads) {
    int64_t total = 0;
    int64_t *gseg = (int64_t *)malloc(sizeof(int64_t) * (n_grooms + 1));
    int64_t **boff = (int64_t **)calloc(n_grooms, sizeof(int64_t *));
    int64_t **soff = (int64_t **)calloc(n_grooms, sizeof(int64_t *));
    if (!gseg || !boff || !soff) return 1;
    gseg[0] = 0;
    for (int32_t gi = 0; gi < n_grooms; ++gi) {
        const orc_groom *g = &grooms[gi];
        boff[gi] = (int64_t *)malloc(sizeof(int64_t) * (g->F + 1));
        soff[gi] = (int64_t *)malloc(sizeof(int64_t) * (g->F + 1));
        if (!boff[gi] || !soff[gi]) return 1;
        bundle_offsets(g, boff[gi]);
        soff[gi][0] = 0;
        for (int32_t f = 0; f < g->F; ++f) {
            int64_t n = g->lod_n[f], c = g->lod_c[f];
            soff[gi][f + 1] = soff[gi][f] + (c >= 2 ? n * (c - 1) : 0);
        }
        gseg[gi + 1] = gseg[gi] + soff[gi][g->F];
    }
    total = gseg[n_grooms];
    seg_t *segs = (seg_t *)malloc(sizeof(seg_t) * (total > 0 ? total : 1));
    if (!segs) return 1;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
    for (int32_t gi = 0; gi < n_grooms; ++gi) {
        const orc_groom *g = &grooms[gi];
#pragma omp parallel for schedule(dynamic, 16)
        for (int32_t f = 0; f < g->F; ++f) {
            int32_t c = g->lod_c[f];
            if (c < 2) continue;
            for (int32_t i = 0; i < g->lod_n[f]; ++i) {
                int64_t s = boff[gi][f] + i;
                strand_segments(g, cam, s, c, &segs[gseg[gi] + soff[gi][f] + (int64_t)i * (c - 1)]);
            }
        }
    }
    const int W = cam->width, H = cam->height;
    const int band = 16;
    const int nb = (H + band - 1) / band;
    int64_t cnt_c = 0, cnt_a = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : cnt_c, cnt_a)
    for (int b = 0; b < nb; ++b) {
        int64_t r0 = (int64_t)b * band, r1 = r0 + band - 1;
        if (r1 > H - 1) r1 = H - 1;
        for (int64_t q = 0; q < total; ++q) {
            const seg_t *sg = &segs[q];
            if (!sg->valid) continue;
            int64_t xmin = sg->XA < sg->XB ? sg->XA : sg->XB, xmax = sg->XA < sg->XB ? sg->XB : sg->XA;
            int64_t ymin = sg->YA < sg->YB ? sg->YA : sg->YB, ymax = sg->YA < sg->YB ? sg->YB : sg->YA;
            int64_t i0 = floor_div256(xmin) - 1, i1 = floor_div256(xmax);
            int64_t m0 = floor_div256(ymin) - 1, m1 = floor_div256(ymax);
            if (i0 < 0) i0 = 0;
            if (i1 > W - 1) i1 = W - 1;
            if (m0 < r0) m0 = r0;
            if (m1 > r1) m1 = r1;
            for (int64_t m = m0; m <= m1; ++m) {
                for (int64_t i = i0; i <= i1; ++i) {
                    int64_t cx = 256 * i + 128, cy = 256 * m + 128;
                    int ca = segment_covers(sg->XA, sg->YA, sg->XB, sg->YB, cx, cy, 128);
                    int cc = segment_covers(sg->XA, sg->YA, sg->XB, sg->YB, cx, cy, sg->hc);
                    if (!ca && !cc) continue;
                    float t = segment_t(sg->XA, sg->YA, sg->XB, sg->YB, cx, cy, 0, 0);
                    uint64_t key = ((uint64_t)depth24(sg->zA, sg->zB, t) << 40) |
                                   (compressed ? cgb_payload(sg, t) : sg->id);
                    int64_t px = m * W + i;
                    if (ca) { ++cnt_a; if (key < vis_a[px]) vis_a[px] = key; }
                    if (cc) { ++cnt_c; if (key < vis_c[px]) vis_c[px] = key; }
                }
            }
        }
    }
    if (counts) { counts[0] += cnt_c; counts[1] += cnt_a; }
    free(segs);
    for (int32_t gi = 0; gi < n_grooms; ++gi) { free(boff[gi]); free(soff[gi]); }
    free(boff); free(soff); free(gseg);
    return 0;
}

/* ---------------------------------------------------------------------------
 * resolve: decode a key back to strand geometry at the pixel (Sec. 3.1.2
 * deferred shading; Sec. 3.3 filter masks)
 * ------------------------------------------------------------------------- */
static int key_empty(uint64_t k) { return (k & ORC_PAYLOAD_MASK) == ORC_PAYLOAD_MASK; }

typedef struct {
    int ok;
    int64_t num, den;
    f3 X, T;                     /* FP32 position and unit tangent at the pixel */
    int iso;                     /* screen tangent degenerate */
    float tsx, tsy;              /* unit screen tangent (pixels, y down) */
} decode_t;

static const orc_groom *find_groom(const orc_groom *gs, int32_t n, uint64_t sgl, int64_t *s_local) {
    for (int32_t i = 0; i < n; ++i) {
        if (sgl >= gs[i].strand_base && sgl < gs[i].strand_base + (uint64_t)gs[i].S) {
            *s_local = (int64_t)(sgl - gs[i].strand_base);
            return &gs[i];
        }
    }
    return 0;
}

/* Screen tangent: the Jacobian of the pixel position with respect to the
 * world position, at X, applied to T, normalized (Code 2's getScreenTangent;
 * reading: analytic Jacobian of the perspective divide and viewport map).
 * Reading: the tangent is degenerate, selecting the isotropic mode of
 * Sec. 3.3.1, when |J T| w < 0.01 focal, i.e. the strand is within about
 * 0.6 degrees of the view ray (|J T| w / focal is the sine of that angle for
 * a tangent at the image centre). */
static int screen_tangent(const orc_camera *cam, f3 X, f3 T, float *tsx, float *tsy) {
    const float *m = cam->m;
    float c0 = clip_row(m, 0, X);
    float c1 = clip_row(m, 1, X);
    float w = clip_row(m, 3, X);
    float a0 = ((m[0] * T.x) + (m[1] * T.y)) + (m[2] * T.z);
    float a1 = ((m[4] * T.x) + (m[5] * T.y)) + (m[6] * T.z);
    float a3 = ((m[12] * T.x) + (m[13] * T.y)) + (m[14] * T.z);
    float w2 = w * w;
    float jx = (((a0 * w) - (c0 * a3)) / w2) * (0.5f * (float)cam->width);
    float jy = -((((a1 * w) - (c1 * a3)) / w2) * (0.5f * (float)cam->height));
    float n = sqrtf((jx * jx) + (jy * jy));
    float focal = (0.5f * (float)cam->height) / cam->tan_half_fovy;
    if (!((n * w) >= (0.01f * focal))) { *tsx = 0.0f; *tsy = 0.0f; return 1; }
    *tsx = jx / n;
    *tsy = jy / n;
    return 0;
}

/* Decode of a key at the sample point (sx, sy) in 1/256 px: the segment's
 * projection parameter there, the FP32 position and unit tangent. */
static decode_t decode_key_at(const orc_groom *gs, int32_t n, const orc_camera *cam, uint64_t key,
                              int64_t sx, int64_t sy) {
    decode_t d;
    memset(&d, 0, sizeof d);
    int64_t s;
    const orc_groom *g = find_groom(gs, n, (key >> 7) & ORC_STRAND_MASK, &s);
    if (!g) return d;
    int j = (int)(key & 127);
    int C = g->lod_c[g->strand_face[s]];
    if (j + 1 >= C) return d;
    f3 P[64], mh[64];
    strand_layer_points(g, s, P);
    layer_tangents(P, g->L, mh);
    f3 pm = (j >= 1) ? control_point(P, mh, g->L, C, j - 1) : mk(0, 0, 0);
    f3 p0 = control_point(P, mh, g->L, C, j);
    f3 p1 = control_point(P, mh, g->L, C, j + 1);
    f3 pp = (j + 2 <= C - 1) ? control_point(P, mh, g->L, C, j + 2) : mk(0, 0, 0);
    proj_t a = project(cam, p0), b = project(cam, p1);
    float t = segment_t(a.X, a.Y, b.X, b.Y, sx, sy, &d.num, &d.den);
    d.X = mk(p0.x + ((p1.x - p0.x) * t), p0.y + ((p1.y - p0.y) * t), p0.z + ((p1.z - p0.z) * t));
    f3 T0 = calc_tangent(j, C, pm, p0, p1);
    f3 T1 = calc_tangent(j + 1, C, p0, p1, pp);
    d.T = normalize3(mk(T0.x + ((T1.x - T0.x) * t), T0.y + ((T1.y - T0.y) * t), T0.z + ((T1.z - T0.z) * t)));
    d.iso = screen_tangent(cam, d.X, d.T, &d.tsx, &d.tsy);
    d.ok = 1;
    return d;
}

static decode_t decode_key(const orc_groom *gs, int32_t n, const orc_camera *cam, uint64_t key,
                           int64_t px, int64_t py) {
    return decode_key_at(gs, n, cam, key, 256 * px + 128, 256 * py + 128);
}

/* Compressed payload decode (Sec. 3.1.2 position reconstruction): the
 * position is the point at the key's depth on the ray through the pixel
 * centre, taken at the middle of the 24-bit depth bin,
 * w = near + ((d24 + 0.5) 2^-24) (far - near), solved from the projection's
 * rows (M0 - xn M3) X = xn M33 - M03, (M1 - yn M3) X = yn M33 - M13,
 * M3 X = w - M33 by Cramer's rule; the tangent is the octahedral decode. */
static f3 cross3(f3 a, f3 b) {
    return mk((a.y * b.z) - (a.z * b.y), (a.z * b.x) - (a.x * b.z), (a.x * b.y) - (a.y * b.x));
}

static f3 unproject(const orc_camera *cam, float xs, float ys, float w) {
    const float *m = cam->m;
    float xn = ((2.0f * xs) / (float)cam->width) - 1.0f;
    float yn = 1.0f - ((2.0f * ys) / (float)cam->height);
    f3 ra = mk(m[0] - (xn * m[12]), m[1] - (xn * m[13]), m[2] - (xn * m[14]));
    f3 rb = mk(m[4] - (yn * m[12]), m[5] - (yn * m[13]), m[6] - (yn * m[14]));
    f3 rc = mk(m[12], m[13], m[14]);
    float ka = (xn * m[15]) - m[3];
    float kb = (yn * m[15]) - m[7];
    float kc = w - m[15];
    f3 bc = cross3(rb, rc), ca = cross3(rc, ra), ab = cross3(ra, rb);
    float det = ((ra.x * bc.x) + (ra.y * bc.y)) + (ra.z * bc.z);
    return mk((((ka * bc.x) + (kb * ca.x)) + (kc * ab.x)) / det,
              (((ka * bc.y) + (kb * ca.y)) + (kc * ab.y)) / det,
              (((ka * bc.z) + (kb * ca.z)) + (kc * ab.z)) / det);
}

static decode_t decode_cgb(const orc_camera *cam, uint64_t key, int64_t px, int64_t py) {
    decode_t d;
    memset(&d, 0, sizeof d);
    float z = ((float)(uint32_t)(key >> 40) + 0.5f) * 5.9604644775390625e-8f;
    float w = cam->near + (z * (cam->far - cam->near));
    d.X = unproject(cam, (float)px + 0.5f, (float)py + 0.5f, w);
    d.T = oct_decode((uint32_t)((key >> 24) & 0xFFFFu));
    d.iso = screen_tangent(cam, d.X, d.T, &d.tsx, &d.tsy);
    d.ok = 1;
    return d;
}

/* Strip membership of window offset (dx, dy) for a unit screen tangent:
 * d_par = d . Ts, e = d - d_par Ts, in iff |e|^2 <= hw^2 (Sec. 3.3.3).
 * Reading: with a degenerate tangent the strip is the pixel itself. */
static int in_strip(int iso, float tsx, float tsy, int dx, int dy, float hw2) {
    if (iso) return dx == 0 && dy == 0;
    float fx = (float)dx, fy = (float)dy;
    float dpar = (fx * tsx) + (fy * tsy);
    float ex = fx - (dpar * tsx);
    float ey = fy - (dpar * tsy);
    return ((ex * ex) + (ey * ey)) <= hw2;
}

/* Per pixel, for the centre key G and the conservative key A when present:
 * the pixel-centre projection parameter as num/den, the isotropic flag and
 * the strip hit counts H_center (centre layer non-empty) and H_cons
 * (conservative layer non-empty) over the (2r+1)^2 window clipped to the
 * screen (Sec. 3.3.3).  Outputs are per pixel, row-major. */
int orc_resolve_decisions(const orc_groom *grooms, int32_t n_grooms, const orc_camera *cam,
                          int32_t radius, float strip_hw, const uint64_t *vis_c, const uint64_t *vis_a,
                          const int64_t *pixels, int64_t n_pixels,
                          int64_t *numG, int64_t *denG, int64_t *numA, int64_t *denA,
                          uint8_t *isoG, uint8_t *isoA, int32_t *HcG, int32_t *HaG,
                          int32_t *HcA, int32_t *HaA, int32_t compressed, int32_t nthreads) {
    const int W = cam->width, H = cam->height;
    const float hw2 = strip_hw * strip_hw;
    int64_t npx = pixels ? n_pixels : (int64_t)W * H;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t q = 0; q < npx; ++q) {
        int64_t p = pixels ? pixels[q] : q;
        int64_t px = p % W, py = p / W;
        numG[q] = denG[q] = numA[q] = denA[q] = 0;
        isoG[q] = isoA[q] = 0;
        HcG[q] = HaG[q] = HcA[q] = HaA[q] = 0;
        for (int layer = 0; layer < 2; ++layer) {
            uint64_t key = layer == 0 ? vis_c[p] : vis_a[p];
            if (key_empty(key)) continue;
            decode_t d = compressed ? decode_cgb(cam, key, px, py) : decode_key(grooms, n_grooms, cam, key, px, py);
            if (!d.ok) continue;
            int hc = 0, ha = 0;
            for (int dy = -radius; dy <= radius; ++dy) {
                int64_t qy = py + dy;
                if (qy < 0 || qy >= H) continue;
                for (int dx = -radius; dx <= radius; ++dx) {
                    int64_t qx = px + dx;
                    if (qx < 0 || qx >= W) continue;
                    if (!in_strip(d.iso, d.tsx, d.tsy, dx, dy, hw2)) continue;
                    int64_t qi = qy * W + qx;
                    hc += !key_empty(vis_c[qi]);
                    ha += !key_empty(vis_a[qi]);
                }
            }
            if (layer == 0) { numG[q] = d.num; denG[q] = d.den; isoG[q] = (uint8_t)d.iso; HcG[q] = hc; HaG[q] = ha; }
            else { numA[q] = d.num; denA[q] = d.den; isoA[q] = (uint8_t)d.iso; HcA[q] = hc; HaA[q] = ha; }
        }
    }
    return 0;
}

/* ---------------------------------------------------------------------------
 * multisample rasterization (Sec. 3.3 keeps a multisampled variant of the
 * software rasterizer, one uint64 layer per sample, as its quality reference)
 *
 * Reading: N point samples per pixel at offsets (ox[k], oy[k]) (1/256 px
 * from the pixel centre); sample k of a pixel is covered by a segment iff the
 * closed box of the segment's centre half-width h_c around the sample point
 * meets it (the centre-sample predicate, moved to the sample), and its key
 * uses the depth at the sample's projection parameter.  Layer k holds the
 * minimum key of sample k: vis_s[k][H*W].
 * ------------------------------------------------------------------------- */
int orc_raster_msaa(const orc_groom *grooms, int32_t n_grooms, const orc_camera *cam, int32_t n_samples,
                    const int32_t *ox, const int32_t *oy, uint64_t *vis_s, int64_t *count, int32_t nthreads) {
    int64_t total = 0;
    int64_t *gseg = (int64_t *)malloc(sizeof(int64_t) * (n_grooms + 1));
    if (!gseg) return 1;
    gseg[0] = 0;
    for (int32_t gi = 0; gi < n_grooms; ++gi) {
        const orc_groom *g = &grooms[gi];
        int64_t t = 0;
        for (int32_t f = 0; f < g->F; ++f) if (g->lod_c[f] >= 2) t += (int64_t)g->lod_n[f] * (g->lod_c[f] - 1);
        gseg[gi + 1] = gseg[gi] + t;
    }
    total = gseg[n_grooms];
    seg_t *segs = (seg_t *)malloc(sizeof(seg_t) * (total > 0 ? total : 1));
    if (!segs) { free(gseg); return 1; }
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
    for (int32_t gi = 0; gi < n_grooms; ++gi) {
        const orc_groom *g = &grooms[gi];
        int64_t *off = (int64_t *)malloc(sizeof(int64_t) * (g->F + 1));
        if (!off) { free(segs); free(gseg); return 1; }
        bundle_offsets(g, off);
        int64_t w = gseg[gi];
        for (int32_t f = 0; f < g->F; ++f) {
            int32_t c = g->lod_c[f];
            if (c < 2) continue;
            for (int32_t i = 0; i < g->lod_n[f]; ++i) {
                strand_segments(g, cam, off[f] + i, c, &segs[w]);
                w += c - 1;
            }
        }
        free(off);
    }
    const int W = cam->width, H = cam->height;
    const int64_t npx = (int64_t)W * H;
    const int band = 16;
    const int nb = (H + band - 1) / band;
    int64_t cnt = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : cnt)
    for (int b = 0; b < nb; ++b) {
        int64_t r0 = (int64_t)b * band, r1 = r0 + band - 1;
        if (r1 > H - 1) r1 = H - 1;
        for (int64_t q = 0; q < total; ++q) {
            const seg_t *sg = &segs[q];
            if (!sg->valid) continue;
            int64_t xmin = sg->XA < sg->XB ? sg->XA : sg->XB, xmax = sg->XA < sg->XB ? sg->XB : sg->XA;
            int64_t ymin = sg->YA < sg->YB ? sg->YA : sg->YB, ymax = sg->YA < sg->YB ? sg->YB : sg->YA;
            /* sample boxes reach at most 240/256 px from the pixel centre */
            int64_t i0 = floor_div256(xmin) - 2, i1 = floor_div256(xmax) + 1;
            int64_t m0 = floor_div256(ymin) - 2, m1 = floor_div256(ymax) + 1;
            if (i0 < 0) i0 = 0;
            if (i1 > W - 1) i1 = W - 1;
            if (m0 < r0) m0 = r0;
            if (m1 > r1) m1 = r1;
            for (int64_t m = m0; m <= m1; ++m) {
                for (int64_t i = i0; i <= i1; ++i) {
                    for (int k = 0; k < n_samples; ++k) {
                        int64_t sx = 256 * i + 128 + ox[k], sy = 256 * m + 128 + oy[k];
                        if (!segment_covers(sg->XA, sg->YA, sg->XB, sg->YB, sx, sy, sg->hc)) continue;
                        float t = segment_t(sg->XA, sg->YA, sg->XB, sg->YB, sx, sy, 0, 0);
                        uint64_t key = ((uint64_t)depth24(sg->zA, sg->zB, t) << 40) | sg->id;
                        uint64_t *dst = &vis_s[(int64_t)k * npx + m * W + i];
                        ++cnt;
                        if (key < *dst) *dst = key;
                    }
                }
            }
        }
    }
    if (count) *count += cnt;
    free(segs);
    free(gseg);
    return 0;
}

/* Projection parameter of every covered sample's key, as num/den (the
 * multisample resolve shades each sample at its own position). */
int orc_msaa_decisions(const orc_groom *grooms, int32_t n_grooms, const orc_camera *cam, int32_t n_samples,
                       const int32_t *ox, const int32_t *oy, const uint64_t *vis_s, int64_t *num, int64_t *den,
                       int32_t nthreads) {
    const int W = cam->width, H = cam->height;
    const int64_t npx = (int64_t)W * H;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t q = 0; q < npx * n_samples; ++q) {
        int k = (int)(q / npx);
        int64_t p = q % npx;
        num[q] = den[q] = 0;
        uint64_t key = vis_s[q];
        if ((key & ORC_PAYLOAD_MASK) == ORC_PAYLOAD_MASK) continue;
        int64_t s;
        const orc_groom *g = find_groom(grooms, n_grooms, (key >> 7) & ORC_STRAND_MASK, &s);
        if (!g) continue;
        int j = (int)(key & 127);
        int C = g->lod_c[g->strand_face[s]];
        if (j + 1 >= C) continue;
        f3 P[64], mh[64];
        strand_layer_points(g, s, P);
        layer_tangents(P, g->L, mh);
        proj_t a = project(cam, control_point(P, mh, g->L, C, j));
        proj_t b = project(cam, control_point(P, mh, g->L, C, j + 1));
        segment_t(a.X, a.Y, b.X, b.Y, 256 * (p % W) + 128 + ox[k], 256 * (p / W) + 128 + oy[k], &num[q], &den[q]);
    }
    return 0;
}

/* ---------------------------------------------------------------------------
 * single-step entry points used by the pin tests
 * ------------------------------------------------------------------------- */
/* ---------------------------------------------------------------------------
 * shadow-map texel of a shaded point (Sec. 3.2 "Depth Comparison Artifact
 * Fix"; Sec. 3.4 queries shadow/opacity maps with that correction)
 *
 * Reading: the FP32 position X decoded from the key at the sample point is
 * projected with the light's camera exactly like a strand control point
 * (same clip rows, divide, guard band and 1/256 px snap); its texel is
 * (floor(X / 256), floor(Y / 256)).  texel[q] = row-major texel index, or -1
 * when X is in front of the light's near plane, off the map, or the key does
 * not decode.  Everything continuous (the depth past the occluder, the
 * visibility) is the value layer's.
 * ------------------------------------------------------------------------- */
int orc_shadow_texels(const orc_groom *grooms, int32_t n_grooms, const orc_camera *cam, const uint64_t *keys,
                      const int64_t *sx, const int64_t *sy, int64_t n_keys, const orc_camera *light,
                      int64_t *texel, int32_t nthreads) {
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t q = 0; q < n_keys; ++q) {
        texel[q] = -1;
        if (key_empty(keys[q])) continue;
        decode_t d = decode_key_at(grooms, n_grooms, cam, keys[q], sx[q], sy[q]);
        if (!d.ok) continue;
        proj_t p = project(light, d.X);
        if (!p.valid) continue;
        int64_t tx = floor_div256(p.X), ty = floor_div256(p.Y);
        if (tx < 0 || ty < 0 || tx >= light->width || ty >= light->height) continue;
        texel[q] = ty * light->width + tx;
    }
    return 0;
}

uint32_t orc_oct_encode(const float *T) { return oct_encode(mk(T[0], T[1], T[2])); }

void orc_oct_decode(uint32_t code, float *T) {
    f3 v = oct_decode(code);
    T[0] = v.x; T[1] = v.y; T[2] = v.z;
}

void orc_unproject(const orc_camera *cam, float xs, float ys, float w, float *X) {
    f3 v = unproject(cam, xs, ys, w);
    X[0] = v.x; X[1] = v.y; X[2] = v.z;
}

int orc_strand_control_points(const orc_groom *g, int64_t s, int32_t C, float *out) {
    f3 P[64], mh[64];
    if (g->L < 2 || g->L > 64 || C < 2) return 1;
    strand_layer_points(g, s, P);
    layer_tangents(P, g->L, mh);
    for (int j = 0; j < C; ++j) {
        f3 p = control_point(P, mh, g->L, C, j);
        out[3 * j + 0] = p.x; out[3 * j + 1] = p.y; out[3 * j + 2] = p.z;
    }
    return 0;
}

int orc_strand_tangents(const orc_groom *g, int64_t s, int32_t C, float *out) {
    f3 P[64], mh[64], p[128];
    if (g->L < 2 || g->L > 64 || C < 2 || C > 128) return 1;
    strand_layer_points(g, s, P);
    layer_tangents(P, g->L, mh);
    for (int j = 0; j < C; ++j) p[j] = control_point(P, mh, g->L, C, j);
    for (int j = 0; j < C; ++j) {
        f3 t = calc_tangent(j, C, j > 0 ? p[j - 1] : p[j], p[j], j < C - 1 ? p[j + 1] : p[j]);
        out[3 * j + 0] = t.x; out[3 * j + 1] = t.y; out[3 * j + 2] = t.z;
    }
    return 0;
}

int orc_project_point(const orc_camera *cam, const float *p, int32_t *XY, float *wz) {
    proj_t r = project(cam, mk(p[0], p[1], p[2]));
    XY[0] = r.X; XY[1] = r.Y;
    wz[0] = r.w; wz[1] = r.z; wz[2] = r.xs; wz[3] = r.ys;
    return r.valid;
}

int orc_segment_covers(int64_t XA, int64_t YA, int64_t XB, int64_t YB, int64_t cx, int64_t cy, int64_t h) {
    return segment_covers(XA, YA, XB, YB, cx, cy, h);
}

uint32_t orc_depth24(int64_t XA, int64_t YA, int64_t XB, int64_t YB, float zA, float zB, int64_t cx, int64_t cy) {
    return depth24(zA, zB, segment_t(XA, YA, XB, YB, cx, cy, 0, 0));
}

int32_t orc_center_halfwidth(const orc_camera *cam, float width_m, float wA, float wB) {
    return center_halfwidth(cam, width_m, wA, wB);
}

int orc_screen_tangent(const orc_camera *cam, const float *X, const float *T, float *ts) {
    return screen_tangent(cam, mk(X[0], X[1], X[2]), mk(T[0], T[1], T[2]), &ts[0], &ts[1]);
}

int orc_in_strip(int iso, float tsx, float tsy, int dx, int dy, float hw) {
    return in_strip(iso, tsx, tsy, dx, dy, hw * hw);
}

void orc_lod_counts(float Lf, int32_t n_full, float delta, int32_t L, int32_t cmax, int32_t *n, int32_t *c) {
    lod_counts(Lf, n_full, delta, L, cmax, n, c);
}
