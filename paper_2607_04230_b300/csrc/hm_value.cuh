// hm_value.cuh -- the continuous ("value") part of the deferred resolve,
// shared by the forward resolve and its adjoint: the shading model (Sec. 3.4)
// and the normalized elliptical bilateral sum with strip hit counts
// (Sec. 3.3.1-3.3.3).  Masks inside come from the exact decision layer in
// hm_device.cuh; the arithmetic here is ordinary FP32 (FMA allowed).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "hm_device.cuh"
#include "hm_kernels.h"

namespace hm {

constexpr int kTileW = 32, kTileH = 16;
constexpr int kResolveThreads = kTileW * kTileH;

// Ambient occlusion at the decoded pixel: the segment's two control points
// interpolated at t.
__device__ __forceinline__ float decoded_ao(const GroomDev &g, const Decoded &d) {
    if (!g.has_ao) return 1.0f;
    const Root r = make_root(g, d.s, __ldg(&g.sface[d.s]));
    const float a = control_ao(g, r, d.C, d.j), b = control_ao(g, r, d.C, d.j + 1);
    return a + (b - a) * d.t;
}

// Shading (Sec. 3.4) with the ambient term darkened by the baked ambient
// occlusion ao.
// Fraction beta = N_LOD / N of the receiver's bundle drawn at the current
// LOD (Sec. 3.2 depth fix); 1 when no shadow map is bound.
__device__ __forceinline__ float receiver_beta(const GroomDev &g, const LightsDev &Ls, int64_t s) {
    if (Ls.n_shadow == 0) return 1.0f;
    const uint32_t f = __ldg(&g.sface[s]);
    const int n = __ldg(&g.faces[f + 1]).w - __ldg(&g.faces[f]).w;
    const uint32_t nl = g.lod[f].x;
    return n > 0 ? __fdiv_rn((float)nl, (float)n) : 1.0f;
}

// Light reaching X through a shadow map: Beer-Lambert exp(-sigma beta d)
// over the depth d travelled past the map's front-most hair (Sec. 3.2: the
// LOD's strand fraction beta shifts log depth by -log beta).  The texel is
// the one under X's snapped projection, a decision taken in the same
// binary32 operations as the rasterizer's projection.  *dvis_dw receives
// dV/dw (w the light-view depth of X) for the adjoint.
__device__ __forceinline__ float shadow_visibility(const ShadowDev &m, float3 X, float beta, float *dvis_dw) {
    *dvis_dw = 0.0f;
    const Proj P = project(m.cam, X);
    if (!P.valid) return 1.0f;
    const int32_t tx = P.X >> 8, ty = P.Y >> 8;
    if (tx < 0 || ty < 0 || tx >= m.cam.W || ty >= m.cam.H) return 1.0f;
    const uint64_t key = __ldg(reinterpret_cast<const unsigned long long *>(m.map) + key_index(m.cam, tx, ty));
    if (key_empty(key)) return 1.0f;
    const float zmap = (float)(uint32_t)(key >> 40) * (1.0f / 16777216.0f);
    const float d = (P.w - m.cam.near_m) - zmap * (m.cam.far_m - m.cam.near_m) - m.bias;
    if (!(d > 0.0f)) return 1.0f;
    const float k = m.sigma * (m.corr ? beta : 1.0f);
    const float v = __expf(-k * d);
    *dvis_dw = -k * v;
    return v;
}

__device__ __forceinline__ float3 shade(float3 X, float3 T, float3 alb, const CamDev &cam, const LightsDev &Ls,
                                        float rough, float tilt, float ao, float beta) {
    float3 V = make_float3(cam.cam_pos[0] - X.x, cam.cam_pos[1] - X.y, cam.cam_pos[2] - X.z);
    float vn = rsqrtf(fmaxf(V.x * V.x + V.y * V.y + V.z * V.z, 1e-30f));
    V = make_float3(V.x * vn, V.y * vn, V.z * vn);
    const float sa = sinf(tilt);
    const float inv2b2 = 1.0f / (2.0f * rough * rough);
    const float amb = Ls.ambient * ao;
    float3 out = make_float3(amb * alb.x, amb * alb.y, amb * alb.z);
    for (int l = 0; l < Ls.n; ++l) {
        const float tl = T.x * Ls.dir[l][0] + T.y * Ls.dir[l][1] + T.z * Ls.dir[l][2];
        const float tv = T.x * V.x + T.y * V.y + T.z * V.z;
        const float sin2 = 1.0f - tl * tl;
        const float kk = Ls.kd * (sin2 > 0.0f ? sqrtf(sin2) : 0.0f);
        const float u = (tl + tv) * 0.5f + sa;
        const float fs = Ls.ks * __expf(-(u * u) * inv2b2);
        float vis = 1.0f;
        if (Ls.shadow_of[l] >= 0) {
            float dvw;
            vis = shadow_visibility(Ls.sh[Ls.shadow_of[l]], X, beta, &dvw);
        }
        out.x += vis * (Ls.rad[l][0] * (alb.x * kk + fs));
        out.y += vis * (Ls.rad[l][1] * (alb.y * kk + fs));
        out.z += vis * (Ls.rad[l][2] * (alb.z * kk + fs));
    }
    return out;
}

struct Recon {
    float3 S;       // sum of w' C over contributing neighbours
    float W;        // sum of w', where w' = w / max w (so W >= 1 when cnt > 0)
    float m;        // exponent of the largest weight: max w = exp(-m)
    int cnt;        // contributing neighbours (exact)
    int hc, ha;     // strip hit counts
};

// Exponent e of the bilateral weight w = exp(-e) of offset (dx, dy) (Eq. 7):
// elliptical spatial term, or the isotropic fallback, plus the colour term.
__device__ __forceinline__ float weight_exponent(bool iso, int dx, int dy, float dpar, float perp2, bool use_color,
                                                 float3 Cp, float3 cq, const FilterDev &fp) {
    float e = iso ? (float)(dx * dx + dy * dy) * fp.inv_siso2 : (dpar * dpar) * fp.inv_spar2 + perp2 * fp.inv_sperp2;
    if (use_color) {
        const float ex = Cp.x - cq.x, ey = Cp.y - cq.y, ez = Cp.z - cq.z;
        e += (ex * ex + ey * ey + ez * ez) * fp.inv_sc2;
    }
    return e;
}

// Staged centre-layer depth of tap i: a separate int array, or the depth
// bits packed into the colour record's w.
__device__ __forceinline__ int tap_depth(const int *s_dg, const float3 *, int i) { return s_dg[i]; }
__device__ __forceinline__ int tap_depth(const int *, const float4 *s_col, int i) { return __float_as_int(s_col[i].w); }

// Strip hit counts H_center, H_cons of Sec. 3.3.3 over the window: taps
// within the strip |d - (d.Ts) Ts| <= hw of the screen tangent (the pixel
// alone for a degenerate tangent).  Only the taps that can be in the strip
// are visited: with the tangent's major axis as k, a tap (k, m) is within
// hw of the line iff |m - k slope| <= hw / |major component| <= hw sqrt(2),
// so per k at most the integers of [k slope - hw sqrt(2) - 0.01,
// k slope + hw sqrt(2) + 0.01] are candidates (0.01 px covers the binary32
// rounding of slope and of the test); each candidate then takes the exact
// test of in_strip, so the counts equal a full-window scan.
__device__ __forceinline__ int2 strip_counts(const int *s_dg, const uint8_t *s_fa, int sw, int lx, int ly, int R,
                                             float tsx, float tsy, bool iso, const FilterDev &fp) {
    int hc = 0, ha = 0;
    if (iso) {
        const int idx = (ly + R) * sw + lx + R;
        return make_int2(s_dg[idx] >= 0 ? 1 : 0, s_fa[idx] ? 1 : 0);
    }
    const bool xmaj = fabsf(tsx) >= fabsf(tsy);
    const float slope = xmaj ? tsy / tsx : tsx / tsy;
    const float half = fp.hw * 1.41422f + 0.01f;
    if (half < 1.0f) {
        // a range narrower than 2 holds at most two integers: m0 and m0 + 1,
        // evaluated without a data-dependent loop (the paper's 0.5 px strip)
#pragma unroll
        for (int k = -R; k <= R; ++k) {
            const float c = (float)k * slope;
            const int m0 = (int)ceilf(c - half), m1 = (int)floorf(c + half);
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                const int m = m0 + j;
                const bool cand = m <= m1 && m >= -R && m <= R;
                const int mc = min(max(m, -R), R);
                const int dx = xmaj ? k : mc, dy = xmaj ? mc : k;
                float dpar, perp2;
                const bool in = cand && in_strip(false, tsx, tsy, dx, dy, fp.hw2, dpar, perp2);
                const int idx = (ly + dy + R) * sw + lx + dx + R;
                hc += (in && s_dg[idx] >= 0) ? 1 : 0;
                ha += (in && s_fa[idx]) ? 1 : 0;
            }
        }
        return make_int2(hc, ha);
    }
    for (int k = -R; k <= R; ++k) {
        const float c = (float)k * slope;
        const int m0 = max((int)ceilf(c - half), -R), m1 = min((int)floorf(c + half), R);
        for (int m = m0; m <= m1; ++m) {
            const int dx = xmaj ? k : m, dy = xmaj ? m : k;
            float dpar, perp2;
            if (!in_strip(false, tsx, tsy, dx, dy, fp.hw2, dpar, perp2)) continue;
            const int idx = (ly + dy + R) * sw + lx + dx + R;
            hc += s_dg[idx] >= 0 ? 1 : 0;
            ha += s_fa[idx] ? 1 : 0;
        }
    }
    return make_int2(hc, ha);
}

__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Bilateral reconstruction of one pixel (Eq. 7).  The spatial exponent is
// written as dpar^2 (1/s_par^2 - 1/s_perp^2) + |d|^2 / s_perp^2
// (perp^2 = |d|^2 - dpar^2), which with the isotropic coefficients
// (0, 1/s_iso^2) and a zero tangent is the isotropic exponent, so one loop
// serves both modes; exponents are scaled by log2(e) for ex2.
// The depth test |d_Q - ref| <= D_rej of Eq. 7's contributors (integer, on
// the staged centre depths s_dg, one 4-byte word per tap so a warp's loads
// hit distinct banks; empty centre-layer taps hold a large negative depth, so
// the test alone rejects them) first builds a bit mask per window
// row, then only the contributing taps are weighted and summed, in (dy, dx)
// order: most windows hold few contributors (a sparse crowd's
// centre-referenced windows about 2 of 121, a close-up's 12).
//  - centre reference (kColor): the pixel itself contributes with exponent 0
//    (zero offset, same depth, same colour) and every exponent is >= 0, so
//    the weights are summed unscaled: each is <= 1 and the sum is >= 1;
//  - conservative reference: the weights are summed unscaled too; when that
//    sum underflows (every contributor far off the strand axis: W < 1e-20)
//    they are summed again relative to the largest, exp(e_min - e) with
//    e_min the smallest exponent of a contributor (m = e_min), so the sum is
//    >= 1 however far off the axis the contributors lie.
template <int R, bool kColor>
__device__ __forceinline__ Recon reconstruct_fast(const int *s_dg, const uint8_t *s_fa, const float4 *s_col, int sw,
                                                  int lx, int ly, int ref, float tsx, float tsy, bool iso, float3 Cp,
                                                  const FilterDev &fp) {
    constexpr float kL2e = 1.4426950408889634f;
    constexpr int D = 2 * R + 1;
    const float a = iso ? 0.0f : (fp.inv_spar2 - fp.inv_sperp2) * kL2e;
    const float b = (iso ? fp.inv_siso2 : fp.inv_sperp2) * kL2e;
    const float c = fp.inv_sc2 * kL2e;
    const float ux = iso ? 0.0f : tsx, uy = iso ? 0.0f : tsy;
    // |dq - ref| <= drej  <=>  (unsigned)(dq - ref + drej) <= 2 drej (no
    // overflow: depths are in [0, 2^24) or -2^30)
    const int lo = fp.drej - ref;
    const unsigned span = 2u * (unsigned)fp.drej;
    const int base = (ly + R) * sw + lx + R;      // the pixel's own staged index
    uint32_t mk[D];
    int cnt = 0;
#pragma unroll
    for (int r = 0; r < D; ++r) {
        const int row = base + (r - R) * sw;
        uint32_t m = 0;
#pragma unroll
        for (int dx = -R; dx <= R; ++dx) {
            const int dq = s_dg[row + dx];                          // staged centre depth
            m |= ((unsigned)(dq + lo) <= span ? 1u : 0u) << (dx + R);
        }
        mk[r] = m;
        cnt += __popc(m);
    }
    // exponent (log2 units) of contributor (dx, dy)
    auto expo = [&](int dx, int dy, const float4 &cq) {
        const float dpar = fmaf((float)dx, ux, (float)dy * uy);
        float e = fmaf(dpar * a, dpar, fmaf((float)(dx * dx), b, (float)(dy * dy) * b));
        if (kColor) {
            const float ex = Cp.x - cq.x, ey = Cp.y - cq.y, ez = Cp.z - cq.z;
            e = fmaf(fmaf(ex, ex, fmaf(ey, ey, ez * ez)), c, e);
        }
        return e;
    };
    float Sx = 0.f, Sy = 0.f, Sz = 0.f, Wt = 0.f;
    auto accumulate = [&](float emin) {
        Sx = Sy = Sz = Wt = 0.f;
#pragma unroll
        for (int r = 0; r < D; ++r) {
            uint32_t m = mk[r];
            while (m) {
                const int k = __ffs(m) - 1;
                m &= m - 1;
                const int dx = k - R;
                const float4 cq = s_col[base + (r - R) * sw + dx];
                const float w = ex2_approx(emin - expo(dx, r - R, cq));
                Sx = fmaf(w, cq.x, Sx);
                Sy = fmaf(w, cq.y, Sy);
                Sz = fmaf(w, cq.z, Sz);
                Wt += w;
            }
        }
    };
    accumulate(0.0f);
    float emin = 0.0f;
    if (!kColor && cnt > 0 && Wt < 1e-20f) {
        emin = __int_as_float(0x7f800000);
#pragma unroll
        for (int r = 0; r < D; ++r) {
            uint32_t m = mk[r];
            while (m) {
                const int k = __ffs(m) - 1;
                m &= m - 1;
                const int dx = k - R;
                emin = fminf(emin, expo(dx, r - R, s_col[base + (r - R) * sw + dx]));
            }
        }
        accumulate(emin);
    }
    const int2 h = strip_counts(s_dg, s_fa, sw, lx, ly, R, tsx, tsy, iso, fp);
    Recon o;
    o.S = make_float3(Sx, Sy, Sz);
    o.W = Wt;
    o.m = emin * (1.0f / kL2e);   // natural-log units: max weight = exp(-m)
    o.cnt = cnt;
    o.hc = h.x;
    o.ha = h.y;
    return o;
}

// reconstruct_fast<R, kColor> for a runtime radius 0..HM_MAX_FILTER_RADIUS.
template <bool kColor>
__device__ __forceinline__ Recon reconstruct_fast_r(int R, const int *s_dg, const uint8_t *s_fa, const float4 *s_col,
                                                    int sw, int lx, int ly, int ref, float tsx, float tsy, bool iso,
                                                    float3 Cp, const FilterDev &fp) {
    switch (R) {
#define HM_RF(r) \
    case r: return reconstruct_fast<r, kColor>(s_dg, s_fa, s_col, sw, lx, ly, ref, tsx, tsy, iso, Cp, fp);
        HM_RF(0) HM_RF(1) HM_RF(2) HM_RF(3) HM_RF(4) HM_RF(5) HM_RF(6) HM_RF(7)
#undef HM_RF
        default: return reconstruct_fast<8, kColor>(s_dg, s_fa, s_col, sw, lx, ly, ref, tsx, tsy, iso, Cp, fp);
    }
}

}  // namespace hm
