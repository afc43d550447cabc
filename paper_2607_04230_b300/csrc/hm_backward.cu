// hm_backward.cu -- adjoint of the deferred resolve (shading + strand
// connection / bilateral filter) with visibility held fixed: the keys, the
// pixel-centre projection parameters and every filter mask and strip count
// are the forward's, so alpha is constant.  Gradients flow to the hair-mesh
// layer vertices (through the pixel position, tangent and screen tangent of
// every decoded strand segment: interpolation, styled tangents, Hermite
// control points, base-spline tangents and chord lengths, barycentric layer
// points) and to the per-strand albedo.
//
// Kernel 1 (tiles, as the forward): recompute the staged colours and each
// tile pixel's reconstruction, then push dL/dC of every contributing
// neighbour into a per-pixel colour-gradient buffer, and dL/d(screen
// tangent) of the pixel's reference segment straight into the geometry.
// Kernel 2 (keys): every key with a gradient (a centre key with a colour or
// screen-tangent gradient, a conservative key with a screen-tangent
// gradient), compacted into job lists per pixel chunk: shading and
// screen-tangent adjoints chained through the strand geometry to the layer
// vertices, plus the albedo gradient.
#include <cstdint>
#include <cuda_runtime.h>

#include "hm_device.cuh"
#include "hm_kernels.h"
#include "hm_value.cuh"

namespace hm {

__device__ __forceinline__ float3 f3(float x, float y, float z) { return make_float3(x, y, z); }
__device__ __forceinline__ float3 add3(float3 a, float3 b) { return f3(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ __forceinline__ float3 sub3(float3 a, float3 b) { return f3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ float3 mul3(float3 a, float k) { return f3(a.x * k, a.y * k, a.z * k); }
__device__ __forceinline__ float dot3(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ float len3(float3 a) { return sqrtf(dot3(a, a)); }

// v -> v / |v|: given the unit result u = v/|v|, |v| and dL/du, dL/dv.
__device__ __forceinline__ float3 unit_adjoint(float3 u, float len, float3 du) {
    if (len == 0.0f) return f3(0.f, 0.f, 0.f);
    return mul3(sub3(du, mul3(u, dot3(u, du))), 1.0f / len);
}

struct Sink {
    float *glv;              // [L][V][3] (global, or this CTA's shared copy) or NULL
    int V;
};

__device__ __forceinline__ void scatter_layer_point(const Sink &sk, const Root &r, int k, float3 dP) {
    if (!sk.glv || (dP.x == 0.f && dP.y == 0.f && dP.z == 0.f)) return;
    float *row = sk.glv + (int64_t)k * sk.V * 3;   // atomicAdd works on either address space
    const int idx[3] = {r.i0, r.i1, r.i2};
    const float b[3] = {r.b0, r.b1, r.b2};
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        float *p = row + 3 * idx[c];
        atomicAdd(p + 0, b[c] * dP.x);
        atomicAdd(p + 1, b[c] * dP.y);
        atomicAdd(p + 2, b[c] * dP.z);
    }
}

// Adjoint of control point j (Hermite with chord-scaled finite-difference
// tangents) to its layer points and on to the layer vertices.
__device__ __noinline__ void control_point_adjoint(const GroomDev &g, const Root &r, int C, int j, float3 dp,
                                                   const Sink &sk) {
    if (dp.x == 0.f && dp.y == 0.f && dp.z == 0.f) return;
    const int L = g.L;
    const int x = j * (L - 1);
    int k = x / (C - 1);
    if (k > L - 2) k = L - 2;
    const float s = (float)(x - k * (C - 1)) / (float)(C - 1);
    const float3 P0 = layer_pt(g, r, k);
    const float3 P1 = layer_pt(g, r, k + 1);
    const bool hm_ = k > 0, hp = k + 2 <= L - 1;
    const float3 Pm = hm_ ? layer_pt(g, r, k - 1) : P0;
    const float3 P2 = hp ? layer_pt(g, r, k + 2) : P1;
    const float3 v0 = (k == 0) ? sub3(P1, P0) : sub3(P1, Pm);
    const float3 v1 = (k + 1 == L - 1) ? sub3(P1, P0) : sub3(P2, P0);
    const float n0 = len3(v0), n1 = len3(v1);
    const float3 t0 = n0 > 0.f ? mul3(v0, 1.f / n0) : f3(0.f, 0.f, 0.f);
    const float3 t1 = n1 > 0.f ? mul3(v1, 1.f / n1) : f3(0.f, 0.f, 0.f);
    const float3 ch = sub3(P1, P0);
    const float ell = len3(ch);
    const float s2 = s * s, s3 = s2 * s;
    const float h00 = 2.f * s3 - 3.f * s2 + 1.f, h10 = s3 - 2.f * s2 + s;
    const float h01 = 3.f * s2 - 2.f * s3, h11 = s3 - s2;
    float3 dP0 = mul3(dp, h00), dP1 = mul3(dp, h01), dPm = f3(0.f, 0.f, 0.f), dP2 = f3(0.f, 0.f, 0.f);
    const float dell = h10 * dot3(t0, dp) + h11 * dot3(t1, dp);
    if (ell > 0.f) {
        const float3 e = mul3(ch, dell / ell);
        dP1 = add3(dP1, e);
        dP0 = sub3(dP0, e);
    }
    const float3 dv0 = unit_adjoint(t0, n0, mul3(dp, h10 * ell));
    if (k == 0) {
        dP1 = add3(dP1, dv0);
        dP0 = sub3(dP0, dv0);
    } else {
        dP1 = add3(dP1, dv0);
        dPm = sub3(dPm, dv0);
    }
    const float3 dv1 = unit_adjoint(t1, n1, mul3(dp, h11 * ell));
    if (k + 1 == L - 1) {
        dP1 = add3(dP1, dv1);
        dP0 = sub3(dP0, dv1);
    } else {
        dP2 = add3(dP2, dv1);
        dP0 = sub3(dP0, dv1);
    }
    scatter_layer_point(sk, r, k, dP0);
    scatter_layer_point(sk, r, k + 1, dP1);
    if (hm_) scatter_layer_point(sk, r, k - 1, dPm);
    if (hp) scatter_layer_point(sk, r, k + 2, dP2);
}

// Adjoint of control points j-1 .. j+2 (dp[c] for point j-1+c; points
// outside [0, C-1] and zero gradients are skipped).  When their layer
// intervals span at most three consecutive intervals, the six layer points
// they read are evaluated once, the four control points' layer-point
// gradients are summed in registers, and each layer point is scattered to
// its vertices once (instead of once per control point); otherwise each
// control point takes control_point_adjoint on its own.
__device__ __forceinline__ float3 pick6(const float3 (&P)[6], int i) {
    float3 v = P[0];
#pragma unroll
    for (int w = 1; w < 6; ++w)
        if (i == w) v = P[w];
    return v;
}

__device__ void control_points_adjoint(const GroomDev &g, const Root &r, int C, int j, const float3 (&dp)[4],
                                       const Sink &sk) {
    const int L = g.L;
    int kc[4];
    float sc[4];
    bool v[4];
    int kmin = L, kmax = -1;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        const int i = j - 1 + c;
        v[c] = i >= 0 && i <= C - 1 && (dp[c].x != 0.f || dp[c].y != 0.f || dp[c].z != 0.f);
        const int x = i * (L - 1);
        int k = v[c] ? x / (C - 1) : 0;
        if (k > L - 2) k = L - 2;
        kc[c] = k;
        sc[c] = (float)(x - k * (C - 1)) / (float)(C - 1);
        if (v[c]) {
            kmin = min(kmin, k);
            kmax = max(kmax, k);
        }
    }
    if (kmax < 0) return;
    if (kmax - kmin > 2) {
#pragma unroll
        for (int c = 0; c < 4; ++c)
            if (v[c]) control_point_adjoint(g, r, C, j - 1 + c, dp[c], sk);
        return;
    }
    const int base = kmin - 1;     // layer of window slot 0
    float3 P[6], acc[6];
#pragma unroll
    for (int w = 0; w < 6; ++w) {
        const int layer = base + w;
        P[w] = (layer >= 0 && layer <= L - 1 && layer <= kmax + 2) ? layer_pt(g, r, layer) : f3(0.f, 0.f, 0.f);
        acc[w] = f3(0.f, 0.f, 0.f);
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        if (!v[c]) continue;
        const int k = kc[c], o = k - kmin;      // slots o .. o+3 hold layers k-1 .. k+2
        const float s = sc[c];
        const float3 P0 = pick6(P, o + 1), P1 = pick6(P, o + 2);
        const float3 Pm = k > 0 ? pick6(P, o) : P0;
        const float3 P2 = k + 2 <= L - 1 ? pick6(P, o + 3) : P1;
        const float3 v0 = (k == 0) ? sub3(P1, P0) : sub3(P1, Pm);
        const float3 v1 = (k + 1 == L - 1) ? sub3(P1, P0) : sub3(P2, P0);
        const float n0 = len3(v0), n1 = len3(v1);
        const float3 t0 = n0 > 0.f ? mul3(v0, 1.f / n0) : f3(0.f, 0.f, 0.f);
        const float3 t1 = n1 > 0.f ? mul3(v1, 1.f / n1) : f3(0.f, 0.f, 0.f);
        const float3 ch = sub3(P1, P0);
        const float ell = len3(ch);
        const float s2 = s * s, s3 = s2 * s;
        const float h00 = 2.f * s3 - 3.f * s2 + 1.f, h10 = s3 - 2.f * s2 + s;
        const float h01 = 3.f * s2 - 2.f * s3, h11 = s3 - s2;
        const float3 d = dp[c];
        float3 dP0 = mul3(d, h00), dP1 = mul3(d, h01), dPm = f3(0.f, 0.f, 0.f), dP2 = f3(0.f, 0.f, 0.f);
        const float dell = h10 * dot3(t0, d) + h11 * dot3(t1, d);
        if (ell > 0.f) {
            const float3 e = mul3(ch, dell / ell);
            dP1 = add3(dP1, e);
            dP0 = sub3(dP0, e);
        }
        const float3 dv0 = unit_adjoint(t0, n0, mul3(d, h10 * ell));
        dP1 = add3(dP1, dv0);
        if (k == 0) dP0 = sub3(dP0, dv0);
        else dPm = sub3(dPm, dv0);
        const float3 dv1 = unit_adjoint(t1, n1, mul3(d, h11 * ell));
        dP0 = sub3(dP0, dv1);
        if (k + 1 == L - 1) dP1 = add3(dP1, dv1);
        else dP2 = add3(dP2, dv1);
#pragma unroll
        for (int oo = 0; oo < 3; ++oo) {
            if (o != oo) continue;
            acc[oo] = add3(acc[oo], dPm);
            acc[oo + 1] = add3(acc[oo + 1], dP0);
            acc[oo + 2] = add3(acc[oo + 2], dP1);
            acc[oo + 3] = add3(acc[oo + 3], dP2);
        }
    }
#pragma unroll
    for (int w = 0; w < 6; ++w) {
        const int layer = base + w;
        if (layer >= 0 && layer <= L - 1) scatter_layer_point(sk, r, layer, acc[w]);
    }
}

// Adjoint of the pixel position X = p_j + (p_{j+1} - p_j) t and unit tangent
// T = unit(T_j + (T_{j+1} - T_j) t), t fixed, to the control points.
__device__ void geometry_adjoint(const GroomDev &g, const Root &r, uint32_t f, int64_t s, int C, int j, float t,
                                 float3 dX, float3 dT, const Sink &sk) {
    float3 cp[4];
    if (g.segpts)    // a decoded key's strand is drawn (checked by the decode)
        recorded_points4(g, f, (uint32_t)(s - (int64_t)__ldg(&g.faces[f]).w), C, j, cp);
    else
        control_pts<4>(g, r, C, j - 1, cp);
    const bool has_m = j >= 1, has_p = j + 2 <= C - 1;
    const float3 pm = cp[0], p0 = cp[1], p1 = cp[2], pp = cp[3];
    const float3 va = (j == 0) ? sub3(p1, p0) : sub3(p1, pm);
    const float3 vb = (j + 1 == C - 1) ? sub3(p1, p0) : sub3(pp, p0);
    const float na = len3(va), nb = len3(vb);
    const float3 Ta = na > 0.f ? mul3(va, 1.f / na) : f3(0.f, 0.f, 0.f);
    const float3 Tb = nb > 0.f ? mul3(vb, 1.f / nb) : f3(0.f, 0.f, 0.f);
    const float3 Tm = add3(Ta, mul3(sub3(Tb, Ta), t));
    const float nm = len3(Tm);
    const float3 T = nm > 0.f ? mul3(Tm, 1.f / nm) : f3(0.f, 0.f, 0.f);
    const float3 dTm = unit_adjoint(T, nm, dT);
    const float3 dTa = mul3(dTm, 1.f - t), dTb = mul3(dTm, t);
    float3 dp0 = mul3(dX, 1.f - t), dp1 = mul3(dX, t), dpm = f3(0.f, 0.f, 0.f), dpp = f3(0.f, 0.f, 0.f);
    const float3 dva = unit_adjoint(Ta, na, dTa);
    if (j == 0) {
        dp1 = add3(dp1, dva);
        dp0 = sub3(dp0, dva);
    } else {
        dp1 = add3(dp1, dva);
        dpm = sub3(dpm, dva);
    }
    const float3 dvb = unit_adjoint(Tb, nb, dTb);
    if (j + 1 == C - 1) {
        dp1 = add3(dp1, dvb);
        dp0 = sub3(dp0, dvb);
    } else {
        dpp = add3(dpp, dvb);
        dp0 = sub3(dp0, dvb);
    }
    const float3 dps[4] = {has_m ? dpm : f3(0.f, 0.f, 0.f), dp0, dp1, has_p ? dpp : f3(0.f, 0.f, 0.f)};
    control_points_adjoint(g, r, C, j, dps, sk);
}

// Adjoint of the screen tangent Ts = J T / |J T| at X (J: Jacobian of the
// pixel position with respect to the world position).
__device__ void screen_tangent_adjoint(const CamDev &cam, float3 X, float3 T, float2 dTs, float3 &dX, float3 &dT) {
    const float *m = cam.m;
    const float3 M0 = f3(m[0], m[1], m[2]), M1 = f3(m[4], m[5], m[6]), M3 = f3(m[12], m[13], m[14]);
    const float c0 = dot3(M0, X) + m[3], c1 = dot3(M1, X) + m[7], w = dot3(M3, X) + m[15];
    const float a0 = dot3(M0, T), a1 = dot3(M1, T), a3 = dot3(M3, T);
    const float hw = 0.5f * (float)cam.W, hh = 0.5f * (float)cam.H;
    const float iw = 1.f / w, iw2 = iw * iw, iw3 = iw2 * iw;
    const float jx = hw * (a0 * iw - c0 * a3 * iw2);
    const float jy = -hh * (a1 * iw - c1 * a3 * iw2);
    const float n = sqrtf(jx * jx + jy * jy);
    dX = f3(0.f, 0.f, 0.f);
    dT = f3(0.f, 0.f, 0.f);
    if (n == 0.f) return;
    const float tx = jx / n, ty = jy / n;
    const float k = tx * dTs.x + ty * dTs.y;
    const float djx = (dTs.x - tx * k) / n, djy = (dTs.y - ty * k) / n;
    // d jx / d T, d jy / d T
    dT = add3(mul3(sub3(mul3(M0, iw), mul3(M3, c0 * iw2)), djx * hw),
              mul3(sub3(mul3(M1, iw), mul3(M3, c1 * iw2)), -djy * hh));
    // d jx / d X = hw (-a0 iw2 M3 - a3 iw2 M0 + 2 c0 a3 iw3 M3), same for jy with -hh, a1, c1, M1
    const float3 gx = add3(mul3(M3, -a0 * iw2 + 2.f * c0 * a3 * iw3), mul3(M0, -a3 * iw2));
    const float3 gy = add3(mul3(M3, -a1 * iw2 + 2.f * c1 * a3 * iw3), mul3(M1, -a3 * iw2));
    dX = add3(mul3(gx, djx * hw), mul3(gy, -djy * hh));
}

// Adjoint of the shading model (Sec. 3.4) at one pixel.
__device__ void shade_adjoint(float3 X, float3 T, float3 alb, const CamDev &cam, const LightsDev &Ls, float rough,
                              float tilt, float ao, float beta, float3 dC, float3 &dX, float3 &dT, float3 &dalb) {
    const float3 Vr = f3(cam.cam_pos[0] - X.x, cam.cam_pos[1] - X.y, cam.cam_pos[2] - X.z);
    const float vl = len3(Vr);
    const float3 V = vl > 0.f ? mul3(Vr, 1.f / vl) : f3(0.f, 0.f, 0.f);
    const float sa = sinf(tilt);
    const float b2 = rough * rough;
    dalb = mul3(dC, Ls.ambient * ao);
    dT = f3(0.f, 0.f, 0.f);
    float3 dV = f3(0.f, 0.f, 0.f);
    float3 dXs = f3(0.f, 0.f, 0.f);       // through the shadow maps' receiver depth
    for (int l = 0; l < Ls.n; ++l) {
        const float3 Ld = f3(Ls.dir[l][0], Ls.dir[l][1], Ls.dir[l][2]);
        const float tl = dot3(T, Ld), tv = dot3(T, V);
        const float sin2 = 1.f - tl * tl;
        const float sq = sin2 > 0.f ? sqrtf(sin2) : 0.f;
        const float u = (tl + tv) * 0.5f + sa;
        const float fs = Ls.ks * __expf(-(u * u) / (2.f * b2));
        float vis = 1.f;
        if (Ls.shadow_of[l] >= 0) {
            const ShadowDev &m = Ls.sh[Ls.shadow_of[l]];
            float dvw;
            vis = shadow_visibility(m, X, beta, &dvw);
            if (dvw != 0.f) {
                // d(out)/dw = dvw E (alb kk + fs), w = row 3 of the light's view_proj . (X, 1)
                const float kk = Ls.kd * sq;
                const float g = dvw * (dC.x * Ls.rad[l][0] * (alb.x * kk + fs) + dC.y * Ls.rad[l][1] * (alb.y * kk + fs) +
                                       dC.z * Ls.rad[l][2] * (alb.z * kk + fs));
                dXs = add3(dXs, f3(g * m.cam.m[12], g * m.cam.m[13], g * m.cam.m[14]));
            }
        }
        const float3 gE = f3(vis * dC.x * Ls.rad[l][0], vis * dC.y * Ls.rad[l][1], vis * dC.z * Ls.rad[l][2]);
        dalb = add3(dalb, mul3(gE, Ls.kd * sq));
        const float dsq = Ls.kd * dot3(gE, alb);
        const float dfs = gE.x + gE.y + gE.z;
        float dtl = sq > 0.f ? -dsq * tl / sq : 0.f;
        const float du = dfs * fs * (-u / b2);
        dtl += 0.5f * du;
        const float dtv = 0.5f * du;
        dT = add3(dT, add3(mul3(Ld, dtl), mul3(V, dtv)));
        dV = add3(dV, mul3(T, dtv));
    }
    dX = add3(mul3(unit_adjoint(V, vl, dV), -1.f), dXs);
}

struct BwdSinks {
    float *glv[HM_MAX_GROOMS_PER_CALL];
    float *galb[HM_MAX_GROOMS_PER_CALL];
};

// Adjoint of one normalized reconstruction R = sum w C / sum w given
// dL/dR: colour gradients of the contributing neighbours (and of the centre
// colour through the colour term) into s_dC, returns dL/d(screen tangent).
template <typename ColT>
__device__ __forceinline__ float2 reconstruct_adjoint(const int *s_dg, const ColT *s_col, float3 *s_dC, int sw,
                                                      int lx, int ly, int gx, int gy, int W, int H, int R, int ref,
                                                      float tsx, float tsy, bool iso, bool use_color, float3 Cp,
                                                      int mid, const Recon &rc, float3 gR, const FilterDev &fp) {
    float2 dTs = make_float2(0.f, 0.f);
    if (rc.cnt == 0) return dTs;
    const float invW = 1.0f / rc.W;
    const float3 Rv = mul3(rc.S, invW);
    float3 dCp = f3(0.f, 0.f, 0.f);
    for (int dy = -R; dy <= R; ++dy) {
        const int qy = gy + dy;
        if (qy < 0 || qy >= H) continue;
        const int row = (ly + dy + R) * sw + R + lx;
        for (int dx = -R; dx <= R; ++dx) {
            const int qx = gx + dx;
            if (qx < 0 || qx >= W) continue;
            const int idx = row + dx;
            const int dq = tap_depth(s_dg, s_col, idx);
            if (dq < 0 || abs(dq - ref) > fp.drej) continue;
            float dpar, perp2;
            in_strip(iso, tsx, tsy, dx, dy, fp.hw2, dpar, perp2);
            const float3 cq = make_float3(s_col[idx].x, s_col[idx].y, s_col[idx].z);
            const float e = weight_exponent(iso, dx, dy, dpar, perp2, use_color, Cp, cq, fp);
            const float om = __expf(rc.m - e) * invW;      // normalized weight
            const float3 dcq = mul3(gR, om);
            // dR/de_Q = -om (C_Q - R)
            const float de = -om * dot3(gR, sub3(cq, Rv));
            float3 dq3 = dcq;
            if (!iso) {
                // e_spatial = dpar^2 / s_par^2 + (|d|^2 - dpar^2) / s_perp^2, dpar = d . Ts
                const float k = de * 2.f * dpar * (fp.inv_spar2 - fp.inv_sperp2);
                dTs.x += k * (float)dx;
                dTs.y += k * (float)dy;
            }
            if (use_color) {
                const float3 dd = mul3(sub3(Cp, cq), 2.f * fp.inv_sc2 * de);
                dCp = add3(dCp, dd);
                dq3 = sub3(dq3, dd);
            }
            atomicAdd(&s_dC[idx].x, dq3.x);
            atomicAdd(&s_dC[idx].y, dq3.y);
            atomicAdd(&s_dC[idx].z, dq3.z);
        }
    }
    if (use_color) {
        atomicAdd(&s_dC[mid].x, dCp.x);
        atomicAdd(&s_dC[mid].y, dCp.y);
        atomicAdd(&s_dC[mid].z, dCp.z);
    }
    return dTs;
}

__global__ void __launch_bounds__(kResolveThreads, 2) resolve_adjoint_kernel(
    CallTable tab, CamDev cam, LightsDev Ls, FilterDev fp, const uint64_t *__restrict__ vis_c,
    const uint64_t *__restrict__ vis_a, const float4 *__restrict__ grad_rgba, float4 *__restrict__ dC,
    float4 *__restrict__ dTs, uint32_t *status, int *list) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int R = fp.enabled ? fp.radius : 0;
    const int sw = kTileW + 2 * R, sh = kTileH + 2 * R, ns = sw * sh;
    uint64_t *s_bases = reinterpret_cast<uint64_t *>(smem);
    float4 *s_col = reinterpret_cast<float4 *>(
        (reinterpret_cast<uintptr_t>(s_bases + HM_MAX_GROOMS_PER_CALL + 1) + 15) & ~(uintptr_t)15);  // rgb, centre depth bits
    float3 *s_dC = reinterpret_cast<float3 *>(s_col + ns);
    uint16_t *s_list = reinterpret_cast<uint16_t *>(s_dC + ns);
    auto dg_at = [&](int i) { return __float_as_int(s_col[i].w); };
    float2 *s_tsG = reinterpret_cast<float2 *>(
        (reinterpret_cast<uintptr_t>(s_list + ((ns + 7) & ~7)) + 15) & ~(uintptr_t)15);
    float2 *s_tsA = s_tsG + kResolveThreads;
    uint8_t *s_isoG = reinterpret_cast<uint8_t *>(s_tsA + kResolveThreads);
    uint8_t *s_isoA = s_isoG + kResolveThreads;
    uint8_t *s_fa = s_isoA + kResolveThreads;
    int *s_dg = reinterpret_cast<int *>((reinterpret_cast<uintptr_t>(s_fa + ns) + 3) & ~(uintptr_t)3);  // centre depth
    __shared__ int s_count, s_nJA, s_nJG, s_tile;
    __shared__ float4 s_dTs[kResolveThreads];    // per tile pixel: d(screen tangent) of G (xy) and A (zw)
    __shared__ float s_gs[kResolveThreads];      // share of the pixel's gradient the centre reconstruction gets
    __shared__ int s_dAv[kResolveThreads];       // conservative-layer depth of the pixel
    __shared__ uint16_t s_jA[kResolveThreads], s_jG[kResolveThreads];

    const int tid = threadIdx.x;
    const int W = cam.W, H = cam.H;
    const int ntx = (W + kTileW - 1) / kTileW;
    const int nlisted = list[0];
    if (tid <= tab.n) {
        uint64_t b = 0;
        for (int i = 0; i < tid; ++i) b += (uint64_t)tab.g[i].S;
        s_bases[tid] = b;
    }
    // persistent: the tiles holding conservative keys, heaviest first, from
    // the work counter list[1] (a keyless tile's pixels have RGBA 0 whatever
    // their neighbours hold, so they pass no gradient)
    for (;;) {
    if (tid == 0) {
        s_tile = atomicAdd(&list[1], 1);
        s_count = 0;
        s_nJA = 0;
        s_nJG = 0;
    }
    __syncthreads();
    if (s_tile >= nlisted) break;
    const int tile = list[2 + s_tile];
    const int x0 = (tile % ntx) * kTileW, y0 = (tile / ntx) * kTileH;
    for (int i = tid; i < ns; i += kResolveThreads) {
        const int gx = x0 - R + i % sw, gy = y0 - R + i / sw;
        int dg = -(1 << 30);                 // far below any d24: the depth test alone rejects it
        uint8_t fa = 0;
        if (gx >= 0 && gx < W && gy >= 0 && gy < H) {
            const uint32_t kp = key_index(cam, gx, gy);
            const uint64_t kg = __ldg(reinterpret_cast<const unsigned long long *>(vis_c + kp));
            const uint64_t ka = __ldg(reinterpret_cast<const unsigned long long *>(vis_a + kp));
            if (!key_empty(kg)) {
                dg = (int)(kg >> 40);
                s_list[atomicAdd(&s_count, 1)] = (uint16_t)i;
            }
            fa = !key_empty(ka);
        }
        s_col[i] = make_float4(0.f, 0.f, 0.f, __int_as_float(dg));
        s_dg[i] = dg;
        s_fa[i] = fa;
        s_dC[i] = f3(0.f, 0.f, 0.f);
    }
    s_isoG[tid] = 1;
    s_isoA[tid] = 1;
    __syncthreads();
    const int ncen = s_count;
    for (int li = tid; li < ncen; li += kResolveThreads) {
        const int i = s_list[li];
        const int lx = i % sw, ly = i / sw;
        const int gx = x0 - R + lx, gy = y0 - R + ly;
        const uint64_t kg = __ldg(reinterpret_cast<const unsigned long long *>(vis_c + key_index(cam, gx, gy)));
        const Decoded d = decode_key(tab, s_bases, cam, kg, gx, gy, status);
        float3 c = f3(0.f, 0.f, 0.f);
        if (d.ok) {
            const GroomDev &g = tab.g[d.gi];
            const float4 a = __ldg(&g.albedo[d.s]);
            c = shade(d.X, d.T, f3(a.x, a.y, a.z), cam, Ls, g.roughness, g.tilt, decoded_ao(g, d),
                      receiver_beta(g, Ls, d.s));
        }
        s_col[i] = make_float4(c.x, c.y, c.z, s_col[i].w);
        const int tx = lx - R, ty = ly - R;
        if (tx >= 0 && tx < kTileW && ty >= 0 && ty < kTileH) {
            const int t = ty * kTileW + tx;
            s_tsG[t] = make_float2(d.tsx, d.tsy);
            s_isoG[t] = d.iso;
        }
    }
    __syncthreads();
    if (tid == 0) s_count = 0;
    __syncthreads();
    const int tx = tid % kTileW, ty = tid / kTileW;
    const int gx = x0 + tx, gy = y0 + ty;
    const bool inside = gx < W && gy < H;
    const int mid = (ty + R) * sw + tx + R;
    uint64_t ka = kEmptyKey;
    int dA = -1;
    if (inside) {
        ka = __ldg(reinterpret_cast<const unsigned long long *>(vis_a + key_index(cam, gx, gy)));
        if (fp.enabled && !key_empty(ka)) {
            dA = (int)(ka >> 40);
            const int dgP = dg_at(mid);
            if (dgP < 0 || dA + fp.dmis <= dgP) s_list[atomicAdd(&s_count, 1)] = (uint16_t)tid;
        }
    }
    __syncthreads();
    const int nA = s_count;
    for (int li = tid; li < nA; li += kResolveThreads) {
        const int t = s_list[li];
        const int px = x0 + t % kTileW, py = y0 + t / kTileW;
        const uint64_t k = __ldg(reinterpret_cast<const unsigned long long *>(vis_a + key_index(cam, px, py)));
        const Decoded d = decode_key(tab, s_bases, cam, k, px, py, status);
        s_tsA[t] = make_float2(d.tsx, d.tsy);
        s_isoA[t] = d.iso;
    }
    __syncthreads();

    // Per-pixel flags, then two compacted job lists so that whole warps run
    // one kind of reconstruction adjoint: first the conservative-referenced
    // ones (promoted pixels and depth mismatches), which also fix the share
    // (1 - al) of a mismatch's gradient the centre reconstruction receives;
    // then the centre-referenced ones that receive any.
    const int lane = tid & 31;
    const unsigned lt = (1u << lane) - 1u;
    float3 g = f3(0.f, 0.f, 0.f);
    bool nz = false;
    if (inside) {
        const float4 g4 = __ldg(&grad_rgba[(int64_t)gy * W + gx]);
        g = f3(g4.x, g4.y, g4.z);
        nz = g.x != 0.f || g.y != 0.f || g.z != 0.f;
    }
    const int dG = dg_at(mid);
    const bool gP = inside && dG >= 0, aP = inside && s_fa[mid];
    s_dTs[tid] = make_float4(0.f, 0.f, 0.f, 0.f);
    s_gs[tid] = 1.0f;
    s_dAv[tid] = dA;
    bool jobA = false;
    if (nz && !fp.enabled) {
        if (gP) {
            atomicAdd(&s_dC[mid].x, g.x);
            atomicAdd(&s_dC[mid].y, g.y);
            atomicAdd(&s_dC[mid].z, g.z);
        }
    } else if (nz) {
        jobA = gP ? (aP && dA + fp.dmis <= dG) : aP;
    }
    {
        const unsigned bal = __ballot_sync(0xFFFFFFFFu, jobA);
        int base = 0;
        if (lane == 0 && bal) base = atomicAdd(&s_nJA, __popc(bal));
        base = __shfl_sync(0xFFFFFFFFu, base, 0);
        if (jobA) s_jA[base + __popc(bal & lt)] = (uint16_t)tid;
    }
    __syncthreads();
    const int nJA = s_nJA;
    for (int li = tid; li < nJA; li += kResolveThreads) {
        const int t = s_jA[li];
        const int jx = t % kTileW, jy = t / kTileW, qx = x0 + jx, qy = y0 + jy;
        const int jm = (jy + R) * sw + jx + R;
        const float4 g4 = __ldg(&grad_rgba[(int64_t)qy * W + qx]);
        float3 gA = f3(g4.x, g4.y, g4.z);
        const int dAq = s_dAv[t];
        const float2 tsa = s_tsA[t];
        const bool isoA = s_isoA[t] != 0;
        const float3 z = f3(0.f, 0.f, 0.f);
        const Recon ra = reconstruct_fast_r<false>(R, s_dg, s_fa, s_col, sw, jx, jy, dAq, tsa.x, tsa.y, isoA, z, fp);
        if (dg_at(jm) >= 0 && ra.cnt > 0) {            // depth mismatch: split al / (1 - al)
            const float al = (float)ra.hc / (float)ra.ha;
            gA = mul3(gA, al);
            s_gs[t] = 1.f - al;                          // exactly 0 when al = 1: no centre adjoint
        }
        if (ra.cnt > 0) {
            const float2 d = reconstruct_adjoint(s_dg, s_col, s_dC, sw, jx, jy, qx, qy, W, H, R, dAq, tsa.x, tsa.y,
                                                 isoA, false, z, jm, ra, gA, fp);
            s_dTs[t].z = d.x;
            s_dTs[t].w = d.y;
        }
    }
    __syncthreads();
    {
        const bool jobG = nz && fp.enabled && gP && s_gs[tid] != 0.0f;
        const unsigned bal = __ballot_sync(0xFFFFFFFFu, jobG);
        int base = 0;
        if (lane == 0 && bal) base = atomicAdd(&s_nJG, __popc(bal));
        base = __shfl_sync(0xFFFFFFFFu, base, 0);
        if (jobG) s_jG[base + __popc(bal & lt)] = (uint16_t)tid;
    }
    __syncthreads();
    const int nJG = s_nJG;
    for (int li = tid; li < nJG; li += kResolveThreads) {
        const int t = s_jG[li];
        const int jx = t % kTileW, jy = t / kTileW, qx = x0 + jx, qy = y0 + jy;
        const int jm = (jy + R) * sw + jx + R;
        const float4 g4 = __ldg(&grad_rgba[(int64_t)qy * W + qx]);
        const float gs = s_gs[t];
        const float3 gG = gs == 1.0f ? f3(g4.x, g4.y, g4.z) : mul3(f3(g4.x, g4.y, g4.z), gs);
        const float4 c4 = s_col[jm];
        const float3 Cp = make_float3(c4.x, c4.y, c4.z);
        const int dGq = __float_as_int(c4.w);
        const float2 ts = s_tsG[t];
        const bool isoG = s_isoG[t] != 0;
        const Recon rg = reconstruct_fast_r<true>(R, s_dg, s_fa, s_col, sw, jx, jy, dGq, ts.x, ts.y, isoG, Cp, fp);
        const float2 d = reconstruct_adjoint(s_dg, s_col, s_dC, sw, jx, jy, qx, qy, W, H, R, dGq, ts.x, ts.y, isoG,
                                             true, Cp, jm, rg, gG, fp);
        s_dTs[t].x = d.x;
        s_dTs[t].y = d.y;
    }
    __syncthreads();
    // colour gradients of the staged pixels to the global buffer
    for (int i = tid; i < ns; i += kResolveThreads) {
        const float3 v = s_dC[i];
        if (v.x == 0.f && v.y == 0.f && v.z == 0.f) continue;
        const int qx = x0 - R + i % sw, qy = y0 - R + i / sw;
        if (qx < 0 || qx >= W || qy < 0 || qy >= H) continue;
        float4 *p = dC + (int64_t)qy * W + qx;
        atomicAdd(&p->x, v.x);
        atomicAdd(&p->y, v.y);
        atomicAdd(&p->z, v.z);
    }
    // screen-tangent gradients of the reference segments, for the geometry pass
    if (inside) dTs[(int64_t)gy * W + gx] = s_dTs[tid];
    __syncthreads();                // shared memory is reused by the next tile
    }
}

// Geometry pass, one thread per key with a gradient (persistent grid over
// pixel chunks compacted into job lists): the shading adjoint of a centre
// key (colour gradient from kernel 1) or the screen-tangent adjoint of a
// reference segment, chained through the strand geometry to the layer
// vertices, and the albedo gradient.  When
// every groom's layer-vertex gradient fits, a CTA accumulates it in shared
// memory and adds it to the global arrays once at the end.
// 256 threads and four CTAs per SM (a 64-register budget): the decode and
// adjoint chains are latency-bound, so 32 resident warps beat fewer warps
// with more registers each (measured: 16 warps at 128 registers were 27%
// slower at 512x512).
constexpr int kGeoThreads = 256, kGeoMinBlocks = 4, kGeoChunk = 2048;

struct GeoLayout {
    int32_t off[HM_MAX_GROOMS_PER_CALL];   // float offset of groom i in the shared copy, -1: none
    int32_t total;                         // floats in the shared copy, 0: accumulate globally
};

__device__ __forceinline__ Sink geo_sink(const GeoLayout &lay, float *s_g, const BwdSinks &sinks, int gi, int V) {
    Sink sk;
    sk.V = V;
    sk.glv = sinks.glv[gi];
    if (sk.glv && lay.total > 0) sk.glv = s_g + lay.off[gi];
    return sk;
}

__global__ void __launch_bounds__(kGeoThreads, kGeoMinBlocks) geometry_adjoint_kernel(CallTable tab, CamDev cam, LightsDev Ls,
                                                                       const uint64_t *__restrict__ vis_c,
                                                                       const uint64_t *__restrict__ vis_a,
                                                                       const float4 *__restrict__ dC,
                                                                       const float4 *__restrict__ dTs,
                                                                       BwdSinks sinks, GeoLayout lay,
                                                                       uint32_t *status) {
    extern __shared__ __align__(16) float s_g[];
    __shared__ uint64_t s_bases[HM_MAX_GROOMS_PER_CALL + 1];
    __shared__ uint16_t s_job[2 * kGeoChunk];
    __shared__ int s_nj;
    if (threadIdx.x <= tab.n) {
        uint64_t b = 0;
        for (int i = 0; i < (int)threadIdx.x; ++i) b += (uint64_t)tab.g[i].S;
        s_bases[threadIdx.x] = b;
    }
    for (int i = threadIdx.x; i < lay.total; i += blockDim.x) s_g[i] = 0.f;
    __syncthreads();
    // Chunks of kGeoChunk pixels: the keys with a gradient (a centre key with
    // a colour or screen-tangent gradient, a conservative key with a
    // screen-tangent gradient) are compacted into a job list so whole warps
    // run the one decode + adjoint path.
    const int64_t npx = (int64_t)cam.W * cam.H;
    // about four chunks per CTA (a multiple of the CTA size, at most kGeoChunk)
    int64_t csz = (npx + 4 * (int64_t)gridDim.x - 1) / (4 * (int64_t)gridDim.x);
    csz = ((csz + kGeoThreads - 1) / kGeoThreads) * kGeoThreads;
    const int chunk_px = (int)(csz < kGeoThreads ? kGeoThreads : (csz > kGeoChunk ? kGeoChunk : csz));
    const int64_t nchunk = (npx + chunk_px - 1) / chunk_px;
    const int lane = threadIdx.x & 31;
    for (int64_t chunk = blockIdx.x; chunk < nchunk; chunk += gridDim.x) {
        const int64_t q0 = chunk * chunk_px;
        if (threadIdx.x == 0) s_nj = 0;
        __syncthreads();
        for (int k = threadIdx.x; k < chunk_px; k += kGeoThreads) {
            const int64_t p = q0 + k;
            bool jg = false, ja = false;
            if (p < npx) {
                const float4 gc = __ldg(&dC[p]);
                const float4 gt = __ldg(&dTs[p]);
                const uint32_t kp = key_index(cam, (int)(p % cam.W), (int)(p / cam.W));
                jg = (gc.x != 0.f || gc.y != 0.f || gc.z != 0.f || gt.x != 0.f || gt.y != 0.f) &&
                     !key_empty(__ldg(reinterpret_cast<const unsigned long long *>(vis_c + kp)));
                ja = (gt.z != 0.f || gt.w != 0.f) &&
                     !key_empty(__ldg(reinterpret_cast<const unsigned long long *>(vis_a + kp)));
            }
#pragma unroll
            for (int layer = 0; layer < 2; ++layer) {
                const bool want = layer ? ja : jg;
                const unsigned bal = __ballot_sync(0xFFFFFFFFu, want);
                int base = 0;
                if (lane == 0 && bal) base = atomicAdd(&s_nj, __popc(bal));
                base = __shfl_sync(0xFFFFFFFFu, base, 0);
                if (want) s_job[base + __popc(bal & ((1u << lane) - 1u))] = (uint16_t)(k | (layer << 15));
            }
        }
        __syncthreads();
        const int nj = s_nj;
        for (int jj = threadIdx.x; jj < nj; jj += kGeoThreads) {
            const int e = s_job[jj];
            const bool cons = (e & 0x8000) != 0;
            const int64_t p = q0 + (e & 0x7FFF);
            const int px = (int)(p % cam.W), py = (int)(p / cam.W);
            const uint64_t key =
                __ldg(reinterpret_cast<const unsigned long long *>((cons ? vis_a : vis_c) + key_index(cam, px, py)));
            const Decoded d = decode_key(tab, s_bases, cam, key, px, py, status);
            if (!d.ok) continue;
            const GroomDev &g = tab.g[d.gi];
            const float4 gt = __ldg(&dTs[p]);
            const float2 gts = cons ? make_float2(gt.z, gt.w) : make_float2(gt.x, gt.y);
            float3 dX = f3(0.f, 0.f, 0.f), dT = f3(0.f, 0.f, 0.f);
            if (!cons) {
                const float4 gc = __ldg(&dC[p]);
                if (gc.x != 0.f || gc.y != 0.f || gc.z != 0.f) {
                    const float4 a = __ldg(&g.albedo[d.s]);
                    float3 dalb;
                    shade_adjoint(d.X, d.T, f3(a.x, a.y, a.z), cam, Ls, g.roughness, g.tilt, decoded_ao(g, d),
                                  receiver_beta(g, Ls, d.s), f3(gc.x, gc.y, gc.z), dX, dT, dalb);
                    float *ga = sinks.galb[d.gi];
                    if (ga) {
                        atomicAdd(ga + 3 * d.s + 0, dalb.x);
                        atomicAdd(ga + 3 * d.s + 1, dalb.y);
                        atomicAdd(ga + 3 * d.s + 2, dalb.z);
                    }
                }
            }
            if ((gts.x != 0.f || gts.y != 0.f) && !d.iso) {
                float3 tX, tT;
                screen_tangent_adjoint(cam, d.X, d.T, gts, tX, tT);
                dX = add3(dX, tX);
                dT = add3(dT, tT);
            }
            const Sink sk = geo_sink(lay, s_g, sinks, d.gi, g.V);
            if (sk.glv) {
                const uint32_t f = __ldg(&g.sface[d.s]);
                geometry_adjoint(g, make_root(g, d.s, f), f, d.s, d.C, d.j, d.t, dX, dT, sk);
            }
        }
        __syncthreads();
    }
    if (lay.total == 0) return;
    __syncthreads();
    for (int gi = 0; gi < tab.n; ++gi) {
        if (lay.off[gi] < 0) continue;
        const int nf = tab.g[gi].L * tab.g[gi].V * 3;
        float *dst = sinks.glv[gi];
        const float *src = s_g + lay.off[gi];
        for (int i = threadIdx.x; i < nf; i += blockDim.x) {
            const float v = src[i];
            if (v != 0.f) atomicAdd(dst + i, v);
        }
    }
}

__global__ void zero_float4_kernel(float4 *p, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = make_float4(0.f, 0.f, 0.f, 0.f);
}

size_t adjoint_smem_bytes(int radius) {
    const int sw = kTileW + 2 * radius, sh = kTileH + 2 * radius, ns = sw * sh;
    size_t b = sizeof(uint64_t) * (HM_MAX_GROOMS_PER_CALL + 1) + 16;   // + alignment of s_col
    b += sizeof(float4) * ns + sizeof(float3) * ns;
    b += sizeof(uint16_t) * ((ns + 7) & ~7) + 16;
    b += sizeof(float2) * 2 * kResolveThreads;
    b += 2 * kResolveThreads;
    b += ns + 3;                      // s_fa, then the alignment of s_dg
    b += sizeof(int) * ns;
    return (b + 15) & ~(size_t)15;
}

// Shared-memory budget for the geometry pass's copy of the layer-vertex
// gradients, sized so that four CTAs still fit on an SM; larger sets (big
// grooms, crowds) accumulate straight into global memory.
constexpr int kGeoSmemFloats = 11 * 1024;

cudaError_t launch_resolve_adjoint(const CallTable &tab, const CamDev &cam, const LightsDev &Ls, const FilterDev &fp,
                                   const uint64_t *vis_c, const uint64_t *vis_a, const float *grad_rgba,
                                   float *const *glv, float *const *galb, void *scratch, uint32_t *status,
                                   cudaStream_t st) {
    const int64_t npx = (int64_t)cam.W * cam.H;
    float4 *dC = static_cast<float4 *>(scratch);
    float4 *dTs = dC + npx;
    int *list = reinterpret_cast<int *>(dTs + npx);     // tile list (resolve_list_bytes)
    BwdSinks sinks;
    GeoLayout lay;
    int32_t total = 0;
    for (int i = 0; i < HM_MAX_GROOMS_PER_CALL; ++i) {
        sinks.glv[i] = (i < tab.n && glv) ? glv[i] : nullptr;
        sinks.galb[i] = (i < tab.n && galb) ? galb[i] : nullptr;
        lay.off[i] = -1;
        if (sinks.glv[i]) {
            lay.off[i] = total;
            total += tab.g[i].L * tab.g[i].V * 3;
        }
    }
    lay.total = total <= kGeoSmemFloats ? total : 0;
    const int sms = num_sms();
    zero_float4_kernel<<<sms * 8, 256, 0, st>>>(dC, 2 * npx);
    const int R = fp.enabled ? fp.radius : 0;
    // per device: the kernels' shared-memory limits (an attribute of the
    // current device) and the persistent tile grid that fits
    static PerDevice<int> resident_tiles;
    const int resident = resident_tiles.get([sms](int) {
        cudaFuncSetAttribute(resolve_adjoint_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)adjoint_smem_bytes(HM_MAX_FILTER_RADIUS));
        cudaFuncSetAttribute(geometry_adjoint_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(kGeoSmemFloats * sizeof(float)));
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, resolve_adjoint_kernel, kResolveThreads,
                                                      adjoint_smem_bytes(HM_MAX_FILTER_RADIUS));
        return (per_sm > 0 ? per_sm : 1) * sms;
    });
    cudaError_t e = launch_tile_list(vis_a, nullptr, cam, kTileH, list, st);
    if (e != cudaSuccess) return e;
    const int ntiles = ((cam.W + kTileW - 1) / kTileW) * ((cam.H + kTileH - 1) / kTileH);
    resolve_adjoint_kernel<<<resident < ntiles ? resident : ntiles, kResolveThreads, adjoint_smem_bytes(R), st>>>(
        tab, cam, Ls, fp, vis_c, vis_a, reinterpret_cast<const float4 *>(grad_rgba), dC, dTs, status, list);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    geometry_adjoint_kernel<<<sms * kGeoMinBlocks, kGeoThreads, (size_t)lay.total * sizeof(float), st>>>(tab, cam, Ls, vis_c, vis_a,
                                                                                          dC, dTs, sinks, lay, status);
    return cudaGetLastError();
}

}  // namespace hm
