// hm_resolve.cu -- deferred resolve of the hair rasterizer (arXiv 2607.04230):
// key decode and shading (Sec. 3.1.2, Sec. 3.4), strand connection,
// elliptical bilateral filter and alpha estimation (Sec. 3.3.1-3.3.3).
//
// One CTA per 32x16 output tile.  The tile plus an r-pixel halo is staged in
// shared memory: per staged pixel the centre-layer depth (or -1 when empty),
// the conservative-layer occupancy and the shaded colour of centre-sample
// pixels.  Decode + shading work is compacted into lists so whole warps stay
// busy, then every thread filters its own tile pixel from shared memory.
#include <cstdint>
#include <cuda_runtime.h>

#include "hm_device.cuh"
#include "hm_kernels.h"
#include "hm_value.cuh"

namespace hm {

__global__ void __launch_bounds__(kResolveThreads) resolve_kernel(CallTable tab, CamDev cam, LightsDev Ls,
                                                                  FilterDev fp, const uint64_t *__restrict__ vis_c,
                                                                  const uint64_t *__restrict__ vis_a,
                                                                  float4 *__restrict__ rgba, uint32_t *status) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int R = fp.enabled ? fp.radius : 0;
    const int sw = kTileW + 2 * R, sh = kTileH + 2 * R, ns = sw * sh;
    // shared layout: bases | s_col[ns] | s_dg[ns] | s_list[ns] | s_fa[ns] | tile arrays
    uint64_t *s_bases = reinterpret_cast<uint64_t *>(smem);
    float3 *s_col = reinterpret_cast<float3 *>(s_bases + HM_MAX_GROOMS_PER_CALL + 1);
    int *s_dg = reinterpret_cast<int *>(s_col + ns);
    uint16_t *s_list = reinterpret_cast<uint16_t *>(s_dg + ns);
    float2 *s_tsG = reinterpret_cast<float2 *>(
        (reinterpret_cast<uintptr_t>(s_list + ((ns + 7) & ~7)) + 15) & ~(uintptr_t)15);
    float2 *s_tsA = s_tsG + kResolveThreads;
    uint8_t *s_isoG = reinterpret_cast<uint8_t *>(s_tsA + kResolveThreads);
    uint8_t *s_isoA = s_isoG + kResolveThreads;
    uint8_t *s_fa = s_isoA + kResolveThreads;
    __shared__ int s_count;

    const int tid = threadIdx.x;
    const int x0 = blockIdx.x * kTileW, y0 = blockIdx.y * kTileH;
    const int W = cam.W, H = cam.H;
    if (tid <= tab.n) {
        uint64_t b = 0;
        for (int i = 0; i < tid; ++i) b += (uint64_t)tab.g[i].S;
        s_bases[tid] = b;
    }
    if (tid == 0) s_count = 0;
    __syncthreads();

    // stage keys of tile + halo; list staged centre-sample pixels
    for (int i = tid; i < ns; i += kResolveThreads) {
        const int gx = x0 - R + i % sw, gy = y0 - R + i / sw;
        int dg = -1;
        uint8_t fa = 0;
        if (gx >= 0 && gx < W && gy >= 0 && gy < H) {
            const int64_t p = (int64_t)gy * W + gx;
            const uint64_t kg = __ldg(reinterpret_cast<const unsigned long long *>(vis_c + p));
            const uint64_t ka = __ldg(reinterpret_cast<const unsigned long long *>(vis_a + p));
            if (!key_empty(kg)) {
                dg = (int)(kg >> 40);
                s_list[atomicAdd(&s_count, 1)] = (uint16_t)i;
            }
            fa = !key_empty(ka);
        }
        s_dg[i] = dg;
        s_fa[i] = fa;
    }
    if (tid < kResolveThreads) s_isoG[tid] = 1, s_isoA[tid] = 1;
    __syncthreads();

    // decode + shade every staged centre-sample pixel
    const int ncen = s_count;
    for (int li = tid; li < ncen; li += kResolveThreads) {
        const int i = s_list[li];
        const int lx = i % sw, ly = i / sw;
        const int gx = x0 - R + lx, gy = y0 - R + ly;
        const uint64_t kg = __ldg(reinterpret_cast<const unsigned long long *>(vis_c + (int64_t)gy * W + gx));
        const Decoded d = decode_key(tab, s_bases, cam, kg, gx, gy, status);
        float3 c = make_float3(0.f, 0.f, 0.f);
        if (d.ok) {
            const GroomDev &g = tab.g[d.gi];
            const float4 a = __ldg(&g.albedo[d.s]);
            c = shade(d.X, d.T, make_float3(a.x, a.y, a.z), cam, Ls, g.roughness, g.tilt);
        }
        s_col[i] = c;
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

    // tile pixels that need the conservative layer as reference: promoted
    // (centre empty) or depth mismatch (a closer conservative strand)
    const int tx = tid % kTileW, ty = tid / kTileW;
    const int gx = x0 + tx, gy = y0 + ty;
    const bool inside = gx < W && gy < H;
    const int mid = (ty + R) * sw + tx + R;
    uint64_t ka = kEmptyKey;
    int dA = -1;
    if (inside && fp.enabled) {
        ka = __ldg(reinterpret_cast<const unsigned long long *>(vis_a + (int64_t)gy * W + gx));
        if (!key_empty(ka)) {
            dA = (int)(ka >> 40);
            const int dgP = s_dg[mid];
            if (dgP < 0 || dA + fp.dmis <= dgP) s_list[atomicAdd(&s_count, 1)] = (uint16_t)tid;
        }
    }
    __syncthreads();
    const int nA = s_count;
    for (int li = tid; li < nA; li += kResolveThreads) {
        const int t = s_list[li];
        const int px = x0 + t % kTileW, py = y0 + t / kTileW;
        const uint64_t k = __ldg(reinterpret_cast<const unsigned long long *>(vis_a + (int64_t)py * W + px));
        const Decoded d = decode_key(tab, s_bases, cam, k, px, py, status);
        s_tsA[t] = make_float2(d.tsx, d.tsy);
        s_isoA[t] = d.iso;
    }
    __syncthreads();
    if (!inside) return;

    // filter the tile pixel
    float4 out = make_float4(0.f, 0.f, 0.f, 0.f);
    const int dG = s_dg[mid];
    const bool gP = dG >= 0, aP = s_fa[mid];
    if (!fp.enabled) {
        if (gP) {
            const float3 c = s_col[mid];
            out = make_float4(c.x, c.y, c.z, 1.0f);
        }
    } else if (gP) {
        const float3 Cp = s_col[mid];
        const float2 ts = s_tsG[tid];
        const Recon rg = reconstruct(s_dg, s_fa, s_col, sw, tx, ty, gx, gy, W, H, R, dG, ts.x, ts.y, s_isoG[tid] != 0,
                                     true, Cp, fp);
        const float invW = 1.0f / rg.W;
        const float3 CG = make_float3(rg.S.x * invW, rg.S.y * invW, rg.S.z * invW);
        if (aP && dA + fp.dmis <= dG) {
            const float2 tsa = s_tsA[tid];
            const Recon ra = reconstruct(s_dg, s_fa, s_col, sw, tx, ty, gx, gy, W, H, R, dA, tsa.x, tsa.y,
                                         s_isoA[tid] != 0, false, Cp, fp);
            float3 c = CG;
            if (ra.cnt > 0) {
                const float al = __fdiv_rn((float)ra.hc, (float)ra.ha);
                const float iw = 1.0f / ra.W;
                c = make_float3(al * (ra.S.x * iw) + (1.0f - al) * CG.x, al * (ra.S.y * iw) + (1.0f - al) * CG.y,
                                al * (ra.S.z * iw) + (1.0f - al) * CG.z);
            }
            out = make_float4(c.x, c.y, c.z, 1.0f);
        } else {
            out = make_float4(CG.x, CG.y, CG.z, __fdiv_rn((float)rg.hc, (float)rg.ha));
        }
    } else if (aP) {
        const float2 tsa = s_tsA[tid];
        const Recon ra = reconstruct(s_dg, s_fa, s_col, sw, tx, ty, gx, gy, W, H, R, dA, tsa.x, tsa.y,
                                     s_isoA[tid] != 0, false, make_float3(0.f, 0.f, 0.f), fp);
        if (ra.cnt > 0) {
            const float iw = 1.0f / ra.W;
            out = make_float4(ra.S.x * iw, ra.S.y * iw, ra.S.z * iw, __fdiv_rn((float)ra.hc, (float)ra.ha));
        }
    }
    rgba[(int64_t)gy * W + gx] = out;
}

size_t resolve_smem_bytes(int radius) {
    const int sw = kTileW + 2 * radius, sh = kTileH + 2 * radius, ns = sw * sh;
    size_t b = sizeof(uint64_t) * (HM_MAX_GROOMS_PER_CALL + 1);
    b += sizeof(float3) * ns;
    b += sizeof(int) * ns;
    b += sizeof(uint16_t) * ((ns + 7) & ~7) + 16;
    b += sizeof(float2) * 2 * kResolveThreads;
    b += 2 * kResolveThreads;
    b += ns;
    return (b + 15) & ~(size_t)15;
}

cudaError_t launch_resolve(const CallTable &tab, const CamDev &cam, const LightsDev &Ls, const FilterDev &fp,
                           const uint64_t *vis_c, const uint64_t *vis_a, float *rgba, uint32_t *status,
                           cudaStream_t st) {
    const int R = fp.enabled ? fp.radius : 0;
    size_t sm = resolve_smem_bytes(R);
    static bool attr_set = false;
    if (!attr_set) {
        cudaFuncSetAttribute(resolve_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)resolve_smem_bytes(HM_MAX_FILTER_RADIUS));
        attr_set = true;
    }
    dim3 grid((cam.W + kTileW - 1) / kTileW, (cam.H + kTileH - 1) / kTileH);
    resolve_kernel<<<grid, kResolveThreads, sm, st>>>(tab, cam, Ls, fp, vis_c, vis_a,
                                                       reinterpret_cast<float4 *>(rgba), status);
    return cudaGetLastError();
}

}  // namespace hm
