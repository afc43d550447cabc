// hm_resolve.cu -- deferred resolve of the hair rasterizer (arXiv 2607.04230):
// key decode and shading (Sec. 3.1.2, Sec. 3.4), strand connection,
// elliptical bilateral filter and alpha estimation (Sec. 3.3.1-3.3.3).
//
// One CTA per 32x32 (or 32x16) output tile.  The tile plus an r-pixel halo
// is staged in shared memory: per staged pixel the centre-layer depth (a
// large negative value when empty), the conservative-layer occupancy and the
// shaded colour of centre-sample pixels.  Decode, shading and the
// reconstructions run over compacted lists so whole warps stay busy.
#include <cstdint>
#include <cuda_runtime.h>

#include "hm_device.cuh"
#include "hm_kernels.h"
#include "hm_value.cuh"

namespace hm {

// Forward resolve tiles: 32x32 output pixels per CTA of 512 threads, so the
// halo recompute is (32 + 2r)^2 / 32^2.  Work runs in uniform phases over
// compacted lists: decode + shade the staged centre-sample pixels; one list
// of centre-referenced reconstructions (centre pixels without a depth
// mismatch) and conservative-key decodes + conservative-referenced
// reconstructions (promoted pixels, depth mismatches); the centre
// reconstruction of the mismatches that blend (weight below 1); then the
// tile is written row-major.
constexpr int kFwdTileW = 32, kFwdThreads = 512;
// staged depth of a pixel without a centre key: far below any d24, so a
// depth-difference test alone rejects it
constexpr int kNoDepth = -(1 << 30);

// Centre-referenced result of tile pixel (tx, ty): the normalized
// reconstruction and alpha H_center / H_cons (Sec. 3.3), or the pixel's
// own colour with alpha 1 when the filter is off.
__device__ __forceinline__ float4 centre_result(int R, const int *s_dg, const uint8_t *s_fa, const float4 *s_col, int sw, int tx,
                                                int ty, float2 ts, bool iso, const FilterDev &fp) {
    const int mid = (ty + R) * sw + tx + R;
    const float4 c4 = s_col[mid];
    const float3 Cp = make_float3(c4.x, c4.y, c4.z);
    if (!fp.enabled) return make_float4(Cp.x, Cp.y, Cp.z, 1.0f);
    const Recon rg = reconstruct_fast_r<true>(R, s_dg, s_fa, s_col, sw, tx, ty, __float_as_int(c4.w), ts.x, ts.y, iso, Cp,
                                              fp);
    const float invW = 1.0f / rg.W;
    return make_float4(rg.S.x * invW, rg.S.y * invW, rg.S.z * invW, __fdiv_rn((float)rg.hc, (float)rg.ha));
}

// kCgb: the keys carry the compressed payload (Sec. 3.1.2) and shading
// reads it alone: position from depth, tangent from its code, albedo from
// the appearance table at (u, v) scaled along w, AO from its code.
// Tile list for sparse frames, first pass: every tile's conservative key
// count goes to weights[tile] (0: no key); a tile without keys is written
// with zeros here when rgba is given (no key: RGBA 0).  One warp per tile,
// lane = column, rows walked.
template <int kFwdTileH>
__global__ void __launch_bounds__(256) resolve_tiles_kernel(const uint64_t *__restrict__ vis_a,
                                                            float4 *__restrict__ rgba, CamDev cam, int ntx,
                                                            int ntiles, int *__restrict__ weights) {
    const int W = cam.W, H = cam.H;
    const int tile = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (tile >= ntiles) return;
    const int gx = (tile % ntx) * kFwdTileW + lane, y0 = (tile / ntx) * kFwdTileH;
    const int y1 = min(y0 + kFwdTileH, H);
    int cnt = 0;
    if (gx < W)
        for (int y = y0; y < y1; ++y)
            cnt += !key_empty(__ldg(reinterpret_cast<const unsigned long long *>(vis_a + key_index(cam, gx, y))));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xFFFFFFFFu, cnt, o);
    if (lane == 0) weights[tile] = cnt;
    if (rgba && cnt == 0 && gx < W)
        for (int y = y0; y < y1; ++y) rgba[(int64_t)y * W + gx] = make_float4(0.f, 0.f, 0.f, 0.f);
}

// Tile list, second pass (one CTA): the tiles with keys, heaviest first, by a
// counting sort of their key counts into kOrderBuckets classes, so that the
// persistent resolve starts its longest tiles first and ends without a long
// tail.  Writes list[0] = listed tiles, list[1] = 0 (the resolve's work
// counter), list[2 ..] = tile indices and *dec_work = 0 (the decode pass's
// work counter).
constexpr int kOrderBuckets = 64, kOrderLoads = 8;
__global__ void __launch_bounds__(1024) resolve_order_kernel(const int *__restrict__ weights, int ntiles,
                                                             int tile_px, int *__restrict__ list,
                                                             int *__restrict__ dec_work) {
    __shared__ int s_hist[kOrderBuckets];
    if (threadIdx.x < kOrderBuckets) s_hist[threadIdx.x] = 0;
    __syncthreads();
    // 1 <= w <= tile_px: class 0 holds the heaviest tiles
    auto bucket = [tile_px](int w) { return kOrderBuckets - 1 - (int)((int64_t)w * kOrderBuckets / (tile_px + 1)); };
    // kOrderLoads weights per thread are loaded before any is used, so a
    // pass over a 4K frame's tiles waits for one round of loads, not eight
    for (int t0 = threadIdx.x; t0 < ntiles; t0 += blockDim.x * kOrderLoads) {
        int w[kOrderLoads];
#pragma unroll
        for (int k = 0; k < kOrderLoads; ++k) {
            const int t = t0 + k * (int)blockDim.x;
            w[k] = t < ntiles ? weights[t] : 0;
        }
#pragma unroll
        for (int k = 0; k < kOrderLoads; ++k)
            if (w[k] > 0) atomicAdd(&s_hist[bucket(w[k])], 1);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int acc = 0;
        for (int c = 0; c < kOrderBuckets; ++c) {
            const int n = s_hist[c];
            s_hist[c] = acc;
            acc += n;
        }
        list[0] = acc;
        list[1] = 0;
        *dec_work = 0;
    }
    __syncthreads();
    for (int t0 = threadIdx.x; t0 < ntiles; t0 += blockDim.x * kOrderLoads) {
        int w[kOrderLoads];
#pragma unroll
        for (int k = 0; k < kOrderLoads; ++k) {
            const int t = t0 + k * (int)blockDim.x;
            w[k] = t < ntiles ? weights[t] : 0;
        }
#pragma unroll
        for (int k = 0; k < kOrderLoads; ++k)
            if (w[k] > 0) list[2 + atomicAdd(&s_hist[bucket(w[k])], 1)] = t0 + k * (int)blockDim.x;
    }
}

// Two-pass resolve with the tile-list scratch, first pass: over strips of 8
// rows of the listed tiles (the tiles heaviest first; the CTAs of a
// persistent grid take strips one at a time from a work counter, so a heavy
// tile is spread over several SMs and no CTA idles while strips remain),
// every centre key is decoded and shaded once
// (px_col = shaded colour, centre depth bits) and every screen tangent the
// filter needs is found once: px_ts.xy of the centre key, px_ts.zw of the
// conservative key of a promoted pixel or a depth mismatch, (0, 0) for a
// degenerate tangent.  The jobs of a strip are listed first (centre decodes,
// then conservative ones) so whole warps run one kind.  Entries of pixels
// without those keys are left unwritten; the filter pass reads only the ones
// its keys say exist.
constexpr int kDecThreads = 256, kDecRows = 8, kDecPx = kFwdTileW * kDecRows;
static_assert(kDecPx == kDecThreads, "one strip pixel per thread");

template <int kFwdTileH>
__global__ void __launch_bounds__(kDecThreads, 4) resolve_decode_kernel(CallTable tab, CamDev cam, LightsDev Ls,
                                                                       FilterDev fp, const uint64_t *__restrict__ vis_c,
                                                                       const uint64_t *__restrict__ vis_a,
                                                                       const int *__restrict__ list,
                                                                       float4 *__restrict__ px_col,
                                                                       float4 *__restrict__ px_ts, uint32_t *status,
                                                                       int *__restrict__ work) {
    constexpr int kStrips = kFwdTileH / kDecRows;
    __shared__ uint64_t s_bases[HM_MAX_GROOMS_PER_CALL + 1];
    __shared__ uint16_t s_job[2 * kDecPx];
    __shared__ int s_ng, s_na, s_wi;
    const int tid = threadIdx.x, lane = tid & 31;
    const int W = cam.W, H = cam.H;
    const int ntx = (W + kFwdTileW - 1) / kFwdTileW;
    if (tid <= tab.n) {
        uint64_t b = 0;
        for (int i = 0; i < tid; ++i) b += (uint64_t)tab.g[i].S;
        s_bases[tid] = b;
    }
    const int nwork = list[0] * kStrips;
    for (;;) {
        if (tid == 0) {
            s_ng = 0;
            s_na = 0;
            s_wi = atomicAdd(work, 1);      // the next strip, heaviest tiles first
        }
        __syncthreads();
        const int wi = s_wi;
        if (wi >= nwork) break;
        const int tile = list[2 + wi / kStrips];
        const int x0 = (tile % ntx) * kFwdTileW, y0 = (tile / ntx) * kFwdTileH + (wi % kStrips) * kDecRows;
        // centre decodes go to s_job[0 ..), conservative ones to s_job[kDecPx ..)
        {
            const int t = tid;                   // one strip pixel per thread
            const int gx = x0 + t % kFwdTileW, gy = y0 + t / kFwdTileW;
            bool gP = false, needA = false;
            if (gx < W && gy < H) {
                const uint32_t kp = key_index(cam, gx, gy);
                const uint64_t kg = __ldg(reinterpret_cast<const unsigned long long *>(vis_c + kp));
                const uint64_t ka = __ldg(reinterpret_cast<const unsigned long long *>(vis_a + kp));
                gP = !key_empty(kg);
                needA = !key_empty(ka) && fp.enabled && (!gP || (int)(ka >> 40) + fp.dmis <= (int)(kg >> 40));
            }
            const unsigned bg = __ballot_sync(0xFFFFFFFFu, gP), ba = __ballot_sync(0xFFFFFFFFu, needA);
            int gb = 0, ab = 0;
            if (lane == 0) {
                if (bg) gb = atomicAdd(&s_ng, __popc(bg));
                if (ba) ab = atomicAdd(&s_na, __popc(ba));
            }
            gb = __shfl_sync(0xFFFFFFFFu, gb, 0);
            ab = __shfl_sync(0xFFFFFFFFu, ab, 0);
            const unsigned below = (1u << lane) - 1u;
            if (gP) s_job[gb + __popc(bg & below)] = (uint16_t)t;
            if (needA) s_job[kDecPx + ab + __popc(ba & below)] = (uint16_t)t;
        }
        __syncthreads();
        const int ng = s_ng, na = s_na;
        for (int j = tid; j < ng + na; j += kDecThreads) {
            const bool cen = j < ng;
            const int t = cen ? s_job[j] : s_job[kDecPx + j - ng];
            const int gx = x0 + t % kFwdTileW, gy = y0 + t / kFwdTileW;
            const int64_t p = (int64_t)gy * W + gx;
            const uint64_t key =
                __ldg(reinterpret_cast<const unsigned long long *>((cen ? vis_c : vis_a) + key_index(cam, gx, gy)));
            const Decoded d = decode_key(tab, s_bases, cam, key, gx, gy, status);
            if (cen) {
                float3 c = make_float3(0.f, 0.f, 0.f);
                if (d.ok) {
                    const GroomDev &g = tab.g[d.gi];
                    const float4 a = __ldg(&g.albedo[d.s]);
                    c = shade(d.X, d.T, make_float3(a.x, a.y, a.z), cam, Ls, g.roughness, g.tilt, decoded_ao(g, d),
                              receiver_beta(g, Ls, d.s));
                }
                px_col[p] = make_float4(c.x, c.y, c.z, __int_as_float((int)(key >> 40)));
                reinterpret_cast<float2 *>(px_ts + p)[0] = make_float2(d.tsx, d.tsy);
            } else {
                reinterpret_cast<float2 *>(px_ts + p)[1] = make_float2(d.tsx, d.tsy);
            }
        }
        __syncthreads();        // s_job and the counters are reused by the next strip
    }
}

// list == nullptr: one CTA per tile (grid = tiles); tiles without keys are
// found and zero-filled here.  list != nullptr: a persistent grid takes the
// listed tiles one at a time from the work counter list[1].
//
// kPre: the decode pass (resolve_decode_kernel) has already shaded every
// centre key of the listed tiles into px_col and found the screen tangents
// the filter needs into px_ts, so the tile stages those instead of decoding
// (no decode of halo keys, which a neighbouring tile decodes again).
template <int kFwdTileH, bool kCgb, bool kPre>
__global__ void __launch_bounds__(kFwdThreads, 2) resolve_kernel(CallTable tab, CamDev cam, LightsDev Ls, FilterDev fp,
                                                              const uint64_t *__restrict__ vis_c,
                                                              const uint64_t *__restrict__ vis_a,
                                                              float4 *__restrict__ rgba, uint32_t *status,
                                                              CgbDev cg, int *list, const float4 *__restrict__ px_col,
                                                              const float4 *__restrict__ px_ts) {
    constexpr int kFwdTilePx = kFwdTileW * kFwdTileH;
    extern __shared__ __align__(16) unsigned char smem[];
    const int R = fp.enabled ? fp.radius : 0;
    const int sw = kFwdTileW + 2 * R, sh = kFwdTileH + 2 * R, ns = sw * sh;
    // shared layout: bases | s_col[ns] (rgb + centre depth bits) | s_list[ns] | s_lg[tile] |
    // s_lb[tile] | s_out[tile] | s_outA[tile] | s_ts[tile] | s_flag[tile] | s_fa[ns] | s_dg[ns]
    uint64_t *s_bases = reinterpret_cast<uint64_t *>(smem);
    float4 *s_col = reinterpret_cast<float4 *>(
        (reinterpret_cast<uintptr_t>(s_bases + HM_MAX_GROOMS_PER_CALL + 1) + 15) & ~(uintptr_t)15);  // 16-byte loads
    uint16_t *s_list = reinterpret_cast<uint16_t *>(s_col + ns);     // staged centre list, then A list
    auto dg_at = [&](int i) { return __float_as_int(s_col[i].w); };    // staged centre depth
    uint16_t *s_lg = s_list + ((ns + 7) & ~7);                         // centre pixels without a mismatch
    uint16_t *s_lb = s_lg + kFwdTilePx;                                // mismatches that blend (al < 1)
    float4 *s_out = reinterpret_cast<float4 *>(
        (reinterpret_cast<uintptr_t>(s_lb + kFwdTilePx) + 15) & ~(uintptr_t)15);  // result (rgb, alpha)
    float4 *s_outA = s_out + kFwdTilePx;                              // conservative result (rgb, alpha or -1)
    float2 *s_ts = reinterpret_cast<float2 *>(s_outA + kFwdTilePx);  // G screen tangent
    uint8_t *s_flag = reinterpret_cast<uint8_t *>(s_ts + kFwdTilePx); // bit0 isoG, bit1 isoA, bit2 needs A
    uint8_t *s_fa = s_flag + kFwdTilePx;
    int *s_dg = reinterpret_cast<int *>((reinterpret_cast<uintptr_t>(s_fa + ns) + 3) & ~(uintptr_t)3);  // centre depth
    __shared__ int s_count, s_ng, s_nb, s_tile, s_jobs;

    const int tid = threadIdx.x, lane = tid & 31;
    const int W = cam.W, H = cam.H;
    const int ntx = (W + kFwdTileW - 1) / kFwdTileW;
    const int nlisted = list ? list[0] : 0;
    // per-tile key counts follow the list (room for the finest, 32 x 16, tiling)
    const int list_cap = ntx * ((H + 15) / 16);
    if (tid <= tab.n) {
        uint64_t b = 0;
        for (int i = 0; i < tid; ++i) b += (uint64_t)tab.g[i].S;
        s_bases[tid] = b;
    }
    for (int it = 0;; ++it) {
    if (tid == 0) {
        if (list) s_tile = atomicAdd(&list[1], 1);
        s_count = 0;
        s_ng = 0;
        s_nb = 0;
        s_jobs = 0;
    }
    int tile;
    if (list) {
        __syncthreads();
        if (s_tile >= nlisted) break;
        tile = list[2 + s_tile];
    } else {
        if (it > 0) break;
        tile = blockIdx.y * ntx + blockIdx.x;
    }
    const int x0 = (tile % ntx) * kFwdTileW, y0 = (tile / ntx) * kFwdTileH;
    if (!list) {
        // 0. a tile whose pixels hold no conservative key has nothing to
        // resolve (no centre key either: centre keys are a subset): zeros
        bool any = false;
        for (int t = tid; t < kFwdTilePx; t += kFwdThreads) {
            const int gx = x0 + t % kFwdTileW, gy = y0 + t / kFwdTileW;
            if (gx < W && gy < H)
                any |= !key_empty(
                    __ldg(reinterpret_cast<const unsigned long long *>(vis_a + key_index(cam, gx, gy))));
        }
        if (!__syncthreads_or(any)) {
            for (int t = tid; t < kFwdTilePx; t += kFwdThreads) {
                const int gx = x0 + t % kFwdTileW, gy = y0 + t / kFwdTileW;
                if (gx < W && gy < H) rgba[(int64_t)gy * W + gx] = make_float4(0.f, 0.f, 0.f, 0.f);
            }
            continue;
        }
    }

    // 1. stage keys of tile + halo; list staged centre-sample pixels
    for (int i = tid; i < ns; i += kFwdThreads) {
        const int gx = x0 - R + i % sw, gy = y0 - R + i / sw;
        int dg = kNoDepth;
        uint8_t fa = 0;
        if (gx >= 0 && gx < W && gy >= 0 && gy < H) {
            const int64_t p = (int64_t)gy * W + gx;
            const uint32_t kp = key_index(cam, gx, gy);
            const uint64_t kg = __ldg(reinterpret_cast<const unsigned long long *>(vis_c + kp));
            const uint64_t ka = __ldg(reinterpret_cast<const unsigned long long *>(vis_a + kp));
            float4 c = make_float4(0.f, 0.f, 0.f, 0.f);
            if (!key_empty(kg)) {
                dg = (int)(kg >> 40);
                if (!kPre) {
                    s_list[atomicAdd(&s_count, 1)] = (uint16_t)i;
                } else if (gx >= x0 && gx < x0 + kFwdTileW && gy >= y0 && gy < y0 + kFwdTileH) {
                    c = px_col[p];
                } else {
                    // a halo key lies in a neighbouring tile, which the decode
                    // pass covered if it is listed (it holds a conservative
                    // key, as every rendered tile with a centre key does)
                    const int nt = (gy / kFwdTileH) * ntx + gx / kFwdTileW;
                    if (__ldg(&list[2 + list_cap + nt]) > 0) c = px_col[p];
                }
            }
            fa = !key_empty(ka);
            s_fa[i] = fa;
            s_dg[i] = dg;
            s_col[i] = make_float4(c.x, c.y, c.z, __int_as_float(dg));
            continue;
        }
        s_fa[i] = fa;
        s_dg[i] = dg;
        s_col[i] = make_float4(0.f, 0.f, 0.f, __int_as_float(dg));
    }
    for (int t = tid; t < kFwdTilePx; t += kFwdThreads) s_flag[t] = 3;
    __syncthreads();

    // 2. decode + shade every staged centre-sample pixel (kPre: the decode
    // pass did; only the tile pixels' centre screen tangents are read)
    if (kPre) {
        for (int t = tid; t < kFwdTilePx; t += kFwdThreads) {
            const int gx = x0 + t % kFwdTileW, gy = y0 + t / kFwdTileW;
            if (gx >= W || gy >= H) continue;
            const int mid = (t / kFwdTileW + R) * sw + t % kFwdTileW + R;
            if (dg_at(mid) < 0) continue;
            const float4 ts = px_ts[(int64_t)gy * W + gx];
            s_ts[t] = make_float2(ts.x, ts.y);
            if (ts.x != 0.0f || ts.y != 0.0f) s_flag[t] = 2;     // a degenerate tangent is stored as (0, 0)
        }
    }
    const int ncen = kPre ? 0 : s_count;
    for (int li = tid; li < ncen; li += kFwdThreads) {
        const int i = s_list[li];
        const int lx = i % sw, ly = i / sw;
        const int gx = x0 - R + lx, gy = y0 - R + ly;
        const uint64_t kg = __ldg(reinterpret_cast<const unsigned long long *>(vis_c + key_index(cam, gx, gy)));
        float3 c = make_float3(0.f, 0.f, 0.f);
        float tsx, tsy;
        bool iso;
        if (kCgb) {
            const DecodedC d = decode_compressed(cam, kg, gx, gy);
            const float4 a = __ldg(&cg.table[d.u * 64u + d.v]);
            const float sc = a.w + (1.0f - a.w) * __fdiv_rn((float)d.w, 63.0f);
            c = shade(d.X, d.T, make_float3(a.x * sc, a.y * sc, a.z * sc), cam, Ls, cg.rough, cg.tilt,
                      __fdiv_rn((float)d.ao, 62.0f), 1.0f);
            tsx = d.tsx;
            tsy = d.tsy;
            iso = d.iso;
        } else {
            const Decoded d = decode_key(tab, s_bases, cam, kg, gx, gy, status);
            if (d.ok) {
                const GroomDev &g = tab.g[d.gi];
                const float4 a = __ldg(&g.albedo[d.s]);
                c = shade(d.X, d.T, make_float3(a.x, a.y, a.z), cam, Ls, g.roughness, g.tilt, decoded_ao(g, d),
                          receiver_beta(g, Ls, d.s));
            }
            tsx = d.tsx;
            tsy = d.tsy;
            iso = d.iso;
        }
        s_col[i] = make_float4(c.x, c.y, c.z, s_col[i].w);
        const int tx = lx - R, ty = ly - R;
        if (tx >= 0 && tx < kFwdTileW && ty >= 0 && ty < kFwdTileH) {
            const int t = ty * kFwdTileW + tx;
            s_ts[t] = make_float2(tsx, tsy);
            if (!iso) s_flag[t] = 2;          // isoG cleared, isoA still set
        }
    }
    __syncthreads();
    if (tid == 0) s_count = 0;
    __syncthreads();

    // 3. lists: centre pixels whose result is the centre reconstruction
    // (row-major per warp); pixels needing the conservative reference
    // (promoted pixels and depth mismatches)
    for (int t = tid; t < kFwdTilePx; t += kFwdThreads) {
        const int tx = t % kFwdTileW, ty = t / kFwdTileW;
        const int gx = x0 + tx, gy = y0 + ty;
        const bool in = gx < W && gy < H;
        const int mid = (ty + R) * sw + tx + R;
        const int dgP = in ? dg_at(mid) : -1;
        const bool gP = dgP >= 0, aP = in && s_fa[mid] != 0;
        bool needA = false;
        if (aP && fp.enabled) {
            const uint64_t ka = __ldg(reinterpret_cast<const unsigned long long *>(vis_a + key_index(cam, gx, gy)));
            needA = dgP < 0 || (int)(ka >> 40) + fp.dmis <= dgP;
        }
        const bool gOnly = gP && !needA;
        const unsigned bal = __ballot_sync(0xFFFFFFFFu, gOnly);
        int wbase = 0;
        if (lane == 0 && bal) wbase = atomicAdd(&s_ng, __popc(bal));
        wbase = __shfl_sync(0xFFFFFFFFu, wbase, 0);
        if (gOnly) s_lg[wbase + __popc(bal & ((1u << lane) - 1u))] = (uint16_t)t;
        const unsigned bala = __ballot_sync(0xFFFFFFFFu, needA);
        int abase = 0;
        if (lane == 0 && bala) abase = atomicAdd(&s_count, __popc(bala));
        abase = __shfl_sync(0xFFFFFFFFu, abase, 0);
        if (needA) {
            s_list[abase + __popc(bala & ((1u << lane) - 1u))] = (uint16_t)t;
            s_flag[t] |= 4;
        }
    }
    __syncthreads();
    const int ng = s_ng, nA = s_count;

    // 4. one pass over the jobs: the centre-referenced reconstruction of the
    // centre pixels without a mismatch, then the decode of the conservative
    // reference and the conservative-referenced reconstruction of every pixel
    // that needs it (as one list, so the few conservative jobs past a
    // multiple of the CTA size share a round with centre jobs).  A mismatch
    // blends al R_A + (1 - al) R_G with al = H_center / H_cons of the
    // conservative strip; when al is exactly 1 (the strip's conservative hits
    // all carry a centre key: most mismatches in dense hair) the result is
    // R_A with alpha 1 and the centre reconstruction is not needed; the
    // others go to a second list.
    // warps claim the jobs 32 at a time from a shared counter, so a warp
    // whose jobs were short takes more instead of waiting at the barrier
    for (;;) {
        int li = 0;
        if (lane == 0) li = atomicAdd(&s_jobs, 32);
        li = __shfl_sync(0xFFFFFFFFu, li, 0) + lane;
        if (li - lane >= ng + nA) break;
        if (li >= ng + nA) continue;
        if (li < ng) {
            const int t = s_lg[li];
            const int tx = t % kFwdTileW, ty = t / kFwdTileW;
            s_out[t] = centre_result(R, s_dg, s_fa, s_col, sw, tx, ty, s_ts[t], (s_flag[t] & 1) != 0, fp);
        } else {
            const int t = s_list[li - ng];
            const int tx = t % kFwdTileW, ty = t / kFwdTileW;
            const int gx = x0 + tx, gy = y0 + ty;
            const uint64_t ka = __ldg(reinterpret_cast<const unsigned long long *>(vis_a + key_index(cam, gx, gy)));
            float tsx, tsy;
            bool iso;
            if (kPre) {
                const float4 ts = px_ts[(int64_t)gy * W + gx];
                tsx = ts.z;
                tsy = ts.w;
                iso = tsx == 0.0f && tsy == 0.0f;
            } else if (kCgb) {
                const DecodedC d = decode_compressed(cam, ka, gx, gy);
                tsx = d.tsx;
                tsy = d.tsy;
                iso = d.iso;
            } else {
                const Decoded d = decode_key(tab, s_bases, cam, ka, gx, gy, status);
                tsx = d.tsx;
                tsy = d.tsy;
                iso = d.iso;
            }
            const int dA = (int)(ka >> 40);
            const float3 z = make_float3(0.f, 0.f, 0.f);
            const Recon ra = reconstruct_fast_r<false>(R, s_dg, s_fa, s_col, sw, tx, ty, dA, tsx, tsy, iso, z, fp);
            float4 oa = make_float4(0.f, 0.f, 0.f, -1.0f);   // no contributor
            if (ra.cnt > 0) {
                const float iw = 1.0f / ra.W;
                oa = make_float4(ra.S.x * iw, ra.S.y * iw, ra.S.z * iw, __fdiv_rn((float)ra.hc, (float)ra.ha));
            }
            const int mid = (ty + R) * sw + tx + R;
            if (dg_at(mid) < 0) {                           // promoted
                s_out[t] = oa.w >= 0.0f ? oa : make_float4(0.f, 0.f, 0.f, 0.f);
            } else if (ra.cnt > 0 && ra.hc == ra.ha) {       // mismatch, al = 1
                s_out[t] = make_float4(oa.x, oa.y, oa.z, 1.0f);
            } else {                                         // mismatch to blend over the centre result
                s_outA[t] = oa;
                s_lb[atomicAdd(&s_nb, 1)] = (uint16_t)t;
            }
        }
    }
    __syncthreads();

    // 5. the blended mismatches: centre reconstruction, then
    // al R_A + (1 - al) R_G (R_G alone without a conservative contributor), alpha 1
    const int nb = s_nb;
    for (int li = tid; li < nb; li += kFwdThreads) {
        const int t = s_lb[li];
        const int tx = t % kFwdTileW, ty = t / kFwdTileW;
        const float4 cg = centre_result(R, s_dg, s_fa, s_col, sw, tx, ty, s_ts[t], (s_flag[t] & 1) != 0, fp);
        const float4 a = s_outA[t];
        float3 c = make_float3(cg.x, cg.y, cg.z);
        if (a.w >= 0.0f) {
            const float al = a.w;
            c = make_float3(al * a.x + (1.0f - al) * c.x, al * a.y + (1.0f - al) * c.y, al * a.z + (1.0f - al) * c.z);
        }
        s_out[t] = make_float4(c.x, c.y, c.z, 1.0f);
    }
    __syncthreads();

    // 6. write the tile row-major
    for (int t = tid; t < kFwdTilePx; t += kFwdThreads) {
        const int tx = t % kFwdTileW, ty = t / kFwdTileW;
        const int gx = x0 + tx, gy = y0 + ty;
        if (gx >= W || gy >= H) continue;
        const int mid = (ty + R) * sw + tx + R;
        const bool written = dg_at(mid) >= 0 || (s_flag[t] & 4);
        rgba[(int64_t)gy * W + gx] = written ? s_out[t] : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    __syncthreads();                // shared memory is reused by the next tile
    }
}

// Multisample resolve: every covered sample is decoded at its own sample
// point and shaded; straight-alpha output with rgb the mean over covered
// samples and alpha the covered fraction (premultiplied: the mean over all).
// The kernel waits mostly on the key, record and albedo loads, so it runs four
// CTAs per SM (64 registers) with every sample layer's key requested first.
template <int N>
__global__ void __launch_bounds__(256, 4) resolve_msaa_kernel(CallTable tab, CamDev cam, LightsDev Ls,
                                                              const uint64_t *__restrict__ vis_s,
                                                              float4 *__restrict__ rgba, uint32_t *status) {
    __shared__ uint64_t s_bases[HM_MAX_GROOMS_PER_CALL + 1];
    if ((int)threadIdx.x <= tab.n) {
        uint64_t b = 0;
        for (int i = 0; i < (int)threadIdx.x; ++i) b += (uint64_t)tab.g[i].S;
        s_bases[threadIdx.x] = b;
    }
    __syncthreads();
    const int64_t npx = (int64_t)cam.W * cam.H;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < npx; p += (int64_t)gridDim.x * blockDim.x) {
        const int px = (int)(p % cam.W), py = (int)(p / cam.W);
        float3 acc = make_float3(0.f, 0.f, 0.f);
        int cnt = 0;
        uint64_t keys[N];   // all sample layers' loads in flight before the first decode
#pragma unroll
        for (int k = 0; k < N; ++k)
            keys[k] = __ldg(reinterpret_cast<const unsigned long long *>(vis_s + (int64_t)k * npx + p));
#pragma unroll
        for (int k = 0; k < N; ++k) {
            const uint64_t key = keys[k];
            if (key_empty(key)) continue;
            int ox, oy;
            sample_offset<N>(k, ox, oy);
            const Decoded d = decode_key_at(tab, s_bases, cam, key, 256 * (int64_t)px + 128 + ox,
                                            256 * (int64_t)py + 128 + oy, status);
            if (!d.ok) continue;
            const GroomDev &g = tab.g[d.gi];
            const float4 a = __ldg(&g.albedo[d.s]);
            const float3 c = shade(d.X, d.T, make_float3(a.x, a.y, a.z), cam, Ls, g.roughness, g.tilt,
                                   decoded_ao(g, d), receiver_beta(g, Ls, d.s));
            acc.x += c.x;
            acc.y += c.y;
            acc.z += c.z;
            ++cnt;
        }
        float4 out = make_float4(0.f, 0.f, 0.f, 0.f);
        if (cnt > 0) {
            const float ic = 1.0f / (float)cnt;
            out = make_float4(acc.x * ic, acc.y * ic, acc.z * ic, __fdiv_rn((float)cnt, (float)N));
        }
        rgba[p] = out;
    }
}

cudaError_t launch_resolve_msaa(const CallTable &tab, const CamDev &cam, const LightsDev &Ls, int samples,
                                const uint64_t *vis_s, float *rgba, uint32_t *status, cudaStream_t st) {
    const int64_t npx = (int64_t)cam.W * cam.H;
    const int64_t want = (npx + 255) / 256;
    const int grid = (int)(want < (int64_t)num_sms() * 16 ? (want > 0 ? want : 1) : (int64_t)num_sms() * 16);
    float4 *out = reinterpret_cast<float4 *>(rgba);
    switch (samples) {
        case 1: resolve_msaa_kernel<1><<<grid, 256, 0, st>>>(tab, cam, Ls, vis_s, out, status); break;
        case 2: resolve_msaa_kernel<2><<<grid, 256, 0, st>>>(tab, cam, Ls, vis_s, out, status); break;
        case 4: resolve_msaa_kernel<4><<<grid, 256, 0, st>>>(tab, cam, Ls, vis_s, out, status); break;
        default: resolve_msaa_kernel<8><<<grid, 256, 0, st>>>(tab, cam, Ls, vis_s, out, status); break;
    }
    return cudaGetLastError();
}

size_t resolve_smem_bytes(int radius, int tile_h) {
    const int tile_px = kFwdTileW * tile_h;
    const int sw = kFwdTileW + 2 * radius, sh = tile_h + 2 * radius, ns = sw * sh;
    size_t b = sizeof(uint64_t) * (HM_MAX_GROOMS_PER_CALL + 1) + 16;   // + alignment of the float4 array
    b += sizeof(float4) * ns;
    b += sizeof(uint16_t) * (((ns + 7) & ~7) + 2 * tile_px) + 16;
    b += 2 * sizeof(float4) * tile_px;
    b += sizeof(float2) * tile_px;
    b += tile_px;
    b += ns + 3;                      // s_fa, then the alignment of s_dg
    b += sizeof(int) * ns;
    return (b + 15) & ~(size_t)15;
}

// Tiles of the finest tiling (32 x 16), the most any tile height can have.
static int resolve_max_tiles(int W, int H) { return ((W + kFwdTileW - 1) / kFwdTileW) * ((H + 15) / 16); }

// list[0], list[1], the ordered tile list, one key count per tile, then the
// decode pass's work counter.
size_t resolve_list_bytes(int W, int H) { return sizeof(int) * (3 + 2 * (size_t)resolve_max_tiles(W, H)); }
static int *decode_work_counter(int *list, int W, int H) { return list + 2 + 2 * (size_t)resolve_max_tiles(W, H); }

cudaError_t launch_tile_list(const uint64_t *vis_a, float4 *rgba, const CamDev &cam, int th, int *list,
                             cudaStream_t st) {
    const int W = cam.W, H = cam.H;
    const int ntx = (W + kFwdTileW - 1) / kFwdTileW, ntiles = ntx * ((H + th - 1) / th);
    int *weights = list + 2 + resolve_max_tiles(W, H);
    if (th == 16)
        resolve_tiles_kernel<16><<<(ntiles + 7) / 8, 256, 0, st>>>(vis_a, rgba, cam, ntx, ntiles, weights);
    else
        resolve_tiles_kernel<32><<<(ntiles + 7) / 8, 256, 0, st>>>(vis_a, rgba, cam, ntx, ntiles, weights);
    resolve_order_kernel<<<1, 1024, 0, st>>>(weights, ntiles, kFwdTileW * th, list, decode_work_counter(list, W, H));
    return cudaGetLastError();
}

// The two-pass resolve's per-pixel arrays follow the tile list in the
// scratch: px_col [H][W] float4, then px_ts [H][W] float4.
static size_t resolve_list_bytes_aligned(int W, int H) { return (resolve_list_bytes(W, H) + 15) & ~(size_t)15; }

size_t resolve_scratch_bytes(int W, int H) {
    return resolve_list_bytes_aligned(W, H) + 2 * sizeof(float4) * (size_t)W * (size_t)H;
}

template <int TH, bool C, bool P>
static int resolve_resident() {
    // per device: the kernel's shared-memory limit (an attribute of the
    // current device) and the persistent tile grid that fits
    static PerDevice<int> resident_tiles;
    return resident_tiles.get([](int) {
        cudaFuncSetAttribute(resolve_kernel<TH, C, P>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)resolve_smem_bytes(HM_MAX_FILTER_RADIUS, TH));
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, resolve_kernel<TH, C, P>, kFwdThreads,
                                                      resolve_smem_bytes(HM_MAX_FILTER_RADIUS, TH));
        return (per_sm > 0 ? per_sm : 1) * num_sms();
    });
}

template <int TH, bool C>
static cudaError_t launch_resolve_t(const CallTable &tab, const CamDev &cam, const LightsDev &Ls, const FilterDev &fp,
                                   const uint64_t *vis_c, const uint64_t *vis_a, float *rgba, uint32_t *status,
                                   cudaStream_t st, const CgbDev &cg, int *tile_list) {
    const int R = fp.enabled ? fp.radius : 0;
    dim3 grid((cam.W + kFwdTileW - 1) / kFwdTileW, (cam.H + TH - 1) / TH);
    float4 *out = reinterpret_cast<float4 *>(rgba);
    if (!tile_list) {
        const int resident = resolve_resident<TH, C, false>();   // sets the shared-memory limit
        (void)resident;
        resolve_kernel<TH, C, false><<<grid, kFwdThreads, resolve_smem_bytes(R, TH), st>>>(
            tab, cam, Ls, fp, vis_c, vis_a, out, status, cg, nullptr, nullptr, nullptr);
        return cudaGetLastError();
    }
    const int ntiles = (int)(grid.x * grid.y);
    cudaError_t e = launch_tile_list(vis_a, out, cam, TH, tile_list, st);
    if (e != cudaSuccess) return e;
    if (C) {
        const int resident = resolve_resident<TH, C, false>();
        resolve_kernel<TH, C, false><<<resident < ntiles ? resident : ntiles, kFwdThreads, resolve_smem_bytes(R, TH),
                                       st>>>(tab, cam, Ls, fp, vis_c, vis_a, out, status, cg, tile_list, nullptr,
                                             nullptr);
        return cudaGetLastError();
    }
    // two passes: decode every key once, then filter the tiles
    float4 *px_col = reinterpret_cast<float4 *>(reinterpret_cast<char *>(tile_list) +
                                                resolve_list_bytes_aligned(cam.W, cam.H));
    float4 *px_ts = px_col + (size_t)cam.W * cam.H;
    const int dec_grid = num_sms() * 4 < ntiles * (TH / kDecRows) ? num_sms() * 4 : ntiles * (TH / kDecRows);
    resolve_decode_kernel<TH><<<dec_grid, kDecThreads, 0, st>>>(tab, cam, Ls, fp, vis_c, vis_a, tile_list, px_col,
                                                                 px_ts, status,
                                                                 decode_work_counter(tile_list, cam.W, cam.H));
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int resident = resolve_resident<TH, false, true>();
    resolve_kernel<TH, false, true><<<resident < ntiles ? resident : ntiles, kFwdThreads, resolve_smem_bytes(R, TH),
                                      st>>>(tab, cam, Ls, fp, vis_c, vis_a, out, status, cg, tile_list, px_col, px_ts);
    return cudaGetLastError();
}


// Resolve tile: 32 x tile_h output pixels per CTA (tile_h 16 or 32).
cudaError_t launch_resolve(const CallTable &tab, const CamDev &cam, const LightsDev &Ls, const FilterDev &fp,
                           const uint64_t *vis_c, const uint64_t *vis_a, float *rgba, uint32_t *status, int tile_h,
                           cudaStream_t st, const CgbDev *compressed, int *tile_list) {
    if (compressed) {
        if (tile_h == 16)
            return launch_resolve_t<16, true>(tab, cam, Ls, fp, vis_c, vis_a, rgba, status, st, *compressed, tile_list);
        return launch_resolve_t<32, true>(tab, cam, Ls, fp, vis_c, vis_a, rgba, status, st, *compressed, tile_list);
    }
    const CgbDev none{nullptr, 0.0f, 0.0f};
    if (tile_h == 16)
        return launch_resolve_t<16, false>(tab, cam, Ls, fp, vis_c, vis_a, rgba, status, st, none, tile_list);
    return launch_resolve_t<32, false>(tab, cam, Ls, fp, vis_c, vis_a, rgba, status, st, none, tile_list);
}

}  // namespace hm
