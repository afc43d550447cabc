// hm_kernels.h -- host-side launchers and the small parameter blocks the
// kernels take by value.
#pragma once

#include <atomic>
#include <cstddef>
#include <cstdint>
#include <mutex>
#include <cuda_runtime.h>

#include "hm_device.cuh"

namespace hm {

struct ShadowDev {
    const uint64_t *map;       // [cam.H][cam.W] keys
    CamDev cam;
    float sigma, bias;
    int32_t corr;              // apply beta = N_LOD / N of the receiver's bundle
};

struct LightsDev {
    int32_t n;
    float dir[HM_MAX_LIGHTS][3];
    float rad[HM_MAX_LIGHTS][3];
    float ambient, kd, ks;
    int32_t n_shadow;
    int32_t shadow_of[HM_MAX_LIGHTS];   // map of each light, -1 none
    ShadowDev sh[HM_MAX_LIGHTS];
};

// Appearance of the compressed payload: per (u, v) code a float4 (tip
// albedo rgb, root / tip ratio), 64 x 64 entries; roughness and tilt.
struct CgbDev {
    const float4 *table;
    float rough, tilt;
};

struct FilterDev {
    int32_t enabled, radius;
    float hw2;                 // strip half-width squared (binary32 product)
    float hw;                  // strip half-width
    float inv_spar2, inv_sperp2, inv_siso2, inv_sc2;
    int32_t drej, dmis;        // depth thresholds in d24 units
};

constexpr int kMaxDevices = 64;

// A value per CUDA device, made on first use with that device current and
// kept for the life of the process (symbol addresses, kernel attributes,
// occupancy-derived grid sizes).  Thread-safe: concurrent first calls on one
// device run `make` once; a zero result (a failed lookup) is not kept, so the
// next call tries again.  The cached device state does not survive
// cudaDeviceReset: a process does not use the library again on a device it
// has reset.
template <typename T>
class PerDevice {
  public:
    template <typename F>
    T get(F &&make) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return T{};
        T v = val_[dev].load(std::memory_order_acquire);
        if (v != T{}) return v;
        std::lock_guard<std::mutex> lock(mu_);
        v = val_[dev].load(std::memory_order_relaxed);
        if (v == T{}) {
            v = make(dev);
            val_[dev].store(v, std::memory_order_release);
        }
        return v;
    }

  private:
    std::mutex mu_;
    std::atomic<T> val_[kMaxDevices] = {};
};

int num_sms();

// Both key layers (nkeys keys each, in cam's key layout) to EMPTY or to the
// scene-depth pre-fill (row-major [H][W] scene_d24, or null); zeroes stats.
cudaError_t launch_clear(uint64_t *vis_c, uint64_t *vis_a, int64_t nkeys, const uint32_t *scene_d24, const CamDev &cam,
                         int do_clear, hm_frame_stats *stats, cudaStream_t st);
cudaError_t launch_lod(const CallTable &tab, const CamDev &cam, hm_frame_stats *stats, cudaStream_t st);
cudaError_t launch_raster(const CallTable &tab, const ViewSet &views, bool precheck, int min_blocks, int ctas_per_sm,
                          hm_frame_stats *stats, cudaStream_t st, bool compressed = false);
// Screen-tile binned rasterizer (the alternative to launch_raster for one
// view with the ID payload): bytes of its workspace for `slots` segment slots
// (32 per work batch of the call's grooms at full detail) at W x H with
// tile_w x tile_h tiles, 0 if out of range; the launch (after the clear and
// the LOD pass, like launch_raster).  tile_w, tile_h in {16, 32}, chunk in
// {256, 1024} segments per unit of the tile pass.
size_t binned_workspace_bytes(uint64_t slots, int W, int H, int tile_w, int tile_h);
cudaError_t launch_raster_binned(const CallTable &tab, const CamDev &cam, uint64_t *vis_c, uint64_t *vis_a, void *ws,
                                 uint64_t slots, int tile_w, int tile_h, int chunk, uint32_t *status,
                                 hm_frame_stats *stats, cudaStream_t st);
cudaError_t launch_probe_atomic_min(uint64_t *buf, int64_t n, int rounds, int pattern, cudaStream_t st);
cudaError_t launch_probe_quotient(const float *num, const float *den, float *out, int64_t n, cudaStream_t st);
cudaError_t launch_resolve(const CallTable &tab, const CamDev &cam, const LightsDev &Ls, const FilterDev &fp,
                           const uint64_t *vis_c, const uint64_t *vis_a, float *rgba, uint32_t *status, int tile_h,
                           cudaStream_t st, const CgbDev *compressed = nullptr, int *tile_list = nullptr);
// Bytes of the tile list alone (list, order, per-tile key counts).
size_t resolve_list_bytes(int W, int H);
// Bytes of the resolve's optional scratch at this resolution: the tile list
// (16-byte aligned) and the two-pass resolve's per-pixel arrays.
size_t resolve_scratch_bytes(int W, int H);
// Tile list of a frame's 32 x th tiles (th 16 or 32) into `list` (resolve_list_bytes):
// per-tile conservative key counts (zero-filling keyless tiles of rgba when it
// is given), then list[0] = occupied tiles, list[1] = 0, list[2 ..] = them,
// heaviest first.
cudaError_t launch_tile_list(const uint64_t *vis_a, float4 *rgba, const CamDev &cam, int th, int *list,
                             cudaStream_t st);
cudaError_t launch_resolve_adjoint(const CallTable &tab, const CamDev &cam, const LightsDev &Ls, const FilterDev &fp,
                                   const uint64_t *vis_c, const uint64_t *vis_a, const float *grad_rgba,
                                   float *const *glv, float *const *galb, void *scratch, uint32_t *status,
                                   cudaStream_t st);
cudaError_t launch_raster_msaa(const CallTable &tab, const CamDev &cam, int samples, uint64_t *vis_s,
                               hm_frame_stats *stats, cudaStream_t st);
cudaError_t launch_resolve_msaa(const CallTable &tab, const CamDev &cam, const LightsDev &Ls, int samples,
                                const uint64_t *vis_s, float *rgba, uint32_t *status, cudaStream_t st);
cudaError_t launch_pack_float3(const float *src, float4 *dst, int64_t n, cudaStream_t st);

}  // namespace hm
