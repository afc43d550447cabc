// hm_api.cu -- the C ABI declared in include/hm.h: argument validation, groom
// upload, per-call groom tables, kernel launches, device status.
#include <cmath>
#include <atomic>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/hm.h"
#include "hm_device.cuh"
#include "hm_kernels.h"

struct hm_groom_s {
    int32_t L, V, F, segs;
    int64_t S;
    float width_m, roughness, tilt;
    hm_lod_params lod;
    int device;
    int has_ao;
    size_t max_batches;
    float4 *d_lv;
    int4 *d_faces;
    uint32_t *d_sface;
    float2 *d_bary;
    float4 *d_albedo;
    float *d_delta;
    uint4 *d_lod;
    uint32_t *d_batch_map;
    uint32_t *d_counters;
    // full-detail LOD state of the shadow-map pass, kept apart from the camera's
    uint4 *d_lod_full;
    uint32_t *d_batch_map_full;
    uint32_t *d_counters_full;
    float2 *d_uv;            // scalp texture coordinates, or null
    // control points of every drawn segment, written by the camera renders
    // (two float4 per segment at full detail); valid while they match the
    // LOD state of the last camera render and the current layer vertices
    float4 *d_segpts;
    bool segpts_valid;
    // workspace of the binned rasterizer when this groom is the first of a
    // call (grown on demand), or null
    void *d_bin_ws;
    size_t bin_ws_bytes;
};

namespace {

thread_local std::string g_last_error;

// One device status word per device (set by device-side consistency checks).
__device__ uint32_t g_device_status;

hm_status fail(hm_status s, const char *msg) {
    g_last_error = msg;
    return s;
}

hm_status cuda_fail(cudaError_t e, const char *where) {
    g_last_error = std::string(where) + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? HM_ERR_OOM : HM_ERR_CUDA;
}

#define HM_CUDA(call, where)                          \
    do {                                              \
        cudaError_t e_ = (call);                      \
        if (e_ != cudaSuccess) return cuda_fail(e_, where); \
    } while (0)

bool finite_all(const float *v, int n) {
    for (int i = 0; i < n; ++i)
        if (!std::isfinite(v[i])) return false;
    return true;
}

uint32_t *status_word() {
    static hm::PerDevice<uint32_t *> addr;
    return addr.get([](int) {
        void *p = nullptr;
        return cudaGetSymbolAddress(&p, g_device_status) == cudaSuccess ? static_cast<uint32_t *>(p) : nullptr;
    });
}

hm_status check_camera(const hm_camera *cam) {
    if (!cam) return fail(HM_ERR_INVALID_ARG, "camera is NULL");
    if (cam->width < 1 || cam->height < 1 || cam->width > HM_MAX_RESOLUTION || cam->height > HM_MAX_RESOLUTION)
        return fail(HM_ERR_INVALID_ARG, "resolution out of range");
    if (!finite_all(cam->view_proj, 16) || !finite_all(cam->cam_pos, 3))
        return fail(HM_ERR_INVALID_ARG, "camera has non-finite values");
    if (!(cam->near_m > 0.0f) || !(cam->far_m > cam->near_m) || !std::isfinite(cam->far_m))
        return fail(HM_ERR_INVALID_ARG, "need 0 < near < far");
    if (!(cam->tan_half_fovy > 0.0f) || !std::isfinite(cam->tan_half_fovy))
        return fail(HM_ERR_INVALID_ARG, "tan_half_fovy must be positive");
    if (cam->key_layout != HM_KEYS_ROW_MAJOR && cam->key_layout != HM_KEYS_BLOCK_2X2)
        return fail(HM_ERR_INVALID_ARG, "key_layout must be HM_KEYS_ROW_MAJOR or HM_KEYS_BLOCK_2X2");
    return HM_OK;
}

// Keys in one key layer of the camera's frames (row-major, or 2 x 2 blocks
// with odd sizes padded); 0 for an invalid size or layout.
int64_t vis_keys(const hm_camera *c) {
    if (!c || c->width < 1 || c->height < 1) return 0;
    if (c->key_layout == HM_KEYS_ROW_MAJOR) return (int64_t)c->width * c->height;
    if (c->key_layout == HM_KEYS_BLOCK_2X2) return 4 * (int64_t)((c->width + 1) / 2) * ((c->height + 1) / 2);
    return 0;
}

hm::CamDev cam_dev(const hm_camera *c) {
    hm::CamDev d;
    std::memcpy(d.m, c->view_proj, sizeof d.m);
    std::memcpy(d.cam_pos, c->cam_pos, sizeof d.cam_pos);
    d.near_m = c->near_m;
    d.far_m = c->far_m;
    d.tan_half = c->tan_half_fovy;
    d.W = c->width;
    d.H = c->height;
    d.layout = c->key_layout;
    d.Wb = (c->width + 1) / 2;
    return d;
}

hm_status build_table(const hm_groom *grooms, int32_t n, hm::CallTable &tab) {
    if (!grooms) return fail(HM_ERR_INVALID_ARG, "grooms is NULL");
    if (n < 1 || n > HM_MAX_GROOMS_PER_CALL) return fail(HM_ERR_INVALID_ARG, "groom count out of range");
    int dev = 0;
    cudaGetDevice(&dev);
    std::memset(&tab, 0, sizeof tab);
    tab.n = n;
    uint64_t base = 0;
    for (int i = 0; i < n; ++i) {
        const hm_groom g = grooms[i];
        if (!g) return fail(HM_ERR_INVALID_ARG, "groom handle is NULL");
        if (g->device != dev) return fail(HM_ERR_INVALID_ARG, "groom lives on another device");
        for (int k = 0; k < i; ++k)
            if (grooms[k] == g) return fail(HM_ERR_INVALID_ARG, "groom appears twice in one call");
        hm::GroomDev &d = tab.g[i];
        d.lv = g->d_lv;
        d.faces = g->d_faces;
        d.sface = g->d_sface;
        d.bary = g->d_bary;
        d.albedo = g->d_albedo;
        d.delta = g->d_delta;
        d.lod = g->d_lod;
        d.batch_map = g->d_batch_map;
        d.counters = g->d_counters;
        d.L = g->L;
        d.V = g->V;
        d.F = g->F;
        d.cmax = g->segs + 1;
        d.S = g->S;
        d.base = base;
        d.width_m = g->width_m;
        d.roughness = g->roughness;
        d.tilt = g->tilt;
        d.lod_lambda = g->lod.lambda;
        d.lod_enabled = g->lod.enabled;
        d.has_ao = g->has_ao;
        d.uv = g->d_uv;
        d.max_batches = (uint32_t)g->max_batches;
        d.segpts = g->segpts_valid ? g->d_segpts : nullptr;
        base += (uint64_t)g->S;
    }
    if (base > (1ull << 33) - 2) return fail(HM_ERR_CAPACITY, "strand ids exceed 33 bits");
    return HM_OK;
}

// Failure injection for tests: with HM_FAIL_ALLOC_AFTER=N in the
// environment, the library's device allocations after the first N report
// HM_ERR_OOM without calling the allocator (read once per process).
bool injected_alloc_failure() {
    static const long limit = [] {
        const char *e = std::getenv("HM_FAIL_ALLOC_AFTER");
        return e ? std::strtol(e, nullptr, 10) : -1L;
    }();
    static std::atomic<long> done{0};
    if (limit < 0) return false;
    return done.fetch_add(1) >= limit;
}

template <typename T>
hm_status dev_alloc(T **p, size_t count, const char *what) {
    *p = nullptr;
    if (count == 0) count = 1;
    if (injected_alloc_failure()) return fail(HM_ERR_OOM, "device allocation failed (injected by HM_FAIL_ALLOC_AFTER)");
    cudaError_t e = cudaMalloc(reinterpret_cast<void **>(p), count * sizeof(T));
    if (e != cudaSuccess) return cuda_fail(e, what);
    return HM_OK;
}

void free_groom(hm_groom g) {
    if (!g) return;
    cudaFree(g->d_lv);
    cudaFree(g->d_faces);
    cudaFree(g->d_sface);
    cudaFree(g->d_bary);
    cudaFree(g->d_albedo);
    cudaFree(g->d_delta);
    cudaFree(g->d_lod);
    cudaFree(g->d_batch_map);
    cudaFree(g->d_counters);
    cudaFree(g->d_segpts);
    cudaFree(g->d_lod_full);
    cudaFree(g->d_batch_map_full);
    cudaFree(g->d_counters_full);
    cudaFree(g->d_uv);
    cudaFree(g->d_bin_ws);
    delete g;
}

thread_local void *g_phase_events[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};

void phase(int i, cudaStream_t s) {
    if (g_phase_events[i]) cudaEventRecord(static_cast<cudaEvent_t>(g_phase_events[i]), s);
}

// Launch-shape tuning shared by every call of the process (hm_set_tuning).
// Defaults: plain atomics (on B300 the read-before-atomic variant is slower:
// 1.28 vs 1.07 ms per 1080p frame), the 64-register raster, as many raster
// CTAs per SM as fit, 32x32 resolve tiles.
hm_tuning g_tuning = {0, 4, 0, 32, 0, 0, 0, 0};   // direct rasterizer

bool valid_tuning(const hm_tuning &t) {
    const bool direct = t.raster_bin_w == 0 && t.raster_bin_h == 0 && t.raster_bin_chunk == 0;
    const bool binned = (t.raster_bin_w == 16 || t.raster_bin_w == 32) &&
                        (t.raster_bin_h == 16 || t.raster_bin_h == 32) &&
                        (t.raster_bin_chunk == 256 || t.raster_bin_chunk == 1024);
    return (t.raster_precheck == 0 || t.raster_precheck == 1) &&
           (t.raster_min_blocks == 3 || t.raster_min_blocks == 4) && t.raster_ctas_per_sm >= 0 &&
           t.raster_ctas_per_sm <= 32 && (t.resolve_tile_h == 16 || t.resolve_tile_h == 32) && (direct || binned);
}

}  // namespace

namespace hm {
int num_sms() {
    static PerDevice<int> count;
    const int v = count.get([](int dev) {
        int n = 0;
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        return n;
    });
    return v > 0 ? v : 1;
}
}  // namespace hm

extern "C" {

const char *hm_status_string(hm_status s) {
    switch (s) {
        case HM_OK: return "HM_OK";
        case HM_ERR_INVALID_ARG: return "HM_ERR_INVALID_ARG";
        case HM_ERR_OOM: return "HM_ERR_OOM";
        case HM_ERR_CUDA: return "HM_ERR_CUDA";
        case HM_ERR_CAPACITY: return "HM_ERR_CAPACITY";
        case HM_ERR_TIMEOUT: return "HM_ERR_TIMEOUT";
        case HM_ERR_NOT_READY: return "HM_ERR_NOT_READY";
        case HM_ERR_DEVICE_CHECK: return "HM_ERR_DEVICE_CHECK";
    }
    return "HM_ERR_UNKNOWN";
}

const char *hm_last_error(void) { return g_last_error.c_str(); }

hm_status hm_create_groom(const hm_groom_desc *d, void *stream, hm_groom *out) {
    if (!d || !out) return fail(HM_ERR_INVALID_ARG, "desc/out is NULL");
    *out = nullptr;
    const int32_t L = d->num_layers, V = d->num_verts, F = d->num_faces, segs = d->segments_per_strand;
    const int64_t S = d->num_strands;
    if (L < 2 || L > HM_MAX_LAYERS) return fail(HM_ERR_INVALID_ARG, "num_layers out of 2..HM_MAX_LAYERS");
    if (V < 3 || F < 1) return fail(HM_ERR_INVALID_ARG, "need V >= 3 and F >= 1");
    if (segs < 1 || segs > HM_MAX_SEGMENTS) return fail(HM_ERR_INVALID_ARG, "segments_per_strand out of range");
    if (S < 0) return fail(HM_ERR_INVALID_ARG, "num_strands < 0");
    if (S > 0x7FFFFFFFll) return fail(HM_ERR_CAPACITY, "more than 2^31 - 1 strands in one groom");
    if ((int64_t)L * V > (1ll << 28)) return fail(HM_ERR_CAPACITY, "hair mesh too large");
    if (!d->layer_verts || !d->faces || !d->bundle_delta)
        return fail(HM_ERR_INVALID_ARG, "layer_verts/faces/bundle_delta is NULL");
    if (S > 0 && (!d->strand_face || !d->strand_bary || !d->strand_albedo))
        return fail(HM_ERR_INVALID_ARG, "strand arrays are NULL");
    if (!finite_all(d->layer_verts, L * V * 3)) return fail(HM_ERR_INVALID_ARG, "non-finite layer vertex");
    if (d->vert_ao)
        for (int64_t i = 0; i < (int64_t)L * V; ++i)
            if (!(d->vert_ao[i] >= 0.0f && d->vert_ao[i] <= 1.0f))
                return fail(HM_ERR_INVALID_ARG, "vert_ao outside [0, 1]");
    if (d->vert_uv)
        for (int64_t i = 0; i < 2ll * V; ++i)
            if (!(d->vert_uv[i] >= 0.0f && d->vert_uv[i] <= 1.0f))
                return fail(HM_ERR_INVALID_ARG, "vert_uv outside [0, 1]");
    if (!(d->strand_width_m > 0.0f) || !std::isfinite(d->strand_width_m) || !(d->roughness > 0.0f) ||
        !std::isfinite(d->tilt))
        return fail(HM_ERR_INVALID_ARG, "strand width / roughness must be positive, tilt finite");
    for (int64_t i = 0; i < 3ll * F; ++i)
        if (d->faces[i] < 0 || d->faces[i] >= V) return fail(HM_ERR_INVALID_ARG, "face index out of range");
    for (int32_t f = 0; f < F; ++f)
        if (!(d->bundle_delta[f] >= 0.0f && d->bundle_delta[f] < 1.0f))
            return fail(HM_ERR_INVALID_ARG, "bundle_delta outside [0, 1)");
    std::vector<int32_t> first(F + 1, 0);
    for (int64_t s = 0; s < S; ++s) {
        uint32_t f = d->strand_face[s];
        if (f >= (uint32_t)F) return fail(HM_ERR_INVALID_ARG, "strand_face out of range");
        if (s > 0 && f < d->strand_face[s - 1]) return fail(HM_ERR_INVALID_ARG, "strand_face not ascending");
        float b1 = d->strand_bary[2 * s], b2 = d->strand_bary[2 * s + 1];
        if (!(b1 >= 0.0f && b1 <= 1.0f && b2 >= 0.0f && b2 <= 1.0f))
            return fail(HM_ERR_INVALID_ARG, "barycentric outside [0, 1]");
        first[f + 1]++;
    }
    for (int32_t f = 0; f < F; ++f) first[f + 1] += first[f];
    // work-list batches at full detail: S (segs + 1) control points, a batch
    // per kBatchStride of them (plus one)
    const uint64_t max_points = (uint64_t)S * (uint64_t)(segs + 1);
    if (max_points > 0xFFFFFF00ull)
        return fail(HM_ERR_CAPACITY, "too many control points in one groom (32-bit index)");
    const size_t max_batches = (size_t)(max_points / hm::kBatchStride + 2);

    // host-side repack to the device layout
    std::vector<float4> lv((size_t)L * V);
    for (size_t i = 0; i < lv.size(); ++i)
        lv[i] = make_float4(d->layer_verts[3 * i], d->layer_verts[3 * i + 1], d->layer_verts[3 * i + 2],
                            d->vert_ao ? d->vert_ao[i] : 1.0f);
    std::vector<int4> faces((size_t)F + 1);
    for (int32_t f = 0; f < F; ++f)
        faces[f] = make_int4(d->faces[3 * f], d->faces[3 * f + 1], d->faces[3 * f + 2], first[f]);
    faces[F] = make_int4(0, 0, 0, first[F]);
    std::vector<float4> alb((size_t)(S > 0 ? S : 1));
    for (int64_t s = 0; s < S; ++s)
        alb[s] = make_float4(d->strand_albedo[3 * s], d->strand_albedo[3 * s + 1], d->strand_albedo[3 * s + 2], 0.0f);

    hm_groom g = new hm_groom_s();
    std::memset(g, 0, sizeof *g);
    g->L = L;
    g->V = V;
    g->F = F;
    g->segs = segs;
    g->S = S;
    g->width_m = d->strand_width_m;
    g->roughness = d->roughness;
    g->tilt = d->tilt;
    g->lod.enabled = 0;
    g->lod.lambda = 3.0f;
    g->has_ao = d->vert_ao ? 1 : 0;
    g->max_batches = max_batches;
    cudaGetDevice(&g->device);
    hm_status st = HM_OK;
#define HM_ALLOC(ptr, n, what) \
    if (st == HM_OK) st = dev_alloc(&(ptr), (n), what);
    HM_ALLOC(g->d_lv, lv.size(), "alloc layer_verts")
    HM_ALLOC(g->d_faces, faces.size(), "alloc faces")
    HM_ALLOC(g->d_sface, (size_t)S, "alloc strand_face")
    HM_ALLOC(g->d_bary, (size_t)S, "alloc strand_bary")
    HM_ALLOC(g->d_albedo, (size_t)S, "alloc strand_albedo")
    HM_ALLOC(g->d_delta, (size_t)F, "alloc bundle_delta")
    HM_ALLOC(g->d_lod, (size_t)F, "alloc lod")
    HM_ALLOC(g->d_batch_map, max_batches, "alloc batch map")
    HM_ALLOC(g->d_counters, (size_t)hm::kCtrWords, "alloc counters")
    HM_ALLOC(g->d_lod_full, (size_t)F, "alloc shadow-pass lod")
    HM_ALLOC(g->d_batch_map_full, max_batches, "alloc shadow-pass batch map")
    HM_ALLOC(g->d_counters_full, (size_t)hm::kCtrWords, "alloc shadow-pass counters")
    if (d->vert_uv) HM_ALLOC(g->d_uv, (size_t)V, "alloc vert_uv")
    HM_ALLOC(g->d_segpts, 2 * (size_t)S * (size_t)segs, "alloc segment records")
#undef HM_ALLOC
    if (st != HM_OK) {
        free_groom(g);
        return st;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaSuccess;
    auto cp = [&](void *dst, const void *src, size_t bytes) {
        if (e == cudaSuccess && bytes) e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, s);
    };
    cp(g->d_lv, lv.data(), lv.size() * sizeof(float4));
    cp(g->d_faces, faces.data(), faces.size() * sizeof(int4));
    cp(g->d_sface, d->strand_face, (size_t)S * sizeof(uint32_t));
    cp(g->d_bary, d->strand_bary, (size_t)S * sizeof(float2));
    cp(g->d_albedo, alb.data(), (size_t)S * sizeof(float4));
    cp(g->d_delta, d->bundle_delta, (size_t)F * sizeof(float));
    if (d->vert_uv) cp(g->d_uv, d->vert_uv, (size_t)V * sizeof(float2));
    if (e == cudaSuccess) e = cudaMemsetAsync(g->d_counters, 0, hm::kCtrWords * sizeof(uint32_t), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(g->d_counters_full, 0, hm::kCtrWords * sizeof(uint32_t), s);
    // LOD state starts at full detail so a resolve before any render decodes safely
    if (e == cudaSuccess) {
        std::vector<uint4> lod0(F);
        for (int32_t f = 0; f < F; ++f) lod0[f] = make_uint4(first[f + 1] - first[f], segs + 1, 0, 0);
        e = cudaMemcpyAsync(g->d_lod, lod0.data(), (size_t)F * sizeof(uint4), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    }
    if (e != cudaSuccess) {
        free_groom(g);
        return cuda_fail(e, "upload groom");
    }
    *out = g;
    return HM_OK;
}

hm_status hm_destroy_groom(hm_groom g) {
    if (!g) return fail(HM_ERR_INVALID_ARG, "groom is NULL");
    free_groom(g);
    return HM_OK;
}

hm_status hm_set_lod(hm_groom g, const hm_lod_params *p) {
    if (!g || !p) return fail(HM_ERR_INVALID_ARG, "groom/params is NULL");
    if (p->enabled && !(p->lambda >= 0.0f && std::isfinite(p->lambda)))
        return fail(HM_ERR_INVALID_ARG, "lambda must be finite and >= 0");
    g->lod = *p;
    return HM_OK;
}

hm_status hm_update_layer_verts(hm_groom g, const float *d_layer_verts, void *stream) {
    if (!g || !d_layer_verts) return fail(HM_ERR_INVALID_ARG, "groom/buffer is NULL");
    g->segpts_valid = false;     // the recorded control points are of the old vertices
    HM_CUDA(hm::launch_pack_float3(d_layer_verts, g->d_lv, (int64_t)g->L * g->V, static_cast<cudaStream_t>(stream)),
            "pack layer verts");
    return HM_OK;
}

hm_status hm_update_albedo(hm_groom g, const float *d_albedo, void *stream) {
    if (!g || (!d_albedo && g->S > 0)) return fail(HM_ERR_INVALID_ARG, "groom/buffer is NULL");
    if (g->S == 0) return HM_OK;
    HM_CUDA(hm::launch_pack_float3(d_albedo, g->d_albedo, g->S, static_cast<cudaStream_t>(stream)), "pack albedo");
    return HM_OK;
}

hm_status hm_render_visibility(const hm_groom *grooms, int32_t n, const hm_camera *cam, uint64_t *d_vis_center,
                               uint64_t *d_vis_cons, const uint32_t *d_scene_d24, int32_t clear,
                               hm_frame_stats *d_stats, void *stream) {
    return hm_render_visibility_range(grooms, n, 0, n, cam, d_vis_center, d_vis_cons, d_scene_d24, clear, d_stats,
                                      stream);
}

// The binned rasterizer's workspace for a call whose first groom is
// `owner`: kept in the groom and grown when a call needs more (after a device
// synchronize, since earlier frames may still use it); never grown during
// stream capture.
static hm_status bin_workspace(hm_groom owner, size_t need, cudaStream_t s, void **ws) {
    if (need == 0) return fail(HM_ERR_CAPACITY, "binned rasterizer: too many segments for its 32-bit pair list");
    if (owner->bin_ws_bytes < need) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        HM_CUDA(cudaStreamIsCapturing(s, &cs), "capture status");
        if (cs != cudaStreamCaptureStatusNone)
            return fail(HM_ERR_CAPACITY, "binned rasterizer workspace must grow: render once outside stream capture");
        HM_CUDA(cudaDeviceSynchronize(), "sync before growing the binned workspace");
        cudaFree(owner->d_bin_ws);
        owner->d_bin_ws = nullptr;
        owner->bin_ws_bytes = 0;
        char *p = nullptr;
        hm_status st = dev_alloc(&p, need, "binned rasterizer workspace");
        if (st != HM_OK) return st;
        owner->d_bin_ws = p;
        owner->bin_ws_bytes = need;
    }
    *ws = owner->d_bin_ws;
    return HM_OK;
}

static hm_status render_views(const hm_groom *grooms, int32_t n, int32_t first, int32_t count, const hm_camera *cams,
                               int32_t n_views, uint64_t *const *d_vis_center, uint64_t *const *d_vis_cons,
                               const uint32_t *const *d_scene_d24, int32_t clear, hm_frame_stats *d_stats,
                               void *stream, bool compressed = false) {
    if (!cams || n_views < 1 || n_views > HM_MAX_VIEWS) return fail(HM_ERR_INVALID_ARG, "view count out of range");
    if (!d_vis_center || !d_vis_cons) return fail(HM_ERR_INVALID_ARG, "visibility buffer array is NULL");
    hm_status st;
    for (int v = 0; v < n_views; ++v) {
        if ((st = check_camera(&cams[v])) != HM_OK) return st;
        if (cams[v].width != cams[0].width || cams[v].height != cams[0].height ||
            cams[v].key_layout != cams[0].key_layout)
            return fail(HM_ERR_INVALID_ARG, "views must share width, height and key layout");
        uint64_t *vc = d_vis_center[v], *va = d_vis_cons[v];
        if (!vc || !va) return fail(HM_ERR_INVALID_ARG, "visibility buffer is NULL");
        if ((reinterpret_cast<uintptr_t>(vc) & 15) || (reinterpret_cast<uintptr_t>(va) & 15))
            return fail(HM_ERR_INVALID_ARG, "visibility buffers must be 16-byte aligned");
        if (vc == va) return fail(HM_ERR_INVALID_ARG, "the two layers must be distinct buffers");
        for (int u = 0; u < v; ++u)
            if (d_vis_center[u] == vc || d_vis_cons[u] == va || d_vis_center[u] == va || d_vis_cons[u] == vc)
                return fail(HM_ERR_INVALID_ARG, "views must use distinct buffers");
    }
    if (first < 0 || count < 1 || first > n - count) return fail(HM_ERR_INVALID_ARG, "groom range outside 0..n");
    hm::CallTable full;
    st = build_table(grooms, n, full);
    if (st != HM_OK) return st;
    hm::CallTable tab;
    std::memset(&tab, 0, sizeof tab);
    tab.n = count;
    for (int i = 0; i < count; ++i) {
        tab.g[i] = full.g[first + i];   // keeps the whole array's strand ids
        tab.g[i].segpts = grooms[first + i]->d_segpts;
    }
    hm::ViewSet views;
    std::memset(&views, 0, sizeof views);
    views.n = n_views;
    for (int v = 0; v < n_views; ++v) {
        views.cam[v] = cam_dev(&cams[v]);
        views.vis_c[v] = d_vis_center[v];
        views.vis_a[v] = d_vis_cons[v];
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int64_t nkeys = vis_keys(&cams[0]);
    const bool binned = g_tuning.raster_bin_w != 0 && n_views == 1 && !compressed;
    void *bin_ws = nullptr;
    uint64_t bin_slots = 0;
    uint32_t *sw = nullptr;
    if (binned) {
        for (int i = 0; i < count; ++i) bin_slots += (uint64_t)tab.g[i].max_batches * hm::kBatchLanes;
        st = bin_workspace(grooms[first],
                           hm::binned_workspace_bytes(bin_slots, cams[0].width, cams[0].height, g_tuning.raster_bin_w,
                                                      g_tuning.raster_bin_h),
                           s, &bin_ws);
        if (st != HM_OK) return st;
        sw = status_word();
        if (!sw) return fail(HM_ERR_CUDA, "device status word unavailable");
    }
    phase(0, s);
    for (int v = 0; v < n_views; ++v)
        HM_CUDA(hm::launch_clear(d_vis_center[v], d_vis_cons[v], nkeys, d_scene_d24 ? d_scene_d24[v] : nullptr,
                                 views.cam[v], clear, v == 0 ? d_stats : nullptr, s),
                "clear");
    phase(1, s);
    for (int i = 0; i < count; ++i) grooms[first + i]->segpts_valid = false;   // until the raster has rewritten them
    HM_CUDA(hm::launch_lod(tab, views.cam[0], d_stats, s), "lod");
    phase(2, s);
    if (binned)
        HM_CUDA(hm::launch_raster_binned(tab, views.cam[0], d_vis_center[0], d_vis_cons[0], bin_ws, bin_slots,
                                         g_tuning.raster_bin_w, g_tuning.raster_bin_h, g_tuning.raster_bin_chunk, sw,
                                         d_stats, s),
                "raster binned");
    else
        HM_CUDA(hm::launch_raster(tab, views, g_tuning.raster_precheck != 0, g_tuning.raster_min_blocks,
                                  g_tuning.raster_ctas_per_sm, d_stats, s, compressed),
                "raster");
    phase(3, s);
    for (int i = 0; i < count; ++i) grooms[first + i]->segpts_valid = true;
    return HM_OK;
}

static hm_status lights_dev(const hm_lights *l, hm::LightsDev &ld);

hm_status hm_render_shadow_map(const hm_groom *grooms, int32_t n, const hm_camera *light_cam,
                               uint64_t *d_map_center, uint64_t *d_map_cons, hm_frame_stats *d_stats,
                               void *stream) {
    hm_status st = check_camera(light_cam);
    if (st != HM_OK) return st;
    if (!d_map_center || !d_map_cons) return fail(HM_ERR_INVALID_ARG, "shadow map buffer is NULL");
    if ((reinterpret_cast<uintptr_t>(d_map_center) & 15) || (reinterpret_cast<uintptr_t>(d_map_cons) & 15))
        return fail(HM_ERR_INVALID_ARG, "shadow map buffers must be 16-byte aligned");
    if (d_map_center == d_map_cons) return fail(HM_ERR_INVALID_ARG, "the two layers must be distinct buffers");
    hm::CallTable tab;
    if ((st = build_table(grooms, n, tab)) != HM_OK) return st;
    for (int i = 0; i < n; ++i) {
        // full geometry into the pass's own LOD buffers
        tab.g[i].lod = grooms[i]->d_lod_full;
        tab.g[i].batch_map = grooms[i]->d_batch_map_full;
        tab.g[i].counters = grooms[i]->d_counters_full;
        tab.g[i].lod_enabled = 0;
        tab.g[i].segpts = nullptr;      // the records follow the camera's LOD state, not this pass's
    }
    hm::ViewSet views;
    std::memset(&views, 0, sizeof views);
    views.n = 1;
    views.cam[0] = cam_dev(light_cam);
    views.vis_c[0] = d_map_center;
    views.vis_a[0] = d_map_cons;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    phase(0, s);
    HM_CUDA(hm::launch_clear(d_map_center, d_map_cons, vis_keys(light_cam), nullptr, views.cam[0], 1, d_stats, s),
            "clear");
    phase(1, s);
    HM_CUDA(hm::launch_lod(tab, views.cam[0], d_stats, s), "lod");
    phase(2, s);
    HM_CUDA(hm::launch_raster(tab, views, g_tuning.raster_precheck != 0, g_tuning.raster_min_blocks,
                              g_tuning.raster_ctas_per_sm, d_stats, s),
            "raster");
    phase(3, s);
    return HM_OK;
}

hm_status hm_render_visibility_msaa(const hm_groom *grooms, int32_t n, const hm_camera *cam, int32_t samples,
                                    uint64_t *d_vis_samples, int32_t clear, hm_frame_stats *d_stats, void *stream) {
    hm_status st = check_camera(cam);
    if (st != HM_OK) return st;
    if (cam->key_layout != HM_KEYS_ROW_MAJOR) return fail(HM_ERR_INVALID_ARG, "sample planes are row-major");
    if (samples != 1 && samples != 2 && samples != 4 && samples != 8)
        return fail(HM_ERR_INVALID_ARG, "samples must be 1, 2, 4 or 8");
    if (!d_vis_samples || (reinterpret_cast<uintptr_t>(d_vis_samples) & 15))
        return fail(HM_ERR_INVALID_ARG, "sample layers NULL or not 16-byte aligned");
    hm::CallTable tab;
    if ((st = build_table(grooms, n, tab)) != HM_OK) return st;
    for (int i = 0; i < n; ++i) tab.g[i].segpts = grooms[i]->d_segpts;
    const hm::CamDev cd = cam_dev(cam);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int64_t npx = (int64_t)cam->width * cam->height;
    // the sample planes are contiguous: cleared as one flat array (one pointer
    // given twice, written once)
    phase(0, s);
    HM_CUDA(hm::launch_clear(d_vis_samples, d_vis_samples, npx * samples, nullptr, cd, clear, d_stats, s), "clear");
    phase(1, s);
    for (int i = 0; i < n; ++i) grooms[i]->segpts_valid = false;   // until the raster has rewritten them
    HM_CUDA(hm::launch_lod(tab, cd, d_stats, s), "lod");
    phase(2, s);
    HM_CUDA(hm::launch_raster_msaa(tab, cd, samples, d_vis_samples, d_stats, s), "raster msaa");
    phase(3, s);
    for (int i = 0; i < n; ++i) grooms[i]->segpts_valid = true;
    return HM_OK;
}

hm_status hm_resolve_msaa(const hm_groom *grooms, int32_t n, const hm_camera *cam, const hm_lights *lights,
                          int32_t samples, const uint64_t *d_vis_samples, float *d_rgba, void *stream) {
    hm_status st = check_camera(cam);
    if (st != HM_OK) return st;
    if (cam->key_layout != HM_KEYS_ROW_MAJOR) return fail(HM_ERR_INVALID_ARG, "sample planes are row-major");
    if (samples != 1 && samples != 2 && samples != 4 && samples != 8)
        return fail(HM_ERR_INVALID_ARG, "samples must be 1, 2, 4 or 8");
    if (!d_vis_samples || !d_rgba || (reinterpret_cast<uintptr_t>(d_rgba) & 15) ||
        (reinterpret_cast<uintptr_t>(d_vis_samples) & 7))
        return fail(HM_ERR_INVALID_ARG, "buffer NULL or misaligned");
    hm::LightsDev ld;
    if ((st = lights_dev(lights, ld)) != HM_OK) return st;
    hm::CallTable tab;
    if ((st = build_table(grooms, n, tab)) != HM_OK) return st;
    uint32_t *sw = status_word();
    if (!sw) return fail(HM_ERR_CUDA, "device status word unavailable");
    phase(4, static_cast<cudaStream_t>(stream));
    HM_CUDA(hm::launch_resolve_msaa(tab, cam_dev(cam), ld, samples, d_vis_samples, d_rgba, sw,
                                    static_cast<cudaStream_t>(stream)),
            "resolve msaa");
    phase(5, static_cast<cudaStream_t>(stream));
    return HM_OK;
}

hm_status hm_render_visibility_multiview(const hm_groom *grooms, int32_t n, const hm_camera *cams, int32_t n_views,
                                         uint64_t *const *d_vis_center, uint64_t *const *d_vis_cons,
                                         const uint32_t *const *d_scene_d24, int32_t clear, hm_frame_stats *d_stats,
                                         void *stream) {
    return render_views(grooms, n, 0, n, cams, n_views, d_vis_center, d_vis_cons, d_scene_d24, clear, d_stats, stream);
}

hm_status hm_render_visibility_range(const hm_groom *grooms, int32_t n, int32_t first, int32_t count,
                                     const hm_camera *cam, uint64_t *d_vis_center, uint64_t *d_vis_cons,
                                     const uint32_t *d_scene_d24, int32_t clear, hm_frame_stats *d_stats,
                                     void *stream) {
    return render_views(grooms, n, first, count, cam, 1, &d_vis_center, &d_vis_cons,
                        d_scene_d24 ? &d_scene_d24 : nullptr, clear, d_stats, stream);
}

hm_status hm_render_visibility_compressed(const hm_groom *grooms, int32_t n, const hm_camera *cam,
                                          uint64_t *d_vis_center, uint64_t *d_vis_cons,
                                          const uint32_t *d_scene_d24, int32_t clear, hm_frame_stats *d_stats,
                                          void *stream) {
    return render_views(grooms, n, 0, n, cam, 1, &d_vis_center, &d_vis_cons, d_scene_d24 ? &d_scene_d24 : nullptr,
                        clear, d_stats, stream, true);
}

static hm_status filter_dev(const hm_filter_params *f, const hm_camera *cam, hm::FilterDev &fd) {
    if (!f) return fail(HM_ERR_INVALID_ARG, "filter params are NULL");
    std::memset(&fd, 0, sizeof fd);
    fd.enabled = f->enabled ? 1 : 0;
    if (!fd.enabled) return HM_OK;
    if (f->radius < 0 || f->radius > HM_MAX_FILTER_RADIUS) return fail(HM_ERR_INVALID_ARG, "radius out of range");
    if (!(f->s_par > 0.0f) || !(f->s_perp > 0.0f) || !(f->sigma_c > 0.0f) || !(f->iso_scale > 0.0f) ||
        !(f->strip_halfwidth >= 0.0f) || !(f->depth_reject_m >= 0.0f) || !(f->depth_mismatch_m >= 0.0f))
        return fail(HM_ERR_INVALID_ARG, "filter widths must be positive");
    fd.radius = f->radius;
    const float r = (float)(f->radius > 0 ? f->radius : 1);
    const float sp = f->s_par * r, sq = f->s_perp * r, si = f->iso_scale * r;
    fd.inv_spar2 = 1.0f / (sp * sp);
    fd.inv_sperp2 = 1.0f / (sq * sq);
    fd.inv_siso2 = 1.0f / (si * si);
    fd.inv_sc2 = 1.0f / (f->sigma_c * f->sigma_c);
    volatile float hw = f->strip_halfwidth;
    fd.hw2 = hw * hw;
    fd.hw = hw;
    const double span = (double)cam->far_m - (double)cam->near_m;
    const double rej = std::floor((double)f->depth_reject_m / span * 16777216.0 + 0.5);
    const double mis = std::floor((double)f->depth_mismatch_m / span * 16777216.0 + 0.5);
    fd.drej = (int32_t)(rej > 16777216.0 ? 16777216.0 : rej);
    fd.dmis = (int32_t)(mis > 16777216.0 ? 16777216.0 : mis);
    return HM_OK;
}

static hm_status lights_dev(const hm_lights *l, hm::LightsDev &ld) {
    if (!l) return fail(HM_ERR_INVALID_ARG, "lights are NULL");
    if (l->count < 0 || l->count > HM_MAX_LIGHTS) return fail(HM_ERR_INVALID_ARG, "light count out of range");
    std::memset(&ld, 0, sizeof ld);
    ld.n = l->count;
    std::memcpy(ld.dir, l->dir, sizeof ld.dir);
    std::memcpy(ld.rad, l->radiance, sizeof ld.rad);
    ld.ambient = l->ambient;
    ld.kd = l->k_d;
    ld.ks = l->k_s;
    for (int i = 0; i < HM_MAX_LIGHTS; ++i) ld.shadow_of[i] = -1;
    if (l->n_shadows < 0 || l->n_shadows > l->count)
        return fail(HM_ERR_INVALID_ARG, "shadow map count out of range");
    if (l->n_shadows > 0 && !l->shadows) return fail(HM_ERR_INVALID_ARG, "shadow maps are NULL");
    ld.n_shadow = l->n_shadows;
    for (int i = 0; i < l->n_shadows; ++i) {
        const hm_shadow_map &m = l->shadows[i];
        if (m.light < 0 || m.light >= l->count) return fail(HM_ERR_INVALID_ARG, "shadow map light out of range");
        if (ld.shadow_of[m.light] >= 0) return fail(HM_ERR_INVALID_ARG, "two shadow maps for one light");
        if (!m.d_map || (reinterpret_cast<uintptr_t>(m.d_map) & 7))
            return fail(HM_ERR_INVALID_ARG, "shadow map NULL or misaligned");
        if (!(m.sigma >= 0.0f) || !std::isfinite(m.sigma) || !(m.bias_m >= 0.0f) || !std::isfinite(m.bias_m) ||
            (m.depth_correction != 0 && m.depth_correction != 1))
            return fail(HM_ERR_INVALID_ARG, "shadow map sigma, bias or depth_correction invalid");
        hm_status st = check_camera(&m.cam);
        if (st != HM_OK) return st;
        ld.shadow_of[m.light] = i;
        ld.sh[i].map = m.d_map;
        ld.sh[i].cam = cam_dev(&m.cam);
        ld.sh[i].sigma = m.sigma;
        ld.sh[i].bias = m.bias_m;
        ld.sh[i].corr = m.depth_correction;
    }
    return HM_OK;
}

hm_status hm_resolve_shade(const hm_groom *grooms, int32_t n, const hm_camera *cam, const hm_lights *lights,
                           const hm_filter_params *filt, const uint64_t *d_vis_center, const uint64_t *d_vis_cons,
                           float *d_rgba, void *d_tile_scratch, void *stream) {
    hm_status st = check_camera(cam);
    if (st != HM_OK) return st;
    if (!d_vis_center || !d_vis_cons || !d_rgba) return fail(HM_ERR_INVALID_ARG, "buffer is NULL");
    if (reinterpret_cast<uintptr_t>(d_tile_scratch) & 15) return fail(HM_ERR_INVALID_ARG, "misaligned tile scratch");
    if ((reinterpret_cast<uintptr_t>(d_rgba) & 15) || (reinterpret_cast<uintptr_t>(d_vis_center) & 7) ||
        (reinterpret_cast<uintptr_t>(d_vis_cons) & 7))
        return fail(HM_ERR_INVALID_ARG, "misaligned buffer");
    hm::LightsDev ld;
    hm::FilterDev fd;
    if ((st = lights_dev(lights, ld)) != HM_OK) return st;
    if ((st = filter_dev(filt, cam, fd)) != HM_OK) return st;
    hm::CallTable tab;
    st = build_table(grooms, n, tab);
    if (st != HM_OK) return st;
    uint32_t *sw = status_word();
    if (!sw) return fail(HM_ERR_CUDA, "device status word unavailable");
    phase(4, static_cast<cudaStream_t>(stream));
    HM_CUDA(hm::launch_resolve(tab, cam_dev(cam), ld, fd, d_vis_center, d_vis_cons, d_rgba, sw,
                               g_tuning.resolve_tile_h, static_cast<cudaStream_t>(stream), nullptr,
                               static_cast<int *>(d_tile_scratch)),
            "resolve");
    phase(5, static_cast<cudaStream_t>(stream));
    return HM_OK;
}

size_t hm_resolve_scratch_bytes(int32_t width, int32_t height) {
    if (width < 1 || height < 1 || width > HM_MAX_RESOLUTION || height > HM_MAX_RESOLUTION) return 0;
    return hm::resolve_scratch_bytes(width, height);
}

hm_status hm_resolve_compressed(const hm_camera *cam, const hm_lights *lights, const hm_filter_params *filt,
                                const hm_appearance *appearance, const uint64_t *d_vis_center,
                                const uint64_t *d_vis_cons, float *d_rgba, void *stream) {
    hm_status st = check_camera(cam);
    if (st != HM_OK) return st;
    if (!d_vis_center || !d_vis_cons || !d_rgba) return fail(HM_ERR_INVALID_ARG, "buffer is NULL");
    if ((reinterpret_cast<uintptr_t>(d_rgba) & 15) || (reinterpret_cast<uintptr_t>(d_vis_center) & 7) ||
        (reinterpret_cast<uintptr_t>(d_vis_cons) & 7))
        return fail(HM_ERR_INVALID_ARG, "misaligned buffer");
    if (!appearance || !appearance->d_table || (reinterpret_cast<uintptr_t>(appearance->d_table) & 15))
        return fail(HM_ERR_INVALID_ARG, "appearance table NULL or not 16-byte aligned");
    if (!(appearance->roughness > 0.0f) || !std::isfinite(appearance->roughness) || !std::isfinite(appearance->tilt))
        return fail(HM_ERR_INVALID_ARG, "appearance roughness must be positive, tilt finite");
    hm::LightsDev ld;
    hm::FilterDev fd;
    if ((st = lights_dev(lights, ld)) != HM_OK) return st;
    if (ld.n_shadow != 0) return fail(HM_ERR_INVALID_ARG, "shadow maps need the strand-id payload");
    if ((st = filter_dev(filt, cam, fd)) != HM_OK) return st;
    hm::CallTable tab;
    std::memset(&tab, 0, sizeof tab);
    const hm::CgbDev cg{reinterpret_cast<const float4 *>(appearance->d_table), appearance->roughness,
                        appearance->tilt};
    uint32_t *sw = status_word();
    if (!sw) return fail(HM_ERR_CUDA, "device status word unavailable");
    phase(4, static_cast<cudaStream_t>(stream));
    HM_CUDA(hm::launch_resolve(tab, cam_dev(cam), ld, fd, d_vis_center, d_vis_cons, d_rgba, sw,
                               g_tuning.resolve_tile_h, static_cast<cudaStream_t>(stream), &cg),
            "resolve compressed");
    phase(5, static_cast<cudaStream_t>(stream));
    return HM_OK;
}

hm_status hm_set_tuning(const hm_tuning *t) {
    if (!t) return fail(HM_ERR_INVALID_ARG, "tuning is NULL");
    if (!valid_tuning(*t)) return fail(HM_ERR_INVALID_ARG, "tuning value out of range");
    g_tuning = *t;
    return HM_OK;
}

hm_status hm_get_tuning(hm_tuning *t) {
    if (!t) return fail(HM_ERR_INVALID_ARG, "tuning is NULL");
    *t = g_tuning;
    return HM_OK;
}

hm_status hm_set_phase_events(void *const *events, int32_t count) {
    if (count < 0 || count > 6) return fail(HM_ERR_INVALID_ARG, "count out of 0..6");
    for (int i = 0; i < 6; ++i) g_phase_events[i] = (events && i < count) ? events[i] : nullptr;
    return HM_OK;
}

hm_status hm_probe_atomic_min(uint64_t *d_buf, int64_t n, int32_t rounds, int32_t pattern, void *stream) {
    if (!d_buf || n < 1 || rounds < 1 || pattern < 0 || pattern > 2)
        return fail(HM_ERR_INVALID_ARG, "bad probe arguments");
    HM_CUDA(hm::launch_probe_atomic_min(d_buf, n, rounds, pattern, static_cast<cudaStream_t>(stream)), "probe");
    return HM_OK;
}

hm_status hm_probe_quotient(const float *d_num, const float *d_den, float *d_out, int64_t n, void *stream) {
    if (n < 0 || (n > 0 && (!d_num || !d_den || !d_out))) return fail(HM_ERR_INVALID_ARG, "bad probe arguments");
    HM_CUDA(hm::launch_probe_quotient(d_num, d_den, d_out, n, static_cast<cudaStream_t>(stream)), "probe");
    return HM_OK;
}

hm_status hm_get_lod(hm_groom g, int32_t *n_lod, int32_t *c, void *stream) {
    if (!g || !n_lod || !c) return fail(HM_ERR_INVALID_ARG, "NULL argument");
    std::vector<uint4> h(g->F);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    HM_CUDA(cudaMemcpyAsync(h.data(), g->d_lod, (size_t)g->F * sizeof(uint4), cudaMemcpyDeviceToHost, s), "copy lod");
    HM_CUDA(cudaStreamSynchronize(s), "sync");
    for (int32_t f = 0; f < g->F; ++f) {
        n_lod[f] = (int32_t)h[f].x;
        c[f] = (int32_t)h[f].y;
    }
    return HM_OK;
}

hm_status hm_groom_info(hm_groom g, int32_t *L, int32_t *V, int32_t *F, int64_t *S, int32_t *segs) {
    if (!g) return fail(HM_ERR_INVALID_ARG, "groom is NULL");
    if (L) *L = g->L;
    if (V) *V = g->V;
    if (F) *F = g->F;
    if (S) *S = g->S;
    if (segs) *segs = g->segs;
    return HM_OK;
}

hm_status hm_get_device_status(void *stream) {
    uint32_t *sw = status_word();
    if (!sw) return fail(HM_ERR_CUDA, "device status word unavailable");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    uint32_t v = 0;
    HM_CUDA(cudaMemcpyAsync(&v, sw, sizeof v, cudaMemcpyDeviceToHost, s), "read status");
    HM_CUDA(cudaMemsetAsync(sw, 0, sizeof v, s), "clear status");
    HM_CUDA(cudaStreamSynchronize(s), "sync");
    if (v) {
        char buf[96];
        std::snprintf(buf, sizeof buf, "device consistency check failed (status bits 0x%x)", v);
        return fail(HM_ERR_DEVICE_CHECK, buf);
    }
    return HM_OK;
}

}  // extern "C"

extern "C" {

size_t hm_vis_buffer_keys(const hm_camera *cam) {
    if (!cam || cam->width > HM_MAX_RESOLUTION || cam->height > HM_MAX_RESOLUTION) return 0;
    return (size_t)vis_keys(cam);
}

size_t hm_backward_scratch_bytes(int32_t width, int32_t height) {
    if (width < 1 || height < 1) return 0;
    // colour gradient + screen-tangent gradients per pixel, then the tile list
    return (size_t)width * (size_t)height * 32 + hm::resolve_list_bytes(width, height);
}

hm_status hm_shade_backward(const hm_groom *grooms, int32_t n, const hm_camera *cam, const hm_lights *lights,
                            const hm_filter_params *filt, const uint64_t *d_vis_center, const uint64_t *d_vis_cons,
                            const float *d_grad_rgba, float *const *d_grad_layer_verts, float *const *d_grad_albedo,
                            void *d_scratch, void *stream) {
    hm_status st = check_camera(cam);
    if (st != HM_OK) return st;
    if (!d_vis_center || !d_vis_cons || !d_grad_rgba || !d_scratch) return fail(HM_ERR_INVALID_ARG, "buffer is NULL");
    if ((reinterpret_cast<uintptr_t>(d_grad_rgba) & 15) || (reinterpret_cast<uintptr_t>(d_scratch) & 15) ||
        (reinterpret_cast<uintptr_t>(d_vis_center) & 7) || (reinterpret_cast<uintptr_t>(d_vis_cons) & 7))
        return fail(HM_ERR_INVALID_ARG, "misaligned buffer");
    hm::LightsDev ld;
    hm::FilterDev fd;
    if ((st = lights_dev(lights, ld)) != HM_OK) return st;
    if ((st = filter_dev(filt, cam, fd)) != HM_OK) return st;
    hm::CallTable tab;
    st = build_table(grooms, n, tab);
    if (st != HM_OK) return st;
    uint32_t *sw = status_word();
    if (!sw) return fail(HM_ERR_CUDA, "device status word unavailable");
    HM_CUDA(hm::launch_resolve_adjoint(tab, cam_dev(cam), ld, fd, d_vis_center, d_vis_cons, d_grad_rgba,
                                       d_grad_layer_verts, d_grad_albedo, d_scratch, sw,
                                       static_cast<cudaStream_t>(stream)),
            "resolve adjoint");
    return HM_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// hm_shade_backward_noalloc: the adjoint with its colour-gradient scratch in
// a static device array instead of caller-allocated memory
// ---------------------------------------------------------------------------
namespace {

// 32 bytes per pixel of the largest frame (the colour gradient and the
// screen-tangent gradients, two float4), then the adjoint's tile list
// (resolve_list_bytes): a frame of at most HM_NOALLOC_MAX_PIXELS pixels with
// sides up to 16384 has fewer than 1,600 tiles of 32 x 16, and the entry
// point checks the list against this room.
constexpr int kNoallocMaxTiles = 4096;
constexpr int kNoallocListFloat4 = (4 * (3 + 2 * kNoallocMaxTiles) + 15) / 16;
static __device__ __align__(256) float4 g_noalloc_scratch[2 * HM_NOALLOC_MAX_PIXELS + kNoallocListFloat4];

// Device address of g_noalloc_scratch on the current device, looked up once
// per device with that device current (the host-side symbol is only a
// stand-in, never a device address); concurrent first calls from several
// host threads look it up once.  nullptr with the CUDA error in `err` when
// the lookup fails (the next call tries again).
float4 *noalloc_scratch(cudaError_t &err) {
    static hm::PerDevice<float4 *> addr;
    err = cudaSuccess;
    float4 *p = addr.get([&err](int) {
        void *q = nullptr;
        err = cudaGetSymbolAddress(&q, g_noalloc_scratch);
        return err == cudaSuccess ? static_cast<float4 *>(q) : nullptr;
    });
    if (!p && err == cudaSuccess) {
        const cudaError_t e = cudaGetLastError();
        err = e != cudaSuccess ? e : cudaErrorInvalidDevice;
    }
    return p;
}

}  // namespace

extern "C" hm_status hm_shade_backward_noalloc(const hm_groom *grooms, int32_t n, const hm_camera *cam,
                                               const hm_lights *lights, const hm_filter_params *filt,
                                               const uint64_t *d_vis_center, const uint64_t *d_vis_cons,
                                               const float *d_grad_rgba, float *const *d_grad_layer_verts,
                                               float *const *d_grad_albedo, void *stream) {
    hm_status st = check_camera(cam);
    if (st != HM_OK) return st;
    if ((int64_t)cam->width * cam->height > (int64_t)HM_NOALLOC_MAX_PIXELS)
        return fail(HM_ERR_CAPACITY, "frame exceeds HM_NOALLOC_MAX_PIXELS pixels of static scratch");
    if (hm::resolve_list_bytes(cam->width, cam->height) > sizeof(float4) * (size_t)kNoallocListFloat4)
        return fail(HM_ERR_CAPACITY, "frame has more tiles than the static scratch's tile list holds");
    if (!d_vis_center || !d_vis_cons || !d_grad_rgba) return fail(HM_ERR_INVALID_ARG, "buffer is NULL");
    if ((reinterpret_cast<uintptr_t>(d_grad_rgba) & 15) || (reinterpret_cast<uintptr_t>(d_vis_center) & 7) ||
        (reinterpret_cast<uintptr_t>(d_vis_cons) & 7))
        return fail(HM_ERR_INVALID_ARG, "misaligned buffer");
    hm::LightsDev ld;
    hm::FilterDev fd;
    if ((st = lights_dev(lights, ld)) != HM_OK) return st;
    if ((st = filter_dev(filt, cam, fd)) != HM_OK) return st;
    hm::CallTable tab;
    st = build_table(grooms, n, tab);
    if (st != HM_OK) return st;
    uint32_t *sw = status_word();
    if (!sw) return fail(HM_ERR_CUDA, "device status word unavailable");
    cudaError_t e = cudaSuccess;
    float4 *scratch = noalloc_scratch(e);
    if (!scratch) return cuda_fail(e, "static scratch address");
    HM_CUDA(hm::launch_resolve_adjoint(tab, cam_dev(cam), ld, fd, d_vis_center, d_vis_cons, d_grad_rgba,
                                       d_grad_layer_verts, d_grad_albedo, scratch, sw,
                                       static_cast<cudaStream_t>(stream)),
            "resolve adjoint (static scratch)");
    return HM_OK;
}
