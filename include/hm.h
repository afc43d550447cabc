/*
 * hm.h -- C ABI of libhm: deferred software rasterization of strand hair
 * generated from hair meshes, on one NVIDIA B300 (sm_103a).
 *
 * The method is arXiv 2607.04230 ("Deferred Software Rasterization for
 * Efficient Real-time Hair Rendering"): strands are generated on the fly from
 * a hair mesh (Sec. 2 "Background: Hair mesh rendering", Sec. 3.1.1),
 * rasterized into a 64-bit depth|ID visibility buffer with atomicMin in two
 * layers, centre sample and conservative (Sec. 3.1.2, Sec. 3.3), shaded in a
 * deferred pass (Sec. 3.4), reconstructed by the strand-connection /
 * bilateral filter with alpha estimation (Sec. 3.3.1-3.3.3) and thinned by
 * the distance/coverage LOD (Sec. 3.2, Eqs. 1-5).
 *
 * Conventions for every entry point:
 *  - Pointers named d_* are DEVICE pointers on the current CUDA device,
 *    allocated and owned by the caller.  Other pointers are host pointers,
 *    read during the call only.
 *  - `stream` is a cudaStream_t passed as void*.  Work is enqueued on it and
 *    the call returns without synchronizing, except where stated.
 *  - Arguments are validated on the host before anything is launched: a bad
 *    argument returns HM_ERR_INVALID_ARG and enqueues nothing.  A CUDA error
 *    returns HM_ERR_CUDA; hm_last_error() gives the message (per thread).
 *  - The library never aborts the process and never traps on the device.
 *    Device-side consistency checks (a key that decodes to no strand, a
 *    segment index out of range) set a device status word that
 *    hm_get_device_status() reads.
 *  - A groom handle is used by at most one stream at a time; calls that share
 *    a groom must be ordered on the host or by stream order.
 *
 * Visibility keys (Sec. 3.1.2, 24-bit depth in the high bits):
 *     key = d24 << 40 | strand_global << 7 | segment,   EMPTY = ~0
 * strand_global < 2^33 - 1, segment < 127.  A key whose low 40 bits are all
 * ones carries no strand (EMPTY, or a scene-depth pre-fill).
 */
#ifndef HM_H_
#define HM_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    HM_OK = 0,
    HM_ERR_INVALID_ARG = 1,
    HM_ERR_OOM = 2,
    HM_ERR_CUDA = 3,
    HM_ERR_CAPACITY = 4,
    HM_ERR_TIMEOUT = 5,
    HM_ERR_NOT_READY = 6,
    HM_ERR_DEVICE_CHECK = 7
} hm_status;

#define HM_MAX_LAYERS 32
#define HM_MAX_SEGMENTS 126        /* control points per strand <= 127 (Sec. 3.2.2) */
#define HM_MAX_GROOMS_PER_CALL 64
#define HM_MAX_LIGHTS 8
#define HM_MAX_FILTER_RADIUS 8
#define HM_MAX_RESOLUTION 16384
#define HM_MAX_VIEWS 8

typedef struct hm_groom_s *hm_groom;

/* A hair mesh plus strand parameters (Sec. 2; Sec. 3.1.1).  Bundles are
 * triangle prisms: scalp triangle f with vertex indices faces[f] on every
 * layer.  Layer 0 holds the roots, layer L-1 the tips.  Strand s grows from
 * bundle strand_face[s] at barycentric (b1, b2) = strand_bary[s], with
 * b0 = 1 - b1 - b2, fixed along the strand.  strand_face must be ascending
 * (strands of a bundle contiguous); the first N_LOD strands of a bundle are
 * the ones drawn under LOD (Eq. 1), so their order within a bundle should be
 * random.  bundle_delta[f] in [0, 1) is the per-bundle LOD offset delta of
 * Eq. 1.  All arrays are HOST pointers, copied to the device by
 * hm_create_groom. */
typedef struct {
    int32_t num_layers;            /* L, 2..HM_MAX_LAYERS */
    int32_t num_verts;             /* V, vertices per layer */
    int32_t num_faces;             /* F, bundles */
    int32_t segments_per_strand;   /* full-detail segments, 1..HM_MAX_SEGMENTS; C_max = segs + 1 */
    int64_t num_strands;           /* S */
    const float *layer_verts;      /* [L][V][3], metres */
    const int32_t *faces;          /* [F][3], indices into a layer's vertices */
    const uint32_t *strand_face;   /* [S], ascending */
    const float *strand_bary;      /* [S][2] */
    const float *strand_albedo;    /* [S][3], linear RGB */
    const float *bundle_delta;     /* [F] */
    float strand_width_m;          /* sets the centre-sample box (Sec. 3.1.2) */
    float roughness;               /* longitudinal lobe width beta (Sec. 3.4) */
    float tilt;                    /* cuticle tilt alpha, radians (Sec. 3.4) */
    const float *vert_ao;          /* [L][V] baked ambient occlusion in [0, 1] per hair-mesh
                                      vertex (Sec. 3.4), or NULL for none (1) */
    const float *vert_uv;          /* [V][2] scalp texture coordinates in [0, 1] (the uv of
                                      the compressed payload's uvw, Sec. 3.1.2), or NULL (0) */
} hm_groom_desc;

/* Pinhole camera: clip = view_proj * (x, y, z, 1), row-major; clip.w is the
 * view-axis depth in metres.  Pixels: x right, y down, centres at +0.5.
 *
 * key_layout: the layout of this camera's two-layer key buffers (the
 * visibility layers and shadow maps; the RGBA image is always row-major
 * [height][width] float4):
 *   HM_KEYS_ROW_MAJOR (0): key of pixel (x, y) at y * width + x;
 *   HM_KEYS_BLOCK_2X2 (1): 2 x 2 pixel blocks of four keys, one 32-byte
 *     sector each, the blocks row-major over ceil(width / 2) block columns:
 *     pixel (x, y) at ((y / 2) * ceil(width / 2) + x / 2) * 4
 *     + (y % 2) * 2 + x % 2.  The rasterizer's atomics then share sectors
 *     (neighbouring lanes reach the two rows or columns of a block), which
 *     the L2 atomic unit serves as one operation.
 * A key buffer holds hm_vis_buffer_keys(cam) keys; the blocked layout pads
 * odd sizes, and its padding keys stay EMPTY.  The multisample calls take
 * row-major sample planes only. */
typedef struct {
    float view_proj[16];
    float cam_pos[3];
    float near_m, far_m;
    float tan_half_fovy;
    int32_t width, height;
    int32_t key_layout;
} hm_camera;

#define HM_KEYS_ROW_MAJOR 0
#define HM_KEYS_BLOCK_2X2 1

/* Keys in one key layer of a frame of this camera (width * height row-major,
 * 4 * ceil(width / 2) * ceil(height / 2) in 2 x 2 blocks), 0 for an invalid
 * size or layout.  No device call. */
size_t hm_vis_buffer_keys(const hm_camera *cam);

/* LOD of Sec. 3.2: enabled = 0 draws every strand at C_max control points. */
typedef struct {
    int32_t enabled;
    float lambda;                  /* LOD sensitivity, Eq. 2 */
} hm_lod_params;

/* A shadow map of one light (Sec. 3.4 queries shadow/opacity maps with the
 * depth correction of Sec. 3.2 "Depth Comparison Artifact Fix").
 * d_map: hm_vis_buffer_keys(&cam) uint64 keys in cam's key layout, the
 * conservative layer of hm_render_shadow_map with the same camera (device
 * memory, caller's, read only).  A shaded point X is projected with cam like a strand control point
 * (16.8 snap); its texel is (floor(X/256), floor(Y/256)).  With z_map the
 * texel's 24-bit depth / 2^24 and w the point's view depth in the light's
 * camera, the light reaching X is
 *     V = exp(-sigma * beta * max(d - bias_m, 0)),  d = (w - near) - z_map (far - near)
 * (Beer-Lambert past the front-most hair; beta = N_LOD / N of the receiver's
 * bundle when depth_correction != 0, which is the shift by
 * Delta = -log(beta) in log depth; else beta = 1).  V = 1 off the map, in
 * front of the light's near plane, and over an empty texel. */
typedef struct {
    const uint64_t *d_map;
    hm_camera cam;
    int32_t light;                 /* index of the light this map shadows */
    float sigma;                   /* hair density, 1/m, >= 0 */
    float bias_m;                  /* >= 0 */
    int32_t depth_correction;      /* 0 or 1 */
} hm_shadow_map;

/* Directional lights plus ambient for the shading model of Sec. 3.4. */
typedef struct {
    int32_t count;                 /* 0..HM_MAX_LIGHTS */
    float dir[HM_MAX_LIGHTS][3];   /* unit, pointing toward the light */
    float radiance[HM_MAX_LIGHTS][3];
    float ambient;
    float k_d, k_s;
    int32_t n_shadows;             /* 0..count shadow maps, at most one per light */
    const hm_shadow_map *shadows;  /* host array of n_shadows, read during the call */
} hm_lights;

/* Reconstruction filter of Sec. 3.3 (defaults in parentheses). */
typedef struct {
    int32_t enabled;               /* 0: centre-sample shading only, alpha 0/1 */
    int32_t radius;                /* r (5), 0..HM_MAX_FILTER_RADIUS */
    float s_par, s_perp;           /* sigma = r * s (0.5, 0.1), Eq. 7 */
    float sigma_c;                 /* colour term (0.9), Eq. 7 */
    float iso_scale;               /* sigma_iso = iso_scale * r (0.4) */
    float strip_halfwidth;         /* alpha strip half-width, px (0.5), Sec. 3.3.3 */
    float depth_reject_m;          /* neighbour depth reject, metres (1.45e-3) */
    float depth_mismatch_m;        /* conservative-in-front threshold, metres (5e-4) */
} hm_filter_params;

/* Per-frame counters written by hm_render_visibility (device memory).
 * covered_* count (pixel, segment) pairs that pass each layer's coverage
 * test, i.e. the atomicMin operations the method performs. */
typedef struct {
    uint64_t strands;              /* strands drawn after LOD */
    uint64_t segments;             /* segments drawn after LOD */
    uint64_t bundles_culled;
    uint64_t covered_center;
    uint64_t covered_cons;
    uint64_t reserved[3];
} hm_frame_stats;

/* Copy a hair mesh to the device and return a handle (allocates device
 * memory with cudaMalloc; enqueues the copies on `stream` and synchronizes
 * it before returning).  LOD starts disabled.  Besides the mesh the groom
 * holds 32 bytes per strand segment at full detail for the control points
 * the camera renders record (see hm_render_visibility).
 * Errors: HM_ERR_INVALID_ARG (null pointer, size out of range, unsorted
 * strand_face, bad face index, bary outside [0, 1], delta outside [0, 1)),
 * HM_ERR_CAPACITY (more than 2^33 - 2 strands), HM_ERR_OOM, HM_ERR_CUDA. */
hm_status hm_create_groom(const hm_groom_desc *desc, void *stream, hm_groom *out);

/* Free the groom's device memory.  The caller must ensure no enqueued work
 * still uses it. */
hm_status hm_destroy_groom(hm_groom g);

/* Store LOD parameters used by every later hm_render_visibility (Sec. 3.2). */
hm_status hm_set_lod(hm_groom g, const hm_lod_params *p);

/* Replace the layer vertices from a DEVICE buffer [L][V][3] (animation or an
 * optimisation step); enqueued on `stream`.  The control points recorded by
 * the last render become stale: until the next render, key decoding
 * regenerates strands from the new vertices.  (A CUDA graph keeps the
 * arguments of the calls it captured: replay a captured resolve only
 * together with the render that rewrites the records.) */
hm_status hm_update_layer_verts(hm_groom g, const float *d_layer_verts, void *stream);

/* Replace the per-strand albedo from a DEVICE buffer [S][3]; enqueued on
 * `stream`. */
hm_status hm_update_albedo(hm_groom g, const float *d_albedo, void *stream);

/* Render the visibility buffers of n grooms into one shared pair of layers
 * (Sec. 3.1-3.2; multiple grooms share depth, Sec. 4 "Multiple Grooms").
 *
 * Steps, all on `stream`, no host synchronization:
 *   clear (if clear != 0): both layers set to EMPTY, or to the scene depth
 *     pre-fill d24 << 40 | 0xFFFFFFFFFF when d_scene_d24 is not NULL;
 *   LOD pre-pass, one thread per bundle (Eqs. 1-5; Sec. 3.2), which also
 *     builds the device work list;
 *   strand generation + projection + 16.8 snap + rasterization with 64-bit
 *     atomicMin into d_vis_center (centre-sample layer) and d_vis_cons
 *     (conservative layer).
 * Strand ids: groom i's strands are numbered after those of grooms 0..i-1
 * in this call.  The LOD result is kept in each groom and used by
 * hm_resolve_shade / hm_shade_backward, which must receive the same groom
 * array in the same order.  The rasterizer also records the two control
 * points of every drawn segment in the groom (device memory it owns); key
 * decoding in the resolves and the adjoint reads them instead of
 * regenerating the strand (bit-identical values) until the groom's layer
 * vertices are replaced or its LOD state is rebuilt by another camera render
 * (hm_render_shadow_map neither writes nor disturbs them).  Both belong to the
 * groom, not to the frame: resolve (or differentiate) a frame before the same
 * grooms are rendered for another camera.
 *
 * d_vis_center, d_vis_cons: hm_vis_buffer_keys(cam) uint64 each, in the
 * camera's key layout, 16-byte aligned.
 * d_scene_d24: [height][width] uint32 (24-bit depth, row-major in every
 * layout) or NULL.
 * d_stats: one hm_frame_stats or NULL.
 * Errors: HM_ERR_INVALID_ARG (n out of 1..HM_MAX_GROOMS_PER_CALL, null or
 * misaligned buffers, resolution out of range, near/far invalid),
 * HM_ERR_CAPACITY (strand ids would exceed 33 bits), HM_ERR_CUDA. */
hm_status hm_render_visibility(const hm_groom *grooms, int32_t n, const hm_camera *cam,
                               uint64_t *d_vis_center, uint64_t *d_vis_cons,
                               const uint32_t *d_scene_d24, int32_t clear,
                               hm_frame_stats *d_stats, void *stream);

/* Multiview rendering (Sec. 5 "Multiview Rendering"): the strands of all
 * grooms are assembled once and projected into n_views views, each with its
 * own camera and pair of key layers (d_vis_center[v], d_vis_cons[v]); all
 * views share width and height.  The LOD pre-pass runs once, for view 0's
 * camera, and its result (kept in the grooms) serves every view, so each
 * view's keys equal a single-view render of that camera under view 0's LOD.
 * Resolve each view with hm_resolve_shade and its own camera.  Both layers
 * of every view are cleared (or pre-filled from d_scene_d24[v] when
 * d_scene_d24 and its entry are not NULL) when clear != 0.  d_stats sums
 * over the views.  Errors as hm_render_visibility; n_views in
 * 1..HM_MAX_VIEWS. */
hm_status hm_render_visibility_multiview(const hm_groom *grooms, int32_t n, const hm_camera *cams,
                                         int32_t n_views, uint64_t *const *d_vis_center,
                                         uint64_t *const *d_vis_cons, const uint32_t *const *d_scene_d24,
                                         int32_t clear, hm_frame_stats *d_stats, void *stream);

/* Compressed G-buffer (Sec. 3.1.2): hm_render_visibility, but the low 40
 * bits of every key hold the shading data instead of the strand-segment id:
 *   bits 39..32 / 31..24  octahedral code of the segment's chord direction
 *                         (8 + 8 bits, Cigolle et al. 2014, sign(0) = +1);
 *   bits 23..18 / 17..12  the root's scalp coordinates u, v (vert_uv), 6 bits;
 *   bits 11..6            w = (j + t) / (C - 1), the position along the strand;
 *   bits 5..0             ambient occlusion, rint(ao 62) (63 unused, so no
 *                         payload equals the all-ones empty marker).
 * Each code is rint(x scale) clamped, ties to even, from binary32 values in
 * fixed operation order.  Same coverage, depths and counts as
 * hm_render_visibility; equal depths are broken by the payload bits.
 * Arguments and errors as hm_render_visibility. */
hm_status hm_render_visibility_compressed(const hm_groom *grooms, int32_t n, const hm_camera *cam,
                                          uint64_t *d_vis_center, uint64_t *d_vis_cons,
                                          const uint32_t *d_scene_d24, int32_t clear, hm_frame_stats *d_stats,
                                          void *stream);

/* Shading parameters of the compressed payload: d_table [64][64][4] float
 * (device), indexed by the (u, v) codes: tip albedo rgb and the root / tip
 * ratio r; albedo = rgb (r + (1 - r) w / 63).  roughness > 0, tilt finite. */
typedef struct {
    const float *d_table;
    float roughness, tilt;
} hm_appearance;

/* Resolve of compressed keys (Sec. 3.1.2 "Position reconstruction"): no
 * hair mesh is read.  Position = the point at depth
 * w = near + ((d24 + 0.5) 2^-24)(far - near) on the ray through the pixel
 * centre; tangent = octahedral decode; AO = code / 62; then shading (Sec.
 * 3.4) and the filter (Sec. 3.3) exactly as hm_resolve_shade.  Shadow maps
 * are not supported here (their depth correction needs the strand's
 * bundle): lights->n_shadows must be 0.  d_rgba [H][W][4] straight alpha,
 * 16-byte aligned. */
hm_status hm_resolve_compressed(const hm_camera *cam, const hm_lights *lights, const hm_filter_params *filt,
                                const hm_appearance *appearance, const uint64_t *d_vis_center,
                                const uint64_t *d_vis_cons, float *d_rgba, void *stream);

/* Shadow map for hm_shadow_map: every groom of grooms[0..n) at full detail
 * (LOD off whatever hm_set_lod holds, no culling: the full geometry set of
 * Sec. 3.2's depth fix), seen from light_cam, into d_map_center /
 * d_map_cons (hm_vis_buffer_keys(light_cam) uint64 each, in light_cam's
 * key layout, 16-byte aligned, cleared first); the
 * conservative layer is the map.  Uses per-groom LOD buffers of its own, so
 * the LOD state of the camera's render is left as it was (the two may run
 * on different streams).  Errors as hm_render_visibility. */
hm_status hm_render_shadow_map(const hm_groom *grooms, int32_t n, const hm_camera *light_cam,
                               uint64_t *d_map_center, uint64_t *d_map_cons, hm_frame_stats *d_stats,
                               void *stream);

/* Multisample software rasterization, the paper's MSAA reference (Sec. 3.3:
 * samples recorded into multiple uint64 layers and resolved later).
 * samples in {1, 2, 4, 8}; sample k of each pixel sits at the standard
 * position for that count (1/16 px units from the centre, y down: 2x (4,4)
 * (-4,-4); 4x (-2,-6) (6,-2) (-6,2) (2,6); 8x (1,-3) (-1,3) (5,1) (-3,-5)
 * (-5,5) (-7,-1) (3,7) (7,-7)) and is covered iff the strand's centre-sample
 * box (the projected half-width) around that point meets the segment; its
 * key's depth is taken at the sample.  d_vis_samples: [samples][H][W]
 * uint64, 16-byte aligned, cleared to EMPTY when clear != 0.  LOD as in
 * hm_render_visibility.  d_stats->covered_center counts covered samples. */
hm_status hm_render_visibility_msaa(const hm_groom *grooms, int32_t n, const hm_camera *cam, int32_t samples,
                                    uint64_t *d_vis_samples, int32_t clear, hm_frame_stats *d_stats, void *stream);

/* Resolve of hm_render_visibility_msaa: each covered sample is decoded at its
 * own sample point and shaded (Sec. 3.4); d_rgba [H][W][4] straight alpha,
 * rgb = mean over covered samples, alpha = covered / samples. */
hm_status hm_resolve_msaa(const hm_groom *grooms, int32_t n, const hm_camera *cam, const hm_lights *lights,
                          int32_t samples, const uint64_t *d_vis_samples, float *d_rgba, void *stream);

/* hm_render_visibility for grooms[first .. first + count) only, with strand
 * ids numbered as in the whole n-groom array, so that per-groom calls into
 * the same buffers (clear only on the first) compose with one
 * hm_resolve_shade over all n grooms: the sequential multi-groom scheme of
 * Sec. 4 "Multiple Grooms".  Same errors as hm_render_visibility, plus
 * HM_ERR_INVALID_ARG when the range is outside 0..n. */
hm_status hm_render_visibility_range(const hm_groom *grooms, int32_t n, int32_t first, int32_t count,
                                     const hm_camera *cam, uint64_t *d_vis_center, uint64_t *d_vis_cons,
                                     const uint32_t *d_scene_d24, int32_t clear, hm_frame_stats *d_stats,
                                     void *stream);

/* Deferred resolve (Sec. 3.1.2 deferred shading, Sec. 3.3 filter, Sec. 3.4
 * shading): decode each key back to its strand segment, shade centre-sample
 * pixels, run the strand-connection / elliptical bilateral filter and alpha
 * estimation, and write straight-alpha RGBA.
 * d_rgba: [height][width][4] float32, 16-byte aligned.
 * d_tile_scratch: NULL, or DEVICE scratch of hm_resolve_scratch_bytes(width,
 * height) bytes (about 32 bytes per pixel), 16-byte aligned, owned by the
 * caller and not used by any other work in flight.  NULL: one CTA per output
 * tile, each finding out whether its tile holds keys, decoding the centre
 * keys of the tile and its filter halo and filtering (best when most tiles
 * hold keys, a single groom filling the frame).  With scratch: a pre-pass
 * counts each tile's conservative keys (zero-filling the tiles without any),
 * a one-CTA pass lists the others heaviest first, a decode pass shades every
 * centre key of the listed tiles and finds every screen tangent the filter
 * needs, once per pixel, into the scratch, and a persistent grid filters the
 * listed tiles in that order.  The image is bit-identical either way for
 * keys written by the render calls, whose centre-layer keys lie at pixels
 * the conservative layer also covers (a centre sample box lies inside the
 * pixel box); with scratch, a centre key in a tile without any conservative
 * key is treated as absent.
 * Same grooms, in the same order, as the render call that wrote the keys.
 * Errors: HM_ERR_INVALID_ARG, HM_ERR_CUDA. */
hm_status hm_resolve_shade(const hm_groom *grooms, int32_t n, const hm_camera *cam,
                           const hm_lights *lights, const hm_filter_params *filt,
                           const uint64_t *d_vis_center, const uint64_t *d_vis_cons,
                           float *d_rgba, void *d_tile_scratch, void *stream);

/* Bytes of hm_resolve_shade's optional tile scratch at this resolution (0
 * for a resolution out of range). */
size_t hm_resolve_scratch_bytes(int32_t width, int32_t height);

/* Adjoint of hm_resolve_shade with the visibility keys, the pixel-centre
 * projection parameters and every filter mask held fixed (the alpha is then
 * constant).  d_grad_rgba [height][width][4] is dLoss/d(rgba) (the alpha
 * channel is ignored).  Gradients are ADDED into d_grad_layer_verts
 * ([L][V][3] of grooms[i], one pointer per groom, NULL to skip) and
 * d_grad_albedo ([S][3] per groom, NULL to skip).
 * d_scratch: device buffer of hm_backward_scratch_bytes(width, height)
 * bytes, 16-byte aligned, contents ignored on entry.
 * Errors: HM_ERR_INVALID_ARG, HM_ERR_CUDA. */
hm_status hm_shade_backward(const hm_groom *grooms, int32_t n, const hm_camera *cam,
                            const hm_lights *lights, const hm_filter_params *filt,
                            const uint64_t *d_vis_center, const uint64_t *d_vis_cons,
                            const float *d_grad_rgba, float *const *d_grad_layer_verts,
                            float *const *d_grad_albedo, void *d_scratch, void *stream);

/* Bytes of scratch hm_shade_backward needs at this resolution. */
size_t hm_backward_scratch_bytes(int32_t width, int32_t height);

/* Largest frame (width * height) hm_shade_backward_noalloc accepts. */
#define HM_NOALLOC_MAX_PIXELS 262144

/* hm_shade_backward for callers that cannot allocate device memory.
 * (The paper has no counterpart: it is a library convenience.)
 * Some callers cannot call cudaMalloc at the point where they need the
 * gradient: code that runs where an allocation's implicit device-wide
 * synchronization is not acceptable (a real-time frame loop), or code whose
 * device memory is owned by another allocator with a fixed budget.  This
 * entry point takes the same inputs and outputs as hm_shade_backward but no
 * d_scratch: its scratch is a static array of the library, held on every GPU
 * that loads libhm until the process exits: HM_NOALLOC_MAX_PIXELS * 32 bytes
 * (8 MiB) of per-pixel colour and screen-tangent gradients, then about
 * 32 KiB for the adjoint's tile list (room for 4,096 tiles of 32 x 16
 * pixels).  It calls no allocator.
 *  - Errors beyond hm_shade_backward's: HM_ERR_CAPACITY, before anything is
 *    launched, for a frame of more than HM_NOALLOC_MAX_PIXELS pixels, or for
 *    one with more tiles than the list room (no frame within the pixel
 *    limit has: at most 1,600 tiles with sides up to HM_MAX_RESOLUTION).
 *  - The first call on a device looks up the array's device address (one
 *    cudaGetSymbolAddress with that device current; concurrent first calls
 *    from several host threads look it up once); make that first call
 *    before any stream capture.  The address is kept for the process: do
 *    not call the library again on a device after cudaDeviceReset.
 *  - Every call on a device shares the one array and clears it on the
 *    stream before use, so calls that overlap on the GPU (different streams
 *    without ordering) race on it; order them.
 * Other arguments, results and errors are those of hm_shade_backward. */
hm_status hm_shade_backward_noalloc(const hm_groom *grooms, int32_t n, const hm_camera *cam,
                                    const hm_lights *lights, const hm_filter_params *filt,
                                    const uint64_t *d_vis_center, const uint64_t *d_vis_cons,
                                    const float *d_grad_rgba, float *const *d_grad_layer_verts,
                                    float *const *d_grad_albedo, void *stream);

/* Copy the groom's current per-bundle LOD result (strands drawn N_LOD and
 * control points C, Eqs. 1-5) to host arrays of num_faces entries.
 * Synchronizes `stream`. */
hm_status hm_get_lod(hm_groom g, int32_t *n_lod, int32_t *c, void *stream);

/* Counts of the groom: layers, verts, faces, strands, segments_per_strand. */
hm_status hm_groom_info(hm_groom g, int32_t *L, int32_t *V, int32_t *F, int64_t *S, int32_t *segs);

/* Synchronize `stream`, read and clear the device status word (set by a
 * failed device-side consistency check): HM_OK or HM_ERR_DEVICE_CHECK. */
hm_status hm_get_device_status(void *stream);

/* Launch shapes of the kernels, process-wide (the project's autotuner,
 * paper_2607_04230_b300/autotune.py, searches these).  Results never depend
 * on them: visibility is bit-identical and colours identical for every
 * setting.
 *   raster_precheck    0/1: read the key before each atomicMin and skip
 *                      atomics that cannot lower it (default 0)
 *   raster_min_blocks  3 or 4 resident 256-thread rasterizer CTAs per SM the
 *                      register budget is sized for (default 4)
 *   raster_ctas_per_sm persistent rasterizer CTAs per SM, 0 = as many as fit
 *   resolve_tile_h     16 or 32: resolve tiles of 32 x tile_h pixels
 *                      (default 32)
 *   raster_bin_w       0: the direct rasterizer (global atomicMin per
 *                      covered pixel, default).  16 or 32: the screen-tile
 *                      binned rasterizer (segments binned to tiles of
 *                      raster_bin_w x raster_bin_h pixels, shared-memory
 *                      atomicMin per tile, one coalesced global atomicMin per
 *                      touched key and chunk) for single-view renders with
 *                      the ID payload; multiview, compressed, multisample
 *                      and shadow-map renders keep the direct rasterizer.
 *                      Its workspace (about 91 B per control point of the
 *                      call's grooms at full detail, plus 12 B per tile)
 *                      belongs to the call's first groom, is allocated on
 *                      first use and grown by later calls, which then
 *                      synchronize the device; a call that must grow it
 *                      during CUDA stream capture returns HM_ERR_CAPACITY
 *                      (render once outside the capture).  A frame whose
 *                      segment-tile pairs exceed 8 per work-list slot sets
 *                      device status bit 4 (hm_get_device_status) and its
 *                      keys are incomplete.
 *   raster_bin_h       16 or 32 when raster_bin_w != 0, else 0
 *   raster_bin_chunk   256 or 1024 segments per unit of the binned tile
 *                      pass when raster_bin_w != 0, else 0
 * Not thread-safe against concurrent render calls on other host threads. */
typedef struct {
    int32_t raster_precheck;
    int32_t raster_min_blocks;
    int32_t raster_ctas_per_sm;
    int32_t resolve_tile_h;
    int32_t raster_bin_w;
    int32_t raster_bin_h;
    int32_t raster_bin_chunk;
    int32_t reserved;
} hm_tuning;

hm_status hm_set_tuning(const hm_tuning *t);
hm_status hm_get_tuning(hm_tuning *t);

/* Profiling: record CUDA events (cudaEvent_t passed as void*) at phase
 * boundaries of later calls on this host thread, on the call's stream:
 * events[0] before the clear, [1] after the clear, [2] after the LOD
 * pre-pass, [3] after the rasterizer (hm_render_visibility and its
 * multiview, multisample and shadow-map forms); [4] before and [5] after
 * the resolve (hm_resolve_shade, hm_resolve_msaa).  count = 0 or events =
 * NULL turns it off; a NULL entry is skipped. */
hm_status hm_set_phase_events(void *const *events, int32_t count);

/* Measurement probe for the roofline denominator, not part of rendering:
 * one launch of 64-bit atomicMin over d_buf[0..n) with `rounds` operations
 * per element, addresses coalesced and distinct within a warp (pattern 0),
 * scattered by a multiplicative hash (pattern 1), or one hashed element per
 * warp, all 32 lanes on it (pattern 2, 32-way contention).  Contents of d_buf
 * are overwritten.  16-byte aligned, n >= 1. */
hm_status hm_probe_atomic_min(uint64_t *d_buf, int64_t n, int32_t rounds, int32_t pattern, void *stream);

/* Arithmetic probe, not part of rendering: d_out[i] = the binary32 quotient
 * d_num[i] / d_den[i] exactly as the rasterizers form the depth parameter of
 * a candidate pixel (Sec. 3.1.2: numerator and |B - A|^2 as floats, one
 * reciprocal per segment, the correctly rounded quotient from it), so tests
 * can compare it with IEEE round-to-nearest division bit for bit.  Device
 * arrays of n floats (n >= 0; n = 0 launches nothing, NULL pointers allowed
 * then); 1 <= d_den[i] < 2^63 and d_num[i] = 0 or 1 <= |d_num[i]| < 2^63,
 * the range the rasterizers use (their numerators and denominators are
 * integers); outside it the values are unspecified (no error).  Errors:
 * HM_ERR_INVALID_ARG for n < 0 or a NULL array with n > 0. */
hm_status hm_probe_quotient(const float *d_num, const float *d_den, float *d_out, int64_t n, void *stream);

const char *hm_status_string(hm_status s);
const char *hm_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* HM_H_ */
