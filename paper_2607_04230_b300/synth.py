"""Seeded synthetic inputs: hair-mesh grooms, cameras and lights.

This module only *makes inputs*.  It holds none of the rendering method's
arithmetic (no strand generation, projection, rasterization, LOD, shading or
filtering), so the CPU oracle and the CUDA path can both consume its output
without sharing any of the computation they are compared on.

A groom is a hair mesh made of triangle-prism bundles (the paper's hair mesh,
Sec. 2 "Background: Hair mesh rendering", uses quad layers; these grooms use
triangle layers, one prism per scalp triangle).  Layer 0 lies on a spherical
scalp cap and layer k is offset along the vertex normal, then displaced by
seeded jitter or a smooth noise field.  Strand roots are per-strand inputs:
the scalp triangle (bundle) and two barycentric coordinates, drawn uniformly
over the triangle, sorted by bundle so that the first N strands of a bundle
are a uniform random subset of it (what the stochastic strand LOD of Eq. 1
needs).  The per-bundle LOD offset delta ~ U[0,1) of Eq. 1 is also an input.

All arrays are numpy, little-endian, C-contiguous.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# Shading constants used by every synthetic workload (Sec. 3.4; the paper
# gives no coefficients, so these are this library's defaults).
K_D = 1.0 / math.pi
K_S = 0.25
AMBIENT = 0.05
ROUGHNESS = 0.15
TILT = -0.05
STRAND_WIDTH_M = 1.0e-4
NEAR_M = 0.05
FAR_M = 256.0


@dataclass
class Groom:
    """One hair mesh plus its strand parameters (host arrays)."""

    layer_verts: np.ndarray      # float32 [L][V][3], metres, world space
    faces: np.ndarray            # int32   [F][3], scalp triangles = bundles
    strand_face: np.ndarray      # uint32  [S], ascending (bundle-contiguous)
    strand_bary: np.ndarray      # float32 [S][2] = (b1, b2)
    strand_albedo: np.ndarray    # float32 [S][3]
    bundle_delta: np.ndarray     # float32 [F], in [0, 1)
    segments_per_strand: int     # full-detail segment count; C_max = segs + 1
    strand_width_m: float = STRAND_WIDTH_M
    roughness: float = ROUGHNESS
    tilt: float = TILT
    vert_ao: np.ndarray | None = None   # float32 [L][V] in [0, 1], baked ambient occlusion, or None
    vert_uv: np.ndarray | None = None   # float32 [V][2] in [0, 1], scalp texture coordinates, or None

    @property
    def num_layers(self) -> int:
        return int(self.layer_verts.shape[0])

    @property
    def num_verts(self) -> int:
        return int(self.layer_verts.shape[1])

    @property
    def num_faces(self) -> int:
        return int(self.faces.shape[0])

    @property
    def num_strands(self) -> int:
        return int(self.strand_face.shape[0])

    def world_aabb(self):
        lv = self.layer_verts.reshape(-1, 3).astype(np.float64)
        return lv.min(0), lv.max(0)


@dataclass
class Camera:
    view_proj: np.ndarray        # float32 [4][4], row-major, clip = M @ (x,y,z,1)
    cam_pos: np.ndarray          # float32 [3]
    near: float
    far: float
    tan_half_fovy: float
    width: int
    height: int
    key_layout: int = 0          # key buffers: 0 row-major, 1 in 2 x 2 blocks (the library's HM_KEYS_*)


@dataclass
class Lights:
    dirs: np.ndarray             # float32 [n][3], unit, pointing toward the light
    radiance: np.ndarray         # float32 [n][3]
    ambient: float = AMBIENT
    k_d: float = K_D
    k_s: float = K_S


@dataclass
class ShadowSpec:
    """A shadow map for one light (Sec. 3.2 depth fix, Sec. 3.4): the light's
    camera, the hair density sigma (1/m) of the Beer-Lambert falloff, a depth
    bias (m) and whether the LOD depth correction is applied."""
    light: int
    cam: "Camera"
    sigma: float = 100.0
    bias_m: float = 0.001
    depth_correction: int = 1


@dataclass
class FilterParams:
    """Reconstruction-filter knobs (Sec. 3.3).  Defaults follow the paper's
    text where it gives a number: r = 5, sigma_c = 0.9, sigma_iso = 0.4 r,
    depth reject 1.45e-3, mismatch 5e-4, strip half-width 0.5 px."""

    enabled: int = 1
    radius: int = 5
    s_par: float = 0.5
    s_perp: float = 0.1
    sigma_c: float = 0.9
    iso_scale: float = 0.4
    strip_halfwidth: float = 0.5
    depth_reject_m: float = 1.45e-3
    depth_mismatch_m: float = 5.0e-4


@dataclass
class LodParams:
    enabled: int = 0
    lam: float = 3.0


@dataclass
class Scene:
    grooms: list
    camera: Camera
    lights: Lights
    filt: FilterParams = field(default_factory=FilterParams)
    lod: LodParams = field(default_factory=LodParams)
    name: str = ""


# --------------------------------------------------------------------------
# scalp cap
# --------------------------------------------------------------------------

def fan_disk(k: int, n: int):
    """Planar k-triangle fan around the origin, midpoint-subdivided n times.

    Returns (verts2d float64 [V][2], faces int32 [F][3]) with F = k * 4**n.
    """
    verts = [(0.0, 0.0)] + [
        (math.cos(2 * math.pi * i / k), math.sin(2 * math.pi * i / k)) for i in range(k)
    ]
    faces = [(0, 1 + i, 1 + (i + 1) % k) for i in range(k)]
    for _ in range(n):
        mids = {}

        def mid(a, b):
            key = (a, b) if a < b else (b, a)
            if key not in mids:
                pa, pb = verts[a], verts[b]
                verts.append(((pa[0] + pb[0]) * 0.5, (pa[1] + pb[1]) * 0.5))
                mids[key] = len(verts) - 1
            return mids[key]

        new = []
        for a, b, c in faces:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            new += [(a, ab, ca), (ab, b, bc), (ca, bc, c), (ab, bc, ca)]
        faces = new
    return np.asarray(verts, np.float64), np.asarray(faces, np.int32)


def scalp_uv(k: int, n: int) -> np.ndarray:
    """Scalp texture coordinates: the planar fan's unit disk mapped to
    [0, 1]^2 (float32 [V][2])."""
    v2, _ = fan_disk(k, n)
    return np.ascontiguousarray(((v2 + 1.0) * 0.5).astype(np.float32))


def scalp_cap(k: int, n: int, radius: float = 0.1, cap_deg: float = 60.0):
    """Map the planar fan onto a spherical cap with its pole along +y.

    Returns (positions float64 [V][3], unit normals float64 [V][3], faces).
    """
    v2, faces = fan_disk(k, n)
    rho = np.sqrt((v2 ** 2).sum(1))
    phi = np.arctan2(v2[:, 1], v2[:, 0])
    theta = rho * math.radians(cap_deg)
    nrm = np.stack([np.sin(theta) * np.cos(phi), np.cos(theta), np.sin(theta) * np.sin(phi)], 1)
    return nrm * radius, nrm, faces


def _tangent_plane(v, nrm):
    return v - (v * nrm).sum(-1, keepdims=True) * nrm


def _smooth_field(rng, pos, n_modes=4, wavelength=0.06):
    """A seeded smooth vector field (sum of random Fourier modes) at pos."""
    out = np.zeros_like(pos)
    for _ in range(n_modes):
        omega = rng.normal(size=3)
        omega *= (2 * math.pi / wavelength) / np.linalg.norm(omega)
        amp = rng.normal(size=3)
        amp /= np.linalg.norm(amp)
        ph = rng.uniform(0, 2 * math.pi)
        out += amp[None, :] * np.sin(pos @ omega + ph)[:, None]
    return out / math.sqrt(n_modes)


def make_groom(seed: int, k: int, n: int, num_layers: int, length_m: float,
               num_strands: int, segments: int, jitter_sigma_m: float = 0.0,
               curl_amp_m: float = 0.0, radius: float = 0.1, cap_deg: float = 60.0,
               offset=(0.0, 0.0, 0.0), albedo_range=(0.2, 0.6)) -> Groom:
    """A seeded prism hair mesh on a spherical cap, plus strand roots."""
    rng = np.random.default_rng(seed)
    pos, nrm, faces = scalp_cap(k, n, radius, cap_deg)
    L = num_layers
    spacing = length_m / (L - 1)
    layers = [pos.copy()]
    for li in range(1, L):
        p = pos + nrm * (spacing * li)
        if jitter_sigma_m > 0:
            p = p + _tangent_plane(rng.normal(scale=jitter_sigma_m, size=pos.shape), nrm)
        if curl_amp_m > 0:
            frac = li / (L - 1)
            p = p + curl_amp_m * frac * _tangent_plane(_smooth_field(rng, pos), nrm)
        layers.append(p)
    lv = np.stack(layers, 0) + np.asarray(offset, np.float64)[None, None, :]
    F = faces.shape[0]
    face = rng.integers(0, F, size=num_strands).astype(np.uint32)
    r1 = rng.random(num_strands)
    r2 = rng.random(num_strands)
    sq = np.sqrt(r1)
    bary = np.stack([sq * (1.0 - r2), sq * r2], 1).astype(np.float32)
    order = np.argsort(face, kind="stable")
    face = face[order]
    bary = bary[order]
    albedo = rng.uniform(albedo_range[0], albedo_range[1], size=(num_strands, 3)).astype(np.float32)
    delta = rng.random(F).astype(np.float32)
    delta = np.minimum(delta, np.float32(np.nextafter(np.float32(1), np.float32(0))))
    return Groom(
        layer_verts=np.ascontiguousarray(lv.astype(np.float32)),
        faces=np.ascontiguousarray(faces.astype(np.int32)),
        strand_face=np.ascontiguousarray(face),
        strand_bary=np.ascontiguousarray(bary),
        strand_albedo=np.ascontiguousarray(albedo),
        bundle_delta=np.ascontiguousarray(delta),
        segments_per_strand=int(segments),
        vert_uv=scalp_uv(k, n),
    )


def appearance_table(seed: int = 0, albedo_range=(0.2, 0.6), ratio_range=(0.5, 1.0)) -> np.ndarray:
    """Shading parameters over the quantized scalp coordinates for the
    compressed payload: float32 [64][64][4], per (u, v) texel the tip albedo
    (rgb) and the root / tip albedo ratio; smooth in (u, v) plus per-texel
    variation, seeded."""
    rng = np.random.default_rng(seed)
    u = np.linspace(0.0, 1.0, 64)
    base = rng.uniform(albedo_range[0], albedo_range[1], size=3)
    grad = rng.normal(scale=0.1, size=(2, 3))
    smooth = base[None, None, :] + u[:, None, None] * grad[0][None, None, :] + u[None, :, None] * grad[1][None, None, :]
    rgb = np.clip(smooth + rng.normal(scale=0.05, size=(64, 64, 3)), albedo_range[0], albedo_range[1])
    ratio = rng.uniform(ratio_range[0], ratio_range[1], size=(64, 64, 1))
    return np.ascontiguousarray(np.concatenate([rgb, ratio], 2).astype(np.float32))


# --------------------------------------------------------------------------
# camera and lights
# --------------------------------------------------------------------------

def make_camera(eye, target, fovy_deg: float, width: int, height: int,
                near: float = NEAR_M, far: float = FAR_M, up=(0.0, 1.0, 0.0)) -> Camera:
    """OpenGL-style look-at plus perspective; clip.w is the view-axis depth."""
    eye = np.asarray(eye, np.float64)
    target = np.asarray(target, np.float64)
    up = np.asarray(up, np.float64)
    f = target - eye
    f /= np.linalg.norm(f)
    s = np.cross(f, up)
    s /= np.linalg.norm(s)
    u = np.cross(s, f)
    view = np.eye(4)
    view[0, :3], view[1, :3], view[2, :3] = s, u, -f
    view[0, 3], view[1, 3], view[2, 3] = -s @ eye, -u @ eye, f @ eye
    t = math.tan(math.radians(fovy_deg) * 0.5)
    aspect = width / height
    proj = np.zeros((4, 4))
    proj[0, 0] = 1.0 / (t * aspect)
    proj[1, 1] = 1.0 / t
    proj[2, 2] = (far + near) / (near - far)
    proj[2, 3] = 2.0 * far * near / (near - far)
    proj[3, 2] = -1.0
    vp = (proj @ view).astype(np.float32)
    return Camera(view_proj=np.ascontiguousarray(vp), cam_pos=eye.astype(np.float32),
                  near=float(np.float32(near)), far=float(np.float32(far)),
                  tan_half_fovy=float(np.float32(t)), width=int(width), height=int(height))


def make_lights(dirs, radiance, ambient=AMBIENT) -> Lights:
    d = np.asarray(dirs, np.float64)
    d = d / np.linalg.norm(d, axis=1, keepdims=True)
    r = np.asarray(radiance, np.float64)
    if r.ndim == 1:
        r = np.repeat(r[:, None], 3, 1)
    return Lights(dirs=np.ascontiguousarray(d.astype(np.float32)),
                  radiance=np.ascontiguousarray(r.astype(np.float32)),
                  ambient=float(np.float32(ambient)))


def light_camera(grooms, light_dir, size: int = 512, dist_m: float = 1.0) -> Camera:
    """A square perspective camera looking at the grooms' AABB centre from
    dist_m along light_dir (toward the light), its field of view fitted to
    the AABB, depth range near 0.05 m to just past the far side."""
    ctr, lo, hi = _aabb_center(grooms)
    rad = 0.5 * float(np.linalg.norm(hi - lo))
    d = np.asarray(light_dir, np.float64)
    d = d / np.linalg.norm(d)
    up = (0.0, 1.0, 0.0) if abs(d[1]) < 0.9 else (1.0, 0.0, 0.0)
    fov = 2.0 * math.degrees(math.atan(1.05 * rad / dist_m))
    return make_camera(ctr + d * dist_m, ctr, fov, size, size, near=NEAR_M, far=dist_m + 2.0 * rad, up=up)


def _aabb_center(grooms):
    lo = np.min([g.world_aabb()[0] for g in grooms], 0)
    hi = np.max([g.world_aabb()[1] for g in grooms], 0)
    return (lo + hi) * 0.5, lo, hi


# --------------------------------------------------------------------------
# the workloads
# --------------------------------------------------------------------------

def tiny_scene(seed: int = 0, width: int = 256, height: int = 256, num_strands: int = 1000,
               segments: int = 8, k: int = 8, n: int = 1, num_layers: int = 4,
               length_m: float = 0.045, dist_m: float = 0.5, jitter_m: float = 0.003,
               curl_m: float = 0.0) -> Scene:
    """Small single-groom scene (the 256x256, 1,000-strand case by default)."""
    g = make_groom(seed, k, n, num_layers, length_m, num_strands, segments,
                   jitter_sigma_m=jitter_m, curl_amp_m=curl_m)
    c, _, _ = _aabb_center([g])
    cam = make_camera(c + np.array([0.0, 0.0, dist_m]), c, 40.0, width, height)
    lights = make_lights([[1.0, 1.0, 1.0]], [1.0])
    return Scene([g], cam, lights, name=f"tiny_s{seed}_{width}x{height}")


def scene_tiny_256() -> Scene:
    """32 scalp triangles, 4 layers (0/1.5/3/4.5 cm, 3 mm jitter), 1,000
    strands x 8 segments, 256x256, one light, LOD off, seed 0."""
    return tiny_scene(0)


def groom_single_1080p() -> Groom:
    return make_groom(1, 8, 4, 8, 0.25, 100_000, 16, curl_amp_m=0.01)


def scene_single_1080p(groom: Groom | None = None, dist_m: float = 0.6,
                       lod: LodParams | None = None) -> Scene:
    """2,048 scalp triangles, 8 layers over 25 cm with 1 cm smooth noise,
    100k strands x 16 segments (1.6M segments), 1920x1080, two lights."""
    g = groom if groom is not None else groom_single_1080p()
    c, _, _ = _aabb_center([g])
    cam = make_camera(c + np.array([0.0, 0.0, dist_m]), c, 40.0, 1920, 1080)
    lights = make_lights([[1.0, 1.0, 1.0], [-1.0, 0.5, 0.5]], [0.8, 0.4])
    return Scene([g], cam, lights, lod=lod or LodParams(0, 3.0), name="single_1080p")


LOD_SWEEP_HEIGHTS_PX = [8.0 * 125.0 ** (i / 7.0) for i in range(8)]


def scene_lod_sweep(i: int, groom: Groom | None = None) -> Scene:
    """The 1080p groom at the distance that makes its world height span
    LOD_SWEEP_HEIGHTS_PX[i] pixels, LOD on with lambda = 3."""
    g = groom if groom is not None else groom_single_1080p()
    _, lo, hi = _aabb_center([g])
    h_world = float(hi[1] - lo[1])
    h_px = LOD_SWEEP_HEIGHTS_PX[i]
    dist = h_world * (0.5 * 1080 / math.tan(math.radians(20.0))) / h_px
    s = scene_single_1080p(g, dist_m=dist, lod=LodParams(1, 3.0))
    s.name = f"lod_sweep_{i}_{h_px:.0f}px"
    return s


def scene_grad_512() -> Scene:
    """256 scalp triangles, 6 layers, 20k strands x 12 segments, 512x512."""
    g = make_groom(3, 4, 3, 6, 0.15, 20_000, 12, curl_amp_m=0.008)
    c, _, _ = _aabb_center([g])
    cam = make_camera(c + np.array([0.0, 0.0, 0.45]), c, 40.0, 512, 512)
    lights = make_lights([[1.0, 1.0, 1.0], [-1.0, 0.5, 0.5]], [0.8, 0.4])
    return Scene([g], cam, lights, name="grad_512")


def perturbed_layer_verts(groom: Groom, sigma_m: float = 0.002, seed: int = 33) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return (groom.layer_verts.astype(np.float64)
            + rng.normal(scale=sigma_m, size=groom.layer_verts.shape)).astype(np.float32)


CROWD_FACES = (512, 1024, 2048, 4096)
_FAN = {256: (4, 3), 512: (8, 3), 1024: (4, 4), 2048: (8, 4), 4096: (4, 5)}


def crowd_grooms(seed: int = 4, n_side: int = 8, pitch_m: float = 1.5,
                 strand_scale: float = 1.0) -> list:
    """n_side x n_side independently seeded grooms on a ground grid."""
    rng = np.random.default_rng(seed)
    grooms = []
    for gi in range(n_side * n_side):
        r, c = divmod(gi, n_side)
        F = int(rng.choice(CROWD_FACES))
        L = int(rng.integers(4, 11))
        S = int(round(math.exp(rng.uniform(math.log(5_000), math.log(200_000))) * strand_scale))
        S = max(S, 1)
        segs = int(rng.integers(8, 25))
        length = float(rng.uniform(0.10, 0.30))
        off = ((c - (n_side - 1) / 2) * pitch_m, 0.0, (r - (n_side - 1) / 2) * pitch_m)
        k, n = _FAN[F]
        grooms.append(make_groom(seed * 1000 + gi, k, n, L, length, S, segs,
                                 curl_amp_m=0.01, offset=off))
    return grooms


def scene_crowd_4k(grooms: list | None = None, width: int = 3840, height: int = 2160) -> Scene:
    """64 grooms on an 8x8 grid 1.5 m apart, camera at (0, 6, 14) m,
    3840x2160, LOD on by distance (lambda = 3)."""
    gs = grooms if grooms is not None else crowd_grooms()
    cam = make_camera((0.0, 6.0, 14.0), (0.0, 0.0, 0.0), 40.0, width, height)
    lights = make_lights([[1.0, 1.0, 1.0], [-1.0, 0.5, 0.5]], [0.8, 0.4])
    return Scene(gs, cam, lights, lod=LodParams(1, 3.0), name="crowd_4k")


def view_offsets(cam: Camera, offsets_m, target=None) -> list:
    """Cameras translated sideways (along the image's right axis) by each
    offset, looking at the same target (stereo / multiview rigs)."""
    vp = cam.view_proj.astype(np.float64)
    right = vp[0, :3] / np.linalg.norm(vp[0, :3])
    eye = np.asarray(cam.cam_pos, np.float64)
    fwd_row = vp[3, :3] / np.linalg.norm(vp[3, :3])
    tgt = eye + fwd_row * 0.5 if target is None else np.asarray(target, np.float64)
    fovy = math.degrees(2 * math.atan(cam.tan_half_fovy))
    return [make_camera(eye + right * o, tgt + right * o, fovy, cam.width, cam.height, cam.near, cam.far)
            for o in offsets_m]


def baked_ao(groom: Groom, seed: int = 0, strength: float = 0.6) -> np.ndarray:
    """A seeded stand-in for baked ambient occlusion per hair-mesh vertex:
    darkest at the roots (inside the hair volume), opening toward the tips,
    with per-vertex variation; float32 [L][V] in [0, 1]."""
    rng = np.random.default_rng(seed)
    L, V = groom.num_layers, groom.num_verts
    depth = 1.0 - np.arange(L)[:, None] / max(L - 1, 1)
    ao = 1.0 - strength * depth * rng.uniform(0.6, 1.0, size=(L, V))
    return np.ascontiguousarray(np.clip(ao, 0.0, 1.0).astype(np.float32))
