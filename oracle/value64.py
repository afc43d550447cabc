"""FP64 value layer of the CPU oracle (TEST INFRASTRUCTURE ONLY).

Plain PyTorch CPU float64 ops.  Given the visibility keys and the FP32
decisions of hm_oracle.c (the pixel-centre projection parameter as an exact
num/den pair, the isotropic flag and the strip hit counts), it computes the
continuous part of the deferred pass:

  * strand geometry at the pixel, recomputed in FP64 from the FP32 inputs
    (Sec. 2 Background; Sec. 3.1.1),
  * the shading model (Sec. 3.4),
  * the elliptical bilateral filter (Eqs. 6-7), the strand connection /
    promotion and depth-mismatch blend (Sec. 3.3.2) and alpha (Sec. 3.3.3).

Everything is differentiable with respect to the hair-mesh layer vertices and
the per-strand albedo, with the keys, t and every mask held fixed; autograd of
this forward is the oracle's reference gradient.

Readings where the paper is silent (each also stated where it is used):
  * shading model: the paper fits a Pekelis-style model to Chiang's BSDF and
    gives no coefficients; this library's model is a Kajiya-Kay diffuse term
    plus one longitudinal Gaussian R lobe with tilt and roughness ("parity
    unpinned" against the paper's images);
  * s_par, s_perp: unspecified ("configurable"), defaults 0.5 / 0.1;
  * depth thresholds in metres of linear view depth;
  * promoted pixels with no contributing neighbour output (0, 0, 0, 0);
  * depth mismatch: rgb = a' C' + (1 - a') C_G with alpha 1.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import depth_thresholds

PAYLOAD_MASK = np.uint64(0xFFFFFFFFFF)
STRAND_MASK = np.uint64(0x1FFFFFFFF)


def key_fields(vis: np.ndarray):
    """(empty, d24, strand_global, seg) of packed keys (Sec. 3.1.2)."""
    vis = np.asarray(vis, np.uint64)
    empty = (vis & PAYLOAD_MASK) == PAYLOAD_MASK
    d24 = (vis >> np.uint64(40)).astype(np.int64)
    sg = ((vis >> np.uint64(7)) & STRAND_MASK).astype(np.int64)
    seg = (vis & np.uint64(127)).astype(np.int64)
    return empty, d24, sg, seg


class GroomT:
    """float64 tensors of one groom for the value layer."""

    def __init__(self, g, lod_c, base, layer_verts=None, albedo=None, lod_n=None):
        self.L = g.num_layers
        self.S = g.num_strands
        self.base = int(base)
        self.lv = layer_verts if layer_verts is not None else torch.from_numpy(
            g.layer_verts.astype(np.float64))
        self.albedo = albedo if albedo is not None else torch.from_numpy(
            g.strand_albedo.astype(np.float64))
        self.faces = torch.from_numpy(g.faces.astype(np.int64))
        self.sface = torch.from_numpy(g.strand_face.astype(np.int64))
        self.bary = torch.from_numpy(g.strand_bary.astype(np.float64))
        self.lod_c = torch.from_numpy(np.asarray(lod_c).astype(np.int64))
        # strands per bundle and, when given, the LOD's strands drawn per bundle
        self.n_face = np.bincount(np.asarray(g.strand_face, np.int64), minlength=g.num_faces)
        self.lod_n = None if lod_n is None else np.asarray(lod_n, np.int64)
        self.roughness = float(np.float32(g.roughness))
        self.tilt = float(np.float32(g.tilt))
        ao = getattr(g, "vert_ao", None)
        self.ao = (torch.ones((self.L, g.num_verts), dtype=torch.float64) if ao is None
                   else torch.from_numpy(np.asarray(ao, np.float64)))


def _normalize(v):
    n2 = (v * v).sum(-1, keepdim=True)
    safe = torch.where(n2 > 0, n2, torch.ones_like(n2))
    return torch.where(n2 > 0, v / torch.sqrt(safe), torch.zeros_like(v))


def layer_points(gt: GroomT, strands):
    """P[n][k] = b0 V_k[i0] + b1 V_k[i1] + b2 V_k[i2], b0 = 1 - b1 - b2."""
    tri = gt.faces[gt.sface[strands]]
    b1 = gt.bary[strands, 0][:, None, None]
    b2 = gt.bary[strands, 1][:, None, None]
    b0 = 1.0 - b1 - b2
    v0 = gt.lv[:, tri[:, 0]].permute(1, 0, 2)
    v1 = gt.lv[:, tri[:, 1]].permute(1, 0, 2)
    v2 = gt.lv[:, tri[:, 2]].permute(1, 0, 2)
    return b0 * v0 + b1 * v1 + b2 * v2


def layer_tangents(P):
    """Forward difference at the root, backward at the tip, central inside."""
    L = P.shape[1]
    nxt = torch.cat([P[:, 1:], P[:, -1:]], 1)
    prv = torch.cat([P[:, :1], P[:, :-1]], 1)
    return _normalize(nxt - prv)


def control_points(P, mh, C, j):
    """Hermite control point j of C per row, chord-length tangent scale."""
    L = P.shape[1]
    x = j * (L - 1)
    k = torch.clamp(torch.div(x, C - 1, rounding_mode="floor"), max=L - 2)
    s = ((x - k * (C - 1)).double() / (C - 1).double())[:, None]
    rows = torch.arange(P.shape[0])
    Pk, Pk1 = P[rows, k], P[rows, k + 1]
    ell = torch.sqrt(((Pk1 - Pk) ** 2).sum(-1, keepdim=True))
    m0, m1 = mh[rows, k] * ell, mh[rows, k + 1] * ell
    s2, s3 = s * s, s * s * s
    h00 = 2 * s3 - 3 * s2 + 1
    h10 = s3 - 2 * s2 + s
    h01 = 3 * s2 - 2 * s3
    h11 = s3 - s2
    return h00 * Pk + h10 * m0 + h01 * Pk1 + h11 * m1


def layer_ao(gt: GroomT, strands):
    """Baked ambient occlusion at every layer point of the strands [N][L]
    (Sec. 3.4: interpolated like the position), barycentric on each layer."""
    tri = gt.faces[gt.sface[strands]]
    b1 = gt.bary[strands, 0][:, None]
    b2 = gt.bary[strands, 1][:, None]
    b0 = 1.0 - b1 - b2
    return b0 * gt.ao[:, tri[:, 0]].T + b1 * gt.ao[:, tri[:, 1]].T + b2 * gt.ao[:, tri[:, 2]].T


def control_ao(A, C, j):
    """Scalar cubic Hermite of layer AO values at control point j of C, on
    the position's interval and parameter, with finite-difference slopes
    (central inside, one-sided at root and tip)."""
    L = A.shape[1]
    x = j * (L - 1)
    k = torch.clamp(torch.div(x, C - 1, rounding_mode="floor"), max=L - 2)
    s = (x - k * (C - 1)).double() / (C - 1).double()
    rows = torch.arange(A.shape[0])
    a0, a1 = A[rows, k], A[rows, k + 1]
    am = A[rows, torch.clamp(k - 1, min=0)]
    a2 = A[rows, torch.clamp(k + 2, max=L - 1)]
    m0 = torch.where(k == 0, a1 - a0, 0.5 * (a1 - am))
    m1 = torch.where(k + 1 == L - 1, a1 - a0, 0.5 * (a2 - a0))
    s2, s3 = s * s, s * s * s
    return (2 * s3 - 3 * s2 + 1) * a0 + (s3 - 2 * s2 + s) * m0 + (3 * s2 - 2 * s3) * a1 + (s3 - s2) * m1


def pixel_ao(gt: GroomT, sg, seg, num, den):
    """Ambient occlusion at the pixel centre: the segment's end values at t."""
    s = torch.as_tensor(sg - gt.base, dtype=torch.long)
    j = torch.as_tensor(seg, dtype=torch.long)
    C = gt.lod_c[gt.sface[s]]
    A = layer_ao(gt, s)
    num_t = torch.as_tensor(num, dtype=torch.float64)
    den_t = torch.as_tensor(den, dtype=torch.float64)
    t = torch.where(den_t > 0, num_t / torch.where(den_t > 0, den_t, torch.ones_like(den_t)),
                    torch.zeros_like(den_t))
    t = torch.clamp(t, 0.0, 1.0)
    a, b = control_ao(A, C, j), control_ao(A, C, j + 1)
    return (a + (b - a) * t)[:, None]


def pixel_geometry(gt: GroomT, sg, seg, num, den):
    """Position X and unit tangent T of the keyed segment at the pixel centre
    (deferred decode; t held fixed from the exact integer projection)."""
    s = torch.as_tensor(sg - gt.base, dtype=torch.long)
    j = torch.as_tensor(seg, dtype=torch.long)
    C = gt.lod_c[gt.sface[s]]
    P = layer_points(gt, s)
    mh = layer_tangents(P)
    jm = torch.clamp(j - 1, min=0)
    jp = torch.minimum(j + 2, C - 1)
    pm = control_points(P, mh, C, jm)
    p0 = control_points(P, mh, C, j)
    p1 = control_points(P, mh, C, j + 1)
    pp = control_points(P, mh, C, jp)
    num_t = torch.as_tensor(num, dtype=torch.float64)
    den_t = torch.as_tensor(den, dtype=torch.float64)
    t = torch.where(den_t > 0, num_t / torch.where(den_t > 0, den_t, torch.ones_like(den_t)),
                    torch.zeros_like(den_t))
    t = torch.clamp(t, 0.0, 1.0)[:, None]
    X = p0 + (p1 - p0) * t
    T0 = torch.where((j == 0)[:, None], _normalize(p1 - p0), _normalize(p1 - pm))
    T1 = torch.where((j + 1 == C - 1)[:, None], _normalize(p1 - p0), _normalize(pp - p0))
    T = _normalize(T0 + (T1 - T0) * t)
    return X, T, s


def shadow_visibility(gt: GroomT, X, s, texels, maps, n_lights):
    """Per-light visibility [N][n_lights] of the shaded points X through the
    shadow maps (1 for lights without one).

    Sec. 3.2's depth fix: light through hair falls off as exp(-sigma d)
    (Beer-Lambert, d the depth travelled past the front-most hair); with only
    a fraction beta = N_remaining / N_total of the strands drawn the density
    is sigma beta, i.e. the depth is shifted by Delta = -log(beta) in log
    space: V = exp(-sigma exp(log d - Delta)) = exp(-sigma beta d).
    Readings: the map is the front-most hair depth of the full geometry (a
    one-layer opacity map with uniform density sigma); d = w_X - near -
    z_map (far - near) in metres of the light's view depth, less a bias,
    clamped at 0; beta is the receiver bundle's N_LOD / N when the map asks
    for the correction, else 1.  `texels` holds, per map, the texel index
    under each point (-1: unshadowed), decided in FP32 by hm_oracle.c."""
    Vis = torch.ones((X.shape[0], n_lights), dtype=torch.float64)
    s_np = np.asarray(s, np.int64)
    face = gt.sface[torch.as_tensor(s_np)].numpy()
    for (spec, keys), tex in zip(maps, texels):
        tex = np.asarray(tex, np.int64)
        keys = np.asarray(keys, np.uint64)
        hit = tex >= 0
        k = np.where(hit, keys[np.maximum(tex, 0)], PAYLOAD_MASK)
        hit &= (k & PAYLOAD_MASK) != PAYLOAD_MASK
        zmap = (k >> np.uint64(40)).astype(np.float64) / float(1 << 24)
        M = torch.from_numpy(np.asarray(spec.cam.view_proj, np.float64))
        w = X @ M[3, :3] + M[3, 3]
        near, far = float(np.float32(spec.cam.near)), float(np.float32(spec.cam.far))
        d = (w - near) - torch.from_numpy(zmap) * (far - near) - float(np.float32(spec.bias_m))
        beta = np.ones(X.shape[0])
        if spec.depth_correction:
            if gt.lod_n is None:
                raise ValueError("depth correction needs the LOD strand counts (GroomT lod_n)")
            beta = gt.lod_n[face] / np.maximum(gt.n_face[face], 1)
        sig = float(np.float32(spec.sigma)) * torch.from_numpy(beta)
        v = torch.exp(-sig * torch.clamp(d, min=0.0))
        v = torch.where(torch.from_numpy(hit), v, torch.ones_like(v))
        Vis = Vis.index_put((torch.arange(X.shape[0]), torch.full((X.shape[0],), int(spec.light))), v)
    return Vis


def shade(X, T, albedo, cam, lights, roughness, tilt, ao=None, vis=None):
    """Sec. 3.4: per directional light, Kajiya-Kay diffuse
    albedo k_d sqrt(1 - (T.L)^2) plus an R lobe
    k_s exp(-((T.L + T.V)/2 + sin(tilt))^2 / (2 beta^2)), times the light's
    visibility vis [N][lights] when given; plus ambient albedo, darkened by
    the baked ambient occlusion ao [N][1] when given."""
    cam_pos = torch.from_numpy(np.asarray(cam.cam_pos, np.float64))
    V = _normalize(cam_pos[None, :] - X)
    kd = float(np.float32(lights.k_d))
    ks = float(np.float32(lights.k_s))
    amb = float(np.float32(lights.ambient))
    sa = math.sin(tilt)
    b2 = 2.0 * roughness * roughness
    out = amb * albedo if ao is None else amb * ao * albedo
    for li in range(lights.dirs.shape[0]):
        Ld = torch.from_numpy(lights.dirs[li].astype(np.float64))
        E = torch.from_numpy(lights.radiance[li].astype(np.float64))
        tl = (T * Ld).sum(-1, keepdim=True)
        tv = (T * V).sum(-1, keepdim=True)
        sin2 = 1.0 - tl * tl
        pos = sin2 > 0
        fd = albedo * kd * torch.where(pos, torch.sqrt(torch.where(pos, sin2, torch.ones_like(sin2))),
                                       torch.zeros_like(sin2))
        u = (tl + tv) * 0.5 + sa
        fs = ks * torch.exp(-(u * u) / b2)
        term = E[None, :] * (fd + fs)
        out = out + (term if vis is None else vis[:, li:li + 1] * term)
    return out


def screen_tangent(X, T, cam):
    """Unit screen-space tangent J T / |J T| (Code 2 getScreenTangent),
    J the Jacobian of the pixel position w.r.t. the world position at X."""
    M = torch.from_numpy(np.asarray(cam.view_proj, np.float64))
    c0 = X @ M[0, :3] + M[0, 3]
    c1 = X @ M[1, :3] + M[1, 3]
    w = X @ M[3, :3] + M[3, 3]
    a0, a1, a3 = T @ M[0, :3], T @ M[1, :3], T @ M[3, :3]
    jx = (a0 * w - c0 * a3) / (w * w) * (0.5 * cam.width)
    jy = -(a1 * w - c1 * a3) / (w * w) * (0.5 * cam.height)
    n2 = jx * jx + jy * jy
    safe = torch.where(n2 > 0, n2, torch.ones_like(n2))
    n = torch.sqrt(safe)
    return torch.stack([jx / n, jy / n], -1)


def _group_by_groom(gts, sg):
    """Index lists of rows per groom (strand ids are numbered groom by groom)."""
    out = []
    for gi, gt in enumerate(gts):
        idx = np.nonzero((sg >= gt.base) & (sg < gt.base + gt.S))[0]
        if idx.size:
            out.append((gi, idx))
    return out


def _geometry_all(gts, sg, seg, num, den):
    n = sg.shape[0]
    X = torch.zeros((n, 3), dtype=torch.float64)
    T = torch.zeros((n, 3), dtype=torch.float64)
    parts_X, parts_T, parts_idx, parts_alb = [], [], [], []
    for gi, idx in _group_by_groom(gts, sg):
        Xg, Tg, s = pixel_geometry(gts[gi], sg[idx], seg[idx], num[idx], den[idx])
        parts_X.append(Xg)
        parts_T.append(Tg)
        parts_idx.append(torch.from_numpy(idx))
        parts_alb.append((gi, s))
    if parts_idx:
        all_idx = torch.cat(parts_idx)
        X = X.index_put((all_idx,), torch.cat(parts_X))
        T = T.index_put((all_idx,), torch.cat(parts_T))
    return X, T, parts_idx, parts_alb


def resolve(gts, cam, lights, filt, vis_c, vis_a, dec, pixels=None, shadows=None):
    """RGBA (straight alpha, float64 [N][4]) for the given pixels (all when
    None), Sec. 3.3-3.4.  Returns (rgba, pixel_index).  shadows: optional
    list of (spec, map keys) with dec["shadow_texels"] the per-map texel of
    every centre key (oracle.centre_shadow_texels)."""
    eG, dG, sgG, segG = key_fields(vis_c)
    eA, dA, sgA, segA = key_fields(vis_a)
    # shading of every centre-sample pixel (the deferred shading pass)
    cen = np.nonzero(~eG)[0]
    Xc, Tc, idxs, albs = _geometry_all(gts, sgG[cen], segG[cen], dec_full(dec, "numG", cen),
                                       dec_full(dec, "denG", cen))
    Ccen = torch.zeros((cen.size, 3), dtype=torch.float64)
    for (gi, s), idx in zip(albs, idxs):
        gt = gts[gi]
        sel = cen[idx.numpy()]
        ao = pixel_ao(gt, sgG[sel], segG[sel], dec_full(dec, "numG", sel), dec_full(dec, "denG", sel))
        vis = None
        if shadows:
            vis = shadow_visibility(gt, Xc[idx], s, [t[sel] for t in dec["shadow_texels"]], shadows,
                                    lights.dirs.shape[0])
        Ccen = Ccen.index_put((idx,), shade(Xc[idx], Tc[idx], gt.albedo[s], cam, lights,
                                            gt.roughness, gt.tilt, ao, vis))

    def geom_a(pix):
        XA, TA, _, _ = _geometry_all(gts, sgA[pix], segA[pix], dec["numA"][pix], dec["denA"][pix])
        return XA, TA

    return _filter(cam, filt, vis_c, vis_a, dec, pixels, cen, Xc, Tc, Ccen, geom_a)


# ---------------------------------------------------------------------------
# compressed G-buffer payload (Sec. 3.1.2): shading from the key alone
# ---------------------------------------------------------------------------

def cgb_fields(vis):
    """(empty, d24, tangent code, u, v, w, ao codes) of compressed keys."""
    vis = np.asarray(vis, np.uint64)
    empty = (vis & PAYLOAD_MASK) == PAYLOAD_MASK
    f = lambda sh, m: ((vis >> np.uint64(sh)) & np.uint64(m)).astype(np.int64)
    return empty, f(40, 0xFFFFFF), f(24, 0xFFFF), f(18, 63), f(12, 63), f(6, 63), f(0, 63)


def cgb_position(cam, pixels, d24):
    """Position at the middle of the key's depth bin on the ray through the
    pixel centre (linear view depth w = near + z (far - near))."""
    W = cam.width
    near, far = float(np.float32(cam.near)), float(np.float32(cam.far))
    w = near + (d24.astype(np.float64) + 0.5) / float(1 << 24) * (far - near)
    xs = (pixels % W).astype(np.float64) + 0.5
    ys = (pixels // W).astype(np.float64) + 0.5
    xn = 2.0 * xs / cam.width - 1.0
    yn = 1.0 - 2.0 * ys / cam.height
    M = np.asarray(cam.view_proj, np.float64)
    # rows: (M0 - xn M3) X = xn M33 - M03, (M1 - yn M3) X = yn M33 - M13, M3 X = w - M33
    A = np.stack([M[0, :3][None, :] - xn[:, None] * M[3, :3][None, :],
                  M[1, :3][None, :] - yn[:, None] * M[3, :3][None, :],
                  np.broadcast_to(M[3, :3], (len(w), 3))], 1)
    b = np.stack([xn * M[3, 3] - M[0, 3], yn * M[3, 3] - M[1, 3], w - M[3, 3]], 1)
    return torch.from_numpy(np.linalg.solve(A, b[:, :, None])[:, :, 0] if len(w) else np.zeros((0, 3)))


def oct_decode64(code):
    """Octahedral unit vector decode (Cigolle et al. 2014) of the 8+8-bit
    codes, in float64."""
    ox = (code >> 8).astype(np.float64) / 255.0 * 2.0 - 1.0
    oy = (code & 255).astype(np.float64) / 255.0 * 2.0 - 1.0
    z = 1.0 - np.abs(ox) - np.abs(oy)
    sx = np.where(ox >= 0, 1.0, -1.0)
    sy = np.where(oy >= 0, 1.0, -1.0)
    fx = np.where(z < 0, (1.0 - np.abs(oy)) * sx, ox)
    fy = np.where(z < 0, (1.0 - np.abs(ox)) * sy, oy)
    return _normalize(torch.from_numpy(np.stack([fx, fy, z], 1)))


def cgb_albedo(table, cu, cv, cw):
    """Appearance query at the quantized uvw: the table's (u, v) texel holds
    the tip albedo (rgb) and the root / tip ratio r; albedo = rgb (r + (1 - r) w)."""
    t = torch.from_numpy(np.asarray(table, np.float64).reshape(64 * 64, 4)[cu * 64 + cv])
    w = torch.from_numpy(cw.astype(np.float64) / 63.0)[:, None]
    return t[:, :3] * (t[:, 3:4] + (1.0 - t[:, 3:4]) * w)


def resolve_cgb(cam, lights, filt, vis_c, vis_a, dec, table, roughness, tilt, pixels=None):
    """resolve() for keys carrying the compressed payload: position from
    depth, tangent from the octahedral code, shading parameters from the
    appearance table at (u, v, w), AO from its 6-bit code."""
    eG, dG, tG, uG, vG, wG, aG = cgb_fields(vis_c)
    eA, dA, tA, _, _, _, _ = cgb_fields(vis_a)
    cen = np.nonzero(~eG)[0]
    Xc = cgb_position(cam, cen, dG[cen])
    Tc = oct_decode64(tG[cen])
    alb = cgb_albedo(table, uG[cen], vG[cen], wG[cen])
    ao = torch.from_numpy(aG[cen].astype(np.float64) / 62.0)[:, None]
    Ccen = shade(Xc, Tc, alb, cam, lights, float(np.float32(roughness)), float(np.float32(tilt)), ao)

    def geom_a(pix):
        return cgb_position(cam, pix, dA[pix]), oct_decode64(tA[pix])

    return _filter(cam, filt, vis_c, vis_a, dec, pixels, cen, Xc, Tc, Ccen, geom_a)


def _filter(cam, filt, vis_c, vis_a, dec, pixels, cen, Xc, Tc, Ccen, geom_a):
    """Strand connection, elliptical bilateral filter and alpha (Sec. 3.3)
    over the shaded centre pixels cen (colours Ccen, geometry Xc, Tc);
    geom_a(pixels) gives the conservative keys' geometry."""
    W, H = cam.width, cam.height
    eG, dG, _, _ = key_fields(vis_c)
    eA, dA, _, _ = key_fields(vis_a)
    npx = W * H
    Cimg = torch.zeros((npx, 3), dtype=torch.float64).index_put((torch.from_numpy(cen),), Ccen)

    if pixels is None:
        pixels = np.nonzero(~eA)[0]
    pixels = np.asarray(pixels, np.int64)
    if not filt.enabled:
        rgb = Cimg[pixels]
        a = torch.from_numpy((~eG[pixels]).astype(np.float64))[:, None]
        return torch.cat([rgb * a, a], 1), pixels

    # per output pixel references
    isc = ~eG[pixels]
    isa = ~eA[pixels]
    # G-referenced geometry for centre pixels, A-referenced for the rest / mismatch
    cpos = np.searchsorted(cen, pixels[isc])
    TsG = torch.zeros((pixels.size, 2), dtype=torch.float64)
    if cpos.size:
        TsG[torch.from_numpy(np.nonzero(isc)[0])] = screen_tangent(Xc[cpos], Tc[cpos], cam)
    rej, mis = depth_thresholds(cam, filt)
    aidx = np.nonzero(isa)[0]
    XA, TA = geom_a(pixels[aidx])
    TsA = torch.zeros((pixels.size, 2), dtype=torch.float64)
    if aidx.size:
        TsA[torch.from_numpy(aidx)] = screen_tangent(XA, TA, cam)

    r = int(filt.radius)
    # Eq. 7 scales the standard deviations by r; reading: a radius-0 window
    # (the pixel alone) uses r = 1 there, where the weights cannot matter
    rs = max(r, 1)
    sp = float(np.float32(filt.s_par)) * rs
    sq = float(np.float32(filt.s_perp)) * rs
    siso = float(np.float32(filt.iso_scale)) * rs
    sc = float(np.float32(filt.sigma_c))
    px = torch.from_numpy(pixels % W)
    py = torch.from_numpy(pixels // W)
    dG_t = torch.from_numpy(dG)
    eG_t = torch.from_numpy(eG)
    CP = Cimg[torch.from_numpy(pixels)]

    def reconstruct(ref_d24, Ts, iso, use_color):
        S = torch.zeros((pixels.size, 3), dtype=torch.float64)
        Wt = torch.zeros((pixels.size, 1), dtype=torch.float64)
        cnt = torch.zeros((pixels.size, 1), dtype=torch.int64)
        for dy in range(-r, r + 1):
            for dx in range(-r, r + 1):
                qx, qy = px + dx, py + dy
                inb = (qx >= 0) & (qx < W) & (qy >= 0) & (qy < H)
                qi = torch.clamp(qy, 0, H - 1) * W + torch.clamp(qx, 0, W - 1)
                ok = inb & ~eG_t[qi] & ((dG_t[qi] - ref_d24).abs() <= rej)
                dpar = dx * Ts[:, 0] + dy * Ts[:, 1]
                ex = dx - dpar * Ts[:, 0]
                ey = dy - dpar * Ts[:, 1]
                ell = torch.exp(-(dpar * dpar) / (sp * sp) - (ex * ex + ey * ey) / (sq * sq))
                isow = math.exp(-(dx * dx + dy * dy) / (siso * siso))
                ws = torch.where(iso, torch.full_like(ell, isow), ell)
                CQ = Cimg[qi]
                if use_color is not None:
                    dc = ((use_color - CQ) ** 2).sum(-1)
                    wc = torch.exp(-dc / (sc * sc))
                else:
                    wc = torch.ones_like(ws)
                w = torch.where(ok, ws * wc, torch.zeros_like(ws))[:, None]
                S = S + w * CQ
                Wt = Wt + w
                cnt = cnt + ok[:, None].long()
        return S, Wt, cnt

    # centre-referenced reconstruction (colour term on)
    isoG = torch.from_numpy(dec_at(dec, "isoG", pixels, None).astype(bool))
    isoA = torch.from_numpy(dec_at(dec, "isoA", pixels, None).astype(bool))
    refG = torch.from_numpy(dG[pixels])
    refA = torch.from_numpy(dA[pixels])
    SG, WG, _ = reconstruct(refG, TsG, isoG, CP)
    SA, WA, nA = reconstruct(refA, TsA, isoA, None)
    safeWG = torch.where(WG > 0, WG, torch.ones_like(WG))
    safeWA = torch.where(WA > 0, WA, torch.ones_like(WA))
    CG = SG / safeWG
    CAh = SA / safeWA
    HcG = dec_at(dec, "HcG", pixels, None).astype(np.float64)
    HaG = dec_at(dec, "HaG", pixels, None).astype(np.float64)
    HcA = dec_at(dec, "HcA", pixels, None).astype(np.float64)
    HaA = dec_at(dec, "HaA", pixels, None).astype(np.float64)
    aG = torch.from_numpy(np.where(HaG > 0, HcG / np.maximum(HaG, 1), 0.0))[:, None]
    aA = torch.from_numpy(np.where(HaA > 0, HcA / np.maximum(HaA, 1), 0.0))[:, None]
    mism = isc & isa & (dA[pixels] + mis <= dG[pixels])
    isc_t = torch.from_numpy(isc)[:, None]
    mism_t = torch.from_numpy(mism)[:, None]
    isa_t = torch.from_numpy(isa)[:, None]
    # a promoted reconstruction exists iff some centre-sample neighbour
    # contributes (every weight exp(-e) is positive), Sec. 3.3.2
    hasA = nA > 0
    blend = torch.where(hasA, aA * CAh + (1.0 - aA) * CG, CG)
    rgb_c = torch.where(mism_t, blend, CG)
    a_c = torch.where(mism_t, torch.ones_like(aG), aG)
    rgb_p = torch.where(hasA, CAh, torch.zeros_like(CAh))
    a_p = torch.where(hasA, aA, torch.zeros_like(aA))
    rgb = torch.where(isc_t, rgb_c, torch.where(isa_t, rgb_p, torch.zeros_like(rgb_p)))
    a = torch.where(isc_t, a_c, torch.where(isa_t, a_p, torch.zeros_like(a_p)))
    return torch.cat([rgb, a], 1), pixels


def dec_full(dec, name, idx):
    return dec[name][idx]


def dec_at(dec, name, pixels, sub):
    """Decision array `name` at output pixels (decisions are full-frame)."""
    v = dec[name][pixels]
    return v if sub is None else v[sub]


def full_image(rgba, pixels, width, height):
    img = torch.zeros((width * height, 4), dtype=torch.float64)
    img[torch.from_numpy(pixels)] = rgba.detach() if rgba.requires_grad else rgba
    return img.reshape(height, width, 4)


def resolve_msaa(gts, cam, lights, vis, num, den, shadows=None, texels=None):
    """Multisample resolve (Sec. 3.3's MSAA reference): every covered sample
    is shaded at its own position; the premultiplied colour is the mean over
    all N samples and alpha the covered fraction.  Returns straight-alpha
    RGBA float64 [H*W][4].  shadows: optional list of (spec, map keys) with
    texels[m][k] the texel of sample layer k's keys in map m."""
    N, npx = vis.shape
    acc = torch.zeros((npx, 3), dtype=torch.float64)
    cov = torch.zeros((npx, 1), dtype=torch.float64)
    for k in range(N):
        e, _, sg, seg = key_fields(vis[k])
        idx = np.nonzero(~e)[0]
        if idx.size == 0:
            continue
        X, T, parts_idx, parts_alb = _geometry_all(gts, sg[idx], seg[idx], num[k][idx], den[k][idx])
        C = torch.zeros((idx.size, 3), dtype=torch.float64)
        for (gi, s), pidx in zip(parts_alb, parts_idx):
            gt = gts[gi]
            sel = idx[pidx.numpy()]
            ao = pixel_ao(gt, sg[sel], seg[sel], num[k][sel], den[k][sel])
            vs = None
            if shadows:
                vs = shadow_visibility(gt, X[pidx], s, [t[k][sel] for t in texels], shadows, lights.dirs.shape[0])
            C = C.index_put((pidx,), shade(X[pidx], T[pidx], gt.albedo[s], cam, lights, gt.roughness, gt.tilt, ao,
                                           vs))
        t = torch.from_numpy(idx)
        acc = acc.index_add(0, t, C)
        cov = cov.index_add(0, t, torch.ones((idx.size, 1), dtype=torch.float64))
    a = cov / N
    rgb = torch.where(cov > 0, acc / torch.where(cov > 0, cov, torch.ones_like(cov)), torch.zeros_like(acc))
    return torch.cat([rgb, a], 1)
