"""Hand-built key buffers for closed-form checks of the filter (Sec. 3.3).

A straight strand lies along world x on the camera's horizontal mid-plane, so
it projects onto the centre row of an odd-height frame, exactly through the
pixel centres: its centre and conservative layers cover the same pixels of
that one row, its screen tangent is horizontal, and every key along it has the
same depth (the view depth is constant along the line).  Three strands share
this geometry (same face, barycentrics (0, 0)) and differ only in albedo, so a
key can be relabelled to another strand, or given another depth, without
changing where it decodes.  With the tangent horizontal, the strip of
Sec. 3.3.3 is the row itself and the elliptical weight of Eq. 7 at horizontal
offset dx is exp(-dx^2 / sigma_par^2): the filter's output at a pixel of the
row has a closed form that the tests below write out by hand.

Used by the CPU pins (oracle only) and by the GPU test that sends the same
buffers through the CUDA resolve.
"""
from __future__ import annotations

import math

import numpy as np

import oracle
from oracle import value64 as v64
from paper_2607_04230_b300 import synth

W, H = 41, 21
ROW = H // 2                      # the row whose centres the strand crosses
ALBEDO = np.float32([[0.20, 0.30, 0.25], [0.60, 0.45, 0.55], [0.35, 0.35, 0.35]])


def line_scene() -> synth.Scene:
    """Three coincident straight strands (4 layers, 6 segments) 0.5 m in front
    of the camera, spanning about 23 columns of a 41 x 21 frame."""
    xs = np.linspace(-0.2, 0.2, 4, dtype=np.float32)
    layers = np.zeros((4, 3, 3), np.float32)
    layers[:, :, 0] = xs[:, None]
    g = synth.Groom(layer_verts=layers, faces=np.int32([[0, 1, 2]]),
                    strand_face=np.zeros(3, np.uint32), strand_bary=np.zeros((3, 2), np.float32),
                    strand_albedo=ALBEDO.copy(), bundle_delta=np.float32([0.5]), segments_per_strand=6)
    cam = synth.make_camera([0.0, 0.0, 0.5], [0.0, 0.0, 0.0], 40.0, W, H)
    lights = synth.make_lights([[0.3, 1.0, 0.6]], [1.0])
    return synth.Scene([g], cam, lights, name="line_41x21")


def raster(sc):
    lods = [oracle.lod(sc.grooms[0], sc.camera, synth.LodParams(0))]
    vc, va, _ = oracle.raster(sc.grooms, sc.camera, lods)
    return vc, va, lods


def px(x: int, y: int = ROW) -> int:
    return y * W + x


def with_depth(key, d24: int):
    return np.uint64((int(d24) << 40) | (int(key) & 0xFFFFFFFFFF))


def with_strand(key, strand: int):
    k = int(key)
    return np.uint64((k & ~(0x1FFFFFFFF << 7)) | (strand << 7))


def span(vc):
    """Columns of ROW that the centre layer covers."""
    cols = [x for x in range(W) if vc[px(x)] != oracle.EMPTY]
    return min(cols), max(cols)


def shaded_colours(sc, lods, vc, va):
    """The shaded colour of every centre key (the filter switched off)."""
    dec = oracle.resolve_decisions(sc.grooms, sc.camera, lods, synth.FilterParams(enabled=0), vc, va)
    gts = [v64.GroomT(sc.grooms[0], lods[0][1], 0)]
    rgba, pix = v64.resolve(gts, sc.camera, sc.lights, synth.FilterParams(enabled=0), vc, va, dec)
    img = v64.full_image(rgba, pix, W, H).numpy().reshape(-1, 4)
    return img[:, :3]


def oracle_filter(sc, lods, vc, va, filt=None):
    filt = filt or synth.FilterParams()
    dec = oracle.resolve_decisions(sc.grooms, sc.camera, lods, filt, vc, va)
    gts = [v64.GroomT(sc.grooms[0], lods[0][1], 0)]
    rgba, pix = v64.resolve(gts, sc.camera, sc.lights, filt, vc, va, dec)
    return v64.full_image(rgba, pix, W, H).numpy().reshape(-1, 4), dec


def expected_row_pixel(x: int, vc, va, colours, filt=None):
    """The filter's output at (x, ROW) written out for a horizontal tangent:
    Eq. 7 over the row's taps |dx| <= r with G non-empty and the depth test
    against the reference key; alpha = H_center / H_cons over the strip (the
    row, no depth test); promotion with the colour term off; the
    depth-mismatch blend a' C' + (1 - a') C_G with alpha 1."""
    filt = filt or synth.FilterParams()
    r = filt.radius
    s_par = float(np.float32(filt.s_par)) * r
    s_c = float(np.float32(filt.sigma_c))
    rej, mis = oracle.depth_thresholds(line_scene().camera, filt)
    d24 = lambda k: int(k) >> 40

    def taps():
        for dx in range(-r, r + 1):
            if 0 <= x + dx < W:
                yield dx, px(x + dx)

    def reconstruct(ref_key, colour_ref):
        num = np.zeros(3)
        den = 0.0
        n = 0
        for dx, q in taps():
            if vc[q] == oracle.EMPTY or abs(d24(vc[q]) - d24(ref_key)) > rej:
                continue
            w = math.exp(-dx * dx / (s_par * s_par))
            if colour_ref is not None:
                w *= math.exp(-float(((colour_ref - colours[q]) ** 2).sum()) / (s_c * s_c))
            num += w * colours[q]
            den += w
            n += 1
        return (num / den if n else np.zeros(3)), n

    hc = sum(vc[q] != oracle.EMPTY for _, q in taps())
    ha = sum(va[q] != oracle.EMPTY for _, q in taps())
    alpha = hc / ha
    p = px(x)
    G, A = vc[p], va[p]
    if G == oracle.EMPTY and A == oracle.EMPTY:
        return np.zeros(4)
    if G == oracle.EMPTY:                           # promoted pixel
        c, n = reconstruct(A, None)
        return np.concatenate([c, [alpha if n else 0.0]])
    cg, _ = reconstruct(G, colours[p])
    if d24(A) + mis <= d24(G):                      # depth mismatch
        ca, n = reconstruct(A, None)
        if n == 0:
            return np.concatenate([cg, [1.0]])
        return np.concatenate([alpha * ca + (1.0 - alpha) * cg, [1.0]])
    return np.concatenate([cg, [alpha]])


def crafted_cases(vc, va, cam, filt=None):
    """The hand-built key buffers of the closed-form pins: (name, vis_c,
    vis_a).  Strand ids 1 and 2 reuse strand 0's geometry."""
    filt = filt or synth.FilterParams()
    rej, mis = oracle.depth_thresholds(cam, filt)
    x0, x1 = span(vc)
    c = (x0 + x1) // 2
    D = int(vc[px(c)]) >> 40
    yield "as_rastered", vc.copy(), va.copy()

    g, a = vc.copy(), va.copy()
    for dx in (1, -3):
        g[px(c + dx)] = oracle.EMPTY
    for x in range(c - 4, c + 5):
        a[px(x, ROW + 1)] = a[px(x)]
    yield "alpha_ratio", g, a

    g, a = vc.copy(), va.copy()
    for x in range(c - 5, c + 6):
        if x not in (c + 1, c - 2, c + 3):
            g[px(x)] = oracle.EMPTY
    g[px(c + 1)] = with_strand(g[px(c + 1)], 1)
    g[px(c + 3)] = with_depth(g[px(c + 3)], D + rej + 1)
    yield "promoted", g, a

    g, a = vc.copy(), va.copy()
    for dx in (-4, -1, 2):
        for buf in (g, a):
            buf[px(c + dx)] = with_strand(buf[px(c + dx)], 1)
    for dx in (3, -5):
        g[px(c + dx)] = oracle.EMPTY
    a[px(c)] = with_strand(with_depth(a[px(c)], D - 50), 2)
    a[px(c + 7)] = with_depth(a[px(c + 7)], D - 500)
    a[px(c - 7)] = with_depth(a[px(c - 7)], D - (mis - 1))
    yield "mismatch", g, a
