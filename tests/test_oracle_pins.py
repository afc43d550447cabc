"""Pins of the CPU oracle against things other than itself.

Each test ties one oracle step to what the paper or the mathematics fixes:
exact rational arithmetic, closed forms, a library routine used as an
independent evaluation, brute force on tiny inputs, or an invariant.  A
plausible slip (dropped term, wrong sign or index, transposed operand) in the
oracle fails at least one of these.  CPU only.
"""
import math
import os
from fractions import Fraction as Fr

import numpy as np
import pytest
import torch
from scipy.interpolate import CubicHermiteSpline
from scipy.ndimage import correlate

import oracle
from oracle import value64 as v64
from paper_2607_04230_b300 import synth

F32_EPS = float(np.finfo(np.float32).eps)


def _groom_from_layers(layers, bary, segs, faces=None):
    """A hand-built groom: layers float [L][V][3], strands with given bary
    (all on face 0)."""
    layers = np.asarray(layers, np.float32)
    L, V, _ = layers.shape
    faces = np.asarray(faces if faces is not None else [[0, 1, 2]], np.int32)
    bary = np.asarray(bary, np.float32).reshape(-1, 2)
    S = bary.shape[0]
    return synth.Groom(layer_verts=np.ascontiguousarray(layers), faces=faces,
                       strand_face=np.zeros(S, np.uint32), strand_bary=np.ascontiguousarray(bary),
                       strand_albedo=np.full((S, 3), 0.4, np.float32),
                       bundle_delta=np.full(faces.shape[0], 0.5, np.float32), segments_per_strand=segs)


# ---------------------------------------------------------------------------
# strand generation (Sec. 2, Sec. 3.1.1)
# ---------------------------------------------------------------------------

def test_layer_point_unit_barycentrics_exact():
    rng = np.random.default_rng(1)
    layers = rng.normal(size=(5, 3, 3)).astype(np.float32)
    g = _groom_from_layers(layers, [[0, 0], [1, 0], [0, 1]], 8)
    for s, vi in enumerate([0, 1, 2]):
        cp = oracle.strand_control_points(g, s, 5)   # C == L: control points are the layer points
        np.testing.assert_array_equal(cp, layers[:, vi])


def test_layer_point_matches_exact_rational():
    rng = np.random.default_rng(2)
    layers = rng.uniform(-0.3, 0.3, size=(4, 3, 3)).astype(np.float32)
    r1, r2 = rng.random(200), rng.random(200)
    bary = np.stack([np.sqrt(r1) * (1 - r2), np.sqrt(r1) * r2], 1).astype(np.float32)
    g = _groom_from_layers(layers, bary, 3)
    for s in range(200):
        cp = oracle.strand_control_points(g, s, 4)
        b1, b2 = Fr(float(bary[s, 0])), Fr(float(bary[s, 1]))
        b0 = 1 - b1 - b2
        for k in range(4):
            for c in range(3):
                terms = [b0 * Fr(float(layers[k, 0, c])), b1 * Fr(float(layers[k, 1, c])),
                         b2 * Fr(float(layers[k, 2, c]))]
                exact = float(sum(terms))
                bound = 6 * F32_EPS * sum(abs(float(t)) for t in terms) + 1e-30
                assert abs(float(cp[k, c]) - exact) <= bound


def test_hermite_straight_line_is_uniform():
    """Collinear, equally spaced layers: with chord-length tangents the
    Hermite spline is the straight line traversed uniformly."""
    A = np.array([0.01, -0.02, 0.03])
    d = np.array([0.011, 0.017, -0.007])
    L = 6
    layers = np.stack([np.stack([A + k * d + off for off in (np.zeros(3), [1e-3, 0, 0], [0, 1e-3, 0])])
                       for k in range(L)]).astype(np.float32)
    g = _groom_from_layers(layers, [[0, 0]], 16)
    for C in (2, 3, 9, 17, 33, 6, 11):
        cp = oracle.strand_control_points(g, 0, C).astype(np.float64)
        P0 = layers[0, 0].astype(np.float64)
        PL = layers[-1, 0].astype(np.float64)
        exp = P0[None] + (np.arange(C)[:, None] / (C - 1)) * (PL - P0)[None]
        np.testing.assert_allclose(cp, exp, atol=2e-8)


def test_hermite_matches_scipy_per_interval():
    """Independent evaluation: scipy's cubic Hermite on each layer interval
    with the finite-difference tangents scaled by the chord length."""
    rng = np.random.default_rng(3)
    L = 7
    base = np.cumsum(rng.normal(scale=0.02, size=(L, 3)), 0)
    layers = np.stack([base, base + [0.002, 0, 0], base + [0, 0.002, 0]], 1).astype(np.float32)
    g = _groom_from_layers(layers, [[0.2, 0.3]], 20)
    P = oracle.strand_control_points(g, 0, L).astype(np.float64)   # layer points
    nrm = lambda v: v / np.linalg.norm(v)
    mh = [nrm(P[1] - P[0])] + [nrm(P[k + 1] - P[k - 1]) for k in range(1, L - 1)] + [nrm(P[-1] - P[-2])]
    for C in (13, 17, 21, 9):
        cp = oracle.strand_control_points(g, 0, C).astype(np.float64)
        for j in range(C):
            u = j * (L - 1) / (C - 1)
            k = min(int(math.floor(u)), L - 2)
            ell = np.linalg.norm(P[k + 1] - P[k])
            spl = CubicHermiteSpline([0.0, 1.0], np.stack([P[k], P[k + 1]]),
                                     np.stack([mh[k] * ell, mh[k + 1] * ell]))
            np.testing.assert_allclose(cp[j], spl(u - k), atol=5e-8)


def test_styled_tangent_rules():
    """Code 1 calcTangent: forward at the root, backward at the tip, central
    otherwise, unit length."""
    sc = synth.tiny_scene(5, num_strands=50)
    g = sc.grooms[0]
    for s in (0, 17, 49):
        C = 9
        p = oracle.strand_control_points(g, s, C).astype(np.float64)
        t = oracle.strand_tangents(g, s, C).astype(np.float64)
        nrm = lambda v: v / np.linalg.norm(v)
        exp = [nrm(p[1] - p[0])] + [nrm(p[j + 1] - p[j - 1]) for j in range(1, C - 1)] + [nrm(p[-1] - p[-2])]
        np.testing.assert_allclose(t, np.stack(exp), atol=3e-6)


def test_value_layer_control_points_agree_with_decision_layer():
    sc = synth.tiny_scene(6, num_strands=64)
    g = sc.grooms[0]
    gt = v64.GroomT(g, np.full(g.num_faces, 9), 0)
    s = torch.arange(64)
    P = v64.layer_points(gt, s)
    mh = v64.layer_tangents(P)
    for C in (9, 5, 4):
        for j in range(C):
            c64 = v64.control_points(P, mh, torch.full((64,), C), torch.full((64,), j)).numpy()
            c32 = np.stack([oracle.strand_control_points(g, i, C)[j] for i in range(64)])
            np.testing.assert_allclose(c64, c32, atol=2e-7)


# ---------------------------------------------------------------------------
# projection and snap (Sec. 3.1.2)
# ---------------------------------------------------------------------------

def test_projection_matches_float64_viewport_map():
    sc = synth.tiny_scene(0, width=320, height=200)
    cam = sc.camera
    rng = np.random.default_rng(4)
    M = cam.view_proj.astype(np.float64)
    for _ in range(400):
        p = (sc.grooms[0].layer_verts.reshape(-1, 3)[rng.integers(0, 100)].astype(np.float64)
             + rng.normal(scale=0.05, size=3)).astype(np.float32)
        valid, X, Y, wz = oracle.project_point(cam, p)
        c = M @ np.r_[p.astype(np.float64), 1.0]
        assert valid == (c[3] >= cam.near)
        if not valid:
            continue
        xs = (c[0] / c[3] + 1) * 0.5 * cam.width
        ys = (1 - c[1] / c[3]) * 0.5 * cam.height
        assert abs(X - xs * 256) <= 1.0 and abs(Y - ys * 256) <= 1.0
        assert abs(wz[1] - (c[3] - cam.near) / (cam.far - cam.near)) < 1e-6


def test_projection_target_is_screen_centre_and_behind_is_invalid():
    sc = synth.tiny_scene(0, width=256, height=128)
    cam = sc.camera
    c, _, _ = synth._aabb_center(sc.grooms)
    valid, X, Y, _ = oracle.project_point(cam, c.astype(np.float32))
    assert valid and abs(X - 128 * 256) <= 2 and abs(Y - 64 * 256) <= 2
    behind = (cam.cam_pos.astype(np.float64) + (cam.cam_pos - c) * 0.5).astype(np.float32)
    assert not oracle.project_point(cam, behind)[0]


# ---------------------------------------------------------------------------
# coverage predicate and depth (Sec. 3.1.2, Sec. 3.3)
# ---------------------------------------------------------------------------

def _lb_intersects(A, B, cx, cy, h):
    """Exact Liang-Barsky clip of segment AB against the closed box."""
    t0, t1 = Fr(0), Fr(1)
    dX, dY = B[0] - A[0], B[1] - A[1]
    for p, q in ((-dX, A[0] - (cx - h)), (dX, (cx + h) - A[0]), (-dY, A[1] - (cy - h)), (dY, (cy + h) - A[1])):
        if p == 0:
            if q < 0:
                return False
            continue
        r = Fr(q, p)
        if p < 0:
            t0 = max(t0, r)
        else:
            t1 = min(t1, r)
        if t0 > t1:
            return False
    return True


def test_coverage_predicate_exact_rational_bruteforce():
    rng = np.random.default_rng(5)
    n = 0
    for _ in range(6000):
        A = [int(v) for v in rng.integers(-700, 700, 2)]
        mode = rng.integers(0, 5)
        if mode == 0:
            B = list(A)                      # degenerate: a point
        elif mode == 1:
            B = [A[0] + int(rng.integers(-900, 900)), A[1]]   # horizontal
        elif mode == 2:
            B = [A[0], A[1] + int(rng.integers(-900, 900))]   # vertical
        else:
            B = [int(v) for v in rng.integers(-700, 700, 2)]
        if rng.random() < 0.5:
            cx, cy = [int(v) * 256 + 128 for v in rng.integers(-3, 3, 2)]
        else:   # a box near a point of the segment
            u = rng.random()
            px, py = A[0] + u * (B[0] - A[0]), A[1] + u * (B[1] - A[1])
            cx = int(np.floor(px / 256 + rng.normal(scale=0.6))) * 256 + 128
            cy = int(np.floor(py / 256 + rng.normal(scale=0.6))) * 256 + 128
        h = int(rng.choice([128, 1, 9, 32, 64, 127]))
        got = oracle.segment_covers(A[0], A[1], B[0], B[1], cx, cy, h)
        assert got == _lb_intersects(A, B, cx, cy, h), (A, B, cx, cy, h)
        n += got
    assert n > 600


def test_coverage_boundary_touches_are_closed():
    # a segment ending exactly on the box edge, and one grazing a corner
    assert oracle.segment_covers(0, 0, 256, 0, 256 + 128, 0, 128)        # ends at x = 256 = cx - h
    assert not oracle.segment_covers(0, 0, 255, 0, 256 + 128, 0, 128)
    assert oracle.segment_covers(0, 512, 512, 0, 384, 384, 128)          # passes through corner (256, 256)
    assert not oracle.segment_covers(0, 511, 511, 0, 384, 384, 128)


def test_coverage_horizontal_segment_analytic():
    """From x0 <= x1 at height Y: conservative rows j satisfy
    |Y - (256 j + 128)| <= 128, columns ceil(x0/256)-1 .. floor(x1/256);
    centre rows |Y - cy| <= hc and x0 - hc <= cx <= x1 + hc."""
    rng = np.random.default_rng(6)
    for _ in range(60):
        x0 = int(rng.integers(-300, 2000))
        x1 = x0 + int(rng.integers(0, 1500))
        Y = int(rng.integers(0, 2000))
        hc = int(rng.choice([1, 9, 32, 128]))
        for j in range(-1, 10):
            cy = 256 * j + 128
            for i in range(-2, 12):
                cx = 256 * i + 128
                cons = abs(Y - cy) <= 128 and math.ceil(x0 / 256) - 1 <= i <= math.floor(x1 / 256)
                cen = abs(Y - cy) <= hc and x0 - hc <= cx <= x1 + hc
                assert oracle.segment_covers(x0, Y, x1, Y, cx, cy, 128) == cons
                assert oracle.segment_covers(x1, Y, x0, Y, cx, cy, hc) == cen


def test_depth24_endpoints_and_quantization():
    # pixel centre at A -> zA; at B -> zB; beyond B clamps to zB
    zA, zB = np.float32(0.25), np.float32(0.75)
    assert oracle.depth24(128, 128, 128 + 2560, 128, zA, zB, 128, 128) == int(0.25 * 2 ** 24)
    assert oracle.depth24(128, 128, 128 + 2560, 128, zA, zB, 128 + 2560, 128) == int(0.75 * 2 ** 24)
    assert oracle.depth24(128, 128, 128 + 2560, 128, zA, zB, 128 + 9000, 128) == int(0.75 * 2 ** 24)
    assert oracle.depth24(0, 0, 0, 0, np.float32(1.5), zB, 100, 100) == 2 ** 24 - 1   # clamp, degenerate
    # halfway, exactly representable
    assert oracle.depth24(0, 0, 512, 0, zA, zB, 256, 0) == int(0.5 * 2 ** 24)


def _brute_segments(g, cam, C, base=0):
    """Every projected segment (XA, YA, XB, YB, zA, zB, h_c, id) recomputed
    from the oracle's control points and projection."""
    segs = []
    f32 = np.float32
    focal = f32(f32(0.5) * f32(cam.height)) / f32(cam.tan_half_fovy)
    for s in range(g.num_strands):
        cp = oracle.strand_control_points(g, s, C)
        pr = [oracle.project_point(cam, p) for p in cp]
        for j in range(C - 1):
            (va, XA, YA, wa), (vb, XB, YB, wb) = pr[j], pr[j + 1]
            if not (va and vb):
                continue
            wm = f32(f32(wa[0] + wb[0]) * f32(0.5))
            r = f32(f32(f32(128.0) * f32(g.strand_width_m)) * focal) / wm
            hc = int(min(max(np.rint(r), 1), 128))
            segs.append((XA, YA, XB, YB, f32(wa[1]), f32(wb[1]), hc, ((base + s) << 7) | j))
    return segs


def _brute_key(XA, YA, XB, YB, zA, zB, sid, cx, cy):
    f32 = np.float32
    dX, dY = XB - XA, YB - YA
    num, den = (cx - XA) * dX + (cy - YA) * dY, dX * dX + dY * dY
    t = f32(0) if den == 0 else min(max(f32(num) / f32(den), f32(0)), f32(1))
    z = min(max(f32(zA + f32(f32(zB - zA) * t)), f32(0)), f32(1))
    d = min(int(np.floor(f32(z * f32(16777216.0)))), 2 ** 24 - 1)
    return np.uint64((d << 40) | sid)


def _brute_force_keys(g, cam, C, base=0):
    """Per-pixel nearest-segment search over every segment of every strand
    (exact rational coverage), recomputing d24 in float32 numpy."""
    W, H = cam.width, cam.height
    segs = _brute_segments(g, cam, C, base)
    vc = np.full(W * H, oracle.EMPTY, np.uint64)
    va = vc.copy()
    for (XA, YA, XB, YB, zA, zB, hc, sid) in segs:
        for m in range(H):
            cy = 256 * m + 128
            if min(YA, YB) > cy + 256 or max(YA, YB) < cy - 256:
                continue
            for i in range(W):
                cx = 256 * i + 128
                if min(XA, XB) > cx + 256 or max(XA, XB) < cx - 256:
                    continue
                ca = _lb_intersects((XA, YA), (XB, YB), cx, cy, 128)
                cc = _lb_intersects((XA, YA), (XB, YB), cx, cy, hc)
                if not (ca or cc):
                    continue
                key = _brute_key(XA, YA, XB, YB, zA, zB, sid, cx, cy)
                px = m * W + i
                if ca:
                    va[px] = min(va[px], key)
                if cc:
                    vc[px] = min(vc[px], key)
    return vc, va


@pytest.mark.parametrize("seed,W,H,C", [(11, 37, 29, 5), (12, 24, 40, 4)])
def test_raster_equals_bruteforce_nearest_segment(seed, W, H, C):
    sc = synth.tiny_scene(seed, width=W, height=H, num_strands=40, segments=C - 1,
                          dist_m=0.35, jitter_m=0.004)
    g = sc.grooms[0]
    lods = [oracle.lod(g, sc.camera, synth.LodParams(0))]
    vc, va, cnt = oracle.raster([g], sc.camera, lods)
    bc, ba = _brute_force_keys(g, sc.camera, C)
    assert (va != oracle.EMPTY).sum() > 50
    np.testing.assert_array_equal(va, ba)
    np.testing.assert_array_equal(vc, bc)


# Standard multisample positions (1/16 px, y down), written out independently
# of the oracle's table.
_MSAA_POS = {2: [(4, 4), (-4, -4)],
             4: [(-2, -6), (6, -2), (-6, 2), (2, 6)],
             8: [(1, -3), (-1, 3), (5, 1), (-3, -5), (-5, 5), (-7, -1), (3, 7), (7, -7)]}


def _brute_force_msaa(g, cam, C, N):
    """Per-sample nearest-segment search: sample k of pixel (i, m) at
    (256 i + 128 + 16 ox_k, 256 m + 128 + 16 oy_k), covered when the closed
    box of half-width h_c around it meets the segment (exact rational clip)."""
    W, H = cam.width, cam.height
    pos = [(0, 0)] if N == 1 else _MSAA_POS[N]
    vis = np.full((N, W * H), oracle.EMPTY, np.uint64)
    for (XA, YA, XB, YB, zA, zB, hc, sid) in _brute_segments(g, cam, C):
        for m in range(H):
            if min(YA, YB) > 256 * m + 512 or max(YA, YB) < 256 * m - 256:
                continue
            for i in range(W):
                if min(XA, XB) > 256 * i + 512 or max(XA, XB) < 256 * i - 256:
                    continue
                for k, (ox, oy) in enumerate(pos):
                    sx, sy = 256 * i + 128 + 16 * ox, 256 * m + 128 + 16 * oy
                    if _lb_intersects((XA, YA), (XB, YB), sx, sy, hc):
                        key = _brute_key(XA, YA, XB, YB, zA, zB, sid, sx, sy)
                        vis[k, m * W + i] = min(vis[k, m * W + i], key)
    return vis


@pytest.mark.parametrize("seed,W,H,C,N", [(21, 23, 19, 4, 2), (22, 30, 17, 5, 4), (23, 19, 21, 4, 8)])
def test_msaa_raster_equals_bruteforce(seed, W, H, C, N):
    """Sec. 3.3's multisample reference: every sample layer against an
    independent per-sample search."""
    sc = synth.tiny_scene(seed, width=W, height=H, num_strands=30, segments=C - 1,
                          dist_m=0.35, jitter_m=0.004)
    g = sc.grooms[0]
    g.strand_width_m = 0.005           # h_c of a few tenths of a pixel: samples both hit and missed
    lods = [oracle.lod(g, sc.camera, synth.LodParams(0))]
    vis, cnt = oracle.raster_msaa([g], sc.camera, lods, N)
    ref = _brute_force_msaa(g, sc.camera, C, N)
    assert (vis != oracle.EMPTY).sum() > 40
    for k in range(N):
        np.testing.assert_array_equal(vis[k], ref[k], err_msg=f"sample {k}")
    assert cnt >= (vis != oracle.EMPTY).sum()


def test_msaa_single_sample_is_the_centre_layer():
    sc = synth.scene_tiny_256()
    lods = oracle.lods_for(sc)
    vc, _, c = oracle.raster(sc.grooms, sc.camera, lods)
    vis, cnt = oracle.raster_msaa(sc.grooms, sc.camera, lods, 1)
    np.testing.assert_array_equal(vis[0], vc)
    assert cnt == c[0]


def test_msaa_resolve_uniform_colour_and_coverage_alpha():
    """With ambient light only and one albedo, every covered sample has the
    colour ambient * albedo: rgb is that constant wherever a sample is
    covered (mean over covered samples, not over all) and alpha is the
    covered fraction."""
    sc = synth.tiny_scene(24, width=40, height=32, num_strands=60, segments=5, dist_m=0.3)
    g = sc.grooms[0]
    g.strand_width_m = 0.004
    g.strand_albedo[:] = np.float32([0.3, 0.5, 0.7])
    lights = synth.Lights(dirs=np.zeros((0, 3), np.float32), radiance=np.zeros((0, 3), np.float32),
                          ambient=float(np.float32(0.5)))
    lods = oracle.lods_for(sc)
    for N in (2, 4):
        vis, _ = oracle.raster_msaa(sc.grooms, sc.camera, lods, N)
        num, den = oracle.msaa_decisions(sc.grooms, sc.camera, lods, N, vis)
        gts = [v64.GroomT(gg, l[1], b) for gg, l, b in zip(sc.grooms, lods, oracle.strand_bases(sc.grooms))]
        out = v64.resolve_msaa(gts, sc.camera, lights, vis, num, den).numpy()
        cov = (vis != oracle.EMPTY).sum(0)
        assert (cov > 0).sum() > 30 and ((cov > 0) & (cov < N)).sum() > 10
        np.testing.assert_allclose(out[:, 3], cov / N, rtol=0, atol=1e-15)
        exp = 0.5 * np.float32([0.3, 0.5, 0.7]).astype(np.float64)
        np.testing.assert_allclose(out[cov > 0, :3], np.broadcast_to(exp, (int((cov > 0).sum()), 3)), rtol=1e-12)
        assert np.all(out[cov == 0] == 0)


def test_raster_invariants_and_thread_independence():
    sc = synth.scene_tiny_256()
    lods = oracle.lods_for(sc)
    vc1, va1, c1 = oracle.raster(sc.grooms, sc.camera, lods, nthreads=1)
    vc4, va4, c4 = oracle.raster(sc.grooms, sc.camera, lods, nthreads=4)
    np.testing.assert_array_equal(vc1, vc4)
    np.testing.assert_array_equal(va1, va4)
    assert tuple(c1) == tuple(c4)
    # centre sample subset of conservative: A <= G everywhere, G set implies A set
    assert np.all(va1 <= vc1)
    eG, dG, sg, seg = v64.key_fields(vc1)
    eA, _, sgA, segA = v64.key_fields(va1)
    assert np.all(~eA[~eG])
    # decoded IDs round-trip into valid strands and segments
    g = sc.grooms[0]
    for e, s_, j_ in ((eG, sg, seg), (eA, sgA, segA)):
        s_ = s_[~e]
        j_ = j_[~e]
        assert np.all(s_ < g.num_strands)
        assert np.all(j_ < lods[0][1][g.strand_face[s_]] - 1)
    # counts are the number of covered (pixel, layer) pairs >= distinct pixels
    assert c1[1] >= (~eA).sum() and c1[0] >= (~eG).sum()


def test_key_packing_round_trip():
    rng = np.random.default_rng(7)
    d = rng.integers(0, 2 ** 24, 1000).astype(np.uint64)
    s = rng.integers(0, 2 ** 33 - 1, 1000).astype(np.uint64)
    j = rng.integers(0, 127, 1000).astype(np.uint64)
    key = (d << np.uint64(40)) | (s << np.uint64(7)) | j
    e, d2, s2, j2 = v64.key_fields(key)
    assert not e.any()
    np.testing.assert_array_equal(d2, d.astype(np.int64))
    np.testing.assert_array_equal(s2, s.astype(np.int64))
    np.testing.assert_array_equal(j2, j.astype(np.int64))
    # smaller depth always wins over any payload
    assert ((np.uint64(5) << np.uint64(40)) | np.uint64(0xFFFFFFFFFE)) < (np.uint64(6) << np.uint64(40))


# ---------------------------------------------------------------------------
# LOD (Sec. 3.2, Eqs. 1-5)
# ---------------------------------------------------------------------------

def test_lod_control_point_snap_table_cmax127():
    """Eqs. 4-5 with C_max = 127: C is a power of two plus one and never
    exceeds 65; the layer count is the lower bound."""
    seen = set()
    for Lf in np.linspace(0.0, 1.0, 2001).astype(np.float32):
        raw64 = math.sqrt(float(Lf)) * 127
        if abs(raw64 - round(raw64)) < 1e-3:
            continue
        craw = max(int(math.floor(raw64)), 4)
        exp = min(2 ** int(math.floor(math.log2(craw - 1))) + 1, 127)
        exp = max(exp, 4)
        _, c = oracle.lod_counts(Lf, 100, 0.5, 4, 127)
        assert c == exp
        seen.add(c)
    assert seen == {5, 9, 17, 33, 65, 4}
    assert oracle.lod_counts(1.0, 10, 0.0, 4, 127)[1] == 65


def test_lod_full_detail_reaches_cmax_only_for_power_of_two_segments():
    assert oracle.lod_counts(1.0, 10, 0.1, 8, 17) == (10, 17)
    assert oracle.lod_counts(1.0, 10, 0.1, 6, 13) == (10, 9)      # 12 segments snap to 8
    assert oracle.lod_counts(0.0, 10, 0.1, 6, 13) == (1, 6)       # floor: layers, at least one strand


def test_lod_strand_count_eq1():
    rng = np.random.default_rng(8)
    for _ in range(3000):
        Lf = np.float32(rng.random())
        N = int(rng.integers(0, 400))
        dl = np.float32(rng.random() * 0.999)
        v = float(Lf) * (N + float(dl))
        if abs(v - round(v)) < 1e-3:
            continue
        exp = 0 if N == 0 else min(max(math.ceil(v), 1), N)
        assert oracle.lod_counts(Lf, N, dl, 4, 9)[0] == exp


def test_lod_disabled_is_full_detail_and_culling():
    sc = synth.tiny_scene(0, num_strands=500)
    g = sc.grooms[0]
    n, c = oracle.lod(g, sc.camera, synth.LodParams(0))
    counts = np.bincount(g.strand_face, minlength=g.num_faces)
    np.testing.assert_array_equal(n, counts)
    assert np.all(c == g.segments_per_strand + 1)
    # camera turned away: every bundle is culled
    ctr, _, _ = synth._aabb_center([g])
    away = synth.make_camera(ctr + np.array([0, 0, 0.5]), ctr + np.array([0, 0, 1.5]), 40, 256, 256)
    n2, _ = oracle.lod(g, away, synth.LodParams(1, 3.0))
    assert n2.sum() == 0
    # groom entirely to the right of the frustum
    right = synth.make_camera(ctr + np.array([-2.0, 0, 0.5]), ctr + np.array([-2.0, 0, 0]), 40, 256, 256)
    assert oracle.lod(g, right, synth.LodParams(1, 3.0))[0].sum() == 0


def test_lod_bundle_aabb_eq2_eq3():
    sc = synth.tiny_scene(9, num_strands=800, width=400, height=300, dist_m=1.2)
    g, cam = sc.grooms[0], sc.camera
    n, c = oracle.lod(g, cam, synth.LodParams(1, 3.0))
    counts = np.bincount(g.strand_face, minlength=g.num_faces)
    M = cam.view_proj.astype(np.float64)
    checked = 0
    for f in range(g.num_faces):
        pts = g.layer_verts[:, g.faces[f]].reshape(-1, 3).astype(np.float64)
        clip = np.c_[pts, np.ones(len(pts))] @ M.T
        xs = (clip[:, 0] / clip[:, 3] + 1) * 0.5 * cam.width
        ys = (1 - clip[:, 1] / clip[:, 3]) * 0.5 * cam.height
        diag = math.hypot(xs.max() - xs.min(), ys.max() - ys.min())
        Lf = min(max(diag / cam.height * 3.0, 0.0), 1.0)
        v = Lf * (counts[f] + float(g.bundle_delta[f]))
        raw = math.sqrt(Lf) * (g.segments_per_strand + 1)
        if abs(v - round(v)) < 1e-3 or abs(raw - round(raw)) < 1e-3:
            continue
        expn = 0 if counts[f] == 0 else min(max(math.ceil(v), 1), counts[f])
        craw = max(int(math.floor(raw)), g.num_layers)
        expc = max(min(2 ** int(math.floor(math.log2(craw - 1))) + 1, g.segments_per_strand + 1), g.num_layers)
        assert n[f] == expn and c[f] == expc
        checked += 1
    assert checked > 20


def test_lod_total_strands_monotone_in_distance():
    g = synth.make_groom(1, 8, 2, 5, 0.2, 6000, 16, curl_amp_m=0.01)
    tot = []
    for i in range(8):
        sc = synth.scene_lod_sweep(i, g)
        tot.append(int(oracle.lod(g, sc.camera, sc.lod)[0].sum()))
    # farthest first: counts grow as the groom gets bigger on screen
    assert all(a <= b for a, b in zip(tot, tot[1:])), tot
    assert tot[0] < tot[-1] <= g.num_strands


# ---------------------------------------------------------------------------
# shading (Sec. 3.4) and screen tangent (Code 2)
# ---------------------------------------------------------------------------

def _shade_one(T, X, albedo, cam_pos, dirs, rad, rough=0.15, tilt=-0.05, amb=0.05):
    cam = synth.Camera(np.eye(4, dtype=np.float32), np.asarray(cam_pos, np.float32), 0.05, 256, 0.5, 8, 8)
    lights = synth.make_lights(dirs, rad, ambient=amb)
    out = v64.shade(torch.tensor(np.array([X], np.float64)), torch.tensor(np.array([T], np.float64)),
                    torch.tensor(np.array([albedo], np.float64)), cam, lights, rough, tilt)
    return out[0].numpy(), lights


def test_shading_closed_forms():
    kd, ks = float(np.float32(1 / math.pi)), float(np.float32(0.25))
    b = 0.15
    sa = math.sin(-0.05)
    alb = np.array([0.3, 0.4, 0.5])
    # T perpendicular to L and V: diffuse = albedo k_d, lobe at T.L = T.V = 0
    c, _ = _shade_one([1, 0, 0], [0, 0, 0], alb, [0, 0, 2], [[0, 1, 0]], [1.0])
    exp = alb * kd + ks * math.exp(-(sa * sa) / (2 * b * b)) + float(np.float32(0.05)) * alb
    np.testing.assert_allclose(c, exp, rtol=1e-12)
    # T parallel to L: no diffuse; T.L = 1, T.V = 0
    c, _ = _shade_one([0, 1, 0], [0, 0, 0], alb, [0, 0, 2], [[0, 1, 0]], [1.0])
    u = 0.5 + sa
    exp = ks * math.exp(-(u * u) / (2 * b * b)) + float(np.float32(0.05)) * alb
    np.testing.assert_allclose(c, exp, rtol=1e-12)
    # two lights add
    c1, _ = _shade_one([0.6, 0.8, 0], [0, 0, 0], alb, [0, 0, 2], [[1, 0, 0]], [0.7], amb=0)
    c2, _ = _shade_one([0.6, 0.8, 0], [0, 0, 0], alb, [0, 0, 2], [[0, 0, 1]], [0.2], amb=0)
    c12, _ = _shade_one([0.6, 0.8, 0], [0, 0, 0], alb, [0, 0, 2], [[1, 0, 0], [0, 0, 1]], [0.7, 0.2], amb=0)
    np.testing.assert_allclose(c12, c1 + c2, rtol=1e-12)


def test_screen_tangent_against_numerical_jacobian_and_signs():
    sc = synth.tiny_scene(0, width=300, height=200)
    cam = sc.camera
    M = cam.view_proj.astype(np.float64)

    def scr(p):
        c = M @ np.r_[p, 1.0]
        return np.array([(c[0] / c[3] + 1) * 0.5 * cam.width, (1 - c[1] / c[3]) * 0.5 * cam.height])

    rng = np.random.default_rng(10)
    ctr, _, _ = synth._aabb_center(sc.grooms)
    for _ in range(50):
        X = ctr + rng.normal(scale=0.03, size=3)
        T = rng.normal(size=3)
        T /= np.linalg.norm(T)
        h = 1e-6
        J = (scr(X + h * T) - scr(X - h * T)) / (2 * h)
        exp = J / np.linalg.norm(J)
        ts64 = v64.screen_tangent(torch.tensor(X[None]), torch.tensor(T[None]), cam)[0].numpy()
        np.testing.assert_allclose(ts64, exp, atol=1e-6)
        iso, ts32 = oracle.screen_tangent(cam, X.astype(np.float32), T.astype(np.float32))
        assert not iso
        np.testing.assert_allclose(ts32, exp, atol=2e-5)
    # camera looks along -z: world +x is screen right, world +y is screen up (y down)
    assert np.allclose(oracle.screen_tangent(cam, ctr.astype(np.float32), np.float32([1, 0, 0]))[1], [1, 0], atol=1e-3)
    assert np.allclose(oracle.screen_tangent(cam, ctr.astype(np.float32), np.float32([0, 1, 0]))[1], [0, -1], atol=1e-3)
    # a tangent along the view ray through X is degenerate; so is one within
    # 0.3 degrees of it, but not one 3 degrees off; a zero tangent is too
    ray = (ctr - cam.cam_pos).astype(np.float64)
    ray /= np.linalg.norm(ray)
    assert oracle.screen_tangent(cam, ctr.astype(np.float32), ray.astype(np.float32))[0]
    side = np.cross(ray, [0.0, 1.0, 0.0])
    side /= np.linalg.norm(side)
    for ang, iso in ((0.005, True), (0.05, False)):
        t = np.cos(ang) * ray + np.sin(ang) * side
        assert oracle.screen_tangent(cam, ctr.astype(np.float32), t.astype(np.float32))[0] == iso
    assert oracle.screen_tangent(cam, ctr.astype(np.float32), np.zeros(3, np.float32))[0]


def test_strip_membership_geometry():
    assert oracle.in_strip(0, 1.0, 0.0, 5, 0, 0.5)
    assert not oracle.in_strip(0, 1.0, 0.0, 0, 1, 0.5)
    r = np.float32(math.sqrt(0.5))
    assert oracle.in_strip(0, r, r, 3, 3, 0.5)
    assert not oracle.in_strip(0, r, r, 1, 0, 0.5)          # distance 0.707 > 0.5
    assert oracle.in_strip(1, 0, 0, 0, 0, 0.5) and not oracle.in_strip(1, 0, 0, 1, 0, 0.5)


# ---------------------------------------------------------------------------
# filter, alpha, reconnection (Sec. 3.3)
# ---------------------------------------------------------------------------

def _resolve_scene(sc, filt=None, lights=None):
    lods = oracle.lods_for(sc)
    filt = filt or sc.filt
    vc, va, _ = oracle.raster(sc.grooms, sc.camera, lods)
    dec = oracle.resolve_decisions(sc.grooms, sc.camera, lods, filt, vc, va)
    gts = [v64.GroomT(g, l[1], b) for g, l, b in zip(sc.grooms, lods, oracle.strand_bases(sc.grooms))]
    rgba, pix = v64.resolve(gts, sc.camera, lights or sc.lights, filt, vc, va, dec)
    return rgba, pix, vc, va, dec, lods


def test_filter_preserves_uniform_colour():
    """Ambient-only light and one albedo: every centre colour is equal, so
    every normalized filter output equals it."""
    sc = synth.tiny_scene(0, num_strands=600)
    sc.grooms[0].strand_albedo[:] = np.float32(0.37)
    lights = synth.make_lights(np.zeros((0, 3)) + [[0, 1, 0]], [0.0], ambient=0.5)
    rgba, pix, vc, va, dec, _ = _resolve_scene(sc, lights=lights)
    c = float(np.float32(0.5)) * float(np.float32(0.37))
    nz = rgba[:, 3] > 0
    assert nz.sum() > 100
    np.testing.assert_allclose(rgba[nz, :3].numpy(), c, rtol=1e-13)
    a = rgba[:, 3].numpy()
    assert np.all((a >= 0) & (a <= 1))


def test_filter_isotropic_unit_weights_is_masked_gaussian_convolution():
    """s_par = s_perp, no colour term, no depth rejection: the filter is a
    normalized Gaussian convolution of the centre-sample image restricted to
    centre pixels (scipy correlate, zero outside the screen)."""
    sc = synth.tiny_scene(1, num_strands=400, width=96, height=80)
    filt = synth.FilterParams(s_par=0.4, s_perp=0.4, sigma_c=1e9, depth_reject_m=1e9, depth_mismatch_m=1e9)
    rgba, pix, vc, va, dec, lods = _resolve_scene(sc, filt=filt)
    W, H = sc.camera.width, sc.camera.height
    eG = v64.key_fields(vc)[0].reshape(H, W)
    # centre colours from the same scene with the filter off
    off = synth.FilterParams(enabled=0)
    gts = [v64.GroomT(g, l[1], b) for g, l, b in zip(sc.grooms, lods, oracle.strand_bases(sc.grooms))]
    img0, pix0 = v64.resolve(gts, sc.camera, sc.lights, off, vc, va, dec)
    C = v64.full_image(img0, pix0, W, H).numpy()[..., :3]
    r = 5
    sig = 0.4 * r
    yy, xx = np.mgrid[-r:r + 1, -r:r + 1]
    k = np.exp(-(xx ** 2 + yy ** 2) / sig ** 2)
    mask = (~eG).astype(np.float64)
    num = np.stack([correlate(C[..., ch] * mask, k, mode="constant") for ch in range(3)], -1)
    den = correlate(mask, k, mode="constant")
    out = v64.full_image(rgba, pix, W, H).numpy()
    sel = ~eG
    den = np.where(den > 0, den, 1.0)
    assert sel.sum() > 50
    np.testing.assert_allclose(out[sel][:, :3], (num / den[..., None])[sel], atol=1e-9)


def test_filter_isolated_centre_pixel_keeps_its_colour():
    """A centre pixel with no other contributing neighbour in its window
    outputs its own shaded colour."""
    sc = synth.tiny_scene(2, num_strands=12, width=200, height=200)
    rgba, pix, vc, va, dec, lods = _resolve_scene(sc)
    W, H = sc.camera.width, sc.camera.height
    eG, dG, _, _ = v64.key_fields(vc)
    gts = [v64.GroomT(g, l[1], b) for g, l, b in zip(sc.grooms, lods, oracle.strand_bases(sc.grooms))]
    img0, pix0 = v64.resolve(gts, sc.camera, sc.lights, synth.FilterParams(enabled=0), vc, va, dec)
    C = v64.full_image(img0, pix0, W, H).numpy().reshape(-1, 4)
    out = v64.full_image(rgba, pix, W, H).numpy().reshape(-1, 4)
    rej, mis = oracle.depth_thresholds(sc.camera, sc.filt)
    eA, dA, _, _ = v64.key_fields(va)
    n = 0
    for p in np.nonzero(~eG)[0]:
        x, y = p % W, p // W
        others = 0
        for dy in range(-5, 6):
            for dx in range(-5, 6):
                qx, qy = x + dx, y + dy
                if (dx or dy) and 0 <= qx < W and 0 <= qy < H:
                    q = qy * W + qx
                    others += (not eG[q]) and abs(dG[q] - dG[p]) <= rej
        if others == 0 and not (dA[p] + mis <= dG[p]):
            np.testing.assert_allclose(out[p, :3], C[p, :3], rtol=1e-13)
            n += 1
    assert n >= 3


def test_strip_counts_equal_window_bruteforce():
    sc = synth.tiny_scene(3, num_strands=300, width=80, height=72)
    rgba, pix, vc, va, dec, lods = _resolve_scene(sc)
    W, H = sc.camera.width, sc.camera.height
    eG = v64.key_fields(vc)[0]
    eA = v64.key_fields(va)[0]
    gts = [v64.GroomT(g, l[1], b) for g, l, b in zip(sc.grooms, lods, oracle.strand_bases(sc.grooms))]
    rng = np.random.default_rng(11)
    cand = np.nonzero(~eG)[0]
    for p in rng.choice(cand, size=min(40, cand.size), replace=False):
        x, y = p % W, p // W
        X, T, _ = v64.pixel_geometry(gts[0], v64.key_fields(vc)[2][[p]], v64.key_fields(vc)[3][[p]],
                                     dec["numG"][[p]], dec["denG"][[p]])
        iso, ts = oracle.screen_tangent(sc.camera, X[0].numpy().astype(np.float32), T[0].numpy().astype(np.float32))
        hc = ha = 0
        for dy in range(-5, 6):
            for dx in range(-5, 6):
                qx, qy = x + dx, y + dy
                if 0 <= qx < W and 0 <= qy < H and oracle.in_strip(iso, ts[0], ts[1], dx, dy, 0.5):
                    hc += not eG[qy * W + qx]
                    ha += not eA[qy * W + qx]
        # the FP64-rounded geometry may sit on a strip boundary; allow that rare case
        assert abs(dec["HcG"][p] - hc) <= 1 and abs(dec["HaG"][p] - ha) <= 1
        assert dec["HaG"][p] >= 1 and 0 <= dec["HcG"][p] <= dec["HaG"][p] + 0


def test_depth_thresholds_in_d24_units():
    cam = synth.tiny_scene(0).camera
    rej, mis = oracle.depth_thresholds(cam, synth.FilterParams())
    span = float(np.float32(256.0)) - float(np.float32(0.05))
    assert rej == round(1.45e-3 / span * 2 ** 24) == 95
    assert mis == round(5e-4 / span * 2 ** 24) == 33


def test_paper_constants_golden():
    here = os.path.dirname(__file__)
    vals = {}
    for line in open(os.path.join(here, "golden", "paper_constants.txt")):
        if line.startswith("#") or not line.strip():
            continue
        name, val = line.split()[:2]
        vals[name] = float(val)
    f = synth.FilterParams()
    assert f.radius == vals["filter_radius"]
    assert f.sigma_c == vals["sigma_c"] and f.iso_scale == vals["iso_scale"]
    assert f.depth_reject_m == vals["depth_reject"] and f.depth_mismatch_m == vals["depth_mismatch"]
    assert f.strip_halfwidth == vals["strip_halfwidth"]
    assert synth.LodParams().lam == vals["lambda_groom1"]
    # with C_max = 127 the full-detail snap of Eq. 5 is 65
    assert oracle.lod_counts(1.0, 1, 0.0, 2, int(vals["c_max"]))[1] == 65


# ---------------------------------------------------------------------------
# gradient of the FP64 value layer (visibility held fixed)
# ---------------------------------------------------------------------------

def test_value_layer_gradient_matches_central_differences():
    sc = synth.tiny_scene(4, num_strands=60, width=64, height=56, dist_m=0.3)
    g = sc.grooms[0]
    lods = oracle.lods_for(sc)
    vc, va, _ = oracle.raster(sc.grooms, sc.camera, lods)
    dec = oracle.resolve_decisions(sc.grooms, sc.camera, lods, sc.filt, vc, va)
    rng = np.random.default_rng(12)
    target = torch.from_numpy(rng.random((64 * 56, 3)) * 0.2)

    def loss(lv, alb):
        gt = v64.GroomT(g, lods[0][1], 0, layer_verts=lv, albedo=alb)
        rgba, pix = v64.resolve([gt], sc.camera, sc.lights, sc.filt, vc, va, dec)
        img = torch.zeros((64 * 56, 3), dtype=torch.float64).index_put((torch.from_numpy(pix),),
                                                                       rgba[:, :3] * rgba[:, 3:4])
        return torch.sqrt(((img - target) ** 2).sum())

    lv = torch.from_numpy(g.layer_verts.astype(np.float64)).requires_grad_(True)
    alb = torch.from_numpy(g.strand_albedo.astype(np.float64)).requires_grad_(True)
    l0 = loss(lv, alb)
    l0.backward()
    glv, galb = lv.grad.numpy(), alb.grad.numpy()
    assert np.abs(glv).max() > 0
    h = 1e-5
    flat = np.argsort(-np.abs(glv).ravel())[:12]
    for idx in list(flat) + list(rng.integers(0, glv.size, 6)):
        e = torch.zeros(glv.size, dtype=torch.float64)
        e[idx] = h
        e = e.reshape(glv.shape)
        with torch.no_grad():
            fd = (loss(lv + e, alb) - loss(lv - e, alb)).item() / (2 * h)
        assert abs(fd - glv.ravel()[idx]) <= 1e-6 + 1e-4 * abs(fd), (idx, fd, glv.ravel()[idx])
    for idx in np.argsort(-np.abs(galb).ravel())[:6]:
        e = torch.zeros(galb.size, dtype=torch.float64)
        e[idx] = h
        e = e.reshape(galb.shape)
        with torch.no_grad():
            fd = (loss(lv, alb + e) - loss(lv, alb - e)).item() / (2 * h)
        assert abs(fd - galb.ravel()[idx]) <= 1e-7 + 1e-5 * abs(fd)


# ---------------------------------------------------------------------------
# baked ambient occlusion (Sec. 3.4)
# ---------------------------------------------------------------------------

def test_ao_interpolation_reproduces_linear_layers_and_layer_values():
    """AO interpolated like the position: at control points that fall on
    layers it equals the layer's barycentric AO, and AO linear in the layer
    index is reproduced exactly (finite-difference slopes make the cubic
    exact for linear data)."""
    sc = synth.tiny_scene(7, num_strands=40, num_layers=5)
    g = sc.grooms[0]
    L, V = g.num_layers, g.num_verts
    ao_lin = (0.2 + 0.15 * np.arange(L)[:, None] * np.ones((1, V))).astype(np.float32)
    g.vert_ao = ao_lin
    gt = v64.GroomT(g, np.full(g.num_faces, 9), 0)
    s = torch.arange(40)
    A = v64.layer_ao(gt, s)
    np.testing.assert_allclose(A.numpy(), np.tile(0.2 + 0.15 * np.arange(L), (40, 1)), atol=1e-7)
    for C in (5, 9, 17, 4):
        for j in range(C):
            a = v64.control_ao(A, torch.full((40,), C), torch.full((40,), j)).numpy()
            np.testing.assert_allclose(a, 0.2 + 0.15 * j * (L - 1) / (C - 1), atol=1e-12)
    rng = np.random.default_rng(3)
    g.vert_ao = rng.uniform(0.3, 1.0, (L, V)).astype(np.float32)
    gt = v64.GroomT(g, np.full(g.num_faces, 5), 0)
    A = v64.layer_ao(gt, s)
    for j in range(5):   # C == L: control points sit on the layers
        np.testing.assert_allclose(v64.control_ao(A, torch.full((40,), 5), torch.full((40,), j)).numpy(),
                                   A[:, j].numpy(), atol=1e-12)


def test_ao_one_is_no_ao_and_scales_only_the_ambient_term():
    sc = synth.tiny_scene(8, num_strands=300, width=96, height=80)
    g = sc.grooms[0]
    rgba0, pix0, vc, va, dec, lods = _resolve_scene(sc)
    g.vert_ao = np.ones((g.num_layers, g.num_verts), np.float32)
    rgba1, pix1, _, _, _, _ = _resolve_scene(sc)
    np.testing.assert_array_equal(rgba0.numpy(), rgba1.numpy())
    # ambient only, shading without the (colour-nonlinear) filter: a uniform
    # AO of 0.25 quarters every shaded pixel
    lights = synth.make_lights([[0.0, 1.0, 0.0]], [0.0], ambient=0.5)
    off = synth.FilterParams(enabled=0)
    g.vert_ao = None
    ra, pa, _, _, _, _ = _resolve_scene(sc, filt=off, lights=lights)
    g.vert_ao = np.full((g.num_layers, g.num_verts), 0.25, np.float32)
    rb, pb, _, _, _, _ = _resolve_scene(sc, filt=off, lights=lights)
    sel = ra[:, 3] > 0
    np.testing.assert_allclose(rb[sel, :3].numpy(), 0.25 * ra[sel, :3].numpy(), rtol=1e-12)


# ---------------------------------------------------------------------------
# shadow maps with the LOD depth correction (Sec. 3.2 "Depth Comparison
# Artifact Fix", queried by the shading of Sec. 3.4)
# ---------------------------------------------------------------------------

def _two_strand_shadow_setup(width_m=0.003):
    """Two straight strands along x (5 collinear, equally spaced layers):
    A at z = 1 cm, B at z = 0, both at y = 0; a light camera 1 m up the z
    axis looking down sees A in front of B; the main camera looks down -y so
    A and B are separate rows of the image."""
    xs = [-0.04 + 0.02 * k for k in range(5)]
    layers = [[[x, -0.01, 0.0], [x, 0.01, 0.0], [x, 0.0, 0.02]] for x in xs]
    g = _groom_from_layers(layers, [[0.25, 0.5], [0.5, 0.0]], 8)      # A: (y, z) = (0, 0.01); B: (0, 0)
    g.strand_width_m = width_m
    light = synth.make_camera([0.0, 0.0, 1.0], [0.0, 0.0, 0.0], 10.0, 256, 256, near=0.05, far=2.0)
    cam = synth.make_camera([0.0, 0.3, 0.005], [0.0, 0.0, 0.005], 40.0, 192, 128, up=(0.0, 0.0, 1.0))
    return g, light, cam


def _shadow_vis_of_centre_keys(g, light, cam, spec, lod_n=None):
    lods = [oracle.lod(g, cam, synth.LodParams(0))]
    vc, _, _ = oracle.raster([g], cam, lods)
    smap = oracle.shadow_map([g], spec)
    tex = oracle.centre_shadow_texels([g], cam, lods, vc, [(spec, smap)])
    e, _, sg, seg = v64.key_fields(vc)
    idx = np.nonzero(~e)[0]
    W = cam.width
    num, den = oracle.msaa_decisions([g], cam, lods, 1, vc[None, :])
    gt = v64.GroomT(g, lods[0][1], 0, lod_n=lod_n)
    X, _, s = v64.pixel_geometry(gt, sg[idx], seg[idx], num[0][idx], den[0][idx])
    V = v64.shadow_visibility(gt, X, s, [tex[0][idx]], [(spec, smap)], 1)
    return V[:, 0].numpy(), sg[idx], tex[0][idx], X, smap


def test_shadow_closed_form_two_strands():
    """The back strand sees exp(-sigma (d - bias)) with d = 1 cm, the depth
    between the strands along the light's view axis; the front strand is
    unshadowed (its own depth, within the bias)."""
    g, light, cam = _two_strand_shadow_setup()
    spec = synth.ShadowSpec(light=0, cam=light, sigma=100.0, bias_m=0.001, depth_correction=0)
    V, sg, tex, X, smap = _shadow_vis_of_centre_keys(g, light, cam, spec)
    a, b = sg == 0, sg == 1
    assert a.sum() > 40 and b.sum() > 40 and np.all(tex >= 0)
    np.testing.assert_allclose(V[a], 1.0, rtol=0, atol=1e-12)
    sig, bias = float(np.float32(100.0)), float(np.float32(0.001))
    np.testing.assert_allclose(V[b], math.exp(-sig * (0.01 - bias)), rtol=2e-4)
    # the map holds A's depth wherever B's points look up
    d24 = (smap[tex[b]] >> np.uint64(40)).astype(np.float64)
    z_a = (0.99 - float(np.float32(0.05))) / (float(np.float32(2.0)) - float(np.float32(0.05)))
    assert np.all(np.abs(d24 / 2 ** 24 - z_a) < 3e-7)
    # the texel column is the floor of the FP64 projection (away from texel edges)
    M = light.view_proj.astype(np.float64)
    Xh = np.c_[X.numpy(), np.ones(len(X))]
    clip = Xh @ M.T
    xs = (clip[:, 0] / clip[:, 3] + 1.0) * 0.5 * light.width
    far = np.abs(xs - np.round(xs)) > 1e-3
    np.testing.assert_array_equal((tex % light.width)[far], np.floor(xs[far]).astype(np.int64))


def test_shadow_depth_correction_is_the_log_depth_shift():
    """With half the bundle's strands drawn (beta = 1/2) the corrected
    visibility is exp(-sigma exp(log d - Delta)), Delta = -log beta; without
    the correction it does not depend on the LOD."""
    g, light, cam = _two_strand_shadow_setup()
    sig, bias = float(np.float32(100.0)), float(np.float32(0.001))
    d = 0.01 - bias
    on = synth.ShadowSpec(light=0, cam=light, sigma=100.0, bias_m=0.001, depth_correction=1)
    V, sg, _, _, _ = _shadow_vis_of_centre_keys(g, light, cam, on, lod_n=[1])
    delta = -math.log(0.5)
    np.testing.assert_allclose(V[sg == 1], math.exp(-sig * math.exp(math.log(d) - delta)), rtol=2e-4)
    V1, sg1, _, _, _ = _shadow_vis_of_centre_keys(g, light, cam, on, lod_n=[2])
    np.testing.assert_allclose(V1[sg1 == 1], math.exp(-sig * d), rtol=2e-4)
    off = synth.ShadowSpec(light=0, cam=light, sigma=100.0, bias_m=0.001, depth_correction=0)
    V0, sg0, _, _, _ = _shadow_vis_of_centre_keys(g, light, cam, off, lod_n=[1])
    np.testing.assert_allclose(V0[sg0 == 1], math.exp(-sig * d), rtol=2e-4)


def test_shadowed_resolve_zero_density_is_unshadowed_and_light_selective():
    """sigma = 0 leaves the image unchanged; a map on one light scales only
    that light's term (with the filter off, where colours pass through)."""
    sc = synth.tiny_scene(3, width=96, height=80, num_strands=500)
    sc.lights = synth.make_lights([[1.0, 1.0, 1.0], [-1.0, 0.5, 0.5]], [0.8, 0.4])
    lods = oracle.lods_for(sc)
    off = synth.FilterParams(enabled=0)
    vc, va, _ = oracle.raster(sc.grooms, sc.camera, lods)
    dec = oracle.resolve_decisions(sc.grooms, sc.camera, lods, off, vc, va)
    gts = [v64.GroomT(g, l[1], b, lod_n=l[0]) for g, l, b in zip(sc.grooms, lods, oracle.strand_bases(sc.grooms))]
    base, pix = v64.resolve(gts, sc.camera, sc.lights, off, vc, va, dec)
    lcam = synth.light_camera(sc.grooms, sc.lights.dirs[0], size=128, dist_m=0.6)
    for sigma in (0.0, 300.0):
        spec = synth.ShadowSpec(light=0, cam=lcam, sigma=sigma, bias_m=0.0005)
        maps = [(spec, oracle.shadow_map(sc.grooms, spec))]
        dec["shadow_texels"] = oracle.centre_shadow_texels(sc.grooms, sc.camera, lods, vc, maps)
        out, _ = v64.resolve(gts, sc.camera, sc.lights, off, vc, va, dec, shadows=maps)
        if sigma == 0.0:
            np.testing.assert_array_equal(out.numpy(), base.numpy())
        else:
            # light 1 alone (light 0 off) is unaffected by light 0's map
            l1 = synth.make_lights(sc.lights.dirs, np.array([[0, 0, 0], [0.4, 0.4, 0.4]], np.float32))
            a, _ = v64.resolve(gts, sc.camera, l1, off, vc, va, dec)
            b, _ = v64.resolve(gts, sc.camera, l1, off, vc, va, dec, shadows=maps)
            np.testing.assert_allclose(b.numpy(), a.numpy(), rtol=0, atol=1e-15)
            darker = (out[:, :3] < base[:, :3] - 1e-6).any(1).sum().item()
            assert darker > 50 and bool((out[:, :3] <= base[:, :3] + 1e-12).all())


# ---------------------------------------------------------------------------
# compressed G-buffer payload (Sec. 3.1.2)
# ---------------------------------------------------------------------------

def test_octahedral_codes_closed_forms_and_error_bound():
    """Cigolle et al.'s octahedral map: the poles and the equator's axis
    points have closed-form codes (0.5 -> 127.5 rounds to even 128), the
    lower hemisphere folds onto the corners, and every unit vector decodes
    within 1 degree of itself at 8 + 8 bits."""
    assert oracle.oct_encode([0, 0, 1]) == (128 << 8) | 128
    assert oracle.oct_encode([1, 0, 0]) == (255 << 8) | 128
    assert oracle.oct_encode([0, -1, 0]) == (128 << 8) | 0
    assert oracle.oct_encode([0, 0, -1]) == (255 << 8) | 255
    np.testing.assert_array_equal(oracle.oct_decode((255 << 8) | 255), np.float32([0, 0, -1]))
    np.testing.assert_allclose(oracle.oct_decode((128 << 8) | 128), [0.00392, 0.00392, 0.99998], atol=1e-4)
    rng = np.random.default_rng(0)
    v = rng.normal(size=(4000, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    worst = 0.0
    for t in v.astype(np.float32):
        code = oracle.oct_encode(t)
        d = oracle.oct_decode(code).astype(np.float64)
        d64 = v64.oct_decode64(np.array([code])).numpy()[0]
        worst = max(worst, math.degrees(math.acos(min(1.0, float(d64 @ t.astype(np.float64))))))
        assert abs(np.linalg.norm(d) - 1.0) < 1e-6 and np.abs(d - d64).max() < 1e-6
    assert worst < 1.0, worst


def test_unproject_inverts_the_projection():
    """The compressed decode's position: projecting it back gives the pixel
    centre and the view depth (FP32 C and FP64 value layer alike)."""
    sc = synth.tiny_scene(5, width=160, height=120)
    cam = sc.camera
    rng = np.random.default_rng(1)
    for _ in range(200):
        px, py = int(rng.integers(0, 160)), int(rng.integers(0, 120))
        w = float(np.float32(rng.uniform(0.2, 3.0)))
        X = oracle.unproject(cam, px + 0.5, py + 0.5, w)
        ok, _, _, wz = oracle.project_point(cam, X)          # wz = (w, z, xs, ys)
        assert ok and abs(wz[2] - (px + 0.5)) < 2e-3 and abs(wz[3] - (py + 0.5)) < 2e-3
        assert abs(wz[0] - w) < 2e-6 * w
    d24 = np.array([1000, 2 ** 23, 2 ** 24 - 1], np.int64)
    pix = np.array([0, 77, 160 * 120 - 1], np.int64)
    X = v64.cgb_position(cam, pix, d24).numpy()
    M = cam.view_proj.astype(np.float64)
    clip = np.c_[X, np.ones(3)] @ M.T
    near, far = float(np.float32(cam.near)), float(np.float32(cam.far))
    np.testing.assert_allclose(clip[:, 3], near + (d24 + 0.5) / 2 ** 24 * (far - near), rtol=1e-12)
    np.testing.assert_allclose((clip[:, 0] / clip[:, 3] + 1) * 0.5 * 160, pix % 160 + 0.5, atol=1e-9)
    np.testing.assert_allclose((1 - clip[:, 1] / clip[:, 3]) * 0.5 * 120, pix // 160 + 0.5, atol=1e-9)


def test_compressed_keys_against_the_segment_they_came_from():
    """Same coverage and depths as the id keys; each payload field, decoded,
    agrees with the FP64 quantity of the segment the id key names (bit
    layout, scales and meaning): root uv and w and AO codes within one step
    of the FP64 rounding, the tangent within 1 degree of the chord."""
    sc = synth.tiny_scene(31, width=120, height=96, num_strands=600, num_layers=5, length_m=0.06)
    g = sc.grooms[0]
    g.vert_ao = synth.baked_ao(g, seed=1)
    lods = oracle.lods_for(sc)
    vc, va, cnt = oracle.raster(sc.grooms, sc.camera, lods)
    cc, ca, cnt2 = oracle.raster(sc.grooms, sc.camera, lods, compressed=True)
    assert tuple(cnt) == tuple(cnt2)
    for idk, ck in ((vc, cc), (va, ca)):
        np.testing.assert_array_equal(idk == oracle.EMPTY, ck == oracle.EMPTY)
        np.testing.assert_array_equal(idk >> np.uint64(40), ck >> np.uint64(40))
    e, _, sg, seg = v64.key_fields(vc)
    ce, _, tcode, cu, cv, cw, cao = v64.cgb_fields(cc)
    idx = np.nonzero(~e)[0]
    # pixels whose minimum depth is held by one segment only carry its payload
    W = sc.camera.width
    C = lods[0][1][g.strand_face[sg[idx]]]
    num, den = oracle.msaa_decisions(sc.grooms, sc.camera, lods, 1, vc[None, :])
    t = np.clip(num[0][idx] / np.maximum(den[0][idx], 1), 0, 1)
    uv = g.vert_uv.astype(np.float64)
    f = g.faces[g.strand_face[sg[idx]]]
    b = g.strand_bary[sg[idx]].astype(np.float64)
    b0 = 1.0 - b[:, 0] - b[:, 1]
    u = b0 * uv[f[:, 0], 0] + b[:, 0] * uv[f[:, 1], 0] + b[:, 1] * uv[f[:, 2], 0]
    v = b0 * uv[f[:, 0], 1] + b[:, 0] * uv[f[:, 1], 1] + b[:, 1] * uv[f[:, 2], 1]
    w = (seg[idx] + t) / (C - 1)
    gt = v64.GroomT(g, lods[0][1], 0)
    ao = v64.pixel_ao(gt, sg[idx], seg[idx], num[0][idx], den[0][idx]).numpy()[:, 0]
    for name, code, ref, scale in (("u", cu[idx], u, 63), ("v", cv[idx], v, 63), ("w", cw[idx], w, 63),
                                   ("ao", cao[idx], ao, 62)):
        err = np.abs(code - np.clip(np.rint(ref * scale), 0, scale))
        assert err.max() <= 1 and (err == 0).mean() > 0.97, (name, err.max(), (err == 0).mean())
    # tangent: the chord of the keyed segment; where two segments of a strand
    # meet they have the same depth and the two payloads break the tie
    # differently, so the neighbouring chord is accepted there
    P = {}
    T = v64.oct_decode64(tcode[idx]).numpy()
    own, best = [], []
    for q, (s, j, c) in enumerate(zip(sg[idx], seg[idx], C)):
        if (s, c) not in P:
            P[(s, c)] = oracle.strand_control_points(g, int(s), int(c)).astype(np.float64)
        angs = []
        for jj in (j, j - 1, j + 1):
            if 0 <= jj < c - 1:
                ch = P[(s, c)][jj + 1] - P[(s, c)][jj]
                ch /= np.linalg.norm(ch)
                angs.append(math.degrees(math.acos(min(1.0, float(ch @ T[q])))))
        own.append(angs[0])
        best.append(min(angs))
    assert max(best) < 1.0 and (np.array(own) < 1.0).mean() > 0.95
    assert np.all(cao[~ce] <= 62)


def test_compressed_resolve_uniform_appearance_and_id_path_agreement():
    """A constant appearance table, ambient light and no AO: every shaded
    colour is ambient * albedo and the filter keeps it; with the synthetic
    lights the compressed image stays close to the id-path image (the
    payload's quantization, chord tangent and depth-bin position)."""
    sc = synth.tiny_scene(32, width=128, height=96, num_strands=800)
    lods = oracle.lods_for(sc)
    cc, ca, _ = oracle.raster(sc.grooms, sc.camera, lods, compressed=True)
    dec = oracle.resolve_decisions(sc.grooms, sc.camera, lods, sc.filt, cc, ca, compressed=True)
    table = np.zeros((64, 64, 4), np.float32)
    table[..., :3] = np.float32([0.3, 0.4, 0.5])
    table[..., 3] = 1.0
    amb = synth.make_lights([[0.0, 1.0, 0.0]], [0.0], ambient=0.5)
    rgba, pix = v64.resolve_cgb(sc.camera, amb, sc.filt, cc, ca, dec, table, 0.15, -0.05)
    on = rgba[:, 3] > 0
    exp = 0.5 * np.float32([0.3, 0.4, 0.5]).astype(np.float64)
    np.testing.assert_allclose(rgba[on, :3].numpy(), np.broadcast_to(exp, (int(on.sum()), 3)), rtol=1e-12)
    # against the id path with per-strand albedo replaced by the table's
    g = sc.grooms[0]
    tab = synth.appearance_table(3)
    vc, va, _ = oracle.raster(sc.grooms, sc.camera, lods)
    deci = oracle.resolve_decisions(sc.grooms, sc.camera, lods, sc.filt, vc, va)
    gt = v64.GroomT(g, lods[0][1], 0)
    ref, rpix = v64.resolve([gt], sc.camera, sc.lights, sc.filt, vc, va, deci)
    got, gpix = v64.resolve_cgb(sc.camera, sc.lights, sc.filt, cc, ca, dec, tab, g.roughness, g.tilt)
    np.testing.assert_array_equal(rpix, gpix)
    # the strip of a promoted pixel follows its (now chord) tangent: a few
    # pixels gain or lose their last contributor
    assert ((ref[:, 3].numpy() > 0) != (got[:, 3].numpy() > 0)).mean() < 0.02
    assert float((ref[:, 3] - got[:, 3]).abs().mean()) < 0.02


# ---------------------------------------------------------------------------
# alpha, promotion and the depth-mismatch blend in closed form (Sec. 3.3.2,
# Sec. 3.3.3, Eq. 7): hand-built keys along a straight horizontal strand
# (tests/_filter_cases.py), where the strip is the row and the weights are
# exp(-dx^2 / sigma_par^2)
# ---------------------------------------------------------------------------

def _line():
    import _filter_cases as fc
    sc = fc.line_scene()
    vc, va, lods = fc.raster(sc)
    return fc, sc, vc, va, lods


def test_alpha_straight_strand_through_centres_is_one():
    """A strand through the pixel centres hits the same pixels in both layers
    along its interior, so alpha = H_center / H_cons = 1 there; where the
    window reaches the conservative-only end pixels it is the exact count
    ratio (e.g. 6/7), never H_center / (H_center + H_cons)."""
    fc, sc, vc, va, lods = _line()
    x0, x1 = fc.span(vc)
    assert va[fc.px(x0 - 1)] != oracle.EMPTY and vc[fc.px(x0 - 1)] == oracle.EMPTY
    out, _ = fc.oracle_filter(sc, lods, vc, va)
    for x in range(x0 + 5, x1 - 4):
        assert out[fc.px(x), 3] == 1.0
    assert out[fc.px(x0), 3] == 6 / 7 and out[fc.px(x1), 3] == 6 / 7
    assert out[fc.px(x0 + 4), 3] == 10 / 11


def test_alpha_is_exact_count_ratio_over_the_strip():
    """Centre keys erased at two pixels of the row (conservative keys kept),
    conservative-only keys added on the next row: alpha at a centre pixel of
    the row is 9/11 (rows off the strip do not count), and every pixel of the
    row matches the closed form."""
    fc, sc, vc, va, lods = _line()
    x0, x1 = fc.span(vc)
    c = (x0 + x1) // 2
    vc = vc.copy()
    va = va.copy()
    for dx in (1, -3):
        vc[fc.px(c + dx)] = oracle.EMPTY
    for x in range(c - 4, c + 5):
        va[fc.px(x, fc.ROW + 1)] = va[fc.px(x)]
    out, dec = fc.oracle_filter(sc, lods, vc, va)
    assert dec["HcG"][fc.px(c)] == 9 and dec["HaG"][fc.px(c)] == 11
    assert out[fc.px(c), 3] == 9 / 11
    cols = fc.shaded_colours(sc, lods, vc, va)
    for x in range(x0 - 1, x1 + 2):
        np.testing.assert_allclose(out[fc.px(x)], fc.expected_row_pixel(x, vc, va, cols), rtol=1e-12, atol=1e-15)


def test_promoted_pixel_is_the_colour_free_average_of_its_contributors():
    """A promoted pixel (conservative key only) with exactly two contributing
    centre neighbours of different colours (dx = +1 relabelled to a second
    strand, dx = -2) and one neighbour beyond the depth-reject threshold
    (dx = +3): Eq. 7 with the colour term off gives
    (w(1) C_1 + w(2) C_2) / (w(1) + w(2)), w(d) = exp(-d^2 / sigma_par^2),
    and alpha = 3 / 11."""
    fc, sc, vc, va, lods = _line()
    x0, x1 = fc.span(vc)
    c = (x0 + x1) // 2
    rej, _ = oracle.depth_thresholds(sc.camera, sc.filt)
    vc = vc.copy()
    keep = {c + 1, c - 2, c + 3}
    for x in range(c - 5, c + 6):
        if x not in keep:
            vc[fc.px(x)] = oracle.EMPTY
    vc[fc.px(c + 1)] = fc.with_strand(vc[fc.px(c + 1)], 1)
    d = int(vc[fc.px(c + 3)]) >> 40
    vc[fc.px(c + 3)] = fc.with_depth(vc[fc.px(c + 3)], d + rej + 1)
    out, _ = fc.oracle_filter(sc, lods, vc, va)
    cols = fc.shaded_colours(sc, lods, vc, va)
    c1, c2 = cols[fc.px(c + 1)], cols[fc.px(c - 2)]
    assert np.abs(c1 - c2).max() > 0.1                       # distinct colours
    sp = 0.5 * 5
    w1, w2 = math.exp(-1 / sp ** 2), math.exp(-4 / sp ** 2)
    np.testing.assert_allclose(out[fc.px(c), :3], (w1 * c1 + w2 * c2) / (w1 + w2), rtol=1e-12)
    assert out[fc.px(c), 3] == 3 / 11
    # the neighbour just inside the threshold contributes
    vc[fc.px(c + 3)] = fc.with_depth(vc[fc.px(c + 3)], d + rej)
    out2, _ = fc.oracle_filter(sc, lods, vc, va)
    c3 = cols[fc.px(c + 3)]
    w3 = math.exp(-9 / sp ** 2)
    np.testing.assert_allclose(out2[fc.px(c), :3], (w1 * c1 + w2 * c2 + w3 * c3) / (w1 + w2 + w3), rtol=1e-12)


def test_depth_mismatch_blend_closed_form():
    """A centre pixel whose conservative key is 50 d24 units closer than its
    centre key (mismatch threshold 33): rgb = a' C' + (1 - a') C_G with alpha
    1, where C' is the colour-free reconstruction at the conservative depth,
    C_G the colour-weighted one at the centre depth, a' = 9/11; a pixel whose
    closer key has no contributor within the reject threshold outputs C_G; a
    difference below the threshold is no mismatch."""
    fc, sc, vc, va, lods = _line()
    x0, x1 = fc.span(vc)
    c = (x0 + x1) // 2
    rej, mis = oracle.depth_thresholds(sc.camera, sc.filt)
    assert mis == 33
    vc = vc.copy()
    va = va.copy()
    for dx in (-4, -1, 2):                       # a second colour in the window
        for buf in (vc, va):
            buf[fc.px(c + dx)] = fc.with_strand(buf[fc.px(c + dx)], 1)
    for dx in (3, -5):                           # two promoted pixels: a' = 9/11
        vc[fc.px(c + dx)] = oracle.EMPTY
    D = int(vc[fc.px(c)]) >> 40
    va[fc.px(c)] = fc.with_strand(fc.with_depth(va[fc.px(c)], D - 50), 2)
    far_px, near_px = c + 7, c - 7
    va[fc.px(far_px)] = fc.with_depth(va[fc.px(far_px)], D - 500)
    va[fc.px(near_px)] = fc.with_depth(va[fc.px(near_px)], D - (mis - 1))
    out, dec = fc.oracle_filter(sc, lods, vc, va)
    cols = fc.shaded_colours(sc, lods, vc, va)
    sp, sc_ = 0.5 * 5, float(np.float32(0.9))     # sigma_c is a binary32 parameter
    CP = cols[fc.px(c)]
    num_g, den_g, num_a, den_a = np.zeros(3), 0.0, np.zeros(3), 0.0
    for dx in range(-5, 6):
        q = fc.px(c + dx)
        if vc[q] == oracle.EMPTY:
            continue
        ws = math.exp(-dx * dx / sp ** 2)
        wc = math.exp(-float(((CP - cols[q]) ** 2).sum()) / sc_ ** 2)
        num_g += ws * wc * cols[q]
        den_g += ws * wc
        num_a += ws * cols[q]
        den_a += ws
    CG, CA = num_g / den_g, num_a / den_a
    assert np.abs(CG - CA).max() > 1e-3
    assert dec["HcA"][fc.px(c)] == 9 and dec["HaA"][fc.px(c)] == 11
    a = 9 / 11
    np.testing.assert_allclose(out[fc.px(c), :3], a * CA + (1 - a) * CG, rtol=1e-12)
    assert out[fc.px(c), 3] == 1.0
    # closer key with no centre neighbour near its depth: C_G, alpha 1
    e = fc.expected_row_pixel(far_px, vc, va, cols)
    np.testing.assert_allclose(out[fc.px(far_px)], e, rtol=1e-12)
    assert e[3] == 1.0
    # a difference of mis - 1 is no mismatch: C_G with alpha H_c / H_a
    e = fc.expected_row_pixel(near_px, vc, va, cols)
    np.testing.assert_allclose(out[fc.px(near_px)], e, rtol=1e-12)
    assert out[fc.px(near_px), 3] == e[3] == dec["HcG"][fc.px(near_px)] / dec["HaG"][fc.px(near_px)]
    for x in range(x0 - 1, x1 + 2):
        np.testing.assert_allclose(out[fc.px(x)], fc.expected_row_pixel(x, vc, va, cols), rtol=1e-12, atol=1e-15)


def test_strand_roots_uniform_over_the_triangle_chi_square():
    """Roots (Sec. 2: strands placed by barycentric coordinates on the base
    mesh) are uniform over each triangle: the sqrt(r1) map gives density 2
    over {b1, b2 >= 0, b1 + b2 <= 1}.  Counts over the 64 congruent
    sub-triangles of a three-level midpoint subdivision pass a chi-square
    test, each barycentric coordinate is Beta(1, 2) distributed, and strands
    are sorted by face (bundle-contiguous) with every coordinate in range."""
    from scipy import stats
    g = synth.make_groom(11, 8, 1, 4, 0.05, 200_000, 8)
    b1 = g.strand_bary[:, 0].astype(np.float64)
    b2 = g.strand_bary[:, 1].astype(np.float64)
    b0 = 1.0 - b1 - b2
    assert np.all(np.diff(g.strand_face.astype(np.int64)) >= 0)
    assert np.all((b1 >= 0) & (b2 >= 0) & (b0 >= -1e-6))
    # sub-triangle of a point at level 3: at each level the point lies in the
    # corner triangle of vertex i when coordinate i exceeds 1/2 (new
    # coordinates 2c with c_i -> 2 c_i - 1), else in the middle one, whose
    # vertices are the edge midpoints (new coordinates 1 - 2c)
    cell = np.zeros(b1.size, np.int64)
    c = np.stack([b0, b1, b2], 1)
    for _ in range(3):
        big = c > 0.5
        corner = np.where(big.any(1), big.argmax(1), 3)
        nxt = 1.0 - 2.0 * c
        rows = np.nonzero(corner < 3)[0]
        nxt[rows] = 2.0 * c[rows]
        nxt[rows, corner[rows]] -= 1.0
        c = nxt
        cell = cell * 4 + corner
    counts = np.bincount(cell, minlength=64)
    assert counts.size == 64
    chi2, p = stats.chisquare(counts)
    assert p > 1e-3, (chi2, p)
    for x in (b0, b1, b2):
        assert stats.kstest(x, stats.beta(1, 2).cdf).pvalue > 1e-3


def test_resolved_frame_alpha_in_unit_interval_and_zero_outside_coverage():
    """Over a whole oracle frame: alpha in [0, 1], colour finite and
    non-negative, exactly zero wherever the conservative layer is empty, and
    positive on every centre pixel (Sec. 3.3.3: alpha is a ratio of strip
    counts H_center / H_cons with H_cons >= H_center)."""
    sc = synth.tiny_scene(31, width=96, height=72, num_strands=400)
    lods = oracle.lods_for(sc)
    vc, va, _ = oracle.raster(sc.grooms, sc.camera, lods)
    dec = oracle.resolve_decisions(sc.grooms, sc.camera, lods, sc.filt, vc, va)
    gts = [v64.GroomT(g, l[1], b) for g, l, b in zip(sc.grooms, lods, oracle.strand_bases(sc.grooms))]
    rgba, pix = v64.resolve(gts, sc.camera, sc.lights, sc.filt, vc, va, dec)
    img = v64.full_image(rgba, pix, sc.camera.width, sc.camera.height).numpy().reshape(-1, 4)
    covered = (va & oracle.PAYLOAD_MASK) != oracle.PAYLOAD_MASK
    assert covered.sum() > 100
    assert np.all(np.isfinite(img))
    assert np.all((img[:, 3] >= 0.0) & (img[:, 3] <= 1.0))
    assert np.all(img[:, :3] >= 0.0)
    assert np.all(img[~covered] == 0.0)
    # a centre pixel counts itself in its strip (H_center >= 1); a promoted
    # pixel without a contributing neighbour is (0, 0, 0, 0)
    centre = (vc & oracle.PAYLOAD_MASK) != oracle.PAYLOAD_MASK
    assert np.all(img[centre, 3] > 0.0)
