"""Shared helpers of the parity tests: run one frame on the GPU through the
C ABI and the same frame through the CPU oracle."""
import numpy as np

import oracle
from oracle import value64 as v64
from paper_2607_04230_b300 import synth

RGBA_TOL = 1e-4          # max abs error of linear RGB(A) vs the FP64 oracle


def gpu_frame(scene, grooms=None, tile_list=False):
    """tile_list: resolve with the tile-list scratch (the two-pass resolve the
    benchmark times) instead of one CTA per tile."""
    import torch
    from paper_2607_04230_b300 import hm
    grooms = grooms or hm.upload_scene(scene)
    frame = hm.Frame(scene.camera.width, scene.camera.height, tile_list=tile_list)
    hm.render(grooms, scene, frame)
    torch.cuda.synchronize()
    hm.get_device_status()
    vc, va = frame.keys_numpy()
    return dict(grooms=grooms, vis_c=vc, vis_a=va, rgba=frame.rgba.cpu().numpy().astype(np.float64),
                stats=hm.stats_dict(frame.stats), lods=[g.get_lod() for g in grooms], frame=frame)


def oracle_keys(scene, nthreads=0):
    lods = oracle.lods_for(scene)
    vc, va, counts = oracle.raster(scene.grooms, scene.camera, lods, nthreads=nthreads)
    return lods, vc, va, counts


def oracle_rgba(scene, lods, vc, va, pixels=None):
    """FP64 oracle RGBA at `pixels` (flat indices; all covered pixels when
    None).  Returns (rgba [N][4], pixels)."""
    dec = oracle.resolve_decisions(scene.grooms, scene.camera, lods, scene.filt, vc, va)
    gts = [v64.GroomT(g, l[1], b) for g, l, b in zip(scene.grooms, lods, oracle.strand_bases(scene.grooms))]
    rgba, pix = v64.resolve(gts, scene.camera, scene.lights, scene.filt, vc, va, dec, pixels=pixels)
    return rgba.numpy(), pix


def assert_keys_equal(got, ref, what):
    if not np.array_equal(got, ref):
        bad = np.nonzero(got != ref)[0]
        raise AssertionError(f"{what}: {bad.size} keys differ, first at {bad[:5]}: "
                             f"gpu {got[bad[:5]]} oracle {ref[bad[:5]]}")


def assert_rgba_close(gpu_rgba, ref_rgba, pixels, tol=RGBA_TOL):
    g = gpu_rgba.reshape(-1, 4)[pixels]
    if len(pixels) == 0:
        return 0.0
    err = np.abs(g - ref_rgba)
    i = np.unravel_index(np.argmax(err), err.shape)
    assert err.max() <= tol, f"max |rgba - oracle| = {err.max():.3e} at pixel {pixels[i[0]]} channel {i[1]}: " \
                             f"gpu {g[i[0]]} oracle {ref_rgba[i[0]]}"
    return float(err.max())


def special_pixels(scene, vc, va):
    """Every pixel whose output is not a plain centre-referenced
    reconstruction: promoted pixels (a conservative key, no centre key) and
    depth mismatches (Sec. 3.3.2), in ascending order."""
    e = oracle.PAYLOAD_MASK
    eG, eA = (vc & e) == e, (va & e) == e
    dG = (vc >> np.uint64(40)).astype(np.int64)
    dA = (va >> np.uint64(40)).astype(np.int64)
    _, mis = oracle.depth_thresholds(scene.camera, scene.filt)
    return np.nonzero(~eA & (eG | (dA + mis <= dG)))[0]


def check_full(scene, sample=None, rng_seed=0, all_special=False, tile_list=False):
    """Keys bit-exact over the whole frame, LOD exact, RGBA within tolerance
    on every covered pixel (or a seeded sample of `sample` covered pixels,
    plus, with all_special, every promoted and depth-mismatch pixel), and
    every uncovered pixel exactly zero."""
    out = gpu_frame(scene, tile_list=tile_list)
    lods, vc, va, counts = oracle_keys(scene)
    for (n, c), (gn, gc) in zip(lods, out["lods"]):
        assert np.array_equal(n, gn), "N_LOD differs"
        assert np.array_equal(c, gc), "C differs"
    assert_keys_equal(out["vis_c"], vc, "centre layer")
    assert_keys_equal(out["vis_a"], va, "conservative layer")
    assert out["stats"]["covered_cons"] == counts[1] and out["stats"]["covered_center"] == counts[0], \
        (out["stats"], counts)
    covered = np.nonzero((va & oracle.PAYLOAD_MASK) != oracle.PAYLOAD_MASK)[0]
    pix = covered
    if sample is not None and covered.size > sample:
        rng = np.random.default_rng(rng_seed)
        pix = np.sort(rng.choice(covered, size=sample, replace=False))
        if all_special:
            pix = np.union1d(pix, special_pixels(scene, vc, va))
    ref, pix = oracle_rgba(scene, lods, vc, va, pixels=pix)
    err = assert_rgba_close(out["rgba"], ref, pix)
    # every pixel outside the conservative layer is exactly zero
    empty = np.ones(va.size, bool)
    empty[covered] = False
    assert np.all(out["rgba"].reshape(-1, 4)[empty] == 0.0)
    return out, err
