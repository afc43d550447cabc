"""Adjoint kernel vs the FP64 oracle's autograd gradient (visibility held
fixed), through hm_shade_backward / the torch.autograd.Function.

Loss: L2 norm of the premultiplied RGB against a target rendered by the
oracle from the same hair mesh with every layer vertex perturbed by
N(0, 2 mm).  Criterion: norm-wise relative error <= 1e-2, and per entry
<= 1e-2 relative for entries above 1e-3 of the largest.
"""
import numpy as np
import pytest
import torch

import oracle
from oracle import value64 as v64
from paper_2607_04230_b300 import synth

from _parity import assert_keys_equal, oracle_keys

pytestmark = pytest.mark.gpu


def _oracle_image(scene, layer_verts):
    g = scene.grooms[0]
    gp = synth.Groom(layer_verts=layer_verts, faces=g.faces, strand_face=g.strand_face, strand_bary=g.strand_bary,
                     strand_albedo=g.strand_albedo, bundle_delta=g.bundle_delta,
                     segments_per_strand=g.segments_per_strand, vert_ao=g.vert_ao)
    sp = synth.Scene([gp], scene.camera, scene.lights, scene.filt, scene.lod)
    lods, vc, va, _ = oracle_keys(sp)
    dec = oracle.resolve_decisions(sp.grooms, sp.camera, lods, sp.filt, vc, va)
    rgba, pix = v64.resolve([v64.GroomT(gp, lods[0][1], 0)], sp.camera, sp.lights, sp.filt, vc, va, dec)
    img = v64.full_image(rgba, pix, sp.camera.width, sp.camera.height).reshape(-1, 4)
    return (img[:, :3] * img[:, 3:4]).numpy()


def _compare(g_gpu, g_ref, what):
    g_gpu = g_gpu.reshape(-1).astype(np.float64)
    g_ref = g_ref.reshape(-1)
    nrm = np.linalg.norm(g_gpu - g_ref) / np.linalg.norm(g_ref)
    assert nrm <= 1e-2, f"{what}: norm-wise relative error {nrm:.3e}"
    big = np.abs(g_ref) > 1e-3 * np.abs(g_ref).max()
    rel = np.abs(g_gpu[big] - g_ref[big]) / np.abs(g_ref[big])
    assert rel.max() <= 1e-2, f"{what}: worst per-entry relative error {rel.max():.3e} over {big.sum()} entries"
    return nrm, rel.max()


def _grad_case(scene, shadow=None):
    """shadow: optional synth.ShadowSpec; its map (rendered once from the
    unperturbed groom) is held fixed on both sides."""
    from paper_2607_04230_b300 import autograd, hm
    g = scene.grooms[0]
    W, H = scene.camera.width, scene.camera.height
    target = _oracle_image(scene, synth.perturbed_layer_verts(g))
    # GPU: forward + hand-written adjoint
    handle = hm.upload_scene(scene)[0]
    frame = hm.Frame(W, H)
    shadows = None
    if shadow is not None:
        npx = shadow.cam.width * shadow.cam.height
        mc = torch.empty(npx, dtype=torch.int64, device="cuda")
        ma = torch.empty(npx, dtype=torch.int64, device="cuda")
        hm.render_shadow_map([handle], shadow.cam, mc, ma)
        shadows = [(shadow, ma)]
    lv = torch.from_numpy(g.layer_verts).cuda().requires_grad_(True)
    alb = torch.from_numpy(g.strand_albedo).cuda().requires_grad_(True)
    rgba = autograd.render(handle, scene, frame, lv, alb, shadows=shadows)
    t = torch.from_numpy(target).float().cuda()
    loss = torch.sqrt(((rgba.reshape(-1, 4)[:, :3] * rgba.reshape(-1, 4)[:, 3:4] - t) ** 2).sum())
    loss.backward()
    torch.cuda.synchronize()
    hm.get_device_status()
    # oracle: FP64 forward with the same (bit-exact) visibility, autograd
    lods, vc, va, _ = oracle_keys(scene)
    gk, ak = frame.keys_numpy()
    assert_keys_equal(gk, vc, "centre layer")
    assert_keys_equal(ak, va, "conservative layer")
    dec = oracle.resolve_decisions(scene.grooms, scene.camera, lods, scene.filt, vc, va)
    lv64 = torch.from_numpy(g.layer_verts.astype(np.float64)).requires_grad_(True)
    alb64 = torch.from_numpy(g.strand_albedo.astype(np.float64)).requires_grad_(True)
    gt = v64.GroomT(g, lods[0][1], 0, layer_verts=lv64, albedo=alb64, lod_n=lods[0][0])
    maps = None
    if shadow is not None:
        maps = [(shadow, oracle.shadow_map(scene.grooms, shadow))]
        assert_keys_equal(shadows[0][1].cpu().numpy().view(np.uint64), maps[0][1], "shadow map")
        dec["shadow_texels"] = oracle.centre_shadow_texels(scene.grooms, scene.camera, lods, vc, maps)
    r64, pix = v64.resolve([gt], scene.camera, scene.lights, scene.filt, vc, va, dec, shadows=maps)
    img = torch.zeros((W * H, 3), dtype=torch.float64).index_put((torch.from_numpy(pix),), r64[:, :3] * r64[:, 3:4])
    l64 = torch.sqrt(((img - torch.from_numpy(target)) ** 2).sum())
    l64.backward()
    assert abs(loss.item() - l64.item()) <= 1e-4 * l64.item()
    out = {}
    out["layer_verts"] = _compare(lv.grad.cpu().numpy(), lv64.grad.numpy(), "layer-vertex gradient")
    out["albedo"] = _compare(alb.grad.cpu().numpy(), alb64.grad.numpy(), "albedo gradient")
    return out


def test_gradient_small_scene():
    sc = synth.tiny_scene(21, width=96, height=80, num_strands=400, dist_m=0.3)
    _grad_case(sc)


def test_gradient_mismatch_and_promoted_heavy():
    # sparse strands far away: mostly promoted pixels and depth mismatches
    sc = synth.tiny_scene(22, width=128, height=96, num_strands=1500, dist_m=0.9, jitter_m=0.006)
    _grad_case(sc)


def test_gradient_512_workload():
    """256 scalp triangles, 6 layers, 20k strands x 12 segments, 512x512."""
    out = _grad_case(synth.scene_grad_512())
    print(out)


def test_gradient_with_baked_ao():
    sc = synth.tiny_scene(23, width=96, height=80, num_strands=500, dist_m=0.3, num_layers=5)
    sc.grooms[0].vert_ao = synth.baked_ao(sc.grooms[0], seed=4)
    sc.lights.ambient = float(np.float32(0.4))
    _grad_case(sc)


def test_gradient_with_shadow_map():
    """A shadow map on light 0 (held fixed): gradients also flow through the
    receiver's depth in the light's view."""
    sc = synth.tiny_scene(24, width=96, height=80, num_strands=600, dist_m=0.3, num_layers=5)
    sc.lod = synth.LodParams(1, 3.0)
    lcam = synth.light_camera(sc.grooms, sc.lights.dirs[0], size=160, dist_m=0.5)
    _grad_case(sc, synth.ShadowSpec(light=0, cam=lcam, sigma=200.0, bias_m=0.0005, depth_correction=1))


def test_gradient_large_layer_vertex_set():
    """2,048 scalp triangles x 4 layers: 13,068 layer-vertex gradient floats,
    more than the geometry pass keeps in shared memory per CTA (11,264), so
    the gradients accumulate straight into global memory."""
    sc = synth.tiny_scene(25, width=96, height=80, num_strands=600, dist_m=0.3, k=8, n=4, num_layers=4)
    assert sc.grooms[0].layer_verts.size > 11 * 1024
    _grad_case(sc)


def test_gradient_vs_central_differences():
    """The GPU layer-vertex and albedo gradients against central differences
    (step 1e-5 m, and 1e-5 in albedo) of the FP64 oracle's forward with the
    GPU's (bit-exact) visibility held fixed, on the largest entries and a
    few random ones."""
    from paper_2607_04230_b300 import autograd, hm
    sc = synth.tiny_scene(26, width=80, height=64, num_strands=300, dist_m=0.3)
    g = sc.grooms[0]
    W, H = sc.camera.width, sc.camera.height
    rng = np.random.default_rng(3)
    target = rng.random((W * H, 3)) * 0.2
    handle = hm.upload_scene(sc)[0]
    frame = hm.Frame(W, H)
    lv = torch.from_numpy(g.layer_verts).cuda().requires_grad_(True)
    alb = torch.from_numpy(g.strand_albedo).cuda().requires_grad_(True)
    rgba = autograd.render(handle, sc, frame, lv, alb)
    t = torch.from_numpy(target).float().cuda()
    loss = torch.sqrt(((rgba.reshape(-1, 4)[:, :3] * rgba.reshape(-1, 4)[:, 3:4] - t) ** 2).sum())
    loss.backward()
    glv, galb = lv.grad.cpu().numpy().astype(np.float64), alb.grad.cpu().numpy().astype(np.float64)
    lods, vc, va, _ = oracle_keys(sc)
    gk, ak = frame.keys_numpy()
    assert_keys_equal(gk, vc, "centre layer")
    assert_keys_equal(ak, va, "conservative layer")
    dec = oracle.resolve_decisions(sc.grooms, sc.camera, lods, sc.filt, vc, va)
    tgt = torch.from_numpy(target)

    def f(lv64, alb64):
        gt = v64.GroomT(g, lods[0][1], 0, layer_verts=lv64, albedo=alb64, lod_n=lods[0][0])
        r, pix = v64.resolve([gt], sc.camera, sc.lights, sc.filt, vc, va, dec)
        img = torch.zeros((W * H, 3), dtype=torch.float64).index_put((torch.from_numpy(pix),), r[:, :3] * r[:, 3:4])
        return torch.sqrt(((img - tgt) ** 2).sum()).item()

    lv0 = torch.from_numpy(g.layer_verts.astype(np.float64))
    alb0 = torch.from_numpy(g.strand_albedo.astype(np.float64))
    h = 1e-5
    scale = np.abs(glv).max()
    for idx in list(np.argsort(-np.abs(glv).ravel())[:8]) + list(rng.integers(0, glv.size, 4)):
        e = torch.zeros(glv.size, dtype=torch.float64)
        e[idx] = h
        e = e.reshape(lv0.shape)
        fd = (f(lv0 + e, alb0) - f(lv0 - e, alb0)) / (2 * h)
        assert abs(fd - glv.ravel()[idx]) <= 1e-2 * max(abs(fd), 1e-3 * scale), (idx, fd, glv.ravel()[idx])
    for idx in np.argsort(-np.abs(galb).ravel())[:4]:
        e = torch.zeros(galb.size, dtype=torch.float64)
        e[idx] = h
        e = e.reshape(alb0.shape)
        fd = (f(lv0, alb0 + e) - f(lv0, alb0 - e)) / (2 * h)
        assert abs(fd - galb.ravel()[idx]) <= 1e-2 * abs(fd), (idx, fd, galb.ravel()[idx])


def test_two_forwards_then_backward():
    """Two differentiable renders of the same groom (different layer
    vertices) before one backward: each backward sees its own forward's
    state, so the gradients equal those of two separate forward/backward
    passes."""
    from paper_2607_04230_b300 import autograd, hm
    sc = synth.tiny_scene(27, width=96, height=80, num_strands=400, dist_m=0.3)
    g = sc.grooms[0]
    W, H = sc.camera.width, sc.camera.height
    handle = hm.upload_scene(sc)[0]
    lv_a = torch.from_numpy(g.layer_verts).cuda()
    lv_b = torch.from_numpy(synth.perturbed_layer_verts(g, sigma_m=0.001, seed=8)).cuda()
    alb = torch.from_numpy(g.strand_albedo).cuda()
    t = torch.rand((W * H, 3), device="cuda", generator=torch.Generator(device="cuda").manual_seed(1)) * 0.2

    def loss_of(rgba):
        r = rgba.reshape(-1, 4)
        return torch.sqrt(((r[:, :3] * r[:, 3:4] - t) ** 2).sum())

    def grads(lv):
        x = lv.clone().requires_grad_(True)
        a = alb.clone().requires_grad_(True)
        loss_of(autograd.render(handle, sc, hm.Frame(W, H), x, a)).backward()
        return x.grad.clone(), a.grad.clone()

    ga, gb = grads(lv_a), grads(lv_b)
    xa, xb = lv_a.clone().requires_grad_(True), lv_b.clone().requires_grad_(True)
    aa, ab = alb.clone().requires_grad_(True), alb.clone().requires_grad_(True)
    la = loss_of(autograd.render(handle, sc, hm.Frame(W, H), xa, aa))
    lb = loss_of(autograd.render(handle, sc, hm.Frame(W, H), xb, ab))
    (la + lb).backward()
    torch.cuda.synchronize()
    for got, ref in ((xa.grad, ga[0]), (aa.grad, ga[1]), (xb.grad, gb[0]), (ab.grad, gb[1])):
        assert torch.allclose(got, ref, rtol=1e-4, atol=1e-7 * float(ref.abs().max())), \
            float((got - ref).abs().max())


def test_unaligned_upstream_gradient():
    """An upstream gradient that is a contiguous view at an odd float offset
    (not 16-byte aligned) gives the same layer-vertex and albedo gradients as
    the same values in an aligned tensor."""
    from paper_2607_04230_b300 import autograd, hm
    sc = synth.tiny_scene(28, width=64, height=48, num_strands=300, dist_m=0.3)
    g = sc.grooms[0]
    W, H = sc.camera.width, sc.camera.height
    handle = hm.upload_scene(sc)[0]
    lv = torch.from_numpy(g.layer_verts).cuda()
    alb = torch.from_numpy(g.strand_albedo).cuda()
    n = H * W * 4
    big = torch.randn(n + 1, device="cuda", generator=torch.Generator(device="cuda").manual_seed(3))
    unaligned = big[1:].view(H, W, 4)
    assert unaligned.is_contiguous() and unaligned.data_ptr() % 16 != 0
    out = []
    for grad in (unaligned, unaligned.clone()):
        x, a = lv.clone().requires_grad_(True), alb.clone().requires_grad_(True)
        rgba = autograd.render(handle, sc, hm.Frame(W, H), x, a)
        torch.autograd.backward(rgba, grad_tensors=grad)
        out.append((x.grad.clone(), a.grad.clone()))
    torch.cuda.synchronize()
    assert float(out[0][0].abs().max()) > 0
    for got, ref in zip(out[0], out[1]):     # float atomics: equal up to summation order
        assert torch.allclose(got, ref, rtol=1e-5, atol=1e-6 * float(ref.abs().max()))
