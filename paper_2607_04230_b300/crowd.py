"""Batched crowd rendering (many grooms, one frame).

The batched path renders every groom of the scene with one
hm_render_visibility call (one LOD pre-pass over all bundles of all grooms,
one persistent rasterizer launch over the joint work list) and one
hm_resolve_shade call, captured once into a CUDA graph and replayed per
frame.  The per-character path is the paper's sequential scheme (Sec. 4,
"Multiple Grooms"): one render call per groom into the shared visibility
buffers, depth preserved between grooms, then one resolve.
"""
from __future__ import annotations

from . import hm


class Crowd:
    def __init__(self, scene, stream=None, key_layout: int = hm.KEYS_ROW_MAJOR):
        import torch
        self.scene = scene
        self.grooms = hm.upload_scene(scene, stream=stream)
        # a crowd covers a small part of the frame: the resolve lists its
        # occupied tiles first
        self.frame = hm.Frame(scene.camera.width, scene.camera.height, tile_list=True, key_layout=key_layout)
        self.graph = None
        self.graph_pc = None
        self._torch = torch

    # -- one call over all grooms ------------------------------------------
    def render_batched(self):
        hm.render(self.grooms, self.scene, self.frame)

    def capture(self):
        """Capture render_batched into a CUDA graph (after a warm-up frame, so
        every lazily initialised launch attribute is set outside capture)."""
        torch = self._torch
        self.render_batched()
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            self.render_batched()
        self.graph = g
        return g

    def replay(self):
        self.graph.replay()

    def capture_per_character(self):
        """The per-character path (one render call per groom, then one
        resolve) captured into a CUDA graph of its own, so the two paths are
        compared without host launch overhead on either side."""
        torch = self._torch
        self.render_per_character()
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            self.render_per_character()
        self.graph_pc = g
        return g

    def replay_per_character(self):
        self.graph_pc.replay()

    # -- one call per groom ------------------------------------------------
    def render_per_character(self):
        sc, fr = self.scene, self.frame
        cam = fr.camera(sc.camera)
        for i in range(len(self.grooms)):
            hm.render_visibility_range(self.grooms, i, 1, cam, fr.vis_center, fr.vis_cons, clear=(i == 0))
        hm.resolve_shade(self.grooms, cam, sc.lights, sc.filt, fr.vis_center, fr.vis_cons, fr.rgba,
                         tile_scratch=fr.tile_scratch)
