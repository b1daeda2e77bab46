"""Device-resident shading pipeline over the C ABI.

One object holds a scene on the GPU (mesh, BVH, probe tables, textures,
cameras, G-buffer, outputs and gradients) and runs the hot path of one
optimisation step as the paper describes it (Sec. 3, Fig. "System"):
probe distribution -> BVH over this iteration's mesh -> primary visibility
(G-buffer) -> Monte Carlo direct illumination forward -> denoiser on c_d and
c_s (Sec. 4.2) -> denoiser input gradient -> shading adjoint.  Every step is
a libmcdi kernel launch on the current torch stream.
"""
from __future__ import annotations

import numpy as np
import torch

from . import mcdi
from .scenes import Scene


class ShadingPipeline:
    def __init__(self, scene: Scene, device="cuda", tau: float = 0.0, ray_eps: float = 1e-4,
                 decorrelate_bwd: bool = False, keep_mask: bool = True, wavefront: bool = True,
                 denoiser_params=None, denoiser_precision=0):
        mcdi.load()
        self.scene = scene
        self.device = torch.device(device)
        dev = self.device
        t = lambda a, dt=torch.float32: torch.from_numpy(np.ascontiguousarray(a)).to(dev, dt)
        self.verts = t(scene.verts)
        self.vnrm = t(scene.vnrm)
        self.tris = t(scene.tris, torch.int32)
        self.env = t(scene.env)
        self.tex_kd = t(scene.tex_kd)
        self.tex_korm = t(scene.tex_korm)
        self.cams = t(scene.cams)
        self.uvmap = [float(x) for x in scene.uvmap]
        self.N, self.H, self.W = scene.n_views, scene.height, scene.width
        self.params = mcdi.make_params(scene.n_light, scene.n_cos, scene.n_ggx, scene.seed, tau, ray_eps,
                                       decorrelate_bwd)
        self.spp = scene.spp
        self.bvh = mcdi.Bvh.allocate(scene.tris.shape[0], dev)
        self.probe = mcdi.Probe.allocate(self.env)
        self.gb = mcdi.GBuffer.allocate(self.N, self.H, self.W, dev)
        shape = (self.N, self.H, self.W, 4)
        # c_d and c_s share one buffer so that the denoiser sees them as a batch of 2N images
        self.terms = torch.zeros((2 * self.N, self.H, self.W, 4), device=dev)
        self.c_d, self.c_s = self.terms[: self.N], self.terms[self.N:]
        self.kd_out = torch.zeros(shape, device=dev)
        self.denoiser = None
        if denoiser_params is not None:
            self.denoiser = mcdi.Denoiser(denoiser_params, 2 * self.N, self.H, self.W, device=dev,
                                          precision=denoiser_precision)
            self.denoised = torch.zeros_like(self.terms)
            self.g_terms = torch.zeros_like(self.terms)
        self.mask = (torch.zeros(self.N, self.H, self.W, (self.spp + 31) // 32, dtype=torch.int32, device=dev)
                     if keep_mask else None)
        self.g_kd, self.g_korm, self.g_nrm = (torch.zeros(shape, device=dev) for _ in range(3))
        self.g_env = torch.zeros_like(self.env)
        self.workspace = None
        if wavefront:
            nbytes = mcdi.shade_workspace_size(self.N, self.H, self.W, self.params)
            self.workspace = torch.empty((nbytes + 255) // 256 * 256, dtype=torch.uint8, device=dev)

    # ---- the steps
    def build_probe(self, stream=None):
        self.probe.build(stream)

    def build_bvh(self, stream=None):
        self.bvh.build(self.verts, self.tris, stream)

    def primary(self, stream=None):
        mcdi.primary_cast(self.bvh, self.verts, self.vnrm, self.tris, self.cams, self.H, self.W, self.tex_kd,
                          self.tex_korm, self.uvmap, self.gb, stream)

    def forward(self, stream=None):
        mcdi.shade_mc_fwd(self.bvh, self.probe, self.gb, self.cams, self.params, self.c_d, self.kd_out, self.c_s,
                          self.mask, self.workspace, stream)

    def backward(self, g_cd, g_kdout, g_cs, stream=None, zero_env_grad=True):
        if zero_env_grad:
            self.g_env.zero_()
        mcdi.shade_mc_bwd(self.bvh, self.probe, self.gb, self.cams, self.params, g_cd, g_kdout, g_cs, self.mask,
                          self.g_kd, self.g_korm, self.g_nrm, self.g_env, stream)

    def denoise(self, stream=None):
        """D(c_d), D(c_s) with k_d,out and the normal as guides (Sec. 4.2)."""
        self.denoiser.forward(self.terms, self.kd_out, self.gb.nrm, self.denoised, stream)

    def denoise_backward(self, g_denoised, stream=None):
        self.denoiser.backward(g_denoised, self.g_terms, stream)

    def step(self, g_cd, g_kdout, g_cs, stream=None):
        """One pass of the hot path: tables, BVH, G-buffer, forward, adjoint.
        With a denoiser, g_cd / g_cs are gradients of the denoised terms and pass
        through the denoiser's input gradient first."""
        self.build_probe(stream)
        self.build_bvh(stream)
        self.primary(stream)
        self.forward(stream)
        if self.denoiser is not None:
            self.denoise(stream)
            g = torch.cat([g_cd, g_cs], 0) if g_cd.shape[0] == self.N else g_cd
            self.denoise_backward(g, stream)
            g_cd, g_cs = self.g_terms[: self.N], self.g_terms[self.N:]
        self.backward(g_cd, g_kdout, g_cs, stream)

    def capture(self, g_cd, g_kdout, g_cs):
        """Capture one `step` into a CUDA graph (its launches, memsets and the
        host-encoded tensor maps are baked in with these buffers); `replay()`
        then reruns the whole step with one launch from the host.  A first step
        runs uncaptured on a side stream so that one-time set-up (kernel
        attributes, device queries) stays outside the graph."""
        dev = self.device
        side = torch.cuda.Stream(dev)
        side.wait_stream(torch.cuda.current_stream(dev))
        with torch.cuda.stream(side):
            self.step(g_cd, g_kdout, g_cs)
        torch.cuda.current_stream(dev).wait_stream(side)
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            self.step(g_cd, g_kdout, g_cs)
        return self.graph

    def replay(self):
        self.graph.replay()

    def covered_pixels(self) -> int:
        return int((self.gb.pos[..., 3] > 0).sum().item())
