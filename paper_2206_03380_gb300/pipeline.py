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


def pixel_spans(P: int, fractions) -> list:
    """Consecutive (first, count) spans of P pixels: each fraction of P rounded to a multiple of 32 pixels (one
    adjoint block) and cut at what is left, the last entry (None) taking the rest; together they cover
    [0, P) once, in order.  The adjoint runs span by span so that each span's gradients can be read back while
    the later ones run."""
    spans, first = [], 0
    for frac in fractions:
        count = P - first if frac is None else min(P - first, int(round(P * frac / 32.0)) * 32)
        spans.append((first, count))
        first += count
    return spans


class ShadingPipeline:
    def __init__(self, scene: Scene, device="cuda", tau: float = 1.0, ray_eps: float = 1e-4,
                 decorrelate_bwd: bool = False, keep_mask: bool = True, wavefront: bool = True,
                 denoiser_params=None, denoiser_precision=0, bilateral_sigma=None, raster: bool = True):
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
        self.bilateral_sigma = bilateral_sigma
        if bilateral_sigma is not None:  # the cross-bilateral denoiser instead of the U-Net
            assert denoiser_params is None
            self.denoiser = "bilateral"
            self.denoised = torch.zeros_like(self.terms)
            self.g_terms = torch.zeros_like(self.terms)
            self.bl_wsum = torch.zeros((self.N, self.H, self.W), device=dev)
        if denoiser_params is not None:
            self.denoiser = mcdi.Denoiser(denoiser_params, 2 * self.N, self.H, self.W, device=dev,
                                          precision=denoiser_precision)
            self.denoised = torch.zeros_like(self.terms)
            self.g_terms = torch.zeros_like(self.terms)
        self.mask = (torch.zeros(self.N, self.H, self.W, (self.spp + 31) // 32, dtype=torch.int32, device=dev)
                     if keep_mask else None)
        self.g_kd, self.g_korm, self.g_nrm = (torch.zeros(shape, device=dev) for _ in range(3))
        self.g_env = torch.zeros_like(self.env)
        self._loss = None
        self.workspace = None
        self._fork = None  # side stream of tables_and_geometry
        self.overlap_generation = True  # see geometry_and_forward
        # pixel spans of the adjoint in loss_step_io (fractions of the image, None = the rest)
        self.bwd_span_fractions = (0.4, 0.3, 0.2, None)
        self._span_streams = []
        if wavefront:
            nbytes = mcdi.shade_workspace_size(self.N, self.H, self.W, self.params)
            self.workspace = torch.empty((nbytes + 255) // 256 * 256, dtype=torch.uint8, device=dev)
        # G-buffer by rasterisation (depth buffer + index map), else by the closest-hit ray cast
        self.raster_ws = None
        if raster:
            nbytes = mcdi.raster_workspace_size(self.N, self.H, self.W)
            self.raster_ws = torch.empty((nbytes + 255) // 256 * 256, dtype=torch.uint8, device=dev)

    # ---- the steps
    def build_probe(self, stream=None):
        self.probe.build(stream)

    def build_bvh(self, stream=None):
        self.bvh.build(self.verts, self.tris, stream)

    def primary(self, stream=None):
        if self.raster_ws is not None:
            mcdi.raster_gbuffer(self.verts, self.vnrm, self.tris, self.cams, self.H, self.W, self.tex_kd,
                                self.tex_korm, self.uvmap, self.gb, self.raster_ws, stream)
        else:
            mcdi.primary_cast(self.bvh, self.verts, self.vnrm, self.tris, self.cams, self.H, self.W, self.tex_kd,
                              self.tex_korm, self.uvmap, self.gb, stream)

    def primary_part(self, part: int, stream=None, tex=None):
        """The rasterised G-buffer in two parts: 1 = depth (mesh only), 2 = resolve (reads the textures:
        ``tex`` = (k_d, k_orm) device textures, (S, S, 4) or packed (S, S, 3); default the pipeline's)."""
        kd, korm = tex if tex is not None else (self.tex_kd, self.tex_korm)
        mcdi.raster_gbuffer_part(self.verts, self.vnrm, self.tris, self.cams, self.H, self.W, kd, korm, self.uvmap,
                                 self.gb, self.raster_ws, part, stream)

    def forward(self, stream=None):
        mcdi.shade_mc_fwd(self.bvh, self.probe, self.gb, self.cams, self.params, self.c_d, self.kd_out, self.c_s,
                          self.mask, self.workspace, stream)

    def forward_part(self, part: int, stream=None):
        mcdi.shade_mc_fwd_part(self.bvh, self.probe, self.gb, self.cams, self.params, self.c_d, self.kd_out, self.c_s,
                               self.mask, self.workspace, part, stream)

    def geometry_and_forward(self, stream=None):
        """`tables_and_geometry` then `forward`.  With the wavefront and the rasterised
        G-buffer, the sample generation, which reads no BVH, follows the G-buffer on the
        forked stream while the BVH is built on a stream of the highest priority (so
        that its chain of small kernels gets SMs before the generation's blocks), and
        the shadow rays follow both (measured: 25 us faster per headline step launched
        kernel by kernel, 20-40 us in the replayed graph, whose nodes keep their
        priorities because the library instantiates it: mcdi.Graph)."""
        if not (self.overlap_generation and self.workspace is not None and self.raster_ws is not None):
            self.tables_and_geometry(stream)
            self.forward(stream)
            return
        cur = stream if stream is not None else torch.cuda.current_stream(self.device)
        if self._fork is None:
            self._fork = torch.cuda.Stream(self.device)
        fork, bs, ps = self._fork, self.bvh_stream(), self.probe_stream()
        for st in (fork, bs, ps):
            st.wait_stream(cur)
        self.build_probe(ps)
        self.primary(fork)
        fork.wait_stream(ps)
        self.forward_part(1, fork)
        self.build_bvh(bs)
        cur.wait_stream(fork)
        cur.wait_stream(bs)
        self.forward_part(2, cur)

    def probe_stream(self):
        """A third stream: the probe tables, beside the G-buffer and the BVH build."""
        if getattr(self, "_probe_stream", None) is None:
            self._probe_stream = torch.cuda.Stream(self.device)
        return self._probe_stream

    def bvh_stream(self):
        """The stream of the highest priority the BVH build runs on beside the sample generation."""
        if getattr(self, "_bvh_stream", None) is None:
            self._bvh_stream = torch.cuda.Stream(self.device, priority=torch.cuda.Stream.priority_range()[1])
        return self._bvh_stream

    def backward(self, g_cd, g_kdout, g_cs, stream=None, zero_env_grad=True):
        if zero_env_grad:
            self.g_env.zero_()
        mcdi.shade_mc_bwd(self.bvh, self.probe, self.gb, self.cams, self.params, g_cd, g_kdout, g_cs, self.mask,
                          self.g_kd, self.g_korm, self.g_nrm, self.g_env, stream)

    def backward_span(self, g_cd, g_kdout, g_cs, first: int, count: int, stream=None):
        """`backward` for the pixels [first, first + count) only; g_env accumulates (zero it first)."""
        mcdi.shade_mc_bwd_span(self.bvh, self.probe, self.gb, self.cams, self.params, g_cd, g_kdout, g_cs,
                               self.mask, self.g_kd, self.g_korm, self.g_nrm, self.g_env, first, count, stream)

    def denoise(self, stream=None):
        """D(c_d), D(c_s): the U-Net with k_d,out and the normal as guides (Sec. 4.2), or
        the cross-bilateral filter with depth and normal as edge-stopping guides (App. B)."""
        if self.bilateral_sigma is not None:
            mcdi.bilateral_fwd(self.gb.pos, self.gb.nrm, self.cams, self.terms, self.bilateral_sigma, self.denoised,
                               self.bl_wsum, stream=stream)
        else:
            self.denoiser.forward(self.terms, self.kd_out, self.gb.nrm, self.denoised, stream)

    def denoise_backward(self, g_denoised, stream=None):
        if self.bilateral_sigma is not None:
            mcdi.bilateral_bwd(self.gb.pos, self.gb.nrm, self.cams, self.bl_wsum, g_denoised, self.bilateral_sigma,
                               self.g_terms, stream=stream)
        else:
            self.denoiser.backward(g_denoised, self.g_terms, stream)

    def tables_and_geometry(self, stream=None):
        """Probe tables and the rasterised G-buffer (which reads the mesh, not the
        BVH) on a forked stream, concurrently with the BVH build (they share no
        buffers), joined before anything reads them; inside a captured graph the
        fork and join become graph edges.  The ray-cast G-buffer needs the BVH and
        follows it on the calling stream."""
        cur = stream if stream is not None else torch.cuda.current_stream(self.device)
        if self._fork is None:
            self._fork = torch.cuda.Stream(self.device)
        self._fork.wait_stream(cur)
        self.build_probe(self._fork)
        if self.raster_ws is not None:
            self.primary(self._fork)
        self.build_bvh(stream)
        if self.raster_ws is None:
            self.primary(stream)
        cur.wait_stream(self._fork)

    def step(self, g_cd, g_kdout, g_cs, stream=None):
        """One pass of the hot path: tables, BVH, G-buffer, forward, adjoint.
        With a denoiser, g_cd / g_cs are gradients of the denoised terms and pass
        through the denoiser's input gradient first."""
        self.tables_and_geometry(stream)
        self.forward(stream)
        if self.denoiser is not None:
            self.denoise(stream)
            g = torch.cat([g_cd, g_cs], 0) if g_cd.shape[0] == self.N else g_cd
            self.denoise_backward(g, stream)
            g_cd, g_cs = self.g_terms[: self.N], self.g_terms[self.N:]
        self.backward(g_cd, g_kdout, g_cs, stream)

    def loss_step(self, ref, stream=None, lambda_light: float = 0.15):
        """One optimisation step driven by the paper's image loss against ``ref``
        ([N][H][W] float4, linear radiance): tables, BVH, G-buffer, forward,
        denoiser, composite + tonemapped L1 loss + lighting regulariser and their
        adjoint, denoiser input gradient, shading adjoint.  (L, L_image, L_light)
        stay on the device in ``self.loss``; the composite is ``self.color``."""
        self.geometry_and_forward(stream)
        self.loss_and_backward(ref, stream, lambda_light)

    def image_loss(self, ref, stream=None, lambda_light: float = 0.15):
        """Composite + image loss + lighting regulariser and their adjoint on the
        denoised terms (the raw terms without a denoiser); gradients land in
        ``self.g_loss_terms`` ([2N] planes: c_d then c_s) and ``self.g_loss_kdout``."""
        N = self.N
        if self._loss is None:
            dev = self.device
            self._loss = dict(loss=torch.zeros(3, dtype=torch.float64, device=dev),
                              g_den=torch.zeros_like(self.terms), g_kdout=torch.zeros_like(self.kd_out),
                              color=torch.zeros_like(self.kd_out),
                              ws=torch.empty(mcdi.image_loss_workspace_size(N * self.H * self.W), dtype=torch.uint8,
                                             device=dev))
        b = self._loss
        self.loss, self.color = b["loss"], b["color"]
        self.g_loss_terms, self.g_loss_kdout = b["g_den"], b["g_kdout"]
        src = self.denoised if self.denoiser is not None else self.terms
        mcdi.image_loss(self.kd_out, src[:N], src[N:], ref, b["loss"], b["g_kdout"], b["g_den"][:N], b["g_den"][N:],
                        b["ws"], lambda_light, b["color"], stream)

    def loss_and_backward(self, ref, stream=None, lambda_light: float = 0.15):
        """The loss part of `loss_step` (after the forward)."""
        N = self.N
        if self.denoiser is not None:
            self.denoise(stream)
        self.image_loss(ref, stream, lambda_light)
        g_cd, g_cs = self.g_loss_terms[:N], self.g_loss_terms[N:]
        if self.denoiser is not None:
            self.denoise_backward(self.g_loss_terms, stream)
            g_cd, g_cs = self.g_terms[:N], self.g_terms[N:]
        self.backward(g_cd, self.g_loss_kdout, g_cs, stream)

    def capture(self, g_cd, g_kdout, g_cs):
        """Capture one `step` (synthetic upstream gradients) into a CUDA graph; see `_capture`."""
        return self._capture(lambda: self.step(g_cd, g_kdout, g_cs))

    def capture_loss_step(self, ref, lambda_light: float = 0.15):
        """Capture one `loss_step` against ``ref`` into a CUDA graph; see `_capture`."""
        return self._capture(lambda: self.loss_step(ref, lambda_light=lambda_light))

    def loss_step_io(self, ref, host_in: dict, host_ref, outputs, stream=None, lambda_light: float = 0.15):
        """`loss_step` with its host I/O overlapped: this step's inputs are copied
        from pinned host memory (``host_in``: verts, vnrm, tris, env, tex_kd,
        tex_korm into the pipeline's buffers — the textures either (S, S, 4) or
        packed (S, S, 3), a quarter fewer bytes, which the rasteriser's resolve
        reads as they are; ``host_ref`` into ``ref``) on one
        copy stream in the order the step first needs them (mesh, probe, the two
        material textures, reference: the host link is the bound, and copies on
        several streams share it, so each input arrives earliest in sequence),
        and every stage waits only for the inputs it reads: the BVH build and the
        rasteriser's depth pass for the mesh, the probe tables for the probe, the
        G-buffer's resolve for the textures, the loss for the reference.
        ``outputs`` lists (device tensor, pinned host tensor) pairs read back as
        soon as their producer has run: the loss and the composite while the
        denoiser input gradient and the adjoint run, the rest at the end (over
        two streams).  Inside a captured graph the waits become graph edges."""
        dev = self.device
        cur = stream if stream is not None else torch.cuda.current_stream(dev)
        if getattr(self, "_io", None) is None:
            self._io = [torch.cuda.Stream(dev) for _ in range(3)]
        up, down, down2 = self._io
        streams = (up, down, down2)
        for st in streams:
            st.wait_stream(cur)
        ev = {k: torch.cuda.Event() for k in ("mesh", "env", "tex", "ref", "loss", "end")}
        tex = (self.tex_kd, self.tex_korm)
        if host_in["tex_kd"].shape[-1] == 3:  # packed RGB: resolved from a packed device copy
            if self.raster_ws is None:
                raise ValueError("packed (S, S, 3) host textures need the rasterised G-buffer")
            shape = tuple(host_in["tex_kd"].shape)
            if getattr(self, "_tex3", None) is None or tuple(self._tex3[0].shape) != shape:
                self._tex3 = tuple(torch.empty(shape, dtype=torch.float32, device=dev) for _ in range(2))
            tex = self._tex3
        with torch.cuda.stream(up):
            for k in ("verts", "tris", "vnrm"):
                getattr(self, k).copy_(host_in[k], non_blocking=True)
            ev["mesh"].record(up)
            self.env.copy_(host_in["env"], non_blocking=True)
            ev["env"].record(up)
            tex[0].copy_(host_in["tex_kd"], non_blocking=True)
            tex[1].copy_(host_in["tex_korm"], non_blocking=True)
            ev["tex"].record(up)
            ref.copy_(host_ref, non_blocking=True)
            ev["ref"].record(up)
        if self._fork is None:
            self._fork = torch.cuda.Stream(dev)
        fork = self._fork
        fork.wait_stream(cur)
        fork.wait_event(ev["mesh"])
        overlap = self.overlap_generation and self.workspace is not None and self.raster_ws is not None
        if self.raster_ws is not None:
            self.primary_part(1, fork)
        ps = self.probe_stream()
        ps.wait_stream(cur)
        ps.wait_event(ev["env"])
        self.build_probe(ps)
        if self.raster_ws is not None:
            fork.wait_event(ev["tex"])
            self.primary_part(2, fork, tex)
        fork.wait_stream(ps)
        if overlap:  # sample generation beside the BVH build, which runs at the highest priority
            self.forward_part(1, fork)
            bs = self.bvh_stream()
            bs.wait_stream(cur)
            bs.wait_event(ev["mesh"])
            self.build_bvh(bs)
            cur.wait_stream(bs)
        else:
            cur.wait_event(ev["mesh"])
            self.build_bvh(cur)
        if self.raster_ws is None:
            cur.wait_event(ev["tex"])
            self.primary(cur)
        cur.wait_stream(fork)
        if overlap:
            self.forward_part(2, cur)
        else:
            self.forward(cur)
        N = self.N
        if self.denoiser is not None:
            self.denoise(cur)
        cur.wait_event(ev["ref"])
        self.image_loss(ref, cur, lambda_light)
        ev["loss"].record(cur)
        early = [(d, h) for d, h in outputs if d is self.loss or d is self.color]
        per_pixel = [(d, h) for d, h in outputs if any(d is t for t in (self.g_kd, self.g_korm, self.g_nrm))]
        late = [(d, h) for d, h in outputs if not any(d is t for t, _ in early + per_pixel)]
        down.wait_event(ev["loss"])
        with torch.cuda.stream(down):
            for d, h in early:
                h.copy_(d, non_blocking=True)
        g_cd, g_cs = self.g_loss_terms[:N], self.g_loss_terms[N:]
        if self.denoiser is not None:
            self.denoise_backward(self.g_loss_terms, cur)
            g_cd, g_cs = self.g_terms[:N], self.g_terms[N:]
        # the adjoint in pixel spans, each span's per-pixel gradients read back while the later ones
        # run; the spans shrink so that little is left to copy after the last (the probe gradient,
        # summed over all pixels, follows it).  The spans write disjoint pixels (and add into the probe
        # gradient by atomics), so each is launched on a stream of its own, earlier spans at higher
        # priority: the block scheduler finishes a span before it starts the next one's blocks, those
        # fill the SMs while the span's last blocks drain, and a read-back waits for its own span only.
        self.g_env.zero_()
        spans = pixel_spans(self.N * self.H * self.W, self.bwd_span_fractions)
        if len(self._span_streams) != len(spans):
            self._span_streams = [torch.cuda.Stream(dev, priority=-(len(spans) - 1 - k)) for k in range(len(spans))]
        for k, (first, count) in enumerate(spans):
            st = self._span_streams[k]
            st.wait_stream(cur)
            self.backward_span(g_cd, self.g_loss_kdout, g_cs, first, count, st)
            e = torch.cuda.Event()
            e.record(st)
            if per_pixel:
                down2.wait_event(e)
                with torch.cuda.stream(down2):
                    for d, h in per_pixel:
                        h.view(-1, 4)[first:first + count].copy_(d.view(-1, 4)[first:first + count], non_blocking=True)
        for k in range(len(spans)):
            cur.wait_stream(self._span_streams[k])
        ev["end"].record(cur)
        down.wait_event(ev["end"])
        with torch.cuda.stream(down):
            for d, h in late:
                h.copy_(d, non_blocking=True)
        for st in streams:
            cur.wait_stream(st)

    def capture_loss_step_io(self, ref, host_in: dict, host_ref, outputs, lambda_light: float = 0.15):
        """Capture one `loss_step_io` into a CUDA graph (its copies included); `replay_io()` reruns it."""
        self._capture(lambda: self.loss_step_io(ref, host_in, host_ref, outputs, lambda_light=lambda_light),
                      "graph_io")
        return self.graph_io

    def _capture(self, fn, attr: str = "graph"):
        """Capture one step into a CUDA graph (its launches, memsets and the
        host-encoded tensor maps are baked in with these buffers) kept as
        ``self.<attr>``; `replay()` then reruns the whole step with one launch
        from the host.  A first step runs uncaptured on a side stream so that
        one-time set-up (kernel attributes, device queries, lazily allocated
        buffers) stays outside the graph."""
        dev = self.device
        side = torch.cuda.Stream(dev)
        side.wait_stream(torch.cuda.current_stream(dev))
        with torch.cuda.stream(side):
            fn()
        torch.cuda.current_stream(dev).wait_stream(side)
        # instantiated by the library with per-node priorities, so that kernels captured from
        # high-priority streams keep their priority in the replay (mcdi.Graph)
        graph = mcdi.Graph.capture(fn)
        setattr(self, attr, graph)
        return graph

    def replay(self):
        self.graph.replay()

    def replay_io(self):
        self.graph_io.replay()

    def covered_pixels(self) -> int:
        return int((self.gb.pos[..., 3] > 0).sum().item())
