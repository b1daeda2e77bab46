"""Python binding of libmcdi (ctypes): argument marshalling only.

Each function carries the C entry point's name without the ``mcdi_`` prefix
and takes torch CUDA tensors (or raw device addresses as ints); all the work
runs in the library's CUDA kernels on the current torch stream.  There is no
CPU fallback: if the library is not built, ``load()`` raises.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libmcdi.so")
_lib = None

OK, INVALID_ARG, UNSUPPORTED, OOM, TIMEOUT, DEVICE_ERROR = range(6)


class McdiError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        super().__init__(f"{where} failed (status {status}): {msg}")
        self.status = status


class BvhView(C.Structure):
    _fields_ = [("nodes", C.c_void_p), ("tri_records", C.c_void_p), ("n_tris", C.c_int)]


class ShadeParams(C.Structure):
    _fields_ = [("n_light", C.c_int), ("n_cos", C.c_int), ("n_ggx", C.c_int), ("decorrelate_bwd", C.c_int),
                ("seed", C.c_ulonglong), ("tau", C.c_float), ("ray_eps", C.c_float)]


EXPORTS = ["mcdi_last_error", "mcdi_version", "mcdi_build_envmap_cdf", "mcdi_bvh_sizes", "mcdi_build_bvh",
           "mcdi_build_bvh_noalloc", "mcdi_primary_cast", "mcdi_shade_workspace_size", "mcdi_shade_mc_fwd",
           "mcdi_shade_mc_bwd", "mcdi_denoise_sizes", "mcdi_denoise_pack_weights", "mcdi_denoise_fwd",
           "mcdi_denoise_bwd", "mcdi_conv3x3_bf16", "mcdi_conv3x3_e4m3", "mcdi_composite",
           "mcdi_image_loss_workspace_size", "mcdi_image_loss", "mcdi_bilateral_fwd", "mcdi_bilateral_bwd",
           "mcdi_shadow_ray_stats", "mcdi_shadow_ray_retrace", "mcdi_read_sweep", "mcdi_refit_bvh",
           "mcdi_edge_table_workspace_size", "mcdi_build_edge_table", "mcdi_shadow_edge_grad",
           "mcdi_raster_workspace_size", "mcdi_raster_gbuffer", "mcdi_denoise_record_plan",
           "mcdi_denoise_wgrad_bytes", "mcdi_denoise_wgrad", "mcdi_conv3x3_wgrad_bytes",
           "mcdi_conv3x3_wgrad", "mcdi_shade_mc_fwd_part", "mcdi_raster_gbuffer_part",
           "mcdi_shade_mc_bwd_span", "mcdi_graph_instantiate", "mcdi_graph_launch", "mcdi_graph_destroy",
           "mcdi_bvh_build_launches", "mcdi_set_graph_dependent_launch"]
BF16, E4M3 = 0, 1  # denoiser operand precisions (MCDI_DENOISE_BF16, MCDI_DENOISE_E4M3)
NOALLOC_MAX_TRIS = 65536


def load(path: str = LIB_PATH):
    """Load libmcdi.so; raises if it has not been built (no fallback path exists)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libmcdi.so not built at {path}: run paper_2206_03380_gb300.build.build()")
    lib = C.CDLL(path)
    P, i, sz, st = C.c_void_p, C.c_int, C.c_size_t, C.c_int
    lib.mcdi_last_error.restype = C.c_char_p
    lib.mcdi_last_error.argtypes = []
    lib.mcdi_version.restype = C.c_int
    lib.mcdi_version.argtypes = []
    lib.mcdi_build_envmap_cdf.restype = st
    lib.mcdi_build_envmap_cdf.argtypes = [P, i, i, P, P, P, P, P]
    lib.mcdi_bvh_sizes.restype = st
    lib.mcdi_bvh_sizes.argtypes = [i, C.POINTER(sz), C.POINTER(sz), C.POINTER(sz)]
    lib.mcdi_build_bvh.restype = st
    lib.mcdi_build_bvh.argtypes = [P, i, P, i, P, P, P, sz, P]
    lib.mcdi_set_graph_dependent_launch.restype = st
    lib.mcdi_set_graph_dependent_launch.argtypes = [i]
    lib.mcdi_bvh_build_launches.restype = st
    lib.mcdi_bvh_build_launches.argtypes = [i, C.POINTER(i)]
    lib.mcdi_refit_bvh.restype = st
    lib.mcdi_refit_bvh.argtypes = [P, i, P, i, P, P, P, sz, P]
    lib.mcdi_build_bvh_noalloc.restype = st
    lib.mcdi_build_bvh_noalloc.argtypes = [P, i, P, i, P, P, P]
    lib.mcdi_primary_cast.restype = st
    lib.mcdi_primary_cast.argtypes = [C.POINTER(BvhView), P, P, P, i, P, i, i, i, P, P, i, C.POINTER(C.c_float),
                                      P, P, P, P, P]
    lib.mcdi_raster_workspace_size.restype = st
    lib.mcdi_raster_workspace_size.argtypes = [i, i, i, C.POINTER(sz)]
    lib.mcdi_raster_gbuffer.restype = st
    lib.mcdi_raster_gbuffer.argtypes = [P, P, P, i, i, P, i, i, i, P, P, i, C.POINTER(C.c_float), P, P, P, P, P, sz,
                                        P]
    lib.mcdi_raster_gbuffer_part.restype = st
    lib.mcdi_raster_gbuffer_part.argtypes = [P, P, P, i, i, P, i, i, i, P, P, i, i, C.POINTER(C.c_float), P, P, P,
                                             P, P, sz, i, P]
    lib.mcdi_shade_workspace_size.restype = st
    lib.mcdi_shade_workspace_size.argtypes = [i, i, i, C.POINTER(ShadeParams), C.POINTER(sz)]
    lib.mcdi_shade_mc_fwd.restype = st
    lib.mcdi_shade_mc_fwd.argtypes = [C.POINTER(BvhView), P, i, i, P, P, P, P, P, P, P, P, i, i, i,
                                      C.POINTER(ShadeParams), P, P, P, P, P, sz, P]
    lib.mcdi_shade_mc_fwd_part.restype = st
    lib.mcdi_shade_mc_fwd_part.argtypes = [C.POINTER(BvhView), P, i, i, P, P, P, P, P, P, P, P, i, i, i,
                                      C.POINTER(ShadeParams), P, P, P, P, P, sz, i, P]
    lib.mcdi_shade_mc_bwd.restype = st
    lib.mcdi_shade_mc_bwd.argtypes = [C.POINTER(BvhView), P, i, i, P, P, P, P, P, P, P, P, i, i, i,
                                      C.POINTER(ShadeParams), P, P, P, P, P, P, P, P, P]
    lib.mcdi_shade_mc_bwd_span.restype = st
    lib.mcdi_shade_mc_bwd_span.argtypes = [C.POINTER(BvhView), P, i, i, P, P, P, P, P, P, P, P, i, i, i,
                                           C.POINTER(ShadeParams), P, P, P, P, P, P, P, P, C.c_longlong,
                                           C.c_longlong, P]
    lib.mcdi_shadow_ray_stats.restype = st
    lib.mcdi_shadow_ray_stats.argtypes = [C.POINTER(BvhView), i, i, i, C.POINTER(ShadeParams), P, sz, P, P]
    lib.mcdi_shadow_ray_retrace.restype = st
    lib.mcdi_shadow_ray_retrace.argtypes = [C.POINTER(BvhView), i, i, i, C.POINTER(ShadeParams), P, sz, P]
    lib.mcdi_read_sweep.restype = st
    lib.mcdi_edge_table_workspace_size.restype = st
    lib.mcdi_edge_table_workspace_size.argtypes = [i, C.POINTER(sz)]
    lib.mcdi_build_edge_table.restype = st
    lib.mcdi_build_edge_table.argtypes = [P, i, P, P, P, sz, P]
    lib.mcdi_shadow_edge_grad.restype = st
    lib.mcdi_shadow_edge_grad.argtypes = [C.POINTER(BvhView), P, i, P, P, i, P, i, i, P, P, P, P, P, i, i, i,
                                          C.POINTER(ShadeParams), i, C.c_float, P, P, P, P, P]
    lib.mcdi_read_sweep.argtypes = [P, sz, i, P, P]
    lib.mcdi_graph_instantiate.restype = st
    lib.mcdi_graph_instantiate.argtypes = [P, C.POINTER(C.c_void_p)]
    lib.mcdi_graph_launch.restype = st
    lib.mcdi_graph_launch.argtypes = [P, P]
    lib.mcdi_graph_destroy.restype = st
    lib.mcdi_graph_destroy.argtypes = [P]
    lib.mcdi_denoise_sizes.restype = st
    lib.mcdi_denoise_sizes.argtypes = [i, i, i, i, C.POINTER(sz), C.POINTER(sz), C.POINTER(sz), C.POINTER(sz)]
    lib.mcdi_denoise_pack_weights.restype = st
    lib.mcdi_denoise_pack_weights.argtypes = [P, P, P]
    lib.mcdi_denoise_fwd.restype = st
    lib.mcdi_denoise_fwd.argtypes = [P, i, i, i, i, P, P, P, i, P, P, sz, P, P]
    lib.mcdi_denoise_bwd.restype = st
    lib.mcdi_denoise_record_plan.restype = st
    lib.mcdi_denoise_record_plan.argtypes = [P, i, P]
    lib.mcdi_denoise_bwd.argtypes = [P, i, i, i, i, P, sz, P, P, P, sz, P, P]
    lib.mcdi_denoise_wgrad_bytes.restype = st
    lib.mcdi_denoise_wgrad_bytes.argtypes = [i, i, i, C.POINTER(sz)]
    lib.mcdi_denoise_wgrad.restype = st
    lib.mcdi_denoise_wgrad.argtypes = [i, i, i, i, P, sz, P, sz, P, P, sz, P, P]
    lib.mcdi_conv3x3_wgrad_bytes.restype = st
    lib.mcdi_conv3x3_wgrad_bytes.argtypes = [i, i, i, i, i, C.POINTER(sz)]
    lib.mcdi_conv3x3_wgrad.restype = st
    lib.mcdi_conv3x3_wgrad.argtypes = [P, P, i, i, i, i, i, i, i, P, P, sz, P, P]
    lib.mcdi_composite.restype = st
    lib.mcdi_composite.argtypes = [P, P, P, C.c_longlong, P, P]
    lib.mcdi_conv3x3_bf16.restype = st
    lib.mcdi_conv3x3_bf16.argtypes = [P, i, i, i, i, P, P, i, i, P, P, P]
    lib.mcdi_bilateral_fwd.restype = st
    lib.mcdi_bilateral_fwd.argtypes = [P, P, P, i, i, i, i, P, C.c_float, i, P, P, P]
    lib.mcdi_bilateral_bwd.restype = st
    lib.mcdi_bilateral_bwd.argtypes = [P, P, P, i, i, i, i, P, P, C.c_float, i, P, P]
    lib.mcdi_image_loss_workspace_size.restype = st
    lib.mcdi_image_loss_workspace_size.argtypes = [C.c_longlong, C.POINTER(sz)]
    lib.mcdi_image_loss.restype = st
    lib.mcdi_image_loss.argtypes = [P, P, P, P, C.c_longlong, C.c_float, P, P, P, P, P, P, sz, P]
    lib.mcdi_conv3x3_e4m3.restype = st
    lib.mcdi_conv3x3_e4m3.argtypes = [P, i, i, i, i, P, P, P, P, i, i, P, P, P]
    _lib = lib
    return lib


def _ptr(t) -> int | None:
    if t is None:
        return None
    if isinstance(t, int):
        return t
    if not t.is_contiguous():
        raise ValueError("tensor arguments must be contiguous")
    return t.data_ptr()


def _stream(stream=None):
    if stream is None:
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, torch.cuda.Stream):
        return C.c_void_p(stream.cuda_stream)
    return C.c_void_p(int(stream))


def _check(status: int, where: str):
    if status != OK:
        raise McdiError(status, where, load().mcdi_last_error().decode())


# ------------------------------------------------------------------ entry points
def version() -> int:
    return load().mcdi_version()


def set_graph_dependent_launch(enable: bool):
    """Whether this thread's captured convolutions keep their programmatic dependence (default True)."""
    _check(load().mcdi_set_graph_dependent_launch(1 if enable else 0), "set_graph_dependent_launch")


def bvh_build_launches(n_tris: int) -> int:
    """Kernels mcdi_build_bvh launches for n_tris triangles on the current device."""
    out = C.c_int()
    _check(load().mcdi_bvh_build_launches(int(n_tris), C.byref(out)), "bvh_build_launches")
    return out.value


class Graph:
    """A step captured by torch into a CUDA graph and instantiated by the library
    with per-node priorities (mcdi_graph_instantiate), so that kernels captured
    from streams of higher priority keep it when the graph is replayed.  Holds
    the torch graph (which owns the captured graph and its memory pool)."""

    def __init__(self, torch_graph):
        self.torch_graph = torch_graph
        raw = torch_graph.raw_cuda_graph()
        if not isinstance(raw, int):
            raise TypeError(f"raw_cuda_graph() returned {type(raw).__name__}, expected an address")
        out = C.c_void_p()
        _check(load().mcdi_graph_instantiate(raw, C.byref(out)), "graph_instantiate")
        self.exec = out.value

    @staticmethod
    def capture(fn):
        """Capture ``fn()`` (on torch's capture stream) and instantiate it with node priorities."""
        g = torch.cuda.CUDAGraph(keep_graph=True)
        with torch.cuda.graph(g):
            fn()
        return Graph(g)

    def replay(self, stream=None):
        _check(load().mcdi_graph_launch(self.exec, _stream(stream)), "graph_launch")

    def __del__(self):
        if getattr(self, "exec", None) and _lib is not None:
            _lib.mcdi_graph_destroy(self.exec)
            self.exec = None


def build_envmap_cdf(env, cond, marg, row_sum, total, stream=None):
    H, W = env.shape[0], env.shape[1]
    _check(load().mcdi_build_envmap_cdf(_ptr(env), W, H, _ptr(cond), _ptr(marg), _ptr(row_sum), _ptr(total),
                                        _stream(stream)), "build_envmap_cdf")


def bvh_sizes(n_tris: int):
    a, b, c = C.c_size_t(), C.c_size_t(), C.c_size_t()
    _check(load().mcdi_bvh_sizes(int(n_tris), C.byref(a), C.byref(b), C.byref(c)), "bvh_sizes")
    return a.value, b.value, c.value


def tracer_structure_bytes(bvh: "Bvh") -> int:
    """Bytes of the structure a shadow ray walks in a built BVH: its four-wide nodes (64 B each;
    the slots of odd-depth nodes are zero and unused) and the triangle records (48 B each).  A
    measurement aid: reads the node array back to count the nodes in use."""
    n = max(int(bvh.n_tris), 1)
    r256 = lambda x: (x + 255) // 256 * 256
    off = r256(r256(max(n - 1, 1) * 64) + (2 * n - 1) * 32)
    scale_x = bvh.nodes[off: off + max(n - 1, 1) * 64].view(torch.float32).reshape(-1, 16)[:, 3]
    return int((scale_x != 0).sum().item()) * 64 + n * 48


def build_bvh(verts, tris, nodes, tri_records, scratch, stream=None):
    _check(load().mcdi_build_bvh(_ptr(verts), verts.shape[0], _ptr(tris), tris.shape[0], _ptr(nodes),
                                 _ptr(tri_records), _ptr(scratch), scratch.numel() * scratch.element_size(),
                                 _stream(stream)), "build_bvh")


def refit_bvh(verts, tris, nodes, tri_records, scratch, stream=None):
    """Bounds-only update after the vertices moved (same triangles as the last build into these buffers)."""
    _check(load().mcdi_refit_bvh(_ptr(verts), verts.shape[0], _ptr(tris), tris.shape[0], _ptr(nodes),
                                 _ptr(tri_records), _ptr(scratch), scratch.numel() * scratch.element_size(),
                                 _stream(stream)), "refit_bvh")


def build_bvh_noalloc(verts, tris, nodes, tri_records, stream=None):
    """BVH build with the library's own fixed scratch (no caller scratch; at most
    NOALLOC_MAX_TRIS triangles; calls that overlap on the GPU must be serialised)."""
    _check(load().mcdi_build_bvh_noalloc(_ptr(verts), verts.shape[0], _ptr(tris), tris.shape[0], _ptr(nodes),
                                         _ptr(tri_records), _stream(stream)), "build_bvh_noalloc")


def primary_cast(bvh: "Bvh", verts, vnrm, tris, cams, H, W, tex_kd, tex_korm, uvmap, gb, stream=None):
    uv = (C.c_float * 3)(*[float(x) for x in uvmap])
    _check(load().mcdi_primary_cast(C.byref(bvh.view), _ptr(verts), _ptr(vnrm), _ptr(tris), verts.shape[0],
                                    _ptr(cams), cams.shape[0], H, W, _ptr(tex_kd), _ptr(tex_korm), tex_kd.shape[0],
                                    uv, _ptr(gb.pos), _ptr(gb.nrm), _ptr(gb.kd), _ptr(gb.korm), _stream(stream)),
           "primary_cast")


def raster_workspace_size(N: int, H: int, W: int) -> int:
    b = C.c_size_t()
    _check(load().mcdi_raster_workspace_size(int(N), int(H), int(W), C.byref(b)), "raster_workspace_size")
    return b.value


def raster_gbuffer(verts, vnrm, tris, cams, H, W, tex_kd, tex_korm, uvmap, gb, workspace, stream=None):
    """The G-buffer by rasterising the mesh (same outputs as primary_cast; no BVH needed)."""
    uv = (C.c_float * 3)(*[float(x) for x in uvmap])
    _check(load().mcdi_raster_gbuffer(_ptr(verts), _ptr(vnrm), _ptr(tris), verts.shape[0], tris.shape[0], _ptr(cams),
                                      cams.shape[0], int(H), int(W), _ptr(tex_kd), _ptr(tex_korm), tex_kd.shape[0], uv,
                                      _ptr(gb.pos), _ptr(gb.nrm), _ptr(gb.kd), _ptr(gb.korm), _ptr(workspace),
                                      workspace.numel() * workspace.element_size(), _stream(stream)),
           "raster_gbuffer")


def raster_gbuffer_part(verts, vnrm, tris, cams, H, W, tex_kd, tex_korm, uvmap, gb, workspace, part: int,
                        stream=None):
    """`raster_gbuffer` in two calls: part 1 (depth; reads the mesh and cameras only), then part 2
    (resolve: attributes and texture lookups into the G-buffer) on a stream ordered after it.  The
    textures are (S, S, 4) or packed (S, S, 3) float32."""
    uv = (C.c_float * 3)(*[float(x) for x in uvmap])
    ch = int(tex_kd.shape[-1])
    if tex_korm.shape[-1] != ch:
        raise ValueError("tex_kd and tex_korm must have the same number of channels")
    _check(load().mcdi_raster_gbuffer_part(_ptr(verts), _ptr(vnrm), _ptr(tris), verts.shape[0], tris.shape[0],
                                           _ptr(cams), cams.shape[0], int(H), int(W), _ptr(tex_kd), _ptr(tex_korm),
                                           tex_kd.shape[0], ch, uv, _ptr(gb.pos), _ptr(gb.nrm), _ptr(gb.kd),
                                           _ptr(gb.korm), _ptr(workspace), workspace.numel() * workspace.element_size(),
                                           int(part), _stream(stream)), "raster_gbuffer_part")


def shade_workspace_size(N: int, H: int, W: int, params: ShadeParams) -> int:
    b = C.c_size_t()
    _check(load().mcdi_shade_workspace_size(int(N), int(H), int(W), C.byref(params), C.byref(b)),
           "shade_workspace_size")
    return b.value


def shade_mc_fwd(bvh: "Bvh", probe: "Probe", gb: "GBuffer", cams, params: ShadeParams, c_d, kd_out, c_s,
                 vis_mask=None, workspace=None, stream=None):
    N, H, W = gb.pos.shape[:3]
    Hp, Wp = probe.env.shape[:2]
    ws_bytes = 0 if workspace is None else workspace.numel() * workspace.element_size()
    _check(load().mcdi_shade_mc_fwd(C.byref(bvh.view), _ptr(probe.env), Wp, Hp, _ptr(probe.cond), _ptr(probe.marg),
                                    _ptr(probe.total), _ptr(gb.pos), _ptr(gb.nrm), _ptr(gb.kd), _ptr(gb.korm),
                                    _ptr(cams), N, H, W, C.byref(params), _ptr(c_d), _ptr(kd_out), _ptr(c_s),
                                    _ptr(vis_mask), _ptr(workspace), ws_bytes, _stream(stream)), "shade_mc_fwd")


def shade_mc_fwd_part(bvh: "Bvh", probe: "Probe", gb: "GBuffer", cams, params: ShadeParams, c_d, kd_out, c_s,
                      vis_mask, workspace, part: int, stream=None):
    """Part 1 (sample generation, reads no BVH) or 2 (shadow rays and accumulation) of shade_mc_fwd."""
    N, H, W = gb.pos.shape[:3]
    Hp, Wp = probe.env.shape[:2]
    _check(load().mcdi_shade_mc_fwd_part(C.byref(bvh.view), _ptr(probe.env), Wp, Hp, _ptr(probe.cond),
                                         _ptr(probe.marg), _ptr(probe.total), _ptr(gb.pos), _ptr(gb.nrm), _ptr(gb.kd),
                                         _ptr(gb.korm), _ptr(cams), N, H, W, C.byref(params), _ptr(c_d), _ptr(kd_out),
                                         _ptr(c_s), _ptr(vis_mask), _ptr(workspace),
                                         workspace.numel() * workspace.element_size(), int(part), _stream(stream)),
           "shade_mc_fwd_part")


def shade_mc_bwd(bvh: "Bvh", probe: "Probe", gb: "GBuffer", cams, params: ShadeParams, g_cd, g_kdout, g_cs,
                 vis_mask, g_kd, g_korm, g_nrm, g_env, stream=None):
    N, H, W = gb.pos.shape[:3]
    Hp, Wp = probe.env.shape[:2]
    _check(load().mcdi_shade_mc_bwd(C.byref(bvh.view), _ptr(probe.env), Wp, Hp, _ptr(probe.cond), _ptr(probe.marg),
                                    _ptr(probe.total), _ptr(gb.pos), _ptr(gb.nrm), _ptr(gb.kd), _ptr(gb.korm),
                                    _ptr(cams), N, H, W, C.byref(params), _ptr(g_cd), _ptr(g_kdout), _ptr(g_cs),
                                    _ptr(vis_mask), _ptr(g_kd), _ptr(g_korm), _ptr(g_nrm), _ptr(g_env),
                                    _stream(stream)), "shade_mc_bwd")


def shade_mc_bwd_span(bvh: "Bvh", probe: "Probe", gb: "GBuffer", cams, params: ShadeParams, g_cd, g_kdout, g_cs,
                      vis_mask, g_kd, g_korm, g_nrm, g_env, first: int, count: int, stream=None):
    """`shade_mc_bwd` for the pixels [first, first + count) of the flattened [N][H][W] image only."""
    N, H, W = gb.pos.shape[:3]
    Hp, Wp = probe.env.shape[:2]
    _check(load().mcdi_shade_mc_bwd_span(C.byref(bvh.view), _ptr(probe.env), Wp, Hp, _ptr(probe.cond),
                                         _ptr(probe.marg), _ptr(probe.total), _ptr(gb.pos), _ptr(gb.nrm), _ptr(gb.kd),
                                         _ptr(gb.korm), _ptr(cams), N, H, W, C.byref(params), _ptr(g_cd),
                                         _ptr(g_kdout), _ptr(g_cs), _ptr(vis_mask), _ptr(g_kd), _ptr(g_korm),
                                         _ptr(g_nrm), _ptr(g_env), int(first), int(count), _stream(stream)),
           "shade_mc_bwd_span")


def shadow_ray_stats(bvh: "Bvh", N: int, H: int, W: int, params: ShadeParams, workspace, stats, stream=None):
    """Counters of the shadow rays a forward pass left in ``workspace``: stats (5 int64, device) gets
    rays, node visits, triangle tests, rays blocked, rays disagreeing with the forward's hit flag."""
    assert stats.dtype == torch.int64 and stats.numel() >= 5
    _check(load().mcdi_shadow_ray_stats(C.byref(bvh.view), int(N), int(H), int(W), C.byref(params),
                                        _ptr(workspace), workspace.numel() * workspace.element_size(), _ptr(stats),
                                        _stream(stream)), "shadow_ray_stats")


def shadow_ray_retrace(bvh: "Bvh", N: int, H: int, W: int, params: ShadeParams, workspace, stream=None):
    """The forward pass's tracer kernel alone, again over the rays left in ``workspace``."""
    _check(load().mcdi_shadow_ray_retrace(C.byref(bvh.view), int(N), int(H), int(W), C.byref(params),
                                          _ptr(workspace), workspace.numel() * workspace.element_size(),
                                          _stream(stream)), "shadow_ray_retrace")


def read_sweep(buf, passes: int, sink, stream=None):
    """Read all of ``buf`` ``passes`` times with L2-cached 16-byte loads (sink: int32 device scalar)."""
    _check(load().mcdi_read_sweep(_ptr(buf), buf.numel() * buf.element_size(), int(passes), _ptr(sink),
                                  _stream(stream)), "read_sweep")


def denoise_sizes(n_img: int, H: int, W: int, precision: int = BF16):
    a, b, c, d = C.c_size_t(), C.c_size_t(), C.c_size_t(), C.c_size_t()
    _check(load().mcdi_denoise_sizes(int(n_img), int(H), int(W), int(precision), C.byref(a), C.byref(b), C.byref(c),
                                     C.byref(d)), "denoise_sizes")
    return a.value, b.value, c.value, d.value


def denoise_pack_weights(params, weights, stream=None):
    _check(load().mcdi_denoise_pack_weights(_ptr(params), _ptr(weights), _stream(stream)), "denoise_pack_weights")


def denoise_fwd(weights, term, kd, nrm, y, acts, err, stream=None, precision: int = BF16):
    n, H, W = term.shape[:3]
    _check(load().mcdi_denoise_fwd(_ptr(weights), int(precision), n, H, W, _ptr(term), _ptr(kd), _ptr(nrm),
                                   kd.shape[0], _ptr(y), _ptr(acts), acts.numel() * acts.element_size(), _ptr(err),
                                   _stream(stream)), "denoise_fwd")


def denoise_bwd(weights, acts, gy, gx, grad_ws, err, stream=None, precision: int = BF16):
    n, H, W = gy.shape[:3]
    _check(load().mcdi_denoise_bwd(_ptr(weights), int(precision), n, H, W, _ptr(acts),
                                   acts.numel() * acts.element_size(), _ptr(gy), _ptr(gx), _ptr(grad_ws),
                                   grad_ws.numel() * grad_ws.element_size(), _ptr(err), _stream(stream)),
           "denoise_bwd")


def composite(kd_out, den_cd, den_cs, c, stream=None):
    n = kd_out.numel() // 4
    _check(load().mcdi_composite(_ptr(kd_out), _ptr(den_cd), _ptr(den_cs), n, _ptr(c), _stream(stream)), "composite")


def conv3x3_bf16(x, w, bias, y, relu, err, stream=None):
    """x: BF16 [n][cin/8][H][W][8] (8-channel planes), w: [cout][9][cin], y: [n][cout/8][H][W][8]."""
    n, g, H, W, _ = x.shape
    cin = 8 * g
    _check(load().mcdi_conv3x3_bf16(_ptr(x), n, H, W, cin, _ptr(w), _ptr(bias), w.shape[0], int(bool(relu)), _ptr(y),
                                    _ptr(err), _stream(stream)), "conv3x3_bf16")


def conv3x3_wgrad_bytes(n: int, H: int, W: int, cin_pad: int, cout_pad: int) -> int:
    b = C.c_size_t()
    _check(load().mcdi_conv3x3_wgrad_bytes(int(n), int(H), int(W), int(cin_pad), int(cout_pad), C.byref(b)),
           "conv3x3_wgrad_bytes")
    return b.value


def conv3x3_wgrad(x, g, cin: int, cout: int, gw, scratch, err, stream=None):
    """x: BF16 [n][cin_pad/8][H][W][8], g: BF16 [n][cout_pad/8][H][W][8] -> gw (float32,
    cout*cin*9 + cout): dW[co][ci][3][3] then db[co]."""
    n, gx_, H, W, _ = x.shape
    _check(load().mcdi_conv3x3_wgrad(_ptr(x), _ptr(g), n, H, W, 8 * gx_, 8 * g.shape[1], int(cin), int(cout), _ptr(gw),
                                     _ptr(scratch), scratch.numel() * scratch.element_size(), _ptr(err),
                                     _stream(stream)), "conv3x3_wgrad")


def bilateral_fwd(gb_pos, gb_nrm, cams, c_in, sigma, c_out, wsum, radius=-1, stream=None):
    """Cross-bilateral filter of the [n_img][H][W] float4 batch c_in with the guides of
    N views (image i uses view i % N); wsum [N][H][W] float32 receives W(p)."""
    N, H, W = gb_pos.shape[:3]
    _check(load().mcdi_bilateral_fwd(_ptr(gb_pos), _ptr(gb_nrm), _ptr(cams), N, H, W, c_in.shape[0], _ptr(c_in),
                                     float(sigma), int(radius), _ptr(c_out), _ptr(wsum), _stream(stream)),
           "bilateral_fwd")


def bilateral_bwd(gb_pos, gb_nrm, cams, wsum, g_out, sigma, g_in, radius=-1, stream=None):
    N, H, W = gb_pos.shape[:3]
    _check(load().mcdi_bilateral_bwd(_ptr(gb_pos), _ptr(gb_nrm), _ptr(cams), N, H, W, g_out.shape[0], _ptr(wsum),
                                     _ptr(g_out), float(sigma), int(radius), _ptr(g_in), _stream(stream)),
           "bilateral_bwd")


def image_loss_workspace_size(n: int) -> int:
    b = C.c_size_t()
    _check(load().mcdi_image_loss_workspace_size(int(n), C.byref(b)), "image_loss_workspace_size")
    return b.value


def image_loss(kd_out, den_cd, den_cs, ref, loss, g_kdout, g_dcd, g_dcs, workspace, lambda_light=0.15, c=None,
               stream=None):
    """Fused composite + tonemapped L1 image loss + lighting regulariser and its adjoint.
    float4 planes of n pixels; loss: device float64 (3,) = (L, L_image, L_light)."""
    n = kd_out.numel() // 4
    _check(load().mcdi_image_loss(_ptr(kd_out), _ptr(den_cd), _ptr(den_cs), _ptr(ref), n, float(lambda_light),
                                  _ptr(c), _ptr(loss), _ptr(g_kdout), _ptr(g_dcd), _ptr(g_dcs), _ptr(workspace),
                                  workspace.numel() * workspace.element_size(), _stream(stream)), "image_loss")


def conv3x3_e4m3(x, w, x_amax, w_amax, bias, y, relu, err, stream=None):
    """x: E4M3 codes (uint8) [n][cin/16][H][W][16], w: codes [cout][9][cin], x_amax / w_amax: device float32
    scalars, y: BF16 [n][cout/8][H][W][8]."""
    n, g, H, W, _ = x.shape
    _check(load().mcdi_conv3x3_e4m3(_ptr(x), n, H, W, 16 * g, _ptr(w), _ptr(x_amax), _ptr(w_amax), _ptr(bias),
                                    w.shape[0], int(bool(relu)), _ptr(y), _ptr(err), _stream(stream)), "conv3x3_e4m3")



def denoise_wgrad_bytes(n_img: int, H: int, W: int) -> int:
    b = C.c_size_t()
    _check(load().mcdi_denoise_wgrad_bytes(int(n_img), int(H), int(W), C.byref(b)), "denoise_wgrad_bytes")
    return b.value


def denoise_wgrad(acts, grad_ws, gw, scratch, err, n_img: int, H: int, W: int, stream=None, precision: int = BF16):
    """gw (device float32, n_params) = the weight and bias gradients of the 15 convolutions, after
    denoise_fwd (acts) and denoise_bwd (grad_ws) of the same images."""
    _check(load().mcdi_denoise_wgrad(int(precision), int(n_img), int(H), int(W), _ptr(acts),
                                     acts.numel() * acts.element_size(), _ptr(grad_ws),
                                     grad_ws.numel() * grad_ws.element_size(), _ptr(gw), _ptr(scratch),
                                     scratch.numel() * scratch.element_size(), _ptr(err), _stream(stream)),
           "denoise_wgrad")


UNET_PLAN = [("enc1a", 9, 32), ("enc1b", 32, 32), ("enc2a", 32, 48), ("enc2b", 48, 48), ("enc3a", 48, 64),
             ("enc3b", 64, 64), ("bot_a", 64, 96), ("bot_b", 96, 96), ("dec3a", 160, 64), ("dec3b", 64, 64),
             ("dec2a", 112, 48), ("dec2b", 48, 48), ("dec1a", 80, 32), ("dec1b", 32, 32), ("out", 32, 3)]


def flatten_unet_params(weights: dict):
    """{name: (W (co, ci, 3, 3), b (co,))} -> one float32 vector in the library's order."""
    import numpy as np

    parts = []
    for name, ci, co in UNET_PLAN:
        W, b = weights[name]
        assert tuple(W.shape) == (co, ci, 3, 3) and tuple(b.shape) == (co,)
        parts += [np.asarray(W, np.float32).ravel(), np.asarray(b, np.float32).ravel()]
    return np.concatenate(parts)


class Denoiser:
    """Device-resident denoiser for n_img images of H x W: packed weights, saved
    activations, gradient scratch and the error word."""

    def __init__(self, params_flat, n_img: int, H: int, W: int, device="cuda", precision: int = BF16):
        wb, ab, gb, n_params = denoise_sizes(n_img, H, W, precision)
        self.precision = precision
        p = torch.as_tensor(params_flat, dtype=torch.float32, device=device).contiguous()
        assert p.numel() == n_params, (p.numel(), n_params)
        self.n_img, self.H, self.W = n_img, H, W
        self.weights = _empty_bytes(wb, device)
        self.acts = _empty_bytes(ab, device)
        self.grad_ws = _empty_bytes(gb, device)
        self.err = torch.zeros(1, dtype=torch.int32, device=device)
        denoise_pack_weights(p, self.weights)
        self._params = p

    def forward(self, term, kd, nrm, y, stream=None):
        denoise_fwd(self.weights, term, kd, nrm, y, self.acts, self.err, stream, self.precision)

    def backward(self, gy, gx, stream=None):
        denoise_bwd(self.weights, self.acts, gy, gx, self.grad_ws, self.err, stream, self.precision)

    def weight_grad(self, gw=None, stream=None):
        """The gradient of the parameters (float32, the order of flatten_unet_params) for the
        last forward/backward pair; the scratch is allocated on first use."""
        if getattr(self, "wgrad_ws", None) is None:
            self.wgrad_ws = _empty_bytes(denoise_wgrad_bytes(self.n_img, self.H, self.W), self.weights.device)
        if gw is None:
            gw = torch.empty(self._params.numel(), dtype=torch.float32, device=self.weights.device)
        denoise_wgrad(self.acts, self.grad_ws, gw, self.wgrad_ws, self.err, self.n_img, self.H, self.W, stream,
                      self.precision)
        return gw


def unflatten_unet_params(flat):
    """One vector in the library's order -> {name: (W (co, ci, 3, 3), b (co,))} (views for tensors)."""
    out, o = {}, 0
    for name, ci, co in UNET_PLAN:
        n = co * ci * 9
        out[name] = (flat[o:o + n].reshape(co, ci, 3, 3), flat[o + n:o + n + co])
        o += n + co
    return out


class denoise_plan_recorder:
    """Context manager: records the launch plan of every convolution the denoiser
    launches from this thread inside the block; ``records`` then holds one dict per
    convolution (pass, conv, level, rows_form, rows, mask_prefetch, pool_fused, e4m3)."""

    KEYS = ("pass", "conv", "level", "rows_form", "rows", "mask_prefetch", "pool_fused", "e4m3")

    def __init__(self, cap: int = 256):
        self.cap = cap
        self.buf = (C.c_int * (8 * cap))()
        self.count = C.c_int(0)
        self.records = []

    def __enter__(self):
        _check(load().mcdi_denoise_record_plan(C.addressof(self.buf), self.cap, C.addressof(self.count)),
               "denoise_record_plan")
        return self

    def __exit__(self, *exc):
        load().mcdi_denoise_record_plan(None, 0, None)
        n = self.count.value
        self.records = [dict(zip(self.KEYS, self.buf[8 * k: 8 * k + 8])) for k in range(n)]


class Denoise(torch.autograd.Function):
    """y = Denoise.apply(term, kd, nrm, denoiser): the U-Net on n_img noisy terms with
    k_d,out and normal guides (image i uses the guides of image i % n_aux).

    Differentiable with respect to the noisy terms only (Sec. 4.2: the gradient
    reaches the shading through the denoiser's input; its weights are locked and
    the guides are constants).  The saved activations live in the Denoiser, so a
    second forward through the same Denoiser before this backward overwrites them.
    """

    @staticmethod
    def forward(ctx, term, kd, nrm, denoiser: "Denoiser"):
        y = torch.empty_like(term)
        denoiser.forward(term.contiguous(), kd.contiguous(), nrm.contiguous(), y)
        ctx.denoiser = denoiser
        return y

    @staticmethod
    def backward(ctx, gy):
        gx = torch.empty_like(gy)
        ctx.denoiser.backward(gy.contiguous(), gx)
        return gx, None, None, None


# ------------------------------------------------------------------ device-resident objects
def edge_table_workspace_size(n_tris: int) -> int:
    b = C.c_size_t()
    _check(load().mcdi_edge_table_workspace_size(int(n_tris), C.byref(b)), "edge_table_workspace_size")
    return b.value


def build_edge_table(tris, edges, n_edges, workspace, stream=None):
    """tris (T, 3) int32 -> edges (3T, 4) int32 records (a, b, c1, c2) in first-half-edge order, n_edges (1,) int32."""
    _check(load().mcdi_build_edge_table(_ptr(tris), tris.shape[0], _ptr(edges), _ptr(n_edges), _ptr(workspace),
                                        workspace.numel() * workspace.element_size(), _stream(stream)),
           "build_edge_table")


def shadow_edge_grad(bvh: "Bvh", verts, edges: "EdgeTable", probe: "Probe", gb: "GBuffer", cams, params: ShadeParams,
                     n_edge_samples: int, g_cd, g_cs, g_verts, sample_w=None, eta=1e-4, stream=None):
    """Edge-sampling estimate of the shadow-visibility gradient, ACCUMULATED into g_verts (V, 3) float32."""
    N, H, W = gb.pos.shape[:3]
    Hp, Wp = probe.env.shape[:2]
    _check(load().mcdi_shadow_edge_grad(C.byref(bvh.view), _ptr(verts), verts.shape[0], _ptr(edges.records),
                                        _ptr(edges.count), edges.records.shape[0], _ptr(probe.env), Wp, Hp,
                                        _ptr(gb.pos), _ptr(gb.nrm), _ptr(gb.kd), _ptr(gb.korm), _ptr(cams), N, H, W,
                                        C.byref(params), int(n_edge_samples), float(eta), _ptr(g_cd), _ptr(g_cs),
                                        _ptr(g_verts), _ptr(sample_w), _stream(stream)), "shadow_edge_grad")


@dataclass
class EdgeTable:
    records: torch.Tensor    # (3 T, 4) int32
    count: torch.Tensor      # (1,) int32, on the device
    workspace: torch.Tensor

    @classmethod
    def allocate(cls, n_tris: int, device="cuda") -> "EdgeTable":
        return cls(torch.empty(3 * n_tris, 4, dtype=torch.int32, device=device),
                   torch.zeros(1, dtype=torch.int32, device=device),
                   _empty_bytes(edge_table_workspace_size(n_tris), device))

    def build(self, tris, stream=None) -> "EdgeTable":
        build_edge_table(tris, self.records, self.count, self.workspace, stream)
        return self


def _empty_bytes(n: int, device) -> torch.Tensor:
    # 256-byte aligned raw buffer
    return torch.empty((max(n, 1) + 255) // 256 * 256, dtype=torch.uint8, device=device)


@dataclass
class Bvh:
    nodes: torch.Tensor
    tri_records: torch.Tensor
    scratch: torch.Tensor
    n_tris: int

    @property
    def view(self) -> BvhView:
        return BvhView(self.nodes.data_ptr(), self.tri_records.data_ptr(), self.n_tris)

    @classmethod
    def allocate(cls, n_tris: int, device="cuda") -> "Bvh":
        nb, tb, sb = bvh_sizes(n_tris)
        return cls(_empty_bytes(nb, device), _empty_bytes(tb, device), _empty_bytes(sb, device), n_tris)

    def build(self, verts, tris, stream=None) -> "Bvh":
        build_bvh(verts, tris, self.nodes, self.tri_records, self.scratch, stream)
        return self

    def refit(self, verts, tris, stream=None) -> "Bvh":
        """New vertex positions, the triangles of the last build: boxes only."""
        refit_bvh(verts, tris, self.nodes, self.tri_records, self.scratch, stream)
        return self


@dataclass
class Probe:
    env: torch.Tensor    # (Hp, Wp, 4) float32
    cond: torch.Tensor   # (Hp, Wp + 1) float32
    marg: torch.Tensor   # (Hp + 1,) float32
    row_sum: torch.Tensor
    total: torch.Tensor  # (1,) float64

    @classmethod
    def allocate(cls, env: torch.Tensor) -> "Probe":
        Hp, Wp = env.shape[:2]
        dev = env.device
        return cls(env, torch.empty(Hp, Wp + 1, device=dev), torch.empty(Hp + 1, device=dev),
                   torch.empty(Hp, dtype=torch.float64, device=dev), torch.empty(1, dtype=torch.float64, device=dev))

    def build(self, stream=None) -> "Probe":
        build_envmap_cdf(self.env, self.cond, self.marg, self.row_sum, self.total, stream)
        return self


@dataclass
class GBuffer:
    pos: torch.Tensor   # (N, H, W, 4)
    nrm: torch.Tensor
    kd: torch.Tensor
    korm: torch.Tensor

    @classmethod
    def allocate(cls, N, H, W, device="cuda") -> "GBuffer":
        return cls(*[torch.empty(N, H, W, 4, device=device) for _ in range(4)])


def make_params(n_light, n_cos, n_ggx, seed, tau=1.0, ray_eps=1e-4, decorrelate_bwd=False) -> ShadeParams:
    """Shading parameters; tau = 1 is binary visibility, where the paper's leakage ramp ends (App. A)."""
    return ShadeParams(int(n_light), int(n_cos), int(n_ggx), int(bool(decorrelate_bwd)), int(seed), float(tau),
                       float(ray_eps))


class ShadeMC(torch.autograd.Function):
    """c_d, kd_out, c_s = ShadeMC.apply(kd, korm, nrm, env, ctx_objects...)

    Differentiable with respect to the G-buffer k_d, k_orm and normal planes and
    the probe texels; the sampling tables, positions and BVH are constants.
    """

    @staticmethod
    def forward(ctx, kd, korm, nrm, env, pos, bvh, probe, cams, params, keep_mask=True, workspace=None):
        gb = GBuffer(pos.contiguous(), nrm.contiguous(), kd.contiguous(), korm.contiguous())
        pr = Probe(env.contiguous(), probe.cond, probe.marg, probe.row_sum, probe.total)
        N, H, W = pos.shape[:3]
        spp = params.n_light + params.n_cos + params.n_ggx
        c_d, kd_out, c_s = (torch.empty_like(pos) for _ in range(3))
        mask = torch.empty(N, H, W, (spp + 31) // 32, dtype=torch.int32, device=pos.device) if keep_mask else None
        shade_mc_fwd(bvh, pr, gb, cams, params, c_d, kd_out, c_s, mask, workspace)
        ctx.bvh, ctx.probe, ctx.params, ctx.gb = bvh, pr, params, gb
        ctx.save_for_backward(cams, mask if mask is not None else torch.empty(0, device=pos.device))
        ctx.has_mask = mask is not None
        return c_d, kd_out, c_s

    @staticmethod
    def backward(ctx, g_cd, g_kdout, g_cs):
        cams, mask = ctx.saved_tensors
        gb = ctx.gb
        zeros = None
        if g_cd is None or g_kdout is None or g_cs is None:
            zeros = torch.zeros_like(gb.pos)
        g_cd = (g_cd if g_cd is not None else zeros).contiguous()
        g_kdout = (g_kdout if g_kdout is not None else zeros).contiguous()
        g_cs = (g_cs if g_cs is not None else zeros).contiguous()
        g_kd, g_korm, g_nrm = (torch.empty_like(gb.pos) for _ in range(3))
        g_env = torch.zeros_like(ctx.probe.env)
        shade_mc_bwd(ctx.bvh, ctx.probe, gb, cams, ctx.params, g_cd, g_kdout, g_cs, mask if ctx.has_mask else None,
                     g_kd, g_korm, g_nrm, g_env)
        return g_kd, g_korm, g_nrm, g_env, None, None, None, None, None, None, None
