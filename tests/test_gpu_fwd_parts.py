"""The shading forward in two calls (mcdi_shade_mc_fwd_part: sample
generation, then shadow rays and accumulation on the same workspace) gives
bitwise the outputs of the single call, also when the generation runs on a
forked stream while the BVH is built on another (pipeline.geometry_and_forward
launched kernel by kernel).  Likewise the rasterised G-buffer in two calls
(mcdi_raster_gbuffer_part: depth from the mesh, then the resolve that reads
the textures), also with the textures written only between the two and with
packed RGB textures, and the
adjoint over disjoint pixel spans (mcdi_shade_mc_bwd_span): per-pixel
gradients bitwise those of one call, the probe gradient (summed by atomics in
no fixed order) to 1e-5 of its largest entry."""
import numpy as np
import pytest
import torch

from paper_2206_03380_gb300 import scenes

pytestmark = pytest.mark.gpu


def _outs(pipe):
    return [t.clone() for t in (pipe.c_d, pipe.kd_out, pipe.c_s, pipe.mask)]


def test_forward_parts_match_the_single_call(cuda_lib):
    from paper_2206_03380_gb300.pipeline import ShadingPipeline

    sc = scenes.parity_scene()
    pipe = ShadingPipeline(sc)
    pipe.overlap_generation = False
    pipe.tables_and_geometry()
    pipe.forward()
    torch.cuda.synchronize()
    ref = _outs(pipe)
    assert float(ref[0].abs().max()) > 0
    for t in (pipe.c_d, pipe.kd_out, pipe.c_s, pipe.mask):
        t.zero_()
    pipe.forward_part(1)
    pipe.forward_part(2)
    torch.cuda.synchronize()
    for a, b in zip(ref, _outs(pipe)):
        assert torch.equal(a, b)
    # the overlapped schedule: generation beside the BVH build, on other streams
    for t in (pipe.c_d, pipe.kd_out, pipe.c_s, pipe.mask):
        t.zero_()
    pipe.bvh.nodes.zero_()
    pipe.overlap_generation = True
    pipe.geometry_and_forward()
    torch.cuda.synchronize()
    for a, b in zip(ref, _outs(pipe)):
        assert torch.equal(a, b)


def test_forward_part_rejects_a_bad_part(cuda_lib):
    from paper_2206_03380_gb300.pipeline import ShadingPipeline

    pipe = ShadingPipeline(scenes.parity_scene())
    with pytest.raises(cuda_lib.McdiError) as e:
        pipe.forward_part(3)
    assert e.value.status == cuda_lib.INVALID_ARG


def _gb(pipe):
    return [t.clone() for t in (pipe.gb.pos, pipe.gb.nrm, pipe.gb.kd, pipe.gb.korm)]


def test_raster_parts_match_the_single_call(cuda_lib):
    from paper_2206_03380_gb300.pipeline import ShadingPipeline

    pipe = ShadingPipeline(scenes.parity_scene())
    assert pipe.raster_ws is not None
    pipe.primary()
    torch.cuda.synchronize()
    ref = _gb(pipe)
    assert float(ref[0][..., 3].sum()) > 0 and float(ref[2].abs().max()) > 0
    tex = pipe.tex_kd.clone(), pipe.tex_korm.clone()
    for t in (pipe.gb.pos, pipe.gb.nrm, pipe.gb.kd, pipe.gb.korm, pipe.tex_kd, pipe.tex_korm):
        t.zero_()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    pipe.primary_part(1, side)  # the depth pass reads no texture
    torch.cuda.current_stream().wait_stream(side)
    pipe.tex_kd.copy_(tex[0])
    pipe.tex_korm.copy_(tex[1])
    pipe.primary_part(2)
    torch.cuda.synchronize()
    for a, b in zip(ref, _gb(pipe)):
        assert torch.equal(a, b)
    # packed RGB textures (the 4th channel dropped): the same G-buffer bit for bit
    tex3 = [t[..., :3].contiguous() for t in tex]
    for t in (pipe.gb.pos, pipe.gb.nrm, pipe.gb.kd, pipe.gb.korm):
        t.zero_()
    cuda_lib.raster_gbuffer_part(pipe.verts, pipe.vnrm, pipe.tris, pipe.cams, pipe.H, pipe.W, tex3[0], tex3[1],
                                 pipe.uvmap, pipe.gb, pipe.raster_ws, 1)
    cuda_lib.raster_gbuffer_part(pipe.verts, pipe.vnrm, pipe.tris, pipe.cams, pipe.H, pipe.W, tex3[0], tex3[1],
                                 pipe.uvmap, pipe.gb, pipe.raster_ws, 2)
    torch.cuda.synchronize()
    for a, b in zip(ref, _gb(pipe)):
        assert torch.equal(a, b)
    with pytest.raises(cuda_lib.McdiError) as e:
        pipe.primary_part(0)
    assert e.value.status == cuda_lib.INVALID_ARG


def test_adjoint_spans_match_the_single_call(cuda_lib):
    from paper_2206_03380_gb300.pipeline import ShadingPipeline

    sc = scenes.parity_scene()
    pipe = ShadingPipeline(sc)
    pipe.tables_and_geometry()
    pipe.forward()
    rng = np.random.default_rng(5)
    g = [torch.from_numpy(rng.normal(size=pipe.c_d.shape).astype(np.float32)).cuda() for _ in range(3)]
    pipe.backward(*g)
    torch.cuda.synchronize()
    outs = (pipe.g_kd, pipe.g_korm, pipe.g_nrm, pipe.g_env)
    ref = [t.clone() for t in outs]
    assert float(ref[0].abs().max()) > 0 and float(ref[3].abs().max()) > 0
    for t in outs:
        t.fill_(float("nan"))
    pipe.g_env.zero_()
    P = pipe.c_d.shape[0] * pipe.c_d.shape[1] * pipe.c_d.shape[2]
    cuts = [0, 37, P // 3, P // 3, P - 1, P]  # ragged spans, an empty one, a single pixel
    for a, b in zip(cuts[:-1], cuts[1:]):
        pipe.backward_span(*g, a, b - a)
    torch.cuda.synchronize()
    for a, b in zip(ref[:3], outs[:3]):
        assert torch.equal(a, b)
    torch.testing.assert_close(outs[3], ref[3], rtol=0, atol=1e-5 * float(ref[3].abs().max()))
    for first, count in ((P, 1), (-1, 2), (0, -1), (P - 3, 4)):
        with pytest.raises(cuda_lib.McdiError) as e:
            pipe.backward_span(*g, first, count)
        assert e.value.status == cuda_lib.INVALID_ARG
