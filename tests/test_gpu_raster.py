"""The rasterised G-buffer (mcdi_raster_gbuffer; the paper rasterises primary
visibility, Sec. 3.1) against the closest-hit ray cast, whose FP32 camera-ray /
triangle test it reuses for every pixel it covers: both must find the same
triangle at the same depth, so their G-buffers agree bit for bit except where
two triangles give the very same FP32 depth (the two break such ties
differently).  Covered: the headline mesh at 512², several ragged views, a
view with geometry behind the eye (near-plane clipping), and one triangle that
covers thousands of pixels (the warp-wide path for large screen boxes)."""
import numpy as np
import pytest
import torch

from paper_2206_03380_gb300 import scenes

pytestmark = pytest.mark.gpu


def _gbuffers(sc):
    from paper_2206_03380_gb300.pipeline import ShadingPipeline

    out = []
    for raster in (True, False):
        pipe = ShadingPipeline(sc, raster=raster)
        pipe.build_bvh()
        pipe.primary()
        torch.cuda.synchronize()
        out.append(torch.cat([pipe.gb.pos, pipe.gb.nrm, pipe.gb.kd, pipe.gb.korm], -1).reshape(-1, 16).cpu().numpy())
    return out


def _agree(r, c, max_ties):
    same = np.all(r.view(np.int32) == c.view(np.int32), axis=1)
    diff = ~same
    assert diff.sum() <= max_ties, diff.sum()
    # a tie: both covered, the same point along the ray (positions agree to rounding)
    both = (r[diff, 3] > 0) & (c[diff, 3] > 0)
    assert np.all(both)
    assert np.abs(r[diff, 0:3] - c[diff, 0:3]).max(initial=0.0) < 1e-4
    return same.mean()


def test_raster_equals_ray_cast_headline(cuda_lib):
    sc = scenes.sphere_union_scene()
    r, c = _gbuffers(sc)
    cov = (c[:, 3] > 0).mean()
    assert 0.2 < cov < 0.95
    assert _agree(r, c, max_ties=int(1e-4 * len(r)) + 2) > 0.9999


def test_raster_equals_ray_cast_ragged_views_and_near_plane(cuda_lib):
    base = scenes.parity_scene()
    # three views of odd sizes; the ground reaches behind the eye in each (clipped at the near plane)
    cams = np.stack([scenes.look_at((0.0, 0.0, 3.0), (0, 0, 0), (0, 1, 0), 45.0, 53 / 37),
                     scenes.look_at((2.5, 0.4, 1.5), (0, -0.3, 0), (0, 1, 0), 60.0, 53 / 37),
                     scenes.look_at((-0.5, -0.6, 2.0), (0.2, -1.0, -1.0), (0, 1, 0), 70.0, 53 / 37)])
    sc = scenes.Scene(**{**base.__dict__, "cams": cams.astype(np.float32), "width": 53, "height": 37})
    r, c = _gbuffers(sc)
    assert (c[:, 3] > 0).sum() > 1000
    _agree(r, c, max_ties=4)


def test_raster_large_triangle(cuda_lib):
    base = scenes.parity_scene(seed=scenes.BASE_SEED + 13)
    verts = np.array([[-3, -1, -3], [3, -1, -3], [0, -1, 4]], np.float32)
    tris = np.array([[0, 1, 2]], np.int32)
    vn = np.tile(np.array([[0, 1, 0]], np.float32), (3, 1))
    cam = scenes.look_at((0, 2.0, 3.0), (0, -1, 0), (0, 1, 0), 45.0, 1.0)[None]
    sc = scenes.Scene(**{**base.__dict__, "verts": verts, "vnrm": vn, "tris": tris, "cams": cam})
    r, c = _gbuffers(sc)
    assert (r[:, 3] > 0).sum() > 1000  # far more than the per-thread limit of 64 pixels
    assert np.array_equal(r.view(np.int32), c.view(np.int32))
