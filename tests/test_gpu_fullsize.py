"""GPU parity at the headline size, in the launch configuration the benchmark
times: 512 x 512, 16 spp (8 light / 4 cosine / 4 GGX), the ~198k-triangle
sphere-union mesh, 1024^2 textures and the 512 x 256 three-lobe probe.  The
whole step (probe tables, BVH, G-buffer, forward, adjoint) runs on the GPU;
the oracle recomputes a seeded sample of pixels one by one (its own G-buffer
rows, brute-force visibility over every triangle) and the adjoint with the
upstream gradient restricted to those pixels."""
import numpy as np
import pytest
import torch

from paper_2206_03380_gb300 import scenes
from tests import parity_util as PU
from tests.test_gpu_shading import check_adjoint, to_np

pytestmark = pytest.mark.gpu

N_SAMPLE = 192


@pytest.fixture(scope="module")
def headline():
    return scenes.sphere_union_scene()


def test_fullsize_step_matches_oracle_on_sampled_pixels(cuda_lib, orc, headline):
    from paper_2206_03380_gb300.pipeline import ShadingPipeline

    sc = headline
    pipe = ShadingPipeline(sc)
    W = H = sc.width
    zeros = torch.zeros(1, H, W, 4, device="cuda")
    pipe.step(zeros, zeros, zeros)  # warm: whole step exactly as timed
    gpos = to_np(pipe.gb.pos).reshape(-1, 4)
    covered = np.nonzero(gpos[:, 3] > 0)[0]
    assert 0.2 * W * H < len(covered) < 0.95 * W * H
    rng = np.random.default_rng(77)
    pix = np.sort(rng.choice(covered, size=N_SAMPLE, replace=False))
    og = orc.primary_cast(sc.verts, sc.vnrm, sc.tris, sc.cams[0], W, H, pix, sc.tex_kd, sc.tex_korm, sc.uvmap)
    gg = np.concatenate([to_np(pipe.gb.pos), to_np(pipe.gb.nrm), to_np(pipe.gb.kd), to_np(pipe.gb.korm)],
                        -1).reshape(-1, 16)[pix]
    same = (og[:, 3] > 0) & (np.abs(og[:, 0:3] - gg[:, 0:3]).max(1) < 1e-4)
    assert same.sum() >= N_SAMPLE - 2
    np.testing.assert_allclose(gg[same][:, 4:7], og[same][:, 4:7], atol=5e-5)
    np.testing.assert_allclose(gg[same][:, 8:15], og[same][:, 8:15], atol=1e-5)
    pix, og = pix[same], og[same]
    rows = og.astype(np.float32)
    o_out, o_vis, recs = PU.oracle_shade(orc, sc, rows, pix, 0)
    gout = np.concatenate([to_np(pipe.c_d), to_np(pipe.kd_out), to_np(pipe.c_s)], -1).reshape(-1, 12)[pix]
    gout = gout[:, [0, 1, 2, 4, 5, 6, 8, 9, 10]]
    np.testing.assert_allclose(gout[:, 3:6], o_out[:, 3:6], rtol=1e-4, atol=1e-6)
    n_bad = 0
    bad_px = np.zeros(len(pix), bool)
    for sl in (slice(0, 3), slice(6, 9)):
        bad, marginal, err = PU.compare_radiance(gout[:, sl], o_out[:, sl], recs)
        assert not (bad & ~marginal).any(), (err[bad & ~marginal], pix[bad & ~marginal])
        n_bad += bad.sum()
        bad_px |= bad
    assert n_bad <= 3
    gbits = PU.mask_bits(to_np(pipe.mask).reshape(W * H, -1)[pix], sc.spp)
    obits = PU.mask_bits(o_vis, sc.spp)
    act = recs["active"].astype(bool)
    mism = (gbits != obits) & act
    assert mism.sum() <= max(1, 1e-4 * act.sum())
    assert np.all(recs["margin"][mism] < PU.MARGIN)
    assert recs["occluded"].sum() > 0.05 * act.sum()
    lo, hi = PU.flipped_samples(gbits, obits, act, bad_px, recs["margin"])
    print(f"headline flipped samples: {lo} (at most {hi}) of {int(act.sum())} active")

    # adjoint: upstream nonzero only on the sampled, non-marginal pixels
    marginal = (recs["margin"] < PU.MARGIN).any(1)
    g = rng.normal(size=(len(pix), 9)).astype(np.float32).astype(np.float64)
    g[marginal] = 0.0
    full = np.zeros((W * H, 12), np.float32)
    full[pix, 0:3], full[pix, 4:7], full[pix, 8:11] = g[:, 0:3], g[:, 3:6], g[:, 6:9]
    ft = torch.from_numpy(full).cuda().reshape(1, H, W, 12)
    pipe.backward(ft[..., 0:4].contiguous(), ft[..., 4:8].contiguous(), ft[..., 8:12].contiguous())
    check_adjoint(orc, sc, pipe, rows, recs, o_out, pix, 0, g)
