"""The optimisation-step batch: 8 of 200 views at 800 x 800, 32 spp (16 light /
8 cosine / 8 GGX), the ~1.3M-triangle union of 32 spheres and 32 boxes
(256^3 grid), 2048^2 textures, a 1024 x 512 probe; the whole step - tables,
BVH, G-buffer, forward, BF16 denoiser forward and input gradient, adjoint -
captured in one CUDA graph and replayed.  The oracle recomputes sampled
pixels of two views one by one (its own G-buffer rows, brute-force visibility
over every triangle)."""
import numpy as np
import pytest
import torch

from paper_2206_03380_gb300 import scenes
from tests import parity_util as PU
from tests.test_gpu_shading import to_np

pytestmark = pytest.mark.gpu

N_PER_VIEW = 40


def test_graph_step_batch_matches_oracle_on_sampled_pixels(cuda_lib, orc):
    from paper_2206_03380_gb300.pipeline import ShadingPipeline

    sc = scenes.union_step_scene()
    assert sc.tris.shape[0] > 1_000_000 and sc.cams.shape[0] == 8 and sc.spp == 32
    den = cuda_lib.flatten_unet_params(scenes.unet_xavier_weights(scenes.BASE_SEED + 3))
    pipe = ShadingPipeline(sc, denoiser_params=den)
    N, H, W = pipe.N, pipe.H, pipe.W
    rng = np.random.default_rng(41)
    g = [torch.from_numpy(rng.normal(size=(N, H, W, 4)).astype(np.float32)).cuda() for _ in range(3)]
    pipe.capture(*g)
    pipe.replay()
    torch.cuda.synchronize()
    assert pipe.denoiser.err.item() == 0
    assert torch.isfinite(pipe.denoised).all() and torch.isfinite(pipe.g_nrm).all()
    gb = np.concatenate([to_np(pipe.gb.pos), to_np(pipe.gb.nrm), to_np(pipe.gb.kd), to_np(pipe.gb.korm)],
                        -1).reshape(N, H * W, 16)
    out = np.concatenate([to_np(pipe.c_d), to_np(pipe.kd_out), to_np(pipe.c_s)], -1).reshape(N, H * W, 12)
    masks = to_np(pipe.mask).reshape(N, H * W, -1)
    n_bad = n_act = n_mism = 0
    for view in (0, 5):
        covered = np.nonzero(gb[view, :, 3] > 0)[0]
        assert 0.1 * H * W < len(covered) < 0.95 * H * W
        pix = np.sort(rng.choice(covered, size=N_PER_VIEW, replace=False))
        og = orc.primary_cast(sc.verts, sc.vnrm, sc.tris, sc.cams[view], W, H, pix, sc.tex_kd, sc.tex_korm,
                              sc.uvmap)
        gg = gb[view, pix]
        same = (og[:, 3] > 0) & (np.abs(og[:, 0:3] - gg[:, 0:3]).max(1) < 1e-4)
        assert same.sum() >= N_PER_VIEW - 2
        np.testing.assert_allclose(gg[same][:, 4:7], og[same][:, 4:7], atol=5e-5)
        pix, og = pix[same], og[same]
        o_out, o_vis, recs = PU.oracle_shade(orc, sc, og.astype(np.float32), pix, view)
        gout = out[view, pix][:, [0, 1, 2, 4, 5, 6, 8, 9, 10]]
        np.testing.assert_allclose(gout[:, 3:6], o_out[:, 3:6], rtol=1e-4, atol=1e-6)
        for sl in (slice(0, 3), slice(6, 9)):
            bad, marginal, err = PU.compare_radiance(gout[:, sl], o_out[:, sl], recs)
            assert not (bad & ~marginal).any(), (err[bad & ~marginal], pix[bad & ~marginal])
            n_bad += bad.sum()
        act = recs["active"].astype(bool)
        mism = (PU.mask_bits(masks[view, pix], sc.spp) != PU.mask_bits(o_vis, sc.spp)) & act
        assert np.all(recs["margin"][mism] < PU.MARGIN)
        n_act += act.sum()
        n_mism += mism.sum()
    assert n_bad <= 2 and n_mism <= max(1, 1e-4 * n_act)
