"""The cross-bilateral denoiser (App. B) against its oracle: forward, the saved
weight sums and the colour adjoint, on G-buffers the oracle rendered itself
(two views, two images per view), plus the identity limit."""
import numpy as np
import pytest
import torch

from oracle import bilateral_ref as B
from paper_2206_03380_gb300 import scenes

pytestmark = pytest.mark.gpu

H, W = 40, 48


@pytest.fixture(scope="module")
def guides(orc):
    sc = scenes.parity_scene()
    cams = np.stack([sc.cams[0], scenes.look_at((1.2, 0.8, 2.6), (0, -0.3, 0), (0, 1, 0), 45.0, W / H)])
    cams[0] = scenes.look_at((0, 0, 3), (0, 0, 0), (0, 1, 0), 45.0, W / H)
    pix = np.arange(H * W)
    rows = [orc.primary_cast(sc.verts, sc.vnrm, sc.tris, c, W, H, pix, sc.tex_kd, sc.tex_korm, sc.uvmap) for c in cams]
    pos = np.stack([r[:, 0:4] for r in rows]).reshape(2, H, W, 4).astype(np.float32)
    nrm = np.stack([r[:, 4:8] for r in rows]).reshape(2, H, W, 4).astype(np.float32)
    assert 0.2 < (pos[..., 3] > 0).mean() < 0.99
    return pos, nrm, cams.astype(np.float32)


@pytest.mark.parametrize("sigma,radius", [(1.5, -1), (2.0, 3)])
def test_bilateral_matches_oracle(cuda_lib, guides, sigma, radius):
    mcdi = cuda_lib
    pos, nrm, cams = guides
    rng = np.random.default_rng(int(sigma * 10))
    c = rng.lognormal(0, 1, size=(4, H, W, 4)).astype(np.float32)
    g = rng.normal(size=(4, H, W, 4)).astype(np.float32)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    out = torch.full((4, H, W, 4), float("nan"), device="cuda")
    gin = torch.full((4, H, W, 4), float("nan"), device="cuda")
    wsum = torch.zeros((2, H, W), device="cuda")
    mcdi.bilateral_fwd(t(pos), t(nrm), t(cams), t(c), sigma, out, wsum, radius=radius)
    mcdi.bilateral_bwd(t(pos), t(nrm), t(cams), wsum, t(g), sigma, gin, radius=radius)
    torch.cuda.synchronize()
    R = None if radius < 0 else radius
    o_out, o_w = B.filter_forward(c[..., :3], pos, nrm, cams, sigma, R)
    o_g = B.filter_backward(g[..., :3], pos, nrm, cams, sigma, R)
    got, gg, gw = out.cpu().numpy(), gin.cpu().numpy(), wsum.cpu().numpy()
    assert np.all(got[..., 3] == 0) and np.all(gg[..., 3] == 0)
    np.testing.assert_allclose(gw, o_w, rtol=1e-4, atol=1e-6)
    np.testing.assert_allclose(got[..., :3], o_out, rtol=1e-4, atol=1e-5 * np.abs(o_out).max())
    np.testing.assert_allclose(gg[..., :3], o_g, rtol=1e-4, atol=1e-5 * np.abs(o_g).max())
    # the filter did something: covered pixels moved
    cov = np.tile(pos[..., 3] > 0, (2, 1, 1))
    assert np.abs(got[..., :3] - c[..., :3])[cov].mean() > 1e-2


def test_tiny_sigma_is_the_identity(cuda_lib, guides):
    mcdi = cuda_lib
    pos, nrm, cams = guides
    c = np.random.default_rng(5).uniform(size=(2, H, W, 4)).astype(np.float32)
    c[..., 3] = 0
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    out = torch.zeros((2, H, W, 4), device="cuda")
    wsum = torch.zeros((2, H, W), device="cuda")
    mcdi.bilateral_fwd(t(pos), t(nrm), t(cams), t(c), 1e-4, out, wsum)
    torch.cuda.synchronize()
    # only the centre weight survives: c w / w, within rounding of the normalisation
    np.testing.assert_allclose(out.cpu().numpy(), c, rtol=1e-6, atol=0)
