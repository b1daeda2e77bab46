"""GPU parity of the shadow-visibility gradient (edge sampling of the boundary
term; the paper's appendix on visibility gradients from shadows) through the
C ABI:

* the edge table is bit-identical to the oracle's (records and order) on the
  parity mesh, the ~198k-triangle headline mesh and a mesh with shuffled
  faces and boundaries;
* on the 64 x 64 parity scene, every edge sample's weight agrees with the
  oracle's (same Philox draws, so the same edge and position on it): the same
  contribute / skip decision wherever the oracle's decision margin is above
  1e-4, values within 1e-3 relative, and the per-vertex gradient sums within
  1e-3 on every vertex that no marginal sample touches;
* at the headline size, in the configuration the benchmark times, sampled
  pixels' edge samples against the oracle run on the same G-buffer rows;
* tau = 0 gives zeros, zero samples leave the accumulator untouched,
  background pixels give zero weights.
"""
import numpy as np
import pytest
import torch

from paper_2206_03380_gb300 import scenes
from tests import parity_util as PU

pytestmark = pytest.mark.gpu

ETA = 1e-4


def weight_tol(margin):
    """A sample's weight is proportional to its cosine n.w and to the
    silhouette and texel measures that the margin bounds from below; FP32
    rounding of the unit direction (about 6e-8) then costs about 6e-8 / margin
    relative: the gradient tolerance plus that term."""
    return PU.GRAD_TOL + 2e-7 / margin


def _gb_rows(pipe):
    return torch.cat([pipe.gb.pos, pipe.gb.nrm, pipe.gb.kd, pipe.gb.korm], -1).reshape(-1, 16).cpu().numpy()


def _upload(pipe, rows):
    g = torch.from_numpy(rows.astype(np.float32)).cuda().reshape(pipe.N, pipe.H, pipe.W, 16)
    for k, t in enumerate((pipe.gb.pos, pipe.gb.nrm, pipe.gb.kd, pipe.gb.korm)):
        t.copy_(g[..., 4 * k:4 * k + 4])


def _gpu_edges(mcdi, tris):
    et = mcdi.EdgeTable.allocate(len(tris), "cuda").build(torch.from_numpy(np.ascontiguousarray(tris)).cuda())
    torch.cuda.synchronize()
    n = int(et.count.item())
    return et, et.records[:n].cpu().numpy()


def _run(mcdi, pipe, et, prm, M, gcd, gcs, want_w=True):
    g = torch.zeros(pipe.verts.shape[0], 3, device="cuda")
    w = torch.full((pipe.N * pipe.H * pipe.W, max(M, 1)), float("nan"), device="cuda") if want_w else None
    mcdi.shadow_edge_grad(pipe.bvh, pipe.verts, et, pipe.probe, pipe.gb, pipe.cams, prm, M, gcd, gcs, g, w, eta=ETA)
    torch.cuda.synchronize()
    return g.cpu().numpy().astype(np.float64), (w.cpu().numpy() if want_w else None)


@pytest.mark.parametrize("which", ["parity", "headline", "shuffled", "single", "fan"])
def test_edge_table_matches_oracle(cuda_lib, orc, which):
    if which == "single":  # three boundary edges
        tris = np.array([[4, 9, 2]], np.int32)
    elif which == "fan":  # four faces on the edge (0, 1): the first two are kept, in half-edge order
        tris = np.array([[0, 1, 2], [1, 0, 3], [0, 1, 4], [5, 1, 0], [2, 3, 4]], np.int32)
    elif which == "parity":
        tris = scenes.parity_scene().tris
    elif which == "headline":
        tris = scenes.sphere_union_scene().tris
    else:
        rng = np.random.default_rng(3)
        _, _, t = scenes.icosphere(3, radius=1.0)
        t = t[rng.permutation(len(t))][: len(t) - 37]  # holes: boundary edges
        tris = np.ascontiguousarray(np.roll(t, 1, axis=1)).astype(np.int32)
    _, got = _gpu_edges(cuda_lib, tris)
    ref = orc.edge_table(tris)
    assert got.shape == ref.shape and np.array_equal(got, ref)


def _parity_case(mcdi, orc, tau=0.7):
    from paper_2206_03380_gb300.pipeline import ShadingPipeline

    sc = scenes.parity_scene()
    W, H = sc.width, sc.height
    rows = orc.primary_cast(sc.verts, sc.vnrm, sc.tris, sc.cams[0], W, H, np.arange(W * H), sc.tex_kd, sc.tex_korm,
                            sc.uvmap).astype(np.float32)
    pipe = ShadingPipeline(sc)
    _upload(pipe, rows)
    pipe.build_probe()
    pipe.build_bvh()
    prm = mcdi.make_params(sc.n_light, sc.n_cos, sc.n_ggx, sc.seed, tau=tau)
    return sc, pipe, rows, prm


def test_parity_scene_matches_oracle(cuda_lib, orc):
    mcdi = cuda_lib
    tau, M = 0.7, 32
    sc, pipe, rows, prm = _parity_case(mcdi, orc, tau)
    W, H = sc.width, sc.height
    rng = np.random.default_rng(11)
    gcd = rng.normal(size=(H * W, 3)).astype(np.float32)
    gcs = rng.normal(size=(H * W, 3)).astype(np.float32)
    pad = lambda a: torch.from_numpy(np.concatenate([a, np.zeros((len(a), 1), np.float32)], 1)).cuda().reshape(
        1, H, W, 4)
    et, _ = _gpu_edges(mcdi, sc.tris)
    edges = orc.edge_table(sc.tris)
    g_gpu, w_gpu = _run(mcdi, pipe, et, prm, M, pad(gcd), pad(gcs))
    pix = np.arange(W * H)
    cam = np.tile(sc.cams[0, :3].astype(np.float64), (len(pix), 1))
    ctr = np.stack([pix, np.zeros_like(pix)], 1).astype(np.uint32)
    g_orc, rec = orc.shadow_edge_grad(sc.verts, sc.tris, edges, sc.env, rows, cam, ctr, gcd, gcs, n_samples=M,
                                      seed=sc.seed, stream=2, tau=tau, ray_eps=1e-4, eta=ETA)
    w_orc, margin = rec[..., 0], rec[..., 1]
    # samples of ground edges seen from ground pixels have coplanar faces and a grazing direction: their
    # silhouette and horizon decisions are marginal; nearly all contributing samples are not
    safe = margin >= PU.MARGIN
    contrib = w_orc != 0
    assert contrib.sum() > 800  # silhouettes of the sphere and the ground's border seen from the pixels
    assert (safe & contrib).sum() >= 0.98 * contrib.sum()
    assert np.array_equal((w_gpu != 0)[safe], contrib[safe])
    floor = 1e-3 * np.abs(w_orc[contrib]).mean()
    err = np.abs(w_gpu - w_orc) / np.maximum(np.abs(w_orc), floor)
    assert np.all(err[safe] <= weight_tol(margin[safe])), (err[safe].max(), margin[safe][err[safe].argmax()])
    # vertex sums, on the vertices no marginal sample touches
    e_idx = rec[..., 2].astype(np.int64)
    unsafe = ~safe & ((w_orc != 0) | (w_gpu != 0))
    touched = np.unique(edges[e_idx[unsafe]][:, :2]) if unsafe.any() else np.zeros(0, np.int64)
    keep = np.ones(len(sc.verts), bool)
    keep[touched] = False
    scale = np.abs(g_orc[keep]).max()
    assert scale > 0
    np.testing.assert_allclose(g_gpu[keep], g_orc[keep], rtol=PU.GRAD_TOL, atol=1e-4 * scale)


def test_degenerate_cases(cuda_lib, orc):
    mcdi = cuda_lib
    sc, pipe, rows, prm = _parity_case(mcdi, orc, 0.7)
    W, H = sc.width, sc.height
    ones = torch.ones(1, H, W, 4, device="cuda")
    et, _ = _gpu_edges(mcdi, sc.tris)
    g, w = _run(mcdi, pipe, et, prm, 4, ones, ones)
    assert np.isfinite(w).all() and np.count_nonzero(w) > 0
    background = rows[:, 3] <= 0
    assert background.any() and np.all(w[background] == 0)
    prm0 = mcdi.make_params(sc.n_light, sc.n_cos, sc.n_ggx, sc.seed, tau=0.0)
    g0, w0 = _run(mcdi, pipe, et, prm0, 4, ones, ones)
    assert np.all(g0 == 0) and np.all(w0 == 0)
    # zero samples: the accumulator is left as it was
    acc = torch.full((pipe.verts.shape[0], 3), 2.5, device="cuda")
    mcdi.shadow_edge_grad(pipe.bvh, pipe.verts, et, pipe.probe, pipe.gb, pipe.cams, prm, 0, ones, ones, acc)
    torch.cuda.synchronize()
    assert torch.all(acc == 2.5)


def test_headline_sampled_pixels_match_oracle(cuda_lib, orc):
    from paper_2206_03380_gb300.pipeline import ShadingPipeline

    mcdi = cuda_lib
    sc = scenes.sphere_union_scene()
    W = H = sc.width
    tau, M = 1.0, 4
    pipe = ShadingPipeline(sc)
    zeros = torch.zeros(1, H, W, 4, device="cuda")
    pipe.step(zeros, zeros, zeros)  # tables, BVH and G-buffer exactly as the timed step builds them
    prm = mcdi.make_params(sc.n_light, sc.n_cos, sc.n_ggx, sc.seed, tau=tau)
    et, _ = _gpu_edges(mcdi, sc.tris)
    rng = np.random.default_rng(5)
    gcd = torch.from_numpy(rng.normal(size=(1, H, W, 4)).astype(np.float32)).cuda()
    gcs = torch.from_numpy(rng.normal(size=(1, H, W, 4)).astype(np.float32)).cuda()
    _, w_gpu = _run(mcdi, pipe, et, prm, M, gcd, gcs)
    covered = np.nonzero(_gb_rows(pipe)[:, 3] > 0)[0]
    # pixels drawn among those with a contributing sample and among all covered ones; the oracle's own
    # G-buffer rows for them replace the GPU's, so that both sides shade identical inputs
    hit = covered[(w_gpu[covered] != 0).any(1)]
    assert len(hit) > 100
    pix = np.unique(np.concatenate([rng.choice(hit, 48, replace=False), rng.choice(covered, 48, replace=False)]))
    rows = orc.primary_cast(sc.verts, sc.vnrm, sc.tris, sc.cams[0], W, H, pix, sc.tex_kd, sc.tex_korm,
                            sc.uvmap).astype(np.float32)
    pix, rows = pix[rows[:, 3] > 0], rows[rows[:, 3] > 0]
    full = _gb_rows(pipe)
    full[pix] = rows
    _upload(pipe, full)
    _, w_gpu = _run(mcdi, pipe, et, prm, M, gcd, gcs)
    cam = np.tile(sc.cams[0, :3].astype(np.float64), (len(pix), 1))
    ctr = np.stack([pix, np.zeros_like(pix)], 1).astype(np.uint32)
    gc, gs = gcd.reshape(-1, 4)[:, :3].cpu().numpy()[pix], gcs.reshape(-1, 4)[:, :3].cpu().numpy()[pix]
    _, rec = orc.shadow_edge_grad(sc.verts, sc.tris, orc.edge_table(sc.tris), sc.env, rows, cam, ctr, gc, gs,
                                  n_samples=M, seed=sc.seed, stream=2, tau=tau, ray_eps=1e-4, eta=ETA)
    w_orc, margin = rec[..., 0], rec[..., 1]
    w_g = w_gpu[pix]
    # many contributing samples are edges of the pixel's own surface seen at a grazing angle (marginal by
    # construction, with weights proportional to their small cosine)
    safe = margin >= PU.MARGIN
    assert np.array_equal((w_g != 0)[safe], (w_orc != 0)[safe])
    c = (w_orc != 0) & safe
    assert c.sum() >= 20
    err = np.abs(w_g[c] - w_orc[c]) / np.abs(w_orc[c])
    assert np.all(err <= weight_tol(margin[c])), err.max()
