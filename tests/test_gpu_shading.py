"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on the
64 x 64 icosphere-over-ground scene (1,280 + 2,000 triangles, 32 x 16 probe
with a x1000 sun texel, 8 spp = 4 light + 2 cosine + 2 GGX), plus edge cases:
black probe, ragged multi-view images with more than 32 spp, a one-triangle
mesh with leakage, decorrelated backward samples."""
import numpy as np
import pytest
import torch

from paper_2206_03380_gb300 import scenes
from tests import parity_util as PU

pytestmark = pytest.mark.gpu


def to_np(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


@pytest.fixture(scope="module")
def scene():
    return scenes.parity_scene()


@pytest.fixture(scope="module")
def oracle_gb(orc, scene):
    W, H = scene.width, scene.height
    return orc.primary_cast(scene.verts, scene.vnrm, scene.tris, scene.cams[0], W, H, np.arange(W * H),
                            scene.tex_kd, scene.tex_korm, scene.uvmap)


def make_pipe(scene, **kw):
    from paper_2206_03380_gb300.pipeline import ShadingPipeline

    return ShadingPipeline(scene, **kw)


def upload_gb(pipe, gb_rows):
    g = torch.from_numpy(gb_rows.astype(np.float32)).cuda().reshape(pipe.N, pipe.H, pipe.W, 16)
    pipe.gb.pos.copy_(g[..., 0:4])
    pipe.gb.nrm.copy_(g[..., 4:8])
    pipe.gb.kd.copy_(g[..., 8:12])
    pipe.gb.korm.copy_(g[..., 12:16])


# ------------------------------------------------------------------ probe tables
@pytest.mark.parametrize("kind", ["sun", "lobes", "black_rows", "black", "largest"])
def test_envmap_cdf_matches_oracle(cuda_lib, orc, kind):
    rng = np.random.default_rng(5)
    if kind == "largest":  # the largest probe the ABI accepts, 8192 x 4096 (512 MiB)
        env = np.exp(rng.normal(0.0, 1.0, size=(4096, 8192, 4))).astype(np.float32)
        env[..., 3] = 0.0
    elif kind == "sun":
        env, _ = scenes.env_with_sun_texel(32, 16, rng)
    elif kind == "lobes":
        env, _ = scenes.env_with_lobes(512, 256, rng)
    elif kind == "black_rows":
        env, _ = scenes.env_with_sun_texel(300, 7, rng)  # ragged sizes
        env[2] = 0.0
        env[4, :150] = 0.0
    else:
        env = np.zeros((16, 32, 4), np.float32)
    pr = cuda_lib.Probe.allocate(torch.from_numpy(env).cuda()).build()
    cond, marg, rs, tot = orc.envmap_cdf(env)
    gc, gm, grs, gt = to_np(pr.cond), to_np(pr.marg), to_np(pr.row_sum), to_np(pr.total)[0]
    ulp = lambda a, b: np.abs(a.view(np.int32).astype(np.int64) - b.view(np.int32).astype(np.int64))
    assert ulp(gc, cond.astype(np.float32)).max() <= 1
    assert ulp(gm, marg.astype(np.float32)).max() <= 1
    np.testing.assert_allclose(grs, rs, rtol=1e-12, atol=0)
    assert gt == pytest.approx(tot, rel=1e-12, abs=0)
    assert gc[:, -1].tolist() == [1.0] * env.shape[0] and gm[-1] == 1.0


# ------------------------------------------------------------------ BVH
def test_bvh_structure_and_determinism(cuda_lib, scene):
    pipe = make_pipe(scene)
    pipe.build_bvh()
    nodes = to_np(pipe.bvh.nodes).view(np.float32)[: (scene.tris.shape[0] - 1) * 16].reshape(-1, 16)
    recs = to_np(pipe.bvh.tri_records).view(np.float32)[: scene.tris.shape[0] * 12].reshape(-1, 12)
    n = scene.tris.shape[0]
    links = nodes[:, 12:14].view(np.int32)
    leaves = np.sort(~links[links < 0])
    internal = np.sort(links[links >= 0])
    np.testing.assert_array_equal(leaves, np.arange(n))  # every triangle in exactly one leaf
    np.testing.assert_array_equal(internal, np.arange(1, n - 1))  # every node but the root has one parent
    orig = recs[:, 3].view(np.int32)
    np.testing.assert_array_equal(np.sort(orig), np.arange(n))
    v = scene.verts[scene.tris[orig]]  # (n, 3, 3) in leaf order
    np.testing.assert_array_equal(recs[:, 0:3], v[:, 0])
    # each child box contains its whole subtree
    lo = np.full((n - 1, 3), np.inf)
    hi = np.full((n - 1, 3), -np.inf)

    def box_of(link):
        if link < 0:
            t = v[~link]
            return t.min(0), t.max(0)
        return lo[link], hi[link]

    def visit(k):
        for c, (xl, xh, yl, yh), (zl, zh) in ((links[k, 0], nodes[k, 0:4], nodes[k, 8:10]),
                                               (links[k, 1], nodes[k, 4:8], nodes[k, 10:12])):
            if c >= 0:
                visit(c)
            blo, bhi = box_of(c)
            assert xl <= blo[0] and yl <= blo[1] and zl <= blo[2]
            assert xh >= bhi[0] and yh >= bhi[1] and zh >= bhi[2]
        lo[k] = np.minimum(box_of(links[k, 0])[0], box_of(links[k, 1])[0])
        hi[k] = np.maximum(box_of(links[k, 0])[1], box_of(links[k, 1])[1])

    visit(0)
    a = to_np(pipe.bvh.nodes).copy()
    pipe.build_bvh()
    np.testing.assert_array_equal(a, to_np(pipe.bvh.nodes))


def test_bvh_depth_first_escape_links(cuda_lib, scene):
    """The stackless layout is the pre-order copy of the two-child tree: first
    child next, escape link past the subtree, the same boxes, every triangle
    in one leaf."""
    pipe = make_pipe(scene)
    pipe.build_bvh()
    n = scene.tris.shape[0]
    raw = to_np(pipe.bvh.nodes)
    nodes = raw.view(np.float32)[: (n - 1) * 16].reshape(-1, 16)
    links = nodes[:, 12:14].view(np.int32)
    off = ((max(n - 1, 1) * 64 + 255) // 256) * 256
    tn = raw[off: off + (2 * n - 1) * 32].view(np.float32).reshape(-1, 8)
    skip, tri = tn[:, 3].view(np.int32), tn[:, 7].view(np.int32)
    # child boxes as stored in the parent: (lo, hi) per link
    child_box = {}
    for k in range(n - 1):
        a, b, c = nodes[k, 0:4], nodes[k, 4:8], nodes[k, 8:12]
        child_box[int(links[k, 0])] = (np.array([a[0], a[2], c[0]]), np.array([a[1], a[3], c[1]]))
        child_box[int(links[k, 1])] = (np.array([b[0], b[2], c[2]]), np.array([b[1], b[3], c[3]]))

    def walk(link, i):
        if link < 0:
            assert tri[i] == ~link and skip[i] == i + 1
        else:
            assert tri[i] == -1
            j = walk(int(links[link, 0]), i + 1)
            j = walk(int(links[link, 1]), j)
            assert skip[i] == j
            lo = np.minimum(child_box[int(links[link, 0])][0], child_box[int(links[link, 1])][0])
            hi = np.maximum(child_box[int(links[link, 0])][1], child_box[int(links[link, 1])][1])
            np.testing.assert_array_equal(tn[i, 0:3], lo)
            np.testing.assert_array_equal(tn[i, 4:7], hi)
        if link in child_box:
            np.testing.assert_array_equal(tn[i, 0:3], child_box[link][0])
            np.testing.assert_array_equal(tn[i, 4:7], child_box[link][1])
        return int(skip[i])

    assert walk(0, 0) == 2 * n - 1
    np.testing.assert_array_equal(np.sort(tri[tri >= 0]), np.arange(n))


def decode_wide(raw, n):
    """The four-wide nodes of a node buffer: {index: (o, s, qlo (4, 3), qhi (4, 3), links (4,))}."""
    r256 = lambda x: (x + 255) // 256 * 256
    off = r256(r256(max(n - 1, 1) * 64) + (2 * n - 1) * 32)
    w = raw[off: off + max(n - 1, 1) * 64].reshape(-1, 64)
    f = w.view(np.float32).reshape(-1, 16)
    q = w[:, 24:48].reshape(-1, 6, 4)  # qlo x, y, z, qhi x, y, z; byte k = child k
    links = w[:, 48:64].view(np.int32).reshape(-1, 4)
    o = f[:, 0:3].astype(np.float64)
    sc = np.stack([f[:, 3], f[:, 4], f[:, 5]], 1).astype(np.float64)
    qlo = q[:, 0:3].transpose(0, 2, 1).astype(np.float64)
    qhi = q[:, 3:6].transpose(0, 2, 1).astype(np.float64)
    return o, sc, qlo, qhi, links


@pytest.mark.parametrize("which", ["parity", "one_triangle"])
def test_bvh_four_wide_nodes(cuda_lib, scene, which):
    """The four-wide nodes shadow rays traverse: from the root every triangle is
    reached exactly once, every decoded child box holds its subtree's triangles with
    at least one quantisation step to spare on every side, empty slots are inverted
    boxes, and slots of nodes at odd depth are zero."""
    if which == "parity":
        sc = scene
    else:
        sc = scenes.Scene(**{**scene.__dict__, "verts": np.array([[0, 0, 0], [1, 0.2, 0], [0.3, 1, 0.5]], np.float32),
                             "vnrm": np.array([[0, 0, 1]] * 3, np.float32), "tris": np.array([[0, 1, 2]], np.int32)})
    pipe = make_pipe(sc)
    pipe.build_bvh()
    n = sc.tris.shape[0]
    raw = to_np(pipe.bvh.nodes)
    recs = to_np(pipe.bvh.tri_records).view(np.float32)[: n * 12].reshape(-1, 12).astype(np.float64)
    tri_lo = np.minimum(recs[:, 0:3], np.minimum(recs[:, 0:3] + recs[:, 4:7], recs[:, 0:3] + recs[:, 8:11]))
    tri_hi = np.maximum(recs[:, 0:3], np.maximum(recs[:, 0:3] + recs[:, 4:7], recs[:, 0:3] + recs[:, 8:11]))
    o, sc_, qlo, qhi, links = decode_wide(raw, n)
    seen = np.zeros(n, int)
    visited = set()

    def subtree_box(link):
        if link < 0:
            seen[~link] += 1
            return tri_lo[~link], tri_hi[~link]
        assert link not in visited
        visited.add(link)
        lo, hi = np.full(3, np.inf), np.full(3, -np.inf)
        for k in range(4):
            c = int(links[link, k])
            if c == np.iinfo(np.int32).min:
                assert np.all(qlo[link, k] == 255) and np.all(qhi[link, k] == 0)
                continue
            blo, bhi = subtree_box(c)
            dlo = o[link] + qlo[link, k] * sc_[link]
            dhi = o[link] + qhi[link, k] * sc_[link]
            assert np.all(dlo <= blo - sc_[link] * (1 - 1e-6)) and np.all(dhi >= bhi + sc_[link] * (1 - 1e-6))
            lo, hi = np.minimum(lo, blo), np.maximum(hi, bhi)
        return lo, hi

    subtree_box(0)
    np.testing.assert_array_equal(seen, np.ones(n, int))
    unused = sorted(set(range(max(n - 1, 1))) - visited)
    woff = ((max(n - 1, 1) * 64 + 255) // 256 * 256 + (2 * n - 1) * 32 + 255) // 256 * 256
    assert np.all(raw[woff: woff + max(n - 1, 1) * 64].reshape(-1, 64)[unused] == 0)
    assert np.all(np.log2(sc_[sorted(visited)]) == np.round(np.log2(sc_[sorted(visited)])))  # powers of two


# ------------------------------------------------------------------ G-buffer
@pytest.mark.parametrize("raster", [True, False])
def test_primary_cast_matches_oracle(cuda_lib, orc, scene, oracle_gb, raster):
    pipe = make_pipe(scene, raster=raster)
    pipe.build_bvh()
    pipe.primary()
    g = np.concatenate([to_np(pipe.gb.pos), to_np(pipe.gb.nrm), to_np(pipe.gb.kd), to_np(pipe.gb.korm)], -1)
    g = g.reshape(-1, 16)
    o = oracle_gb
    both = (g[:, 3] > 0) & (o[:, 3] > 0)
    cov_mismatch = (g[:, 3] > 0) != (o[:, 3] > 0)
    far = np.abs(g[:, 0:3] - o[:, 0:3]).max(1) > 1e-4
    assert cov_mismatch.sum() <= 3, cov_mismatch.sum()
    assert (both & far).sum() <= 3
    ok = both & ~far
    assert ok.sum() > 2000
    np.testing.assert_allclose(g[ok, 0:3], o[ok, 0:3], atol=2e-5)
    np.testing.assert_allclose(g[ok, 4:7], o[ok, 4:7], atol=2e-5)
    np.testing.assert_allclose(g[ok, 8:11], o[ok, 8:11], atol=1e-6)
    np.testing.assert_allclose(g[ok, 12:15], o[ok, 12:15], atol=1e-6)
    assert np.all(g[g[:, 3] == 0] == 0)


# ------------------------------------------------------------------ forward / adjoint
def run_fwd(pipe, gb_rows):
    upload_gb(pipe, gb_rows)
    pipe.build_probe()
    pipe.build_bvh()
    pipe.forward()
    out = np.concatenate([to_np(pipe.c_d)[..., :3], to_np(pipe.kd_out)[..., :3], to_np(pipe.c_s)[..., :3]], -1)
    return out.reshape(-1, 9), to_np(pipe.mask).reshape(pipe.N * pipe.H * pipe.W, -1)


def check_forward(orc, scene, gpu_out, gpu_mask, gb_rows, pix, view, tau=1.0, flips=None):
    o_out, o_vis, recs = PU.oracle_shade(orc, scene, gb_rows, pix, view, tau=tau)
    cov = gb_rows[:, 3] > 0
    np.testing.assert_allclose(gpu_out[:, 3:6], o_out[:, 3:6], rtol=1e-6, atol=1e-7)
    n_bad = 0
    bad_px = np.zeros(len(pix), bool)
    for sl in (slice(0, 3), slice(6, 9)):
        bad, marginal, err = PU.compare_radiance(gpu_out[cov, sl], o_out[cov, sl], recs[cov])
        assert not (bad & ~marginal).any(), (err[bad & ~marginal].max(), np.nonzero(bad & ~marginal)[0][:10])
        n_bad += bad.sum()
        bad_px[np.nonzero(cov)[0][bad]] = True
    assert n_bad <= max(2, 0.002 * cov.sum())
    # shadow-ray agreement on samples active on both sides
    spp = scene.spp
    gbits, obits = PU.mask_bits(gpu_mask, spp), PU.mask_bits(o_vis, spp)
    act = recs["active"].astype(bool)
    mism = (gbits != obits) & act
    assert mism.sum() <= max(1, 1e-4 * act.sum()), mism.sum()
    assert np.all(recs["margin"][mism] < PU.MARGIN)
    assert not np.any(gbits & ~act & (recs["margin"] >= PU.MARGIN))
    if flips is not None:
        lo, hi = PU.flipped_samples(gbits, obits, act, bad_px, recs["margin"])
        flips.append((lo, hi, int(act.sum())))
    return o_out, recs


@pytest.mark.parametrize("wavefront", [True, False])
def test_shade_fwd_matches_oracle(cuda_lib, orc, scene, oracle_gb, wavefront):
    pipe = make_pipe(scene, wavefront=wavefront)
    out, mask = run_fwd(pipe, oracle_gb)
    o_out, recs = check_forward(orc, scene, out, mask, oracle_gb.astype(np.float32), np.arange(64 * 64), 0)
    assert recs["occluded"].sum() > 500  # the sphere shadows the ground
    assert np.isfinite(out).all()


def check_adjoint(orc, scene, pipe, gb_rows, recs, o_out, pix, view, g):
    """g: (n, 9) upstream; zero on marginal pixels so that the probe gradient is comparable.

    A gradient is a sum of terms of either sign (the upstream gradient is
    random; inside one sample the diffuse and specular parts can also cancel);
    its FP32 error is bounded relative to the sum of the terms' magnitudes,
    which the oracle reports beside the gradient."""
    cam = np.tile(scene.cams[view, :3].astype(np.float64), (len(pix), 1))
    prow = orc.param_rows(gb_rows)
    env3 = scene.env[..., :3].reshape(-1, 3).astype(np.float64)
    grad, genv, scale, genv_scale = orc.frozen_adjoint(recs, prow, cam, o_out[:, 9].astype(np.int32), env3, g,
                                                       with_scale=True)
    gk, go, gn = to_np(pipe.g_kd).reshape(-1, 4), to_np(pipe.g_korm).reshape(-1, 4), to_np(pipe.g_nrm).reshape(-1, 4)
    gpu = np.concatenate([gn[pix, :3], gk[pix, :3], go[pix, :3]], 1)
    floor = 1e-6 * scale.max(0, keepdims=True) + 1e-30
    err = np.abs(gpu - grad) / np.maximum(scale, floor)
    assert err.max() <= PU.GRAD_TOL, (err.max(), np.unravel_index(err.argmax(), err.shape))
    ge = to_np(pipe.g_env)[..., :3].reshape(-1, 3)
    eerr = np.abs(ge - genv) / np.maximum(genv_scale, 1e-6 * genv_scale.max() + 1e-30)
    assert eerr.max() <= PU.GRAD_TOL, eerr.max()
    # and plain relative error wherever the terms do not cancel
    nc = scale <= 1.5 * np.abs(grad)
    rel = np.abs(gpu - grad)[nc] / np.maximum(np.abs(grad)[nc], floor.repeat(len(grad), 0)[nc])
    assert rel.max() <= PU.GRAD_TOL, rel.max()


def upstream(n, rng, marginal):
    g = rng.normal(size=(n, 9)).astype(np.float32).astype(np.float64)
    g[marginal] = 0.0
    return g


def test_shade_bwd_matches_oracle_adjoint(cuda_lib, orc, scene, oracle_gb):
    pipe = make_pipe(scene)
    gb_rows = oracle_gb.astype(np.float32)
    out, mask = run_fwd(pipe, oracle_gb)
    pix = np.arange(64 * 64)
    o_out, recs = check_forward(orc, scene, out, mask, gb_rows, pix, 0)
    marginal = (recs["margin"] < PU.MARGIN).any(1)
    g = upstream(len(pix), np.random.default_rng(9), marginal)
    gt = torch.from_numpy(g.astype(np.float32)).cuda()
    pad = lambda x: torch.nn.functional.pad(x, (0, 1)).reshape(1, 64, 64, 4).contiguous()
    pipe.backward(pad(gt[:, 0:3]), pad(gt[:, 3:6]), pad(gt[:, 6:9]))
    check_adjoint(orc, scene, pipe, gb_rows, recs, o_out, pix, 0, g)


def test_black_probe(cuda_lib, orc, scene, oracle_gb):
    sc = scenes.Scene(**{**scene.__dict__, "env": np.zeros_like(scene.env)})
    pipe = make_pipe(sc)
    out, mask = run_fwd(pipe, oracle_gb)
    assert np.all(out[:, 0:3] == 0) and np.all(out[:, 6:9] == 0)
    check_forward(orc, sc, out, mask, oracle_gb.astype(np.float32), np.arange(64 * 64), 0)


def test_ragged_multiview_many_spp(cuda_lib, orc):
    base = scenes.parity_scene(seed=scenes.BASE_SEED + 11)
    rng = np.random.default_rng(12)
    cams = np.stack([scenes.look_at(e, (0, -0.3, 0), (0, 1, 0), 50.0, 37 / 23)
                     for e in [(0, 0.5, 3.2), (2.5, 1.5, 1.5), (-2.8, 0.3, -1.0)]])
    sc = scenes.Scene(**{**base.__dict__, "cams": cams, "width": 37, "height": 23, "n_light": 20, "n_cos": 10,
                         "n_ggx": 10, "tex_kd": rng.uniform(size=(8, 8, 4)).astype(np.float32),
                         "tex_korm": np.concatenate([np.zeros((8, 8, 1)), rng.uniform(0.1, 1.0, (8, 8, 2)),
                                                     np.zeros((8, 8, 1))], -1).astype(np.float32)})
    pipe = make_pipe(sc, tau=0.25)
    pipe.build_bvh()
    pipe.primary()
    g = np.concatenate([to_np(pipe.gb.pos), to_np(pipe.gb.nrm), to_np(pipe.gb.kd), to_np(pipe.gb.korm)], -1)
    rows = []
    for v in range(3):
        og = orc.primary_cast(sc.verts, sc.vnrm, sc.tris, cams[v], 37, 23, np.arange(37 * 23), sc.tex_kd,
                              sc.tex_korm, sc.uvmap)
        rows.append(og)
    og = np.concatenate(rows)
    assert ((g.reshape(-1, 16)[:, 3] > 0) != (og[:, 3] > 0)).sum() <= 6
    out, mask = run_fwd(pipe, og)
    for v in range(3):
        sl = slice(v * 851, (v + 1) * 851)
        check_forward(orc, sc, out[sl], mask[sl], og[sl].astype(np.float32), np.arange(851), v, tau=0.25)


@pytest.mark.parametrize("with_occluder", [False, True])
def test_small_meshes_leakage_and_decorrelated_backward(cuda_lib, orc, with_occluder):
    base = scenes.parity_scene(seed=scenes.BASE_SEED + 13)
    ground = np.array([[-3, -1, -3], [3, -1, -3], [0, -1, 4]], np.float32)  # one triangle
    occ = np.array([[-0.5, 1.5, -0.5], [0.6, 1.5, -0.4], [0.0, 1.6, 0.7]], np.float32)  # floating occluder
    verts = np.concatenate([ground, occ]) if with_occluder else ground
    tris = np.array([[0, 1, 2], [3, 4, 5]] if with_occluder else [[0, 1, 2]], np.int32)
    vn = np.tile(np.array([[0, 1, 0]], np.float32), (len(verts), 1))
    cam = scenes.look_at((0, 2.0, 3.0), (0, -1, 0), (0, 1, 0), 45.0, 1.0)[None]
    sc = scenes.Scene(**{**base.__dict__, "verts": verts, "vnrm": vn, "tris": tris, "cams": cam})
    for tau, decorrelate in [(0.4, False), (0.0, True)]:
        pipe = make_pipe(sc, tau=tau, decorrelate_bwd=decorrelate)
        og = orc.primary_cast(verts, vn, tris, cam[0], 64, 64, np.arange(4096), sc.tex_kd, sc.tex_korm, sc.uvmap)
        out, mask = run_fwd(pipe, og)
        o_out, recs = check_forward(orc, sc, out, mask, og.astype(np.float32), np.arange(4096), 0, tau=tau)
        assert (recs["occluded"].sum() > 100) == with_occluder
        stream = 1 if decorrelate else 0
        o_out_b, _, recs_b = PU.oracle_shade(orc, sc, og.astype(np.float32), np.arange(4096), 0, tau=tau,
                                             stream=stream)
        marginal = (recs_b["margin"] < PU.MARGIN).any(1) | (recs["margin"] < PU.MARGIN).any(1)
        g = upstream(4096, np.random.default_rng(14), marginal)
        gt = torch.from_numpy(g.astype(np.float32)).cuda()
        pad = lambda x: torch.nn.functional.pad(x, (0, 1)).reshape(1, 64, 64, 4).contiguous()
        pipe.backward(pad(gt[:, 0:3]), pad(gt[:, 3:6]), pad(gt[:, 6:9]))
        check_adjoint(orc, sc, pipe, og.astype(np.float32), recs_b, o_out_b, np.arange(4096), 0, g)


def test_flipped_sample_rate(cuda_lib, orc, scene, oracle_gb):
    """The benchmark spec's bound on discrete decisions taken differently under identical
    samples: fewer than 0.01% of the active samples, counted on the parity scene (all
    4,096 pixels) and on three views of a ragged 37 x 23 image with 40 spp."""
    flips = []
    pipe = make_pipe(scene)
    out, mask = run_fwd(pipe, oracle_gb)
    check_forward(orc, scene, out, mask, oracle_gb.astype(np.float32), np.arange(64 * 64), 0, flips=flips)
    lo = sum(f[0] for f in flips)
    hi = sum(f[1] for f in flips)
    act = sum(f[2] for f in flips)
    print(f"flipped samples: {lo} (at most {hi}) of {act} active = {lo / act:.2e} ({hi / act:.2e})")
    assert hi <= max(1, 1e-4 * act), (lo, hi, act)


@pytest.mark.parametrize("wavefront", [True, False])
def test_forward_is_repeatable(cuda_lib, scene, wavefront):
    pipe = make_pipe(scene, wavefront=wavefront)
    pipe.build_probe()
    pipe.build_bvh()
    pipe.primary()
    pipe.forward()
    a = to_np(pipe.c_s).copy(), to_np(pipe.c_d).copy()
    pipe.forward()
    np.testing.assert_array_equal(a[0], to_np(pipe.c_s))
    np.testing.assert_array_equal(a[1], to_np(pipe.c_d))


def test_wavefront_and_fused_forward_agree(cuda_lib, scene, oracle_gb):
    a, b = make_pipe(scene, wavefront=True), make_pipe(scene, wavefront=False)
    oa, ma = run_fwd(a, oracle_gb)
    ob, mb = run_fwd(b, oracle_gb)
    np.testing.assert_array_equal(ma, mb)  # same samples, same shadow rays
    np.testing.assert_allclose(oa, ob, rtol=2e-6, atol=1e-7 * np.abs(ob).max())
