"""Pins for the oracle's shadow-visibility gradient (edge sampling of the
boundary term; the paper's appendix on visibility gradients from shadows,
Sec. 3.1 "Shadow gradients").

Independent facts used:
* Lambert's formula: the cosine-weighted solid angle of a polygon seen from a
  point is half the sum over its edges of the edge's subtended angle times the
  normal component of the edge plane's unit normal.  Under a constant probe a
  diffuse point with one polygon occluder therefore has
  c_d = L (1 - tau Phi / pi), and its vertex gradient is the (smooth) closed
  form's derivative, taken here by central differences of the formula.
* Occluders hidden behind (or in front of and inside) a larger one do not
  move the blocked set: their vertex gradients vanish.
* The gradient of the forward estimator's expectation, estimated by central
  differences of the oracle's own forward pass with common random numbers
  (the sampling does not depend on the mesh), with the specular lobe on, a
  textured probe and leakage tau < 1.
* Euler's formula and face adjacency for the edge table.
"""
import numpy as np
import pytest

from paper_2206_03380_gb300 import scenes


def gb_row(p, n, kd=(0.5, 0.5, 0.5), r=0.5, m=0.0):
    return np.array([*p, 1.0, *n, 0.0, *kd, 0.0, 0.0, r, m, 0.0], np.float32)


def lambert_phi(poly, o, n):
    """Cosine-weighted solid angle of the polygon (rows of vertices) seen from o."""
    r = poly - o
    r = r / np.linalg.norm(r, axis=1, keepdims=True)
    tot = 0.0
    for i in range(len(r)):
        a, b = r[i], r[(i + 1) % len(r)]
        c = np.cross(a, b)
        tot += 0.5 * np.arccos(np.clip(a @ b, -1.0, 1.0)) * (n @ c) / np.linalg.norm(c)
    return abs(tot)


def lambert_grad(poly, o, n, h=1e-6):
    g = np.zeros_like(poly)
    for k in range(len(poly)):
        for c in range(3):
            d = np.zeros_like(poly)
            d[k, c] = h
            g[k, c] = (lambert_phi(poly + d, o, n) - lambert_phi(poly - d, o, n)) / (2 * h)
    return g


def replicate_grads(orc, verts, tris, env, row, cam, gcd, gcs, *, reps=8, M=25000, tau=1.0, ray_eps=0.0):
    edges = orc.edge_table(tris)
    runs = []
    for k in range(reps):
        g, _ = orc.shadow_edge_grad(verts, tris, edges, env, row[None], np.asarray(cam)[None], np.array([[0, 0]]),
                                    np.asarray(gcd)[None], np.asarray(gcs)[None], n_samples=M, seed=1000 + k,
                                    tau=tau, ray_eps=ray_eps, want_records=False)
        runs.append(g)
    runs = np.array(runs)
    return runs.mean(0), runs.std(0, ddof=1) / np.sqrt(reps)


CONST_ENV = np.ones((4, 8, 4), np.float32)
UP = np.array([0.0, 1.0, 0.0])


@pytest.mark.parametrize("tau", [1.0, 0.6])
def test_single_triangle_matches_lambert(orc, tau):
    verts = np.array([[-0.3, 1.0, -0.2], [0.4, 1.1, -0.1], [0.0, 0.9, 0.5]], np.float32)
    tris = np.array([[0, 1, 2]], np.int32)
    o = np.zeros(3)
    row = gb_row(o, UP)
    mean, se = replicate_grads(orc, verts, tris, CONST_ENV, row, (0, 3, 3), (1.0, 0.0, 0.0), (0, 0, 0), tau=tau)
    ref = -tau / np.pi * lambert_grad(verts.astype(np.float64), o, UP)
    scale = np.abs(ref).max()
    assert np.all(np.abs(mean - ref) <= 5 * se + 1e-3 * scale), (mean, ref, se)
    assert np.abs(mean - ref).max() < 0.02 * scale


def test_quad_interior_edge_is_not_a_silhouette(orc):
    verts = np.array([[-0.4, 1.0, -0.3], [0.5, 1.0, -0.35], [0.45, 1.2, 0.4], [-0.35, 1.1, 0.3]], np.float32)
    tris = np.array([[0, 1, 2], [0, 2, 3]], np.int32)
    o = np.zeros(3)
    row = gb_row(o, UP)
    mean, se = replicate_grads(orc, verts, tris, CONST_ENV, row, (0, 3, 3), (0.0, 2.0, 0.0), (0, 0, 0))
    ref = -2.0 / np.pi * lambert_grad(verts.astype(np.float64), o, UP)
    scale = np.abs(ref).max()
    assert np.all(np.abs(mean - ref) <= 5 * se + 1e-3 * scale), (mean, ref, se)
    # the shared diagonal (edge 2 in first-half-edge order) never contributes
    edges = orc.edge_table(tris)
    diag = [k for k, e in enumerate(edges) if e[3] >= 0]
    assert len(diag) == 1
    _, rec = orc.shadow_edge_grad(verts, tris, edges, CONST_ENV, row[None], np.array([[0, 3, 3]]),
                                  np.array([[0, 0]]), np.array([[0, 2.0, 0]]), np.zeros((1, 3)), n_samples=4000,
                                  seed=5, ray_eps=0.0)
    on_diag = rec[0, :, 2] == diag[0]
    assert on_diag.sum() > 500 and np.all(rec[0, on_diag, 0] == 0.0)
    assert np.count_nonzero(rec[0, ~on_diag, 0]) > 0.9 * (~on_diag).sum()


@pytest.mark.parametrize("small_in_front", [True, False])
def test_hidden_occluder_edges_contribute_nothing(orc, small_in_front):
    big = np.array([[-0.8, 1.5, -0.7], [0.9, 1.5, -0.6], [0.0, 1.5, 1.0]])
    y = 0.8 if small_in_front else 2.5
    s = y / 1.5 * 0.25  # well inside the big triangle's projection
    small = np.array([[-s, y, -s], [s, y, -s * 0.8], [0.0, y, s]])
    verts = np.concatenate([big, small]).astype(np.float32)
    tris = np.array([[0, 1, 2], [3, 4, 5]], np.int32)
    o = np.zeros(3)
    row = gb_row(o, UP)
    mean, se = replicate_grads(orc, verts, tris, CONST_ENV, row, (0, 3, 3), (1.0, 1.0, 1.0), (0, 0, 0), reps=6)
    assert np.all(mean[3:] == 0.0)
    ref = -3.0 / np.pi * lambert_grad(big, o, UP)
    scale = np.abs(ref).max()
    assert np.all(np.abs(mean[:3] - ref) <= 5 * se[:3] + 1e-3 * scale)


@pytest.mark.parametrize("case", ["diffuse+specular", "specular"])
def test_matches_finite_differences_of_the_forward_estimator(orc, case):
    """Specular lobe on, log-normal probe, tau = 0.5: the edge-sampling gradient
    of one vertex coordinate against central differences of the forward MC
    estimator's expectation (common random numbers, independent replicates).
    The second case weights only c_s, seen at cos_o = 0.53 off a metal."""
    rng = np.random.default_rng(77)
    env = np.exp(rng.normal(0.0, 0.5, size=(16, 32, 4))).astype(np.float32)
    env[..., 3] = 0.0
    cond, marg, _, total = orc.envmap_cdf(env)
    cond32, marg32 = cond.astype(np.float32), marg.astype(np.float32)
    verts = np.array([[-0.5, 0.9, -0.2], [0.4, 1.0, -0.4], [0.3, 0.8, 0.5], [-0.4, 1.1, 0.4]], np.float32)
    tris = np.array([[0, 1, 2], [0, 2, 3]], np.int32)
    n = np.array([0.2, 1.0, 0.1])
    n /= np.linalg.norm(n)
    gcs = np.array([0.3, 0.5, -0.6])
    if case == "specular":
        row = gb_row((0.05, 0.0, -0.02), n, kd=(0.6, 0.4, 0.3), r=0.3, m=1.0)
        cam, gcd = np.array([0.4, 1.2, 2.5]), np.zeros(3)
    else:
        row = gb_row((0.05, 0.0, -0.02), n, kd=(0.6, 0.4, 0.3), r=0.35, m=0.5)
        cam, gcd = np.array([0.4, 2.5, 2.0]), np.array([0.7, -0.2, 0.4])
    tau = 0.5
    mean, se = replicate_grads(orc, verts, tris, env, row, cam, gcd, gcs, reps=6, M=40000, tau=tau, ray_eps=1e-4)
    k, c = np.unravel_index(np.abs(mean).argmax(), mean.shape)
    h = 2e-3
    fd = []
    for rep in range(6):
        vals = []
        for sgn in (1, -1):
            v = verts.copy()
            v[k, c] += sgn * h
            out, _, _ = orc.shade_fwd(v, tris, env, cond32, marg32, total, row[None], cam[None], np.array([[0, 0]]),
                                      n_light=1 << 16, n_cos=1 << 15, n_ggx=1 << 15, seed=500 + rep, tau=tau,
                                      ray_eps=1e-4, want_records=False)
            vals.append(gcd @ out[0, 0:3] + gcs @ out[0, 6:9])
        fd.append((vals[0] - vals[1]) / (2 * h))
    fd = np.array(fd)
    fd_mean, fd_se = fd.mean(), fd.std(ddof=1) / np.sqrt(len(fd))
    assert abs(mean[k, c] - fd_mean) <= 5 * np.hypot(se[k, c], fd_se), (mean[k, c], fd_mean, se[k, c], fd_se)
    assert abs(mean[k, c] - fd_mean) <= 0.15 * abs(fd_mean)


def test_zero_leakage_and_linearity(orc):
    verts = np.array([[-0.3, 1.0, -0.2], [0.4, 1.1, -0.1], [0.0, 0.9, 0.5]], np.float32)
    tris = np.array([[0, 1, 2]], np.int32)
    edges = orc.edge_table(tris)
    row = gb_row((0, 0, 0), UP)
    args = (verts, tris, edges, CONST_ENV, row[None], np.array([[0, 3, 3]]), np.array([[3, 0]]))
    g1, _ = orc.shadow_edge_grad(*args, np.array([[1.0, 0.5, 0.0]]), np.zeros((1, 3)), n_samples=500, seed=9)
    g2, _ = orc.shadow_edge_grad(*args, np.array([[2.0, 1.0, 0.0]]), np.zeros((1, 3)), n_samples=500, seed=9)
    g0, _ = orc.shadow_edge_grad(*args, np.array([[1.0, 0.5, 0.0]]), np.zeros((1, 3)), n_samples=500, seed=9,
                                 tau=0.0)
    assert np.abs(g1).max() > 0 and np.array_equal(g2, 2 * g1) and np.all(g0 == 0)


def test_edge_table_closed_and_open_meshes(orc):
    v, _, t = scenes.icosphere(2, radius=1.0)
    e = orc.edge_table(t)
    assert len(e) == 3 * len(t) // 2 and np.all(e[:, 3] >= 0)
    assert len(v) - len(e) + len(t) == 2  # Euler characteristic of a sphere
    faces = {tuple(np.roll(f, -i)) for f in t.tolist() for i in range(3)}
    for a, b, c1, c2 in e.tolist():
        assert (a, b, c1) in faces  # the owner's face, in its orientation
        assert (b, a, c2) in faces or (a, b, c2) in faces  # the other face (either orientation)
    # first-half-edge order: brute force over the half-edges
    seen, order = set(), []
    for f in t.tolist():
        for i in range(3):
            k = frozenset((f[i], f[(i + 1) % 3]))
            if k not in seen:
                seen.add(k)
                order.append((f[i], f[(i + 1) % 3]))
    assert [tuple(r[:2]) for r in e.tolist()] == order
    # an open grid of nx x nz quads: boundary edges on its perimeter only
    nx, nz = 5, 3
    idx = np.arange((nx + 1) * (nz + 1)).reshape(nz + 1, nx + 1)
    quads = [(idx[j, i], idx[j, i + 1], idx[j + 1, i + 1], idx[j + 1, i]) for j in range(nz) for i in range(nx)]
    grid = np.array([[a, b, c] for a, b, c, d in quads] + [[a, c, d] for a, b, c, d in quads], np.int32)
    eg = orc.edge_table(grid)
    assert (eg[:, 3] < 0).sum() == 2 * (nx + nz)
    assert len(eg) == nx * (nz + 1) + nz * (nx + 1) + nx * nz
