"""Pins for the oracle's MIS estimator (Sec. 3.1 Monte Carlo estimator, Sec. 4.1
MIS with the balance heuristic, Sec. 4.2 light separation, App. A leakage).

Closed forms and invariants, none of which retype the oracle's formulas:
* zero-variance furnace: cosine sampling under a constant probe returns the
  probe radiance exactly in every pixel (the integrand is proportional to the
  density);
* unbiasedness: for an unoccluded, up-facing point under ANY lat-long probe with
  nearest lookup the diffuse integral is the finite sum
  sum_texels L_t (sin^2 theta_j+1 - sin^2 theta_j) / W over the upper bands;
  every technique alone and the MIS mix converge to it;
* polar cap of half-angle theta_c: L sin^2 theta_c;
* mirror limit: a smooth (alpha -> 0) conductor with F0 = 1 reflects the probe
  texel in the mirror direction;
* specular albedo: the estimator converges to an FP64 quadrature of the lobe;
* visibility: inside a closed mesh every active sample is blocked and the
  result scales by (1 - tau) exactly.
"""
import numpy as np
import pytest

from paper_2206_03380_gb300 import scenes

EMPTY_V = np.zeros((3, 3), np.float32)
EMPTY_T = np.zeros((0, 3), np.int32)


def gb_rows(n_pix, p, N, kd, korm):
    g = np.zeros((n_pix, 16), np.float32)
    g[:, 0:3] = p
    g[:, 3] = 1.0
    g[:, 4:7] = N
    g[:, 8:11] = kd
    g[:, 12:15] = korm
    return g


def run(orc, env, n_pix, p, N, cam, kd, korm, split, seed=1, verts=EMPTY_V, tris=EMPTY_T, tau=0.0, records=False):
    cond, marg, _, tot = orc.envmap_cdf(env)
    g = gb_rows(n_pix, p, N, kd, korm)
    ctr = np.stack([np.arange(n_pix), np.zeros(n_pix)], axis=1).astype(np.uint32)
    cam_rows = np.tile(np.asarray(cam, np.float64), (n_pix, 1))
    return orc.shade_fwd(verts, tris, env, cond.astype(np.float32), marg.astype(np.float32), tot, g, cam_rows, ctr,
                         n_light=split[0], n_cos=split[1], n_ggx=split[2], seed=seed, tau=tau,
                         want_records=records)


def diffuse_closed_form(env):
    H, W = env.shape[:2]
    th = np.pi * np.arange(H + 1) / H
    band = (np.sin(th[1:]) ** 2 - np.sin(th[:-1]) ** 2) / W
    up = np.arange(H) < H // 2
    return (env[up, :, :3].astype(np.float64) * band[up, None, None]).sum(axis=(0, 1))


def test_cosine_furnace_zero_variance(orc):
    env = np.zeros((16, 32, 4), np.float32)
    env[..., :3] = (0.5, 1.0, 2.0)
    out, _, _ = run(orc, env, 64, [0, 0, 0], [0.3, 0.9, -0.2], [0, 3, 1], [0.2, 0.3, 0.4], [0, 0.5, 0], (0, 8, 0))
    np.testing.assert_allclose(out[:, 0:3], np.tile([0.5, 1.0, 2.0], (64, 1)), rtol=1e-12)


@pytest.mark.parametrize("split", [(8, 0, 0), (0, 8, 0), (0, 0, 8), (4, 2, 2)])
def test_diffuse_converges_to_closed_form(orc, split):
    rng = np.random.default_rng(30)
    env, _ = scenes.env_with_sun_texel(32, 16, rng, gain=50.0)
    exact = diffuse_closed_form(env)
    # roughness 1 so that the GGX technique alone covers the hemisphere
    out, _, _ = run(orc, env, 60000, [0, 0, 0], [0, 1, 0], [0.4, 2.0, 0.7], [0.5, 0.5, 0.5], [0, 1.0, 0], split)
    m = out[:, 0:3].mean(0)
    se = out[:, 0:3].std(0) / np.sqrt(len(out))
    assert np.all(np.abs(m - exact) < 4.5 * se + 1e-9 * exact), (m, exact, se)


def test_polar_cap_closed_form(orc):
    H, W, k = 16, 32, 5
    env = np.zeros((H, W, 4), np.float32)
    env[:k, :, :3] = 3.0
    out, _, _ = run(orc, env, 40000, [0, 0, 0], [0, 1, 0], [0, 2.0, 0], [1, 1, 1], [0, 0.5, 0], (4, 2, 2))
    exact = 3.0 * np.sin(np.pi * k / H) ** 2
    m = out[:, 0].mean()
    se = out[:, 0].std() / np.sqrt(len(out))
    assert abs(m - exact) < 4.5 * se, (m, exact, se)


def test_mirror_limit_reflects_probe_texel(orc):
    H, W = 32, 64
    env = np.zeros((H, W, 4), np.float32)
    jj, ii = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
    env[..., 0] = 1.0 + 0.02 * ii
    env[..., 1] = 2.0 + 0.05 * jj
    env[..., 2] = 0.5
    # reflect toward the centre of texel (i, j) = (10, 9)
    r = orc.dir_from_uv(10.5 / W, 9.5 / H)
    n = np.array([0.0, 1.0, 0.0])
    wo = 2 * (r @ n) * n - r
    out, _, _ = run(orc, env, 64, [0, 0, 0], n, wo * 4.0, [1, 1, 1], [0, 0.0, 1.0], (0, 0, 4))
    np.testing.assert_allclose(out[:, 6:9], np.tile(env[9, 10, :3], (64, 1)), rtol=2e-4)


@pytest.mark.parametrize("alpha,theta_o", [(0.25, 0.5), (0.6, 1.2)])
def test_specular_albedo_matches_quadrature(orc, alpha, theta_o):
    env = np.ones((16, 32, 4), np.float32)
    n = np.array([0.0, 1.0, 0.0])
    wo = np.array([np.sin(theta_o), np.cos(theta_o), 0.0])
    out, _, _ = run(orc, env, 40000, [0, 0, 0], n, wo * 3, [1, 1, 1], [0, np.sqrt(alpha), 1.0], (4, 2, 2))
    est = out[:, 6].mean()
    se = out[:, 6].std() / np.sqrt(len(out))
    # quadrature of f_s cos_i = D G2 / (4 cos_o) with F = 1 over the upper hemisphere
    nm, nphi = 3000, 1024
    s = (np.arange(nm) + 0.5) / nm
    mu = 1 - s ** 2  # nodes dense near the pole
    wmu = 2 * s / nm
    phi = (np.arange(nphi) + 0.5) * 2 * np.pi / nphi
    M, P = np.meshgrid(mu, phi, indexing="ij")
    st = np.sqrt(1 - M ** 2)
    wi = np.stack([st * np.cos(P), M, st * np.sin(P)], -1).reshape(-1, 3)
    h = wi + wo
    h /= np.linalg.norm(h, axis=1, keepdims=True)
    D = orc.ggx_D_n(h @ n, alpha)
    G2 = orc.ggx_G2_n(wi @ n, np.full(len(wi), wo @ n), alpha)
    f = (D * G2 / (4 * (wo @ n))).reshape(M.shape)
    exact = (f.sum(1) * (2 * np.pi / nphi) * wmu).sum()
    assert abs(est - exact) < 4.5 * se + 1e-4, (est, exact, se)
    assert exact < 1.0


@pytest.mark.parametrize("tau", [0.0, 0.3, 1.0])
def test_closed_mesh_blocks_everything(orc, tau):
    rng = np.random.default_rng(31)
    env, _ = scenes.env_with_sun_texel(32, 16, rng)
    v, _, t = scenes.icosphere(2, radius=2.0, center=(0.1, 0.2, 0.0))
    args = (orc, env, 500, [0, 0, 0], [0.2, 1, 0.1], [0, 1, 3], [0.6, 0.4, 0.2], [0, 0.5, 0.3], (4, 2, 2))
    free, _, _ = run(*args)
    blocked, vis, rec = run(*args, verts=v, tris=t, tau=tau, records=True)
    light = [0, 1, 2, 6, 7, 8]  # c_d and c_s scale by (1 - tau); k_d,out does not
    np.testing.assert_allclose(blocked[:, light], (1 - tau) * free[:, light], rtol=1e-12, atol=1e-300)
    act = rec["active"].astype(bool)
    assert act.sum() > 1000
    bits = ((vis[:, :1] >> np.arange(8, dtype=np.uint32)[None, :]) & 1).astype(bool)
    np.testing.assert_array_equal(bits, act)
    # k_d,out = k_d (1 - m) regardless of light
    np.testing.assert_allclose(blocked[:, 3:6], np.tile([0.6 * 0.7, 0.4 * 0.7, 0.2 * 0.7], (500, 1)), rtol=1e-6)


def test_background_pixel_is_zero(orc):
    rng = np.random.default_rng(32)
    env, _ = scenes.env_with_sun_texel(32, 16, rng)
    cond, marg, _, tot = orc.envmap_cdf(env)
    g = np.zeros((3, 16), np.float32)
    g[1, 3] = 1.0  # covered but zero normal: degenerate, treated as background
    out, vis, _ = orc.shade_fwd(EMPTY_V, EMPTY_T, env, cond.astype(np.float32), marg.astype(np.float32), tot, g,
                                np.zeros((3, 3)), np.zeros((3, 2), np.uint32), n_light=4, n_cos=2, n_ggx=2, seed=3)
    assert np.all(out == 0) and np.all(vis == 0)


def test_surface_does_not_shadow_itself(orc):
    # a point on a ground grid facing up, nothing else in the scene: the grid
    # lies below the offset shadow-ray origin, so the result is unoccluded
    rng = np.random.default_rng(33)
    env, _ = scenes.env_with_sun_texel(32, 16, rng)
    v, _, t = scenes.ground_grid(4, 4, -2.0, 2.0, -2.0, 2.0, 0.0)
    args = (orc, env, 2000, [0.13, 0.0, -0.27], [0, 1, 0], [0, 2, 3], [0.5, 0.5, 0.5], [0, 0.6, 0], (4, 2, 2))
    free, _, _ = run(*args)
    on_grid, vis, _ = run(*args, verts=v, tris=t)
    np.testing.assert_array_equal(on_grid, free)
    assert np.all(vis == 0)
