"""Pins for the oracle's light-probe distribution (Sec. 4.1 light importance
sampling with a piecewise-constant 2D distribution; App. D).

What fixes it, independent of the oracle's own formulas:
* the density integrates to one over the sphere (uniform-sphere Monte Carlo,
  a parameterisation the oracle does not use);
* sampled directions land in solid-angle bins with the frequency the density
  predicts (chi-square against an independent integral of the density);
* importance is proportional to luminance Y = (r+g+b)/3 times solid angle:
  equal-luminance texels of different colour are drawn equally often, texels
  in different polar bands in proportion to their solid angle;
* a black probe switches the technique off.
"""
import numpy as np
import pytest
from scipy import stats

from paper_2206_03380_gb300 import scenes


def uniform_sphere(n, rng):
    v = rng.normal(size=(n, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def tables(orc, env):
    cond, marg, rs, tot = orc.envmap_cdf(env)
    return cond.astype(np.float32), marg.astype(np.float32), cond, marg, rs, tot


def test_cdf_shape_monotone_and_total(orc):
    rng = np.random.default_rng(1)
    env, _ = scenes.env_with_sun_texel(32, 16, rng)
    env[3, :, :3] = 0.0  # a black row
    env[5, 7, :3] = 0.0  # a black texel
    c32, m32, cond, marg, rs, tot = tables(orc, env)
    assert cond.shape == (16, 33) and marg.shape == (17,)
    assert np.all(np.diff(cond, axis=1) >= 0) and np.all(np.diff(marg) >= 0)
    assert np.all(cond[:, 0] == 0) and np.all(cond[:, -1] == 1) and marg[0] == 0 and marg[-1] == 1
    assert np.isclose(tot, rs.sum(), rtol=1e-14)
    assert rs[3] == 0.0 and marg[4] == marg[3]  # black row has no marginal mass
    np.testing.assert_array_equal(cond[3], np.arange(33) / 32)  # and a uniform conditional
    assert cond[5, 8] == cond[5, 7]  # black texel has no conditional mass


@pytest.mark.parametrize("W,H", [(32, 16), (64, 32)])
def test_light_pdf_integrates_to_one(orc, W, H):
    rng = np.random.default_rng(2)
    env = scenes.env_lognormal(W, H, rng, sigma=0.5)
    c32, m32, *_rest, tot = tables(orc, env)
    d = uniform_sphere(2_000_000, rng)
    p = orc.pdf_light_n(c32, m32, tot, d)
    est = 4 * np.pi * p.mean()
    err = 4 * np.pi * p.std() / np.sqrt(len(p))
    assert abs(est - 1.0) < 5 * err + 1e-3, (est, err)


def test_light_samples_follow_density(orc):
    rng = np.random.default_rng(3)
    env, _ = scenes.env_with_sun_texel(32, 16, rng, gain=20.0)
    c32, m32, *_rest, tot = tables(orc, env)
    n = 400_000
    d, tex, pdf = orc.sample_light_n(c32, m32, tot, rng.uniform(size=(n, 2)))
    # bins: 8 bands equal in z (= equal area) x 12 azimuth sectors
    def bins(v):
        zb = np.clip(((v[:, 1] + 1) / 2 * 8).astype(int), 0, 7)
        pb = np.clip(((np.arctan2(v[:, 2], v[:, 0]) % (2 * np.pi)) / (2 * np.pi) * 12).astype(int), 0, 11)
        return zb * 12 + pb
    counts = np.bincount(bins(d), minlength=96)
    q = uniform_sphere(4_000_000, rng)
    pq = orc.pdf_light_n(c32, m32, tot, q)
    expected_p = np.bincount(bins(q), weights=pq, minlength=96) * (4 * np.pi / len(q))
    expected_p /= expected_p.sum()
    keep = expected_p * n > 20
    chi = ((counts[keep] - n * expected_p[keep]) ** 2 / (n * expected_p[keep])).sum()
    dof = keep.sum() - 1
    # the expected probabilities are themselves Monte Carlo estimates (4M points): allow a margin
    assert chi < dof + 6 * np.sqrt(2 * dof), (chi, dof)
    # density reported with a sample equals the density evaluated at its direction
    sel = np.arange(0, n, 97)
    pe = orc.pdf_light_n(c32, m32, tot, d[sel])
    np.testing.assert_allclose(pdf[sel], pe, rtol=1e-9)


def test_importance_is_luminance_times_solid_angle(orc):
    W, H = 16, 8
    env = np.zeros((H, W, 4), np.float32)
    env[2, 3, :3] = (3.0, 0.0, 0.0)   # Y = 1
    env[2, 9, :3] = (0.0, 0.0, 3.0)   # Y = 1, other colour, same band
    env[2, 12, :3] = (2.0, 2.0, 2.0)  # Y = 2
    env[0, 5, :3] = (1.0, 1.0, 1.0)   # Y = 1 in the polar band
    c32, m32, *_rest, tot = tables(orc, env)
    rng = np.random.default_rng(4)
    n = 400_000
    _, tex, _ = orc.sample_light_n(c32, m32, tot, rng.uniform(size=(n, 2)))
    f = np.bincount(tex, minlength=W * H) / n
    a, b, c, pole = f[2 * W + 3], f[2 * W + 9], f[2 * W + 12], f[0 * W + 5]
    assert set(np.nonzero(f)[0]) == {2 * W + 3, 2 * W + 9, 2 * W + 12, 5}
    assert abs(a / b - 1.0) < 0.03
    assert abs(c / a - 2.0) < 0.06
    # texels of equal luminance are drawn in proportion to their solid angle,
    # (cos(theta_j) - cos(theta_j+1)) * 2 pi / W
    sa = lambda j: np.cos(np.pi * j / H) - np.cos(np.pi * (j + 1) / H)
    ratio = pole / a
    assert abs(ratio / (sa(0) / sa(2)) - 1.0) < 0.03, ratio


def test_black_probe_disables_light_technique(orc):
    env = np.zeros((8, 16, 4), np.float32)
    c32, m32, *_rest, tot = tables(orc, env)
    assert tot == 0.0
    ok, _, _, pdf = orc.sample_light(c32, m32, tot, 0.3, 0.6)
    assert not ok and pdf == 0.0
    assert orc.pdf_light(c32, m32, tot, [0.0, 1.0, 0.0]) == 0.0


def test_texel_lookup_matches_parameterisation(orc):
    W, H = 32, 16
    for j in range(H):
        for i in range(0, W, 5):
            d = orc.dir_from_uv((i + 0.5) / W, (j + 0.5) / H)
            t, bd = orc.texel_of_dir(d, W, H)
            assert t == j * W + i and abs(bd - 0.5) < 1e-9
    # y up: the first band is around +y, u = 0 is +x, u = 1/4 is +z
    np.testing.assert_allclose(orc.dir_from_uv(0.0, 0.0), [0, 1, 0], atol=1e-15)
    np.testing.assert_allclose(orc.dir_from_uv(0.0, 0.5), [1, 0, 0], atol=1e-15)
    np.testing.assert_allclose(orc.dir_from_uv(0.25, 0.5), [0, 0, 1], atol=1e-15)
