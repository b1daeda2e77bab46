"""Pins of the cross-bilateral denoiser oracle (App. B): limits where the
filter reduces to the identity or to a library Gaussian blur, edge stopping on
depth and normals, exact depth gradients on planes, and the adjoint by the
dot-product identity."""
import numpy as np
import pytest
from scipy import ndimage

from oracle import bilateral_ref as B

H, W = 12, 14


def camera():
    # eye at origin, looking down -z: right +x, up +y, forward -z
    return np.array([[0, 0, 0, 1, 0, 0, 0, 1, 0, 0, 0, -1, 0.5, W / H]], np.float64)


def gbuffer(depth, normal, cov=None):
    """Positions with camera-space depth `depth` (H, W) and the given normals."""
    ys, xs = np.mgrid[0:H, 0:W].astype(np.float64)
    pos = np.zeros((1, H, W, 4))
    pos[0, ..., 0] = 0.01 * xs
    pos[0, ..., 1] = -0.01 * ys
    pos[0, ..., 2] = -depth
    pos[0, ..., 3] = 1.0 if cov is None else cov
    nrm = np.zeros((1, H, W, 4))
    nrm[0, ..., 0:3] = normal
    return pos, nrm


def test_depth_gradient_is_exact_on_planes_and_one_sided_at_borders():
    ys, xs = np.mgrid[0:H, 0:W].astype(np.float64)
    pos, nrm = gbuffer(3.0 + 0.05 * xs - 0.02 * ys, [0, 0, 1])
    cov, z, gx, gy, n = B.guides(pos, nrm, camera())
    np.testing.assert_allclose(z[0], 3.0 + 0.05 * xs - 0.02 * ys, rtol=1e-14)
    np.testing.assert_allclose(gx[0], 0.05, rtol=1e-10)
    np.testing.assert_allclose(gy[0], -0.02, rtol=1e-10)


def test_tiny_sigma_is_the_identity():
    rng = np.random.default_rng(0)
    pos, nrm = gbuffer(np.full((H, W), 2.0), [0, 0, 1])
    c = rng.uniform(size=(1, H, W, 3))
    out, _ = B.filter_forward(c, pos, nrm, camera(), 1e-4)
    np.testing.assert_array_equal(out, c)


def test_constant_colour_is_preserved():
    rng = np.random.default_rng(1)
    pos, nrm = gbuffer(2.0 + rng.uniform(0, 0.3, size=(H, W)), rng.normal(size=(H, W, 3)))
    c = np.ones((1, H, W, 3)) * np.array([0.3, 1.7, 5.0])
    out, _ = B.filter_forward(c, pos, nrm, camera(), 1.5)
    np.testing.assert_allclose(out, c, rtol=1e-13)


def test_fronto_parallel_plane_is_a_normalised_gaussian_blur():
    rng = np.random.default_rng(2)
    pos, nrm = gbuffer(np.full((H, W), 2.5), [0, 0, 1])
    c = rng.uniform(size=(1, H, W, 3))
    sigma = 1.2
    R = B.footprint_radius(sigma)
    k = np.exp(-(np.arange(-R, R + 1) ** 2) / (2 * sigma ** 2))
    k2 = np.outer(k, k)
    norm = ndimage.correlate(np.ones((H, W)), k2, mode="constant", cval=0.0)
    ref = np.stack([ndimage.correlate(c[0, ..., ch], k2, mode="constant", cval=0.0) / norm for ch in range(3)], -1)
    out, wsum = B.filter_forward(c, pos, nrm, camera(), sigma)
    np.testing.assert_allclose(out[0], ref, rtol=1e-12)
    np.testing.assert_allclose(wsum[0], norm, rtol=1e-12)


def test_depth_and_normal_edges_stop_the_filter():
    ys, xs = np.mgrid[0:H, 0:W]
    left = xs < W // 2
    c = np.where(left[None, ..., None], 1.0, 4.0) * np.ones((1, H, W, 3))
    # depth step between two fronto-parallel planes: the central difference of the two columns at the
    # step straddles it (its linear prediction covers half the step there), every other column is cut off
    pos, nrm = gbuffer(np.where(left, 2.0, 2.6), [0, 0, 1])
    out, _ = B.filter_forward(c, pos, nrm, camera(), 2.0)
    away = (xs < W // 2 - 1) | (xs > W // 2)
    np.testing.assert_allclose(out[0][away], c[0][away], rtol=1e-12)
    assert np.all(np.abs(out[0][~away] - c[0][~away]) > 0.1)
    # equal depth, orthogonal normals
    pos, nrm = gbuffer(np.full((H, W), 2.0), np.where(left[..., None], [0, 0, 1.0], [1.0, 0, 0]))
    out, _ = B.filter_forward(c, pos, nrm, camera(), 2.0)
    np.testing.assert_allclose(out, c, rtol=1e-12)


def test_uncovered_pixels_pass_through_and_are_not_neighbours():
    rng = np.random.default_rng(3)
    cov = (rng.uniform(size=(H, W)) > 0.3).astype(np.float64)
    pos, nrm = gbuffer(np.full((H, W), 2.0), [0, 0, 1], cov)
    c = rng.uniform(size=(1, H, W, 3))
    c_mod = c.copy()
    c_mod[0][cov == 0] = 1e6          # uncovered values must not leak
    out, _ = B.filter_forward(c_mod, pos, nrm, camera(), 1.0)
    assert np.all(out[0][cov == 0] == 1e6)
    assert np.all(out[0][cov > 0] < 1.0 + 1e-12)


def test_adjoint_by_the_dot_product_identity():
    rng = np.random.default_rng(4)
    ys, xs = np.mgrid[0:H, 0:W].astype(np.float64)
    cov = (rng.uniform(size=(H, W)) > 0.15).astype(np.float64)
    pos, nrm = gbuffer(2.0 + 0.03 * xs + 0.2 * (ys > 6), rng.normal(size=(H, W, 3)) * 0.2 + [0, 0, 1], cov)
    cams = camera()
    c = rng.normal(size=(2, H, W, 3))
    g = rng.normal(size=(2, H, W, 3))
    out, _ = B.filter_forward(c, pos, nrm, cams, 1.4)
    gin = B.filter_backward(g, pos, nrm, cams, 1.4)
    assert (out * g).sum() == pytest.approx((c * gin).sum(), rel=1e-12)
