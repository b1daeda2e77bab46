"""Pins for the oracle's BSDF and BSDF sampling (Sec. 3: Disney diffuse + isotropic
GGX; Sec. 4.1: cosine sampling and GGX importance sampling after Heitz 2018).

Independent facts used:
* cosine-weighted directions have cos^2(theta) uniform on [0, 1] and uniform azimuth;
* the GGX normal distribution is normalised, int D(h) (n.h) dw_h = 1, and is the
  constant 1/pi at alpha = 1;
* Smith masking satisfies the visible-normal normalisation
  int G1(wo) max(0, wo.h) D(h) dw_h = n.wo (Heitz 2014), and at alpha = 1 has the
  closed form G1(c) = 2c / (1 + c);
* the GGX technique's density integrates to one over the sphere and predicts the
  histogram of its own samples;
* Schlick's Fresnel equals F0 at normal incidence and 1 at grazing.
"""
import numpy as np
import pytest
from scipy import integrate, stats


def uniform_sphere(n, rng):
    v = rng.normal(size=(n, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


NORMALS = [np.array([0.0, 0.0, 1.0]), np.array([0.0, 0.0, -1.0]), np.array([0.0, 1.0, 0.0]),
           np.array([0.48, -0.6, 0.64]), np.array([-0.36, 0.48, -0.8])]


@pytest.mark.parametrize("k", range(len(NORMALS)))
def test_frame_orthonormal(orc, k):
    n = NORMALS[k] / np.linalg.norm(NORMALS[k])
    b1, b2 = orc.frame(n)
    M = np.stack([b1, b2, n])
    np.testing.assert_allclose(M @ M.T, np.eye(3), atol=1e-14)
    np.testing.assert_allclose(np.cross(b1, b2), n, atol=1e-14)


@pytest.mark.parametrize("k", range(len(NORMALS)))
def test_cosine_sampler_distribution(orc, k):
    n = NORMALS[k] / np.linalg.norm(NORMALS[k])
    rng = np.random.default_rng(10 + k)
    d = orc.sample_cosine_n(n, rng.uniform(size=(100_000, 2)))
    np.testing.assert_allclose(np.linalg.norm(d, axis=1), 1.0, atol=1e-14)
    c = d @ n
    assert np.all(c > 0)
    assert stats.kstest(c ** 2, "uniform").pvalue > 1e-4
    b1, b2 = orc.frame(n)
    phi = np.arctan2(d @ b2, d @ b1)
    assert stats.kstest((phi + np.pi) / (2 * np.pi), "uniform").pvalue > 1e-4
    # density integrates to one (uniform-sphere Monte Carlo)
    q = uniform_sphere(1_000_000, rng)
    p = orc.pdf_cosine_n(n, q)
    assert abs(4 * np.pi * p.mean() - 1.0) < 5 * 4 * np.pi * p.std() / 1000 + 1e-3


@pytest.mark.parametrize("alpha", [0.02, 0.1, 0.4, 1.0])
def test_ggx_D_normalised(orc, alpha):
    # int D(h) cos dw = 2 pi int_0^1 D(mu) mu dmu
    f = lambda mu: orc.ggx_D(mu, alpha) * mu
    val, err = integrate.quad(f, 0.0, 1.0, points=[1.0 - 10 * alpha ** 2] if alpha < 0.3 else None, limit=400,
                              epsabs=1e-13, epsrel=1e-11)
    assert abs(2 * np.pi * val - 1.0) < 1e-8
    assert orc.ggx_D(-0.2, alpha) == 0.0


def test_ggx_D_alpha1_constant(orc):
    for mu in [0.01, 0.3, 0.77, 1.0]:
        assert abs(orc.ggx_D(mu, 1.0) - 1.0 / np.pi) < 1e-15


@pytest.mark.parametrize("alpha,theta_o", [(0.1, 0.3), (0.35, 1.0), (0.7, 1.3), (1.0, 0.6)])
def test_smith_visible_normal_normalisation(orc, alpha, theta_o):
    # int G1(wo) max(0, wo.h) D(h) dw_h = n.wo, in spherical coordinates of h about n = z
    wo = np.array([np.sin(theta_o), 0.0, np.cos(theta_o)])
    mu, wmu = np.polynomial.legendre.leggauss(400)
    mu = 0.5 * (mu + 1.0)
    wmu = 0.5 * wmu
    # concentrate nodes near mu = 1 where D peaks: mu = 1 - s^2
    s, ws = np.polynomial.legendre.leggauss(400)
    s = 0.5 * (s + 1.0)
    ws = 0.5 * ws
    mu = 1.0 - s ** 2
    wmu = 2.0 * s * ws
    nphi = 512
    phi = (np.arange(nphi) + 0.5) * 2 * np.pi / nphi
    M, P = np.meshgrid(mu, phi, indexing="ij")
    st = np.sqrt(np.maximum(0.0, 1 - M ** 2))
    h = np.stack([st * np.cos(P), st * np.sin(P), M], axis=-1)
    wh = np.maximum(0.0, h @ wo)
    D = orc.ggx_D_n(M.ravel(), alpha).reshape(M.shape)
    integrand = orc.ggx_G1(wo[2], alpha) * wh * D
    val = (integrand.sum(axis=1) * (2 * np.pi / nphi) * wmu).sum()
    assert abs(val - wo[2]) < 2e-6 * max(1.0, 1 / alpha), (val, wo[2])


def test_smith_G1_alpha1_closed_form(orc):
    for c in [0.05, 0.2, 0.5, 0.9, 1.0]:
        assert abs(orc.ggx_G1(c, 1.0) - 2 * c / (1 + c)) < 1e-14
    # masking vanishes for a smooth surface
    assert abs(orc.ggx_G1(0.3, 1e-6) - 1.0) < 1e-10


@pytest.mark.parametrize("alpha,theta_o", [(0.2, 0.4), (0.5, 1.1), (1.0, 0.2)])
def test_ggx_pdf_integrates_to_one_and_predicts_samples(orc, alpha, theta_o):
    n = np.array([0.0, 1.0, 0.0])
    wo = np.array([np.sin(theta_o), np.cos(theta_o), 0.0])
    rng = np.random.default_rng(int(alpha * 100))
    # 1) normalisation over the sphere: grid in (mu, phi) about n, refined toward the reflection lobe
    nm, nphi = 4000, 2000
    mu = -1 + (np.arange(nm) + 0.5) * 2 / nm
    phi = (np.arange(nphi) + 0.5) * 2 * np.pi / nphi
    M, P = np.meshgrid(mu, phi, indexing="ij")
    st = np.sqrt(np.maximum(0.0, 1 - M ** 2))
    dirs = np.stack([st * np.cos(P), M, st * np.sin(P)], axis=-1).reshape(-1, 3)
    p = orc.pdf_ggx_n(n, wo, alpha, dirs)
    total = p.sum() * (2 / nm) * (2 * np.pi / nphi)
    assert abs(total - 1.0) < 2e-3, total
    # 2) samples: chi-square in 10 mu-bins x 12 phi-bins against the density
    d = orc.sample_ggx_n(n, wo, alpha, rng.uniform(size=(300_000, 2)))
    def bins(v):
        mb = np.clip(((v[:, 1] + 1) / 2 * 10).astype(int), 0, 9)
        pb = np.clip(((np.arctan2(v[:, 2], v[:, 0]) % (2 * np.pi)) / (2 * np.pi) * 12).astype(int), 0, 11)
        return mb * 12 + pb
    counts = np.bincount(bins(d), minlength=120)
    exp = np.bincount(bins(dirs), weights=p, minlength=120) * (2 / nm) * (2 * np.pi / nphi)
    exp = exp / exp.sum() * len(d)
    keep = exp > 30
    chi = ((counts[keep] - exp[keep]) ** 2 / exp[keep]).sum()
    dof = keep.sum() - 1
    assert chi < dof + 6 * np.sqrt(2 * dof), (chi, dof)
    assert counts[~keep].sum() < 0.002 * len(d)


def test_schlick_limits(orc):
    for f0 in [0.04, 0.5, 1.0]:
        assert orc.schlick(f0, 1.0) == f0
        assert abs(orc.schlick(f0, 0.0) - 1.0) < 1e-15
        assert f0 <= orc.schlick(f0, 0.6) <= 1.0


def test_alpha_is_squared_roughness_with_floor(orc):
    assert orc.alpha_of(0.5) == 0.25
    assert orc.alpha_of(0.0) == 1e-4


def test_schlick_spot_values(orc):
    # Schlick 1994: F = F0 + (1 - F0)(1 - cos)^5; at cos = 1/2 the factor is 1/32
    assert abs(orc.schlick(0.04, 0.5) - (0.04 + 0.96 / 32)) < 1e-15
    assert abs(orc.schlick(0.5, 0.0) - 1.0) < 1e-15
