"""Pins for the oracle's adjoint of the frozen-sample estimator (Sec. 4.1 detached
importance sampling, correlated seeds in forward and backward; Sec. 3.1
detached shadow visibility).

* The frozen estimator evaluated at the forward parameters reproduces the
  forward outputs (same samples, same visibility).
* Its analytic FP64 adjoint matches central finite differences of the frozen
  estimator on every per-pixel parameter (normal, k_d, roughness, metallic;
  the occlusion channel has no effect) and on probe texels.
* The outputs are exactly linear in the probe texels, so the probe gradient
  satisfies <g, out(env + delta)> - <g, out(env)> = <grad_env, delta> for any
  delta, however large.
"""
import numpy as np
import pytest

from paper_2206_03380_gb300 import scenes


@pytest.fixture(scope="module")
def frozen_case(orc):
    return make_frozen_case(orc)


def make_frozen_case(orc):
    sc = scenes.parity_scene()
    rng = np.random.default_rng(40)
    W, H = sc.width, sc.height
    pix = np.arange(0, W * H, 37)
    gb = orc.primary_cast(sc.verts, sc.vnrm, sc.tris, sc.cams[0], W, H, pix, sc.tex_kd, sc.tex_korm, sc.uvmap)
    gb = gb[gb[:, 3] > 0]
    n = len(gb)
    gb[:, 8:11] = rng.uniform(0.05, 0.95, size=(n, 3))  # spatially varying materials
    gb[:, 13] = rng.uniform(0.15, 0.9, size=n)
    gb[:, 14] = rng.uniform(0.0, 1.0, size=n)
    gb[:, 4:7] *= rng.uniform(0.7, 1.4, size=(n, 1))  # unnormalised normals
    g32 = gb.astype(np.float32)
    cond, marg, _, tot = orc.envmap_cdf(sc.env)
    cam = np.tile(sc.cams[0, :3].astype(np.float64), (n, 1))
    ctr = np.stack([np.arange(n), np.zeros(n)], 1).astype(np.uint32)
    out, vis, rec = orc.shade_fwd(sc.verts, sc.tris, sc.env, cond.astype(np.float32), marg.astype(np.float32), tot,
                                  g32, cam, ctr, n_light=4, n_cos=2, n_ggx=2, seed=77, tau=0.2)
    prow = orc.param_rows(g32)
    spec_on = out[:, 9].astype(np.int32)
    env3 = sc.env[..., :3].reshape(-1, 3).astype(np.float64)
    g = rng.normal(size=(n, 9))
    return dict(rec=rec, prow=prow, cam=cam, spec_on=spec_on, env3=env3, out=out, g=g)


def test_frozen_eval_reproduces_forward(orc, frozen_case):
    c = frozen_case
    fe = orc.frozen_eval(c["rec"], c["prow"], c["cam"], c["spec_on"], c["env3"])
    np.testing.assert_allclose(fe, c["out"][:, :9], rtol=1e-12, atol=1e-12 * np.abs(c["out"]).max())
    assert (c["rec"]["active"].sum() > 100) and (c["rec"]["occluded"].sum() > 0)


def _loss(orc, c, prow=None, env3=None):
    fe = orc.frozen_eval(c["rec"], c["prow"] if prow is None else prow, c["cam"], c["spec_on"],
                         c["env3"] if env3 is None else env3)
    return float((fe * c["g"]).sum())


def test_adjoint_matches_central_differences(orc, frozen_case):
    c = frozen_case
    grad, genv = orc.frozen_adjoint(c["rec"], c["prow"], c["cam"], c["spec_on"], c["env3"], c["g"])
    rng = np.random.default_rng(41)
    pixels = rng.choice(len(c["prow"]), size=12, replace=False)
    worst = 0.0
    for q in pixels:
        for k in range(9):  # N.xyz, k_d.rgb, o, r, m
            eps = 1e-6
            pp, pm = c["prow"].copy(), c["prow"].copy()
            pp[q, k] += eps
            pm[q, k] -= eps
            fd = (_loss(orc, c, prow=pp) - _loss(orc, c, prow=pm)) / (2 * eps)
            an = grad[q, k]
            scale = max(abs(fd), abs(an), 1e-6 * np.abs(grad[q]).max(), 1e-12)
            worst = max(worst, abs(fd - an) / scale)
    assert worst < 1e-6, worst
    assert np.all(grad[:, 6] == 0.0)  # occlusion channel unused
    # probe texels touched by samples
    touched = np.unique(c["rec"]["texel"][c["rec"]["active"] == 1])
    for t in rng.choice(touched, size=min(10, len(touched)), replace=False):
        for ch in range(3):
            ep, em = c["env3"].copy(), c["env3"].copy()
            ep[t, ch] += 1e-3
            em[t, ch] -= 1e-3
            fd = (_loss(orc, c, env3=ep) - _loss(orc, c, env3=em)) / 2e-3
            assert abs(fd - genv[t, ch]) <= 1e-9 * max(1.0, abs(fd))


def test_probe_gradient_exactly_linear(orc, frozen_case):
    c = frozen_case
    _, genv = orc.frozen_adjoint(c["rec"], c["prow"], c["cam"], c["spec_on"], c["env3"], c["g"])
    rng = np.random.default_rng(42)
    delta = rng.normal(size=c["env3"].shape) * 50.0
    lhs = _loss(orc, c, env3=c["env3"] + delta) - _loss(orc, c)
    rhs = float((genv * delta).sum())
    assert abs(lhs - rhs) < 1e-9 * max(abs(lhs), 1.0)


def test_adjoint_of_black_pixels_is_zero(orc, frozen_case):
    c = frozen_case
    rec = c["rec"].copy()
    rec["active"][:5] = 0
    g = c["g"].copy()
    g[:5, 3:6] = 0.0  # no upstream on k_d,out either
    grad, _ = orc.frozen_adjoint(rec, c["prow"], c["cam"], c["spec_on"], c["env3"], g)
    assert np.all(grad[:5] == 0.0)


def test_adjoint_scale_bounds_gradient(orc, frozen_case):
    c = frozen_case
    grad, genv, scale, gscale = orc.frozen_adjoint(c["rec"], c["prow"], c["cam"], c["spec_on"], c["env3"], c["g"],
                                                   with_scale=True)
    g0, e0 = orc.frozen_adjoint(c["rec"], c["prow"], c["cam"], c["spec_on"], c["env3"], c["g"])
    np.testing.assert_array_equal(grad, g0)
    np.testing.assert_array_equal(genv, e0)
    assert np.all(scale >= np.abs(grad) * (1 - 1e-12)) and np.all(gscale >= np.abs(genv) * (1 - 1e-12))
    # the scale is homogeneous in the upstream gradient and blind to its sign
    g2 = -2.0 * c["g"]
    _, _, s2, gs2 = orc.frozen_adjoint(c["rec"], c["prow"], c["cam"], c["spec_on"], c["env3"], g2, with_scale=True)
    np.testing.assert_allclose(s2, 2.0 * scale, rtol=1e-12)
    np.testing.assert_allclose(gs2, 2.0 * gscale, rtol=1e-12)
