"""Pins of the image-loss oracle (App. A): the sRGB transfer function's
published constants, the tonemap's fixed points, exact zeros where prediction
and reference agree, and the autograd adjoint against central differences."""
import numpy as np
import pytest
import torch

from oracle import loss_ref as LR


def test_srgb_transfer_function_constants():
    knee = LR.SRGB_KNEE
    lin = 12.92 * knee
    pw = 1.055 * knee ** (1 / 2.4) - 0.055
    assert abs(lin - pw) < 1e-7          # the two segments meet at the knee (value 0.04045)
    assert lin == pytest.approx(0.040449936, abs=1e-8)
    assert float(LR.srgb(1.0)) == pytest.approx(1.0, abs=1e-15)
    assert float(LR.srgb(0.0)) == 0.0
    y = torch.linspace(0, 2, 2001, dtype=torch.float64)
    assert torch.all(torch.diff(LR.srgb(y)) > 0)


def test_tonemap_fixed_points_and_clamp():
    assert float(LR.tonemap(0.0)) == 0.0
    assert float(LR.tonemap(np.e - 1.0)) == pytest.approx(1.0, abs=1e-14)   # log(e) = 1, Gamma(1) = 1
    assert float(LR.tonemap(-3.0)) == 0.0                                      # negative radiance clamps


def test_loss_vanishes_when_the_composite_matches_a_grey_reference():
    rng = np.random.default_rng(1)
    grey = np.repeat(rng.uniform(0, 5, size=(1, 6, 7, 1)), 3, axis=-1)
    dcd, dcs = grey.copy(), np.zeros_like(grey)  # composite and light sum equal the reference exactly
    kd = np.ones_like(grey)
    L, li, ll, gk, ga, gb = LR.loss_and_grads(kd, dcd, dcs, grey, lam=0.0)
    assert li == 0.0 and L == 0.0
    assert np.all(gk == 0) and np.all(ga == 0) and np.all(gb == 0)   # |0| has zero gradient
    # luminance of a grey light sum equals the value of the grey reference (up to the mean's rounding)
    assert LR.loss_and_grads(kd, dcd, dcs, grey)[2] < 1e-15


def test_adjoint_matches_central_differences():
    rng = np.random.default_rng(2)
    shp = (1, 5, 4, 3)
    kd = rng.uniform(0.05, 1, size=shp)
    dcd = rng.lognormal(0, 1, size=shp)
    dcs = rng.lognormal(-1, 1, size=shp)
    ref = rng.lognormal(0, 1, size=shp)
    L, _, _, gk, ga, gb = LR.loss_and_grads(kd, dcd, dcs, ref)
    eps = 1e-6
    for arr, g in ((kd, gk), (dcd, ga), (dcs, gb)):
        for idx in [(0, 1, 2, 0), (0, 4, 0, 2), (0, 2, 3, 1)]:
            p, m = arr.copy(), arr.copy()
            p[idx] += eps
            m[idx] -= eps
            if arr is kd:
                fp, fm = LR.loss(torch.tensor(p), torch.tensor(dcd), torch.tensor(dcs), torch.tensor(ref))[0], \
                    LR.loss(torch.tensor(m), torch.tensor(dcd), torch.tensor(dcs), torch.tensor(ref))[0]
            elif arr is dcd:
                fp, fm = LR.loss(torch.tensor(kd), torch.tensor(p), torch.tensor(dcs), torch.tensor(ref))[0], \
                    LR.loss(torch.tensor(kd), torch.tensor(m), torch.tensor(dcs), torch.tensor(ref))[0]
            else:
                fp, fm = LR.loss(torch.tensor(kd), torch.tensor(dcd), torch.tensor(p), torch.tensor(ref))[0], \
                    LR.loss(torch.tensor(kd), torch.tensor(dcd), torch.tensor(m), torch.tensor(ref))[0]
            fd = (float(fp) - float(fm)) / (2 * eps)
            assert g[idx] == pytest.approx(fd, rel=1e-6, abs=1e-12)


def test_single_element_gradient_is_the_tonemap_slope():
    # one differing element: dL/dc = sign * T'(c) / (3 N H W), T'(x) = Gamma'(log(x + 1)) / (x + 1)
    n = 2 * 3 * 3
    ref = np.zeros((1, 2, 3, 3))
    dcs = np.zeros_like(ref)
    dcs[0, 1, 2, 1] = 0.7
    _, _, _, _, _, gb = LR.loss_and_grads(np.zeros_like(ref), np.zeros_like(ref), dcs, ref, lam=0.0)
    y = np.log(1.7)
    slope = 1.055 / 2.4 * y ** (1 / 2.4 - 1) / 1.7
    assert gb[0, 1, 2, 1] == pytest.approx(slope / n, rel=1e-12)
    assert np.count_nonzero(gb) == 1
