"""Pins for the denoiser oracle (Sec. 4.2 neural denoiser, a U-Net; Sec. 4.2's
gradient-sharing argument dL/dX = dL/dO conv F^T).

* the library convolution equals the textbook zero-padded cross-correlation
  written as explicit loops over taps;
* the input gradient of a convolution is the convolution of the output
  gradient with the flipped, channel-transposed filter (the paper's identity,
  which the CUDA backward implements);
* routing weights that pass one channel straight through pin the wiring: the
  skip path returns the input exactly, the deep path returns the 8x8 block
  maximum upsampled back (three 2x2 max-pools then three nearest 2x upsamples);
* the adjoint equals central differences of the forward (float64);
* Xavier-uniform initialisation stays within its bound with the right variance.
"""
import numpy as np
import pytest
import torch
import torch.nn.functional as F

from oracle import denoise_ref as D


def test_library_conv_is_textbook_cross_correlation():
    rng = np.random.default_rng(0)
    x = rng.normal(size=(2, 5, 7, 9))
    W = rng.normal(size=(4, 5, 3, 3))
    b = rng.normal(size=4)
    got = D.conv3x3(torch.from_numpy(x), torch.from_numpy(W), torch.from_numpy(b)).numpy()
    np.testing.assert_allclose(got, D.conv3x3_direct(x, W, b), rtol=1e-12, atol=1e-12)


def test_input_gradient_is_flipped_transposed_conv():
    rng = np.random.default_rng(1)
    x = torch.from_numpy(rng.normal(size=(2, 6, 8, 10))).requires_grad_(True)
    W = torch.from_numpy(rng.normal(size=(5, 6, 3, 3)))
    g = torch.from_numpy(rng.normal(size=(2, 5, 8, 10)))
    (D.conv3x3(x, W, None) * g).sum().backward()
    flipped = W.flip(2, 3).transpose(0, 1).contiguous()  # (6, 5, 3, 3)
    np.testing.assert_allclose(x.grad.numpy(), D.conv3x3(g, flipped, None).numpy(), rtol=1e-12, atol=1e-12)


def routing_weights(deep: bool):
    """Every conv copies channel 0 of its input (centre tap 1) except the first
    decoder conv of each level, which copies either the upsampled (deep) or the
    skip part of its concatenated input."""
    plan = D.unet_plan()
    w = {}
    for name, ci, co, _ in plan:
        W = np.zeros((co, ci, 3, 3), np.float32)
        src = 0
        if name.startswith("dec") and name.endswith("a"):
            up = ci - {"dec3a": 64, "dec2a": 48, "dec1a": 32}[name]
            src = 0 if deep else up
        W[0, src, 1, 1] = 1.0
        w[name] = (W, np.zeros(co, np.float32))
    return w


@pytest.mark.parametrize("deep", [False, True])
def test_unet_wiring(deep):
    rng = np.random.default_rng(2)
    x = np.abs(rng.normal(size=(2, 9, 16, 24)))  # non-negative: ReLU passes it
    y = D.unet_forward(torch.from_numpy(x), routing_weights(deep)).numpy()
    if not deep:
        np.testing.assert_allclose(y[:, 0], x[:, 0], rtol=0, atol=0)
    else:
        blk = x[:, 0].reshape(2, 2, 8, 3, 8).max(axis=(2, 4))
        np.testing.assert_allclose(y[:, 0], np.repeat(np.repeat(blk, 8, 1), 8, 2), rtol=0, atol=0)
    assert np.all(y[:, 1:] == 0)


def test_unet_adjoint_matches_central_differences():
    rng = np.random.default_rng(3)
    w = D.xavier_weights(7)
    x = rng.normal(size=(1, 9, 8, 8))
    gy = rng.normal(size=(1, 3, 8, 8))
    y, gx, gw = D.unet_forward_backward(x, w, gy)
    loss = lambda xx: float((D.unet_forward(torch.from_numpy(xx), w).numpy() * gy).sum())
    for _ in range(12):
        idx = tuple(rng.integers(0, s) for s in x.shape)
        xp, xm = x.copy(), x.copy()
        xp[idx] += 1e-6
        xm[idx] -= 1e-6
        fd = (loss(xp) - loss(xm)) / 2e-6
        assert abs(fd - gx.numpy()[idx]) <= 1e-6 * max(1.0, abs(fd))
    # one weight entry per conv (float64 copies, small steps: ReLU and max-pool kinks)
    w64 = {n: (a.astype(np.float64), c.astype(np.float64)) for n, (a, c) in w.items()}
    for name, (W, b) in list(w64.items())[::3]:
        k = tuple(rng.integers(0, s) for s in W.shape)
        wp = {n: (a.copy(), c) for n, (a, c) in w64.items()}
        wm = {n: (a.copy(), c) for n, (a, c) in w64.items()}
        wp[name][0][k] += 1e-7
        wm[name][0][k] -= 1e-7
        fd = (float((D.unet_forward(torch.from_numpy(x), wp).numpy() * gy).sum())
              - float((D.unet_forward(torch.from_numpy(x), wm).numpy() * gy).sum())) / 2e-7
        assert abs(fd - gw[name][0].numpy()[k]) <= 1e-5 * max(1.0, abs(fd))


def test_xavier_initialisation():
    w = D.xavier_weights(11)
    for name, ci, co, _ in D.unet_plan():
        W, b = w[name]
        a = np.sqrt(6.0 / (9 * ci + 9 * co))
        assert W.shape == (co, ci, 3, 3) and np.abs(W).max() <= a
        if W.size > 2000:
            assert abs(W.var() / (a * a / 3) - 1) < 0.1
    assert D.rel_l2([1.0, 2.0], [1.0, 2.0]) == 0.0 and D.psnr([1.0, 2.0], [1.0, 2.0]) == float("inf")


def test_bf16_storage_rounds_and_stays_close():
    rng = np.random.default_rng(4)
    w = D.xavier_weights(3)
    x = np.abs(rng.normal(size=(1, 9, 16, 16)))
    gy = rng.normal(size=(1, 3, 16, 16))
    y64, g64, _ = D.unet_forward_backward(x, w, gy)
    y16, g16, _ = D.unet_forward_backward(x, w, gy, storage="bf16")
    assert 1e-4 < D.rel_l2(y16, y64) < 5e-2  # rounding happened, and stays bounded
    # the routing network is exact in either precision when values are representable
    xr = np.round(np.abs(rng.normal(size=(1, 9, 16, 24))) * 8) / 8
    yr = D.unet_forward(xr, routing_weights(False), storage="bf16").numpy()
    np.testing.assert_array_equal(yr[:, 0], xr[:, 0])


# ------------------------------------------------------------------ E4M3 (the FP8 path's quantiser)
def _e4m3_value(code: int) -> float:
    """The OCP FP8 E4M3 format written out: sign, 4 exponent bits (bias 7), 3
    mantissa bits; exponent 0 is subnormal; S.1111.111 is NaN, no infinities."""
    s = -1.0 if code & 0x80 else 1.0
    e, m = (code >> 3) & 0xF, code & 0x7
    if e == 0:
        return s * (m / 8.0) * 2.0 ** -6
    return s * (1.0 + m / 8.0) * 2.0 ** (e - 7)


def test_e4m3_codes_match_the_format_definition():
    codes = [c for c in range(256) if (c & 0x7F) != 0x7F]  # 254 finite codes
    vals = np.array([_e4m3_value(c) for c in codes])
    dec = torch.tensor(codes, dtype=torch.uint8).view(torch.float8_e4m3fn).to(torch.float64).numpy()
    np.testing.assert_array_equal(dec, vals)
    assert vals.max() == 448.0 and np.min(np.abs(vals[vals != 0])) == 2.0 ** -9
    # every finite value is a fixed point of the quantiser at scale 1 (amax = 448)
    t = torch.tensor(vals)
    np.testing.assert_array_equal(D.e4m3_quantize(t, 448.0).numpy(), vals)


def test_e4m3_quantiser_rounds_to_nearest_even_and_saturates():
    q = lambda v: D.e4m3_quantize(torch.tensor([v], dtype=torch.float64), 448.0).item()
    assert q(1.0625) == 1.0      # halfway between 1 and 1.125: even mantissa
    assert q(1.1875) == 1.25     # halfway between 1.125 and 1.25: even mantissa
    assert q(17.0) == 16.0 and q(19.0) == 20.0
    assert q(232.0) == 224.0 and q(248.0) == 256.0
    assert q(500.0) == 448.0 and q(-1e6) == -448.0
    assert q(2.0 ** -10) == 0.0 and q(1.5 * 2.0 ** -10) == 2.0 ** -9
    # per-tensor scale: the largest magnitude maps onto 448 and back onto itself
    t = torch.tensor([0.3, -2.5, 7.25, 0.0])
    out = D.e4m3_quantize(t, 7.25).numpy()
    assert out[2] == pytest.approx(7.25, rel=1e-7) and out[3] == 0.0
    assert np.all(np.abs(out - t.numpy()) <= 7.25 / 448 * 8 + 1e-12)  # within half a step of the coarsest binade
    assert np.all(D.e4m3_quantize(t, 0.0).numpy() == 0.0)


def test_e4m3_storage_network_stays_close_and_its_gradient_is_straight_through():
    rng = np.random.default_rng(12)
    weights = D.xavier_weights(77)
    x = rng.normal(size=(2, 9, 16, 16))
    gy = rng.normal(size=(2, 3, 16, 16))
    y64, gx64, _ = D.unet_forward_backward(x, weights, gy)
    y8, gx8, _ = D.unet_forward_backward(x, weights, gy, storage="e4m3")
    yb, gxb, _ = D.unet_forward_backward(x, weights, gy, storage="bf16")
    e8, eb = D.rel_l2(y8, y64), D.rel_l2(yb, y64)
    assert eb < e8 < 0.1  # coarser than bfloat16 (3 mantissa bits against 7), still the same network
    # the input gradient runs through 15 quantised convolutions and as many ReLU masks: coarser still
    assert D.rel_l2(gxb, gx64) < D.rel_l2(gx8, gx64) < 0.6
    # the same quantisation twice gives the same result (deterministic emulation)
    y8b = D.unet_forward(x, weights, storage="e4m3")
    np.testing.assert_array_equal(y8b.numpy(), y8.numpy())
