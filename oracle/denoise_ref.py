"""Denoiser oracle: the U-Net of 3x3 convolutions applied to c_d and c_s
(Sec. 4.2 "Neural denoisers": a direct-prediction U-Net, fully convolutional
and therefore differentiable; App. B: random (Xavier) initialisation for the
live-trained variant), written with plain PyTorch CPU float64 library ops
(conv2d, max_pool2d, nearest interpolate, cat) and autograd for the adjoint.

TEST INFRASTRUCTURE: only the test suite, the smoke check and the benchmark's
CPU-baseline leg may import it.

Reading of the network (the paper names a U-Net, not its exact layers): four
levels of widths (32, 48, 64, 96); two 3x3 zero-padded convolutions per level,
each followed by ReLU; 2x2 max-pool down; nearest 2x upsample, then
concatenation of [upsampled, skip] along channels; a final linear 3x3
convolution to 3 channels.  Input 9 channels per image: the noisy term (c_d or
c_s), k_d and the normal; the two terms form a batch of two images.
"""
from __future__ import annotations

import math

import numpy as np
import torch
import torch.nn.functional as F


def unet_plan(cin: int = 9, cout: int = 3, widths=(32, 48, 64, 96)):
    """Ordered list of (name, c_in, c_out, relu) for the 15 convolutions."""
    w1, w2, w3, w4 = widths
    return [
        ("enc1a", cin, w1, True), ("enc1b", w1, w1, True),
        ("enc2a", w1, w2, True), ("enc2b", w2, w2, True),
        ("enc3a", w2, w3, True), ("enc3b", w3, w3, True),
        ("bot_a", w3, w4, True), ("bot_b", w4, w4, True),
        ("dec3a", w4 + w3, w3, True), ("dec3b", w3, w3, True),
        ("dec2a", w3 + w2, w2, True), ("dec2b", w2, w2, True),
        ("dec1a", w2 + w1, w1, True), ("dec1b", w1, w1, True),
        ("out", w1, cout, False),
    ]


def xavier_weights(seed: int):
    """The seeded denoiser weights both sides receive (from the shared input generator)."""
    from paper_2206_03380_gb300 import scenes

    return scenes.unet_xavier_weights(seed)


def _t(a):
    return torch.as_tensor(np.asarray(a), dtype=torch.float64)


def conv3x3(x, W, b):
    """3x3 convolution with zero padding 1 (cross-correlation, as the library defines it)."""
    return F.conv2d(x, W, b, padding=1)


E4M3_MAX = 448.0


def e4m3_quantize(t, amax):
    """Per-tensor E4M3 quantisation as the FP8 path defines it: scale s = 448 / amax
    (float32), codes = round-to-nearest-even of v * s in float32, saturated to
    +-448 (the OCP FP8 E4M3 format: 4 exponent bits, bias 7, 3 mantissa bits, no
    infinities); returns the dequantised float64 values codes * amax / 448."""
    amax = float(amax)
    if not amax > 0:
        return torch.zeros_like(t, dtype=torch.float64)
    s = torch.tensor(E4M3_MAX, dtype=torch.float32) / torch.tensor(amax, dtype=torch.float32)
    v = (t.to(torch.float32) * s).clamp(-E4M3_MAX, E4M3_MAX)
    return v.to(torch.float8_e4m3fn).to(torch.float64) * (amax / E4M3_MAX)


class _QuantX(torch.autograd.Function):
    """Forward: per-tensor E4M3 quantisation of a convolution input; backward:
    the gradient passes unchanged (the input gradient is computed from the
    quantised operands, not through the rounding)."""

    @staticmethod
    def forward(ctx, x):
        return e4m3_quantize(x, x.abs().max())

    @staticmethod
    def backward(ctx, g):
        return g


class _QuantG(torch.autograd.Function):
    """Forward: identity on a convolution output; backward: the gradient
    arriving there (stored in bfloat16) is quantised per tensor to E4M3 before
    the input-gradient convolution uses it."""

    @staticmethod
    def forward(ctx, z):
        return z.view_as(z)

    @staticmethod
    def backward(ctx, g):
        g = g.to(torch.bfloat16).to(torch.float64)
        return e4m3_quantize(g, g.abs().max())


class _RoundBF16(torch.autograd.Function):
    """Identity up to rounding to bfloat16, in the forward value and in the
    backward gradient: marks a tensor that is stored in bfloat16."""

    @staticmethod
    def forward(ctx, x):
        return x.to(torch.bfloat16).to(x.dtype)

    @staticmethod
    def backward(ctx, g):
        return g.to(torch.bfloat16).to(g.dtype)


def _unet(x, P, storage=None):
    """The network on float64 tensors; P = {name: (W, b)}.  storage="bf16" rounds
    every stored tensor (input, each activation after its ReLU, pooled and
    concatenated tensors) and every gradient of those to bfloat16, which is
    where a bfloat16 implementation takes its discrete decisions (ReLU masks,
    max-pool winners); arithmetic stays float64.  storage="e4m3" stores the
    same way and in addition quantises each convolution's input (per tensor,
    forward) and the gradient entering each input-gradient convolution (per
    tensor, backward) to E4M3; the weights arrive quantised in P."""
    r = _RoundBF16.apply if storage in ("bf16", "e4m3") else (lambda t: t)
    fp8 = storage == "e4m3"

    def conv(name, h, relu):
        z = conv3x3(_QuantX.apply(h) if fp8 else h, *P[name])
        if fp8:
            z = _QuantG.apply(z)
        return r(F.relu(z)) if relu else z

    up = lambda t: F.interpolate(t, scale_factor=2, mode="nearest")
    pool = lambda t: r(F.max_pool2d(t, 2))
    cat = lambda a, b: r(torch.cat([a, b], 1))
    x = r(x)
    e1 = conv("enc1b", conv("enc1a", x, True), True)
    e2 = conv("enc2b", conv("enc2a", pool(e1), True), True)
    e3 = conv("enc3b", conv("enc3a", pool(e2), True), True)
    bt = conv("bot_b", conv("bot_a", pool(e3), True), True)
    d3 = conv("dec3b", conv("dec3a", cat(up(bt), e3), True), True)
    d2 = conv("dec2b", conv("dec2a", cat(up(d3), e2), True), True)
    d1 = conv("dec1b", conv("dec1a", cat(up(d2), e1), True), True)
    return conv("out", d1, False)


def _params(weights, storage, grad=False):
    def w(a):
        t = _t(a)
        if storage == "bf16":
            t = t.to(torch.bfloat16).to(torch.float64)
        elif storage == "e4m3":  # per weight tensor, from the float32 parameters
            t32 = t.to(torch.float32)
            t = e4m3_quantize(t32, t32.abs().max())
        return t.clone().requires_grad_(grad)

    return {k: (w(W), _t(b).clone().requires_grad_(grad)) for k, (W, b) in weights.items()}


def unet_forward(x, weights, storage=None):
    """x: (N, 9, H, W) (H, W divisible by 8) -> y (N, 3, H, W), float64.
    storage="bf16" also rounds the weights to bfloat16."""
    with torch.no_grad():
        return _unet(_t(x), _params(weights, storage), storage)


def unet_forward_backward(x, weights, gy, storage=None):
    """Forward and the adjoint of the scalar <gy, y>: returns (y, gx, {name: (gW, gb)}).
    With storage="bf16" or "e4m3" the upstream gradient is rounded to bfloat16 too."""
    x = _t(x).clone().requires_grad_(True)
    P = _params(weights, storage, grad=True)
    y = _unet(x, P, storage)
    g = _t(gy)
    if storage in ("bf16", "e4m3"):
        g = g.to(torch.bfloat16).to(torch.float64)
    (y * g).sum().backward()
    return y.detach(), x.grad.detach(), {k: (v[0].grad.detach(), v[1].grad.detach()) for k, v in P.items()}


def conv3x3_direct(x, W, b):
    """Textbook 3x3 cross-correlation with zero padding, by explicit loops over taps
    (numpy float64); used to pin the library convolution on tiny inputs."""
    x = np.asarray(x, np.float64)
    N, C, H, Wd = x.shape
    co = W.shape[0]
    xp = np.zeros((N, C, H + 2, Wd + 2))
    xp[:, :, 1:-1, 1:-1] = x
    y = np.zeros((N, co, H, Wd)) + np.asarray(b, np.float64)[None, :, None, None]
    for dy in range(3):
        for dx in range(3):
            patch = xp[:, :, dy:dy + H, dx:dx + Wd]  # (N, C, H, W)
            y += np.einsum("nchw,oc->nohw", patch, np.asarray(W[:, :, dy, dx], np.float64))
    return y


def denoiser_input(term, kd, nrm):
    """(N, H, W, 3) planes -> (N, 9, H, W) float64 network input [term, k_d, normal]."""
    x = np.concatenate([term, kd, nrm], axis=-1).astype(np.float64)
    return torch.from_numpy(np.ascontiguousarray(x.transpose(0, 3, 1, 2)))


def rel_l2(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def psnr(a, ref):
    a = np.asarray(a, np.float64)
    ref = np.asarray(ref, np.float64)
    peak = np.abs(ref).max()
    mse = np.mean((a - ref) ** 2)
    return float("inf") if mse == 0 else float(10 * np.log10(peak * peak / mse))
