"""Image-space loss of the optimisation step, restated from the paper in plain
PyTorch CPU float64 (autograd gives the adjoint).

TEST INFRASTRUCTURE: only the test suite, the smoke check and the benchmark's
CPU-baseline leg may import it.

- Composite (Sec. 4.2 "light separation"): c = k_d,out * D(c_d) + D(c_s).
- Image loss (App. A "Image Loss"): L1 norm of tonemapped colours, tonemap
  T(x) = Gamma(log(x + 1)) with Gamma the sRGB transfer function (linear
  segment 12.92 x up to 0.0031308, else 1.055 x^(1/2.4) - 0.055).
- Lighting regulariser (App. A "Regularizers"): L1 norm between the luminance
  Y = (r + g + b) / 3 of T(D(c_d) + D(c_s)) and the HSV value V = max(r, g, b)
  of T(reference); the final loss weighs it by lambda_light = 0.15.

Readings (the paper does not state them): an "L1 norm" is the mean absolute
difference over all pixels (and colour channels, for the image loss); radiance
below zero, which a denoiser may output, is clamped to 0 before the tonemap
(zero gradient there); |0| has zero gradient.
"""
from __future__ import annotations

import numpy as np
import torch

SRGB_A = 0.055
SRGB_KNEE = 0.0031308
LAMBDA_LIGHT = 0.15


def srgb(y):
    """Gamma: the sRGB transfer function on linear values y >= 0."""
    y = torch.as_tensor(y, dtype=torch.float64)
    return torch.where(y <= SRGB_KNEE, 12.92 * y, (1.0 + SRGB_A) * torch.clamp(y, min=SRGB_KNEE) ** (1.0 / 2.4) - SRGB_A)


def tonemap(x):
    """T(x) = Gamma(log(max(x, 0) + 1))."""
    x = torch.as_tensor(x, dtype=torch.float64)
    return srgb(torch.log(torch.clamp(x, min=0.0) + 1.0))


def loss(kd_out, dcd, dcs, ref, lam: float = LAMBDA_LIGHT):
    """(N, H, W, 3) tensors -> (L, L_image, L_light) as float64 scalars (tensors)."""
    c = kd_out * dcd + dcs
    l_img = (tonemap(c) - tonemap(ref)).abs().mean()
    y = tonemap(dcd + dcs).mean(dim=-1)
    v = tonemap(ref).max(dim=-1).values
    l_light = (y - v).abs().mean()
    return l_img + lam * l_light, l_img, l_light


def loss_and_grads(kd_out, dcd, dcs, ref, lam: float = LAMBDA_LIGHT):
    """Returns (L, L_image, L_light, dL/dk_d,out, dL/dD(c_d), dL/dD(c_s)) as float64 numpy."""
    t = lambda a: torch.as_tensor(np.asarray(a), dtype=torch.float64).clone().requires_grad_(True)
    k, a, b = t(kd_out), t(dcd), t(dcs)
    r = torch.as_tensor(np.asarray(ref), dtype=torch.float64)
    L, li, ll = loss(k, a, b, r, lam)
    L.backward()
    return (L.item(), li.item(), ll.item(), k.grad.numpy(), a.grad.numpy(), b.grad.numpy())
