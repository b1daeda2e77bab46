"""Cross-bilateral denoiser (App. B "Bilateral Denoiser": the spatial part of
SVGF evaluated densely in the footprint, gradients to the colours only),
restated in numpy float64.

TEST INFRASTRUCTURE: only the test suite, the smoke check and the benchmark's
CPU-baseline leg may import it.

    c_hat(p) = sum_q c(q) w(p, q) / sum_q w(p, q)
    w(p, q)  = exp(-|p - q|^2 / (2 sigma^2))
             * exp(-|z(p) - z(q)| / (sigma_z |grad z(p) . (p - q)| + eps(p)))
             * max(0, n(p) . n(q)) ^ sigma_n
with sigma_z = 1 and sigma_n = 128 as in the paper.

Readings (the paper does not state them): the footprint is the square of
radius R = ceil(2 sigma) pixels; z is the camera-space depth (pos - eye) .
forward of the G-buffer position; grad z(p) is the central difference of z
over the two neighbours in x and in y, one-sided where one neighbour is
uncovered or outside the image, 0 where both are; eps(p) = 1e-3 z(p) keeps
the depth test finite where the predicted difference vanishes; n is the
normalised G-buffer normal; uncovered pixels are neither filtered (their
output is their input) nor used as neighbours.  The filter of view v applies
to images v, v + N, v + 2N, ... of the batch.
"""
from __future__ import annotations

import math

import numpy as np

SIGMA_Z = 1.0
SIGMA_N = 128.0
EPS_REL = 1e-3


def footprint_radius(sigma: float) -> int:
    return max(0, int(math.ceil(2.0 * sigma)))


def guides(gb_pos, gb_nrm, cams):
    """(N, H, W, 4) position / normal planes and (N, 14) cameras -> covered (N,H,W) bool,
    depth z, depth gradient (gx, gy), unit normals (N, H, W, 3); float64."""
    pos = np.asarray(gb_pos, np.float64)
    cov = pos[..., 3] > 0
    eye = np.asarray(cams, np.float64)[:, None, None, 0:3]
    fwd = np.asarray(cams, np.float64)[:, None, None, 9:12]
    z = np.where(cov, ((pos[..., 0:3] - eye) * fwd).sum(-1), 0.0)
    n = np.asarray(gb_nrm, np.float64)[..., 0:3]
    ln = np.linalg.norm(n, axis=-1, keepdims=True)
    n = np.where(ln > 0, n / np.where(ln > 0, ln, 1.0), 0.0)

    def grad(axis):
        zp, cp = np.roll(z, -1, axis=axis), np.roll(cov, -1, axis=axis)   # neighbour at +1
        zm, cm = np.roll(z, 1, axis=axis), np.roll(cov, 1, axis=axis)     # neighbour at -1
        size = z.shape[axis]
        idx = np.arange(size).reshape([-1 if a == axis else 1 for a in range(3)])
        cp = cp & (idx < size - 1)
        cm = cm & (idx > 0)
        return np.where(cp & cm, 0.5 * (zp - zm), np.where(cp, zp - z, np.where(cm, z - zm, 0.0)))

    return cov, z, grad(2), grad(1), n


def weights(cov, z, gx, gy, n, sigma, p_y, p_x, view, radius):
    """Weights w(p, q) of pixel p = (p_y, p_x) of `view` over its footprint, as a
    (2R+1, 2R+1) float64 array (0 outside the image and on uncovered q)."""
    H, W = z.shape[1:]
    R = radius
    out = np.zeros((2 * R + 1, 2 * R + 1))
    zp = z[view, p_y, p_x]
    eps = EPS_REL * abs(zp)
    for dy in range(-R, R + 1):
        for dx in range(-R, R + 1):
            qy, qx = p_y + dy, p_x + dx
            if not (0 <= qy < H and 0 <= qx < W) or not cov[view, qy, qx]:
                continue
            ws = math.exp(-(dx * dx + dy * dy) / (2.0 * sigma * sigma))
            pred = abs(gx[view, p_y, p_x] * dx + gy[view, p_y, p_x] * dy)
            wz = math.exp(-abs(zp - z[view, qy, qx]) / (SIGMA_Z * pred + eps))
            d = float(np.dot(n[view, p_y, p_x], n[view, qy, qx]))
            wn = max(0.0, d) ** SIGMA_N
            out[dy + R, dx + R] = ws * wz * wn
    return out


def filter_forward(c, gb_pos, gb_nrm, cams, sigma, radius=None):
    """c: (n_img, H, W, 3) -> (c_hat, wsum (N, H, W)); loops over pixels (small images only)."""
    c = np.asarray(c, np.float64)
    N = gb_pos.shape[0]
    R = footprint_radius(sigma) if radius is None else radius
    cov, z, gx, gy, n = guides(gb_pos, gb_nrm, cams)
    H, W = z.shape[1:]
    out = c.copy()
    wsum = np.zeros((N, H, W))
    for v in range(N):
        for y in range(H):
            for x in range(W):
                if not cov[v, y, x]:
                    continue
                w = weights(cov, z, gx, gy, n, sigma, y, x, v, R)
                wsum[v, y, x] = w.sum()
                ys, xs = np.nonzero(w)
                for i in range(v, c.shape[0], N):
                    acc = (w[ys, xs, None] * c[i, y + ys - R, x + xs - R]).sum(0)
                    out[i, y, x] = acc / wsum[v, y, x]
    return out, wsum


def filter_backward(g_out, gb_pos, gb_nrm, cams, sigma, radius=None):
    """Adjoint with respect to the colours (the weights are constants): scatters
    g(p) w(p, q) / W(p) onto q; uncovered pixels pass their gradient through."""
    g_out = np.asarray(g_out, np.float64)
    N = gb_pos.shape[0]
    R = footprint_radius(sigma) if radius is None else radius
    cov, z, gx, gy, n = guides(gb_pos, gb_nrm, cams)
    H, W = z.shape[1:]
    g_in = np.zeros_like(g_out)
    for v in range(N):
        unc = ~cov[v]
        for i in range(v, g_out.shape[0], N):
            g_in[i][unc] += g_out[i][unc]
        for y in range(H):
            for x in range(W):
                if not cov[v, y, x]:
                    continue
                w = weights(cov, z, gx, gy, n, sigma, y, x, v, R)
                w = w / w.sum()
                ys, xs = np.nonzero(w)
                for i in range(v, g_out.shape[0], N):
                    g_in[i, y + ys - R, x + xs - R] += w[ys, xs, None] * g_out[i, y, x]
    return g_in
