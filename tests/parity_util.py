"""Helpers shared by the GPU parity tests: run the oracle on chosen pixels and
compare with the CUDA outputs under the stated tolerances.

Tolerances (north star, identical samples): radiance relative error <= 1e-4;
shadow-ray hit/miss agreement >= 99.99% with every mismatch near a triangle
edge; gradient relative error <= 1e-3.  A pixel whose samples include a
discrete decision (CDF bin, texel, horizon test, shadow hit) that the FP32 and
FP64 computations may take differently is "marginal" and compared only through
the counts of such pixels.
"""
import numpy as np

RAD_TOL = 1e-4
GRAD_TOL = 1e-3
MARGIN = 1e-4  # decision margin below which FP32 and FP64 may legitimately differ


def oracle_tables(orc, env):
    cond, marg, rs, tot = orc.envmap_cdf(env)
    return cond.astype(np.float32), marg.astype(np.float32), tot


def rel_err(g, o, floor):
    return np.abs(g - o) / np.maximum(np.abs(o), floor)


def oracle_shade(orc, scene, gb_rows, pix, view, tau=1.0, ray_eps=1e-4, stream=0, margin=True):
    c32, m32, tot = oracle_tables(orc, scene.env)
    cam = np.tile(scene.cams[view, :3].astype(np.float64), (len(pix), 1))
    ctr = np.stack([pix, np.full(len(pix), view)], axis=1).astype(np.uint32)
    return orc.shade_fwd(scene.verts, scene.tris, scene.env, c32, m32, tot, gb_rows, cam, ctr,
                         n_light=scene.n_light, n_cos=scene.n_cos, n_ggx=scene.n_ggx, seed=scene.seed, stream=stream,
                         tau=tau, ray_eps=ray_eps, want_margin=margin)


def compare_radiance(gpu, ora, recs):
    """gpu, ora: (n, 3) of one output; returns (bad mask, marginal mask)."""
    floor = 1e-3 * max(np.abs(ora).mean(), 1e-30)
    err = rel_err(gpu, ora, floor).max(axis=1)
    marginal = (recs["margin"] < MARGIN).any(axis=1)
    return err > RAD_TOL, marginal, err


def mask_bits(words, spp):
    words = np.asarray(words).astype(np.uint32).reshape(len(words), -1)
    j = np.arange(spp)
    return ((words[:, j // 32] >> (j % 32).astype(np.uint32)) & 1).astype(bool)


def flipped_samples(gbits, obits, active, bad_pixels, margin):
    """Samples whose discrete decisions the GPU and the oracle took differently:
    (lower, upper) = (hit flips on active samples + one per pixel outside the
    radiance tolerance, hit flips + every marginal sample of those pixels).  A
    pixel outside the tolerance holds at least one flipped decision (texel, CDF
    bin); flips that leave every pixel inside the tolerance (a sample grazing the
    horizon contributes ~0 either way) are not counted."""
    hits = int(((gbits != obits) & active).sum())
    near = (margin < MARGIN) & ~((gbits != obits) & active)
    return hits + int(bad_pixels.sum()), hits + int(near[bad_pixels].sum())
