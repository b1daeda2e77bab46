"""The GPU adjoint against the GPU forward itself (Sec. 4.1 detached sampling
with reused seeds; Sec. 3.1 detached shadows), independently of the oracle:

(iii) central differences (eps = 1e-3) of the GPU forward against the GPU
      adjoint, per pixel, for k_d, roughness, metallic and the normal, and per
      texel for a seeded subset of probe texels;
(iv)  the dot-product identity <J v, w> = <v, J^T w> for random directions v,
      with J v from central differences of the GPU forward and J^T w from the
      GPU adjoint with upstream gradient w.

The adjoint differentiates the estimator with sample directions, MIS
denominators and visibility frozen at the current parameters.  The GPU forward
is that frozen estimator wherever its sampling does not depend on the
perturbed parameter, so each parameter is perturbed in a configuration where
this holds: k_d, metallic and probe texels (with the sampling tables built
once) in the full 4 light / 2 cosine / 2 GGX split; roughness with the GGX
technique off (4 light / 4 cosine); the normal with probe samples only (8
light), pixels whose visibility or specular-lobe switch changes under the
perturbation excluded.  For the normal, the finite step must also be small
against the scale on which the integrand bends: the roughness is drawn from
[0.5, 0.9] (a GGX lobe of width alpha = r^2 >= 0.25) and pixels with a sample
within 2e-2 of the horizon (n . w_i, the directions taken from the oracle's
sample records) are left out, where the clamped cosine and the Smith term
change faster than a step of 1e-3 resolves; and since a lobe lit by the x1000
sun texel still bends within 1e-3, the normal's difference quotient is taken
at eps and eps / 2 and extrapolated, (4 D(eps/2) - D(eps)) / 3 (Richardson),
which removes the eps^2 term of central differences.  The scene is the 64 x 64 icosphere over the ground
plane with its rasterised G-buffer, k_d and k_orm replaced by seeded values
inside (0, 1).

Rounding: each output is an FP32 sum of S non-negative terms, so its error is
at most (S + 32) u |out| (u = 2^-24; the 32 bounds the roundings inside one
term: the GGX distribution, two Smith terms, Fresnel and the products).
A per-pixel difference quotient therefore carries at most
sum_c |w_c| (S + 32) u (|out+| + |out-|) / (2 eps) of rounding; the checks in
(iii) add that bound to the 1e-3 relative tolerance.  The dot products in
(iv) sum such errors over all pixels with random signs; their tolerance adds 4
standard deviations of that sum (the per-pixel bounds taken as independent).
"""
import numpy as np
import pytest
import torch

from paper_2206_03380_gb300 import scenes
from tests import parity_util as PU

pytestmark = pytest.mark.gpu

EPS = 1e-3
REL = 1e-3
U = 2.0 ** -24


def _np(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy().astype(np.float64)


class Setup:
    def __init__(self, split, seed=41, rough=(0.25, 0.9)):
        from paper_2206_03380_gb300.pipeline import ShadingPipeline

        base = scenes.parity_scene()
        nl, nc, ng = split
        self.sc = scenes.Scene(**{**base.__dict__, "n_light": nl, "n_cos": nc, "n_ggx": ng})
        self.pipe = p = ShadingPipeline(self.sc)
        p.build_probe()
        p.build_bvh()
        p.primary()
        torch.cuda.synchronize()
        rng = np.random.default_rng(seed)
        shape = p.gb.kd.shape
        kd = rng.uniform(0.1, 0.9, size=shape).astype(np.float32)
        korm = np.stack([np.zeros(shape[:3]), rng.uniform(*rough, shape[:3]), rng.uniform(0.1, 0.9, shape[:3]),
                         np.zeros(shape[:3])], -1).astype(np.float32)
        kd[..., 3] = 0
        p.gb.kd.copy_(torch.from_numpy(kd))
        p.gb.korm.copy_(torch.from_numpy(korm))
        self.P = p.N * p.H * p.W
        self.S = self.sc.spp
        self.cov = _np(p.gb.pos)[..., 3].reshape(-1) > 0
        # upstream gradient w of (c_d, kd_out, c_s), zero on uncovered pixels
        w = rng.normal(size=(self.P, 9))
        w[~self.cov] = 0.0
        self.w = w
        wt = torch.from_numpy(w.astype(np.float32)).cuda()
        pad = lambda x: torch.nn.functional.pad(x, (0, 1)).reshape(shape).contiguous()
        self.w32 = w.astype(np.float32).astype(np.float64)
        self.base, self.mask = self.forward()
        p.backward(pad(wt[:, 0:3]), pad(wt[:, 3:6]), pad(wt[:, 6:9]))
        self.g_kd = _np(p.g_kd).reshape(self.P, 4)
        self.g_korm = _np(p.g_korm).reshape(self.P, 4)
        self.g_nrm = _np(p.g_nrm).reshape(self.P, 4)
        self.g_env = _np(p.g_env).reshape(-1, 4)

    def forward(self):
        p = self.pipe
        p.forward()
        out = np.concatenate([_np(p.c_d)[..., :3], _np(p.kd_out)[..., :3], _np(p.c_s)[..., :3]], -1)
        return out.reshape(self.P, 9), _np(p.mask).reshape(self.P, -1).astype(np.int64)

    def central(self, apply, eps):
        """apply(+1 / -1 / 0) sets the perturbed (or base) parameters; returns the per-pixel
        difference quotient of <w, F>, its rounding bound, and whether the pixel's
        visibility changed."""
        apply(+1)
        fp, mp = self.forward()
        apply(-1)
        fm, mm = self.forward()
        apply(0)
        q = (self.w32 * (fp - fm)).sum(1) / (2 * eps)
        bound = (np.abs(self.w32) * (self.S + 32) * U * (np.abs(fp) + np.abs(fm))).sum(1) / (2 * eps)
        flips = (mp != self.mask).any(1) | (mm != self.mask).any(1)
        return q, bound, flips


def _perturb_plane(t, ch, eps, v=None):
    base = t[..., ch].clone()
    d = eps if v is None else eps * v

    def apply(s):
        t[..., ch] = base + s * d

    return apply


def _check_pixels(q, bound, adj, ok, what):
    err = np.abs(q - adj)
    tol = REL * np.abs(adj) + bound + 1e-6 * np.abs(adj).max()
    bad = ok & (err > tol)
    assert ok.sum() > 1000, what
    worst = np.argmax(np.where(ok, err - tol, -np.inf))
    assert not bad.any(), (what, int(bad.sum()), "worst pixel", int(worst), "fd", q[worst], "adjoint", adj[worst],
                           "rounding bound", bound[worst])


@pytest.fixture(scope="module")
def full():
    return Setup((4, 2, 2))


@pytest.mark.parametrize("ch", [0, 1, 2])
def test_fd_kd_matches_adjoint(cuda_lib, full, ch):
    s = full
    q, bound, flips = s.central(_perturb_plane(s.pipe.gb.kd, ch, EPS), EPS)
    assert not flips.any()  # k_d does not move a shadow ray
    _check_pixels(q, bound, s.g_kd[:, ch], s.cov, f"k_d[{ch}]")


def test_fd_metallic_matches_adjoint(cuda_lib, full):
    s = full
    q, bound, flips = s.central(_perturb_plane(s.pipe.gb.korm, 2, EPS), EPS)
    assert not flips.any()
    _check_pixels(q, bound, s.g_korm[:, 2], s.cov, "metallic")
    assert np.all(s.g_korm[:, 0] == 0)  # occlusion has no effect


def test_fd_roughness_matches_adjoint(cuda_lib):
    s = Setup((4, 4, 0))  # GGX technique off: the samples do not depend on the roughness
    q, bound, flips = s.central(_perturb_plane(s.pipe.gb.korm, 1, EPS), EPS)
    assert not flips.any()
    _check_pixels(q, bound, s.g_korm[:, 1], s.cov, "roughness")


def smooth_pixels(orc, s):
    """Pixels whose probe samples all stay 2e-2 away from the horizon, active or not
    (an inactive sample just below it switches on under a small turn of the normal),
    and whose view direction stays 1e-2 away from the specular-lobe switch.  The
    sample directions are the oracle's: its Philox uniforms through its inversion of
    the probe distribution."""
    rows = np.concatenate([_np(t).reshape(-1, 4) for t in (s.pipe.gb.pos, s.pipe.gb.nrm)], 1)
    c32, m32, tot = PU.oracle_tables(orc, s.sc.env)
    S = s.sc.n_light
    u = np.array([orc.sample_uniforms(s.sc.seed, p, 0, j) for p in range(s.P) for j in range(S)])
    dirs, _, _ = orc.sample_light_n(c32, m32, tot, u)
    n = rows[:, 4:7]
    n = n / np.maximum(np.linalg.norm(n, axis=1, keepdims=True), 1e-30)
    cos_i = np.einsum("pjc,pc->pj", dirs.reshape(s.P, S, 3), n)
    wo = s.sc.cams[0, :3][None].astype(np.float64) - rows[:, 0:3]
    wo /= np.maximum(np.linalg.norm(wo, axis=1, keepdims=True), 1e-30)
    return (np.abs(cos_i) >= 2e-2).all(1) & ((n * wo).sum(1) > 1e-2)


@pytest.fixture(scope="module")
def normal_setup(orc):
    s = Setup((8, 0, 0), seed=47, rough=(0.5, 0.9))  # probe samples only: directions and densities fixed
    s.smooth = smooth_pixels(orc, s)
    return s


def richardson(s, make_apply):
    """Central differences at EPS and EPS / 2 extrapolated to remove the eps^2 term;
    the rounding bound of the combination; pixels whose visibility changed at either step."""
    q1, b1, f1 = s.central(make_apply(EPS), EPS)
    q2, b2, f2 = s.central(make_apply(EPS / 2), EPS / 2)
    return (4 * q2 - q1) / 3, (4 * b2 + b1) / 3, f1 | f2


@pytest.mark.parametrize("ch", [0, 1, 2])
def test_fd_normal_matches_adjoint(cuda_lib, normal_setup, ch):
    s = normal_setup
    q, bound, flips = richardson(s, lambda e: _perturb_plane(s.pipe.gb.nrm, ch, e))
    ok = s.cov & ~flips & s.smooth
    assert flips.sum() <= 0.01 * s.cov.sum()
    print(f"normal[{ch}]: {int(ok.sum())} of {int(s.cov.sum())} covered pixels away from the horizon and "
          f"the lobe switch")
    assert ok.sum() >= 0.4 * s.cov.sum()
    _check_pixels(q, bound, s.g_nrm[:, ch], ok, f"normal[{ch}]")


def test_fd_probe_texels_match_adjoint(cuda_lib, full):
    """Probe texels, with the sampling tables of the unperturbed probe (the
    estimator is linear in the texel values it looks up)."""
    s = full
    env = s.pipe.env
    Hp, Wp = env.shape[:2]
    rng = np.random.default_rng(3)
    used = np.nonzero(np.abs(s.g_env[:, :3]).sum(1) > 0)[0]
    top = used[np.argsort(-np.abs(s.g_env[used, :3]).sum(1))[:6]]
    pick = np.unique(np.concatenate([top, rng.choice(used, size=min(10, len(used)), replace=False)]))
    flat = env.view(-1, 4)
    checked = 0
    for t in pick:
        for c in range(3):
            v0 = float(flat[t, c].item())
            eps = EPS * max(abs(v0), 1.0)

            def apply(sg, t=t, c=c, v0=v0, eps=eps):
                flat[t, c] = v0 + sg * eps

            q, bound, flips = s.central(apply, eps)
            assert not flips.any()
            fd, b = q.sum(), bound.sum()
            adj = s.g_env[t, c]
            assert abs(fd - adj) <= REL * abs(adj) + b + 1e-9, (t // Wp, t % Wp, c, fd, adj, b)
            checked += 1
    assert checked >= 30 and Hp * Wp == 32 * 16


def _dot_test(s, perturb, v_dot_adj, eps, extrapolate=False):
    """perturb(sign) applies theta + sign * eps * v (perturb(eps) makes it when extrapolating);
    returns (<Jv, w>, <v, J^T w>, 4-sigma rounding bound)."""
    if extrapolate:
        q, bound, flips = richardson(s, perturb)
    else:
        q, bound, flips = s.central(perturb, eps)
    keep = ~flips
    jv_w = q[keep].sum()
    sigma = np.sqrt((bound[keep] ** 2).sum())
    return jv_w, v_dot_adj(keep), 4 * sigma


def test_dot_product_identity(cuda_lib, full, normal_setup):
    """<J v, w> = <v, J^T w> for random v over (k_d, metallic) jointly, over all
    probe texels, over the roughness and over the normal (each in a split where the
    forward is the frozen estimator)."""
    results = {}
    rng = np.random.default_rng(11)
    # (k_d, metallic): the estimator is bilinear in them (F0 = 0.04 (1 - m) + k_d m), so central
    # differences are exact up to rounding at any step
    s = full
    p = s.pipe
    vkd = rng.normal(size=tuple(p.gb.kd.shape)).astype(np.float32)
    vkd[..., 3] = 0
    vm = rng.normal(size=tuple(p.gb.korm.shape[:3])).astype(np.float32)
    kd0, km0 = p.gb.kd.clone(), p.gb.korm[..., 2].clone()
    vkd_t, vm_t = torch.from_numpy(vkd).cuda(), torch.from_numpy(vm).cuda()
    eps = 1e-2

    def pert_a(sg):
        p.gb.kd.copy_(kd0 + sg * eps * vkd_t)
        p.gb.korm[..., 2] = km0 + sg * eps * vm_t

    def adj_a(keep):
        return ((vkd.reshape(-1, 4)[:, :3] * s.g_kd[:, :3]).sum(1) + vm.reshape(-1) * s.g_korm[:, 2])[keep].sum()

    results["kd_metallic"] = _dot_test(s, pert_a, adj_a, eps)
    # probe texels (linear)
    env0 = p.env.clone()
    venv = rng.normal(size=tuple(p.env.shape)).astype(np.float32) * np.maximum(np.abs(env0.cpu().numpy()), 1.0)
    venv[..., 3] = 0
    venv_t = torch.from_numpy(venv).cuda()

    def pert_e(sg):
        p.env.copy_(env0 + sg * EPS * venv_t)

    results["probe"] = _dot_test(s, pert_e, lambda keep: (venv.reshape(-1, 4)[:, :3] * s.g_env[:, :3]).sum(), EPS)
    # roughness (GGX off)
    sr = Setup((4, 4, 0), seed=43)
    vr = rng.normal(size=tuple(sr.pipe.gb.korm.shape[:3])).astype(np.float32)
    r0, vr_t = sr.pipe.gb.korm[..., 1].clone(), torch.from_numpy(vr).cuda()

    def pert_r(sg):
        sr.pipe.gb.korm[..., 1] = r0 + sg * EPS * vr_t

    results["roughness"] = _dot_test(sr, pert_r, lambda keep: (vr.reshape(-1) * sr.g_korm[:, 1])[keep].sum(), EPS)
    # normal (probe samples only), on the pixels where a step of 1e-3 resolves the integrand
    sn = normal_setup
    vn = rng.normal(size=tuple(sn.pipe.gb.nrm.shape)).astype(np.float32)
    vn[..., 3] = 0
    vn.reshape(-1, 4)[~sn.smooth] = 0
    n0, vn_t = sn.pipe.gb.nrm.clone(), torch.from_numpy(vn).cuda()

    def pert_n(e):
        def apply(sg):
            sn.pipe.gb.nrm.copy_(n0 + sg * e * vn_t)

        return apply

    results["normal"] = _dot_test(sn, pert_n, lambda keep: (vn.reshape(-1, 4)[:, :3] * sn.g_nrm[:, :3])[keep].sum(),
                                  EPS, extrapolate=True)
    for k, (a, b, r) in results.items():
        print(f"dot-product identity {k}: <Jv,w> {a:.9e}  <v,J^T w> {b:.9e}  rel {abs(a - b) / abs(b):.2e}  "
              f"rounding bound {r / abs(b):.2e}")
        assert abs(a - b) <= REL * abs(b) + r, (k, a, b, r)
