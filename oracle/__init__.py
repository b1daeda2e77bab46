"""FP64 CPU oracle for the Monte Carlo direct-illumination estimator.

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The product path
(``paper_2206_03380_gb300``) never imports it, and this package imports
nothing from the product path: the two share no code.

The arithmetic lives in ``mcdi_oracle.c`` (plain C, double precision, one
pixel and one sample at a time, each function citing the passage of the
paper it follows).  This module only compiles it with gcc and marshals numpy
arrays through ctypes.  ``denoise_ref`` holds the denoiser oracle (PyTorch CPU
float64 library convolutions).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mcdi_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False, src: str = _SRC, out: str = _LIB_PATH) -> str:
    """Compile the oracle with gcc (-O2, IEEE semantics, no FMA contraction)."""
    os.makedirs(os.path.dirname(out), exist_ok=True)
    if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(src):
        return out
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-fno-fast-math", "-o", tmp, src, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


REC_DTYPE = np.dtype([("wi", "<f8", (3,)), ("inv_denom", "<f8"), ("vis", "<f8"), ("margin", "<f8"),
                      ("texel", "<i4"), ("active", "<i4"), ("technique", "<i4"), ("occluded", "<i4")])


class _EdgeParams(C.Structure):
    _fields_ = [("seed", C.c_uint64), ("stream", C.c_uint32), ("n_samples", C.c_int), ("tau", C.c_double),
                ("ray_eps", C.c_double), ("eta", C.c_double)]


class _Params(C.Structure):
    _fields_ = [("n_light", C.c_int), ("n_cos", C.c_int), ("n_ggx", C.c_int), ("stream", C.c_uint32),
                ("seed", C.c_uint64), ("tau", C.c_double), ("ray_eps", C.c_double), ("want_margin", C.c_int)]


def load(path: str | None = None):
    """Load (building if needed) the oracle library; returns the ctypes handle."""
    global _lib
    with _lock:
        if path is not None:
            return _declare(C.CDLL(path))
        if _lib is None:
            _lib = _declare(C.CDLL(build()))
        return _lib


def _declare(lib):
    P = C.c_void_p
    d, i, u32, u64 = C.c_double, C.c_int, C.c_uint32, C.c_uint64
    sig = {
        "orc_philox4x32_10": (None, [P, P, P]),
        "orc_sample_uniforms": (None, [u64, u32, u32, u32, u32, P]),
        "orc_dir_from_uv": (None, [d, d, P]),
        "orc_uv_from_dir": (None, [P, P, P]),
        "orc_texel_of_dir": (i, [P, i, i, P]),
        "orc_envmap_cdf": (None, [P, i, i, P, P, P, P]),
        "orc_sample_light": (i, [P, P, i, i, d, d, d, P, P, P, P]),
        "orc_pdf_light": (d, [P, P, i, i, d, P]),
        "orc_frame": (None, [P, P, P]),
        "orc_sample_cosine": (None, [P, d, d, P]),
        "orc_pdf_cosine": (d, [P, P]),
        "orc_alpha": (d, [d]),
        "orc_ggx_D": (d, [d, d]),
        "orc_ggx_lambda": (d, [d, d]),
        "orc_ggx_G1": (d, [d, d]),
        "orc_ggx_G2": (d, [d, d, d]),
        "orc_schlick": (d, [d, d]),
        "orc_sample_vndf_local": (None, [P, d, d, d, P]),
        "orc_sample_ggx": (None, [P, P, d, d, d, P]),
        "orc_pdf_ggx": (d, [P, P, d, P]),
        "orc_ray_triangle": (i, [P, P, P, P, P, P, P, P]),
        "orc_any_hit": (i, [P, P, i, P, P, P, P]),
        "orc_closest_hit": (i, [P, P, i, P, P, P, P, P]),
        "orc_camera_ray": (None, [P, i, i, i, i, P]),
        "orc_texture_bilinear": (None, [P, i, d, d, P]),
        "orc_primary_cast": (None, [P, P, P, i, P, i, i, P, i, P, P, i, P, P]),
        "orc_shade_fwd": (None, [P, P, i, P, i, i, P, P, d, P, P, P, i, _Params, P, P, P]),
        "orc_frozen_eval": (None, [P, i, i, P, P, P, P, P]),
        "orc_frozen_adjoint": (None, [P, i, i, P, P, P, P, P, P, P, P, P]),
        "orc_sample_rec_size": (i, []),
        "orc_edge_table": (i, [P, i, P]),
        "orc_shadow_edge_grad": (None, [P, P, i, P, i, P, i, i, P, P, P, i, P, P, _EdgeParams, P, P]),
        "orc_pdf_light_n": (None, [P, P, i, i, d, P, i, P]),
        "orc_sample_light_n": (None, [P, P, i, i, d, P, i, P, P, P]),
        "orc_sample_cosine_n": (None, [P, P, i, P]),
        "orc_pdf_cosine_n": (None, [P, P, i, P]),
        "orc_sample_ggx_n": (None, [P, P, d, P, i, P]),
        "orc_pdf_ggx_n": (None, [P, P, d, P, i, P]),
        "orc_ggx_D_n": (None, [P, i, d, P]),
        "orc_ggx_G2_n": (None, [P, P, i, d, P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    assert lib.orc_sample_rec_size() == REC_DTYPE.itemsize, "record layout mismatch"
    return lib


def _p(a):
    return a.ctypes.data_as(C.c_void_p)


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a if shape is None else a.reshape(shape)


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


# ---------------------------------------------------------------- random numbers
def philox4x32_10(ctr, key):
    lib = load()
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, np.uint32)
    lib.orc_philox4x32_10(_p(c), _p(k), _p(out))
    return out


def sample_uniforms(seed, pixel, view, sample, stream=0):
    lib = load()
    u = np.zeros(2)
    lib.orc_sample_uniforms(int(seed), int(pixel), int(view), int(sample), int(stream), _p(u))
    return u


# ---------------------------------------------------------------- probe
def dir_from_uv(u, v):
    out = np.zeros(3)
    load().orc_dir_from_uv(float(u), float(v), _p(out))
    return out


def texel_of_dir(d, W, H):
    d = _f64(d)
    bd = np.zeros(1)
    t = load().orc_texel_of_dir(_p(d), W, H, _p(bd))
    return t, bd[0]


def envmap_cdf(env):
    """env: (H, W, 4) float32 -> (cond (H, W+1), marg (H+1), row_sum (H), total) in float64."""
    env = _f32(env)
    H, W = env.shape[:2]
    cond = np.zeros((H, W + 1))
    marg = np.zeros(H + 1)
    rs = np.zeros(H)
    tot = np.zeros(1)
    load().orc_envmap_cdf(_p(env), W, H, _p(cond), _p(marg), _p(rs), _p(tot))
    return cond, marg, rs, tot[0]


def sample_light(cond32, marg32, total, u0, u1):
    cond32, marg32 = _f32(cond32), _f32(marg32)
    H, W1 = cond32.shape
    d = np.zeros(3)
    t = np.zeros(1, np.int32)
    pdf = np.zeros(1)
    sm = np.zeros(1)
    ok = load().orc_sample_light(_p(cond32), _p(marg32), W1 - 1, H, float(total), float(u0), float(u1), _p(d),
                                 _p(t), _p(pdf), _p(sm))
    return bool(ok), d, int(t[0]), pdf[0]


def pdf_light(cond32, marg32, total, d):
    cond32, marg32 = _f32(cond32), _f32(marg32)
    H, W1 = cond32.shape
    d = _f64(d)
    return load().orc_pdf_light(_p(cond32), _p(marg32), W1 - 1, H, float(total), _p(d))


# ---------------------------------------------------------------- BSDF sampling
def frame(n):
    n = _f64(n)
    b1, b2 = np.zeros(3), np.zeros(3)
    load().orc_frame(_p(n), _p(b1), _p(b2))
    return b1, b2


def sample_cosine(n, u0, u1):
    n = _f64(n)
    d = np.zeros(3)
    load().orc_sample_cosine(_p(n), float(u0), float(u1), _p(d))
    return d


def pdf_cosine(n, d):
    return load().orc_pdf_cosine(_p(_f64(n)), _p(_f64(d)))


def ggx_D(nh, alpha):
    return load().orc_ggx_D(float(nh), float(alpha))


def ggx_lambda(c, alpha):
    return load().orc_ggx_lambda(float(c), float(alpha))


def ggx_G1(c, alpha):
    return load().orc_ggx_G1(float(c), float(alpha))


def ggx_G2(ci, co, alpha):
    return load().orc_ggx_G2(float(ci), float(co), float(alpha))


def schlick(f0, vh):
    return load().orc_schlick(float(f0), float(vh))


def alpha_of(r):
    return load().orc_alpha(float(r))


def sample_ggx(n, wo, alpha, u0, u1):
    d = np.zeros(3)
    load().orc_sample_ggx(_p(_f64(n)), _p(_f64(wo)), float(alpha), float(u0), float(u1), _p(d))
    return d


def pdf_ggx(n, wo, alpha, d):
    return load().orc_pdf_ggx(_p(_f64(n)), _p(_f64(wo)), float(alpha), _p(_f64(d)))


# ---------------------------------------------------------------- visibility
def ray_triangle(o, d, v0, v1, v2):
    t, u, v = np.zeros(1), np.zeros(1), np.zeros(1)
    hit = load().orc_ray_triangle(_p(_f64(o)), _p(_f64(d)), _p(_f64(v0)), _p(_f64(v1)), _p(_f64(v2)), _p(t), _p(u),
                                  _p(v))
    return bool(hit), t[0], u[0], v[0]


def any_hit(verts, tris, o, d, want_margin=False):
    verts, tris = _f32(verts), _i32(tris)
    em, tm = np.zeros(1), np.zeros(1)
    h = load().orc_any_hit(_p(verts), _p(tris), len(tris), _p(_f64(o)), _p(_f64(d)),
                           _p(em) if want_margin else None, _p(tm) if want_margin else None)
    return (bool(h), em[0], tm[0]) if want_margin else bool(h)


def closest_hit(verts, tris, o, d):
    verts, tris = _f32(verts), _i32(tris)
    t, u, v = np.zeros(1), np.zeros(1), np.zeros(1)
    k = load().orc_closest_hit(_p(verts), _p(tris), len(tris), _p(_f64(o)), _p(_f64(d)), _p(t), _p(u), _p(v))
    return k, t[0], u[0], v[0]


# ---------------------------------------------------------------- G-buffer
def camera_ray(cam14, W, H, x, y):
    d = np.zeros(3)
    load().orc_camera_ray(_p(_f64(cam14)), W, H, x, y, _p(d))
    return d


def texture_bilinear(tex, u, v):
    tex = _f32(tex)
    out = np.zeros(4)
    load().orc_texture_bilinear(_p(tex), tex.shape[0], float(u), float(v), _p(out))
    return out


def primary_cast(verts, vnrm, tris, cam14, W, H, pix, tex_kd, tex_korm, uvmap):
    """G-buffer rows (n_pix, 16) float64 for pixels ``pix`` (y*W + x)."""
    verts, vnrm, tris = _f32(verts), _f32(vnrm), _i32(tris)
    pix = _i32(pix)
    tex_kd, tex_korm = _f32(tex_kd), _f32(tex_korm)
    gb = np.zeros((len(pix), 16))
    load().orc_primary_cast(_p(verts), _p(vnrm), _p(tris), len(tris), _p(_f64(cam14)), W, H, _p(pix), len(pix),
                            _p(tex_kd), _p(tex_korm), tex_kd.shape[0], _p(_f64(uvmap)), _p(gb))
    return gb


# ---------------------------------------------------------------- estimator
def shade_fwd(verts, tris, env, cond32, marg32, total, gb_rows, cam_pos_rows, ctr_rows, *, n_light, n_cos, n_ggx,
              seed, stream=0, tau=0.0, ray_eps=1e-4, want_margin=False, want_records=True):
    """Shade listed pixels.

    gb_rows: (n, 16) float32 G-buffer rows (pos4 nrm4 kd4 korm4); cam_pos_rows: (n, 3);
    ctr_rows: (n, 2) uint32 (pixel index in its view, view index).
    Returns (out (n, 12), vis (n, words) uint32, recs (n, spp) REC_DTYPE or None).
    """
    verts, tris, env = _f32(verts), _i32(tris), _f32(env)
    cond32, marg32 = _f32(cond32), _f32(marg32)
    gb_rows = _f32(gb_rows).reshape(-1, 16)
    n = gb_rows.shape[0]
    cam = _f64(cam_pos_rows).reshape(n, 3)
    ctr = np.ascontiguousarray(ctr_rows, dtype=np.uint32).reshape(n, 2)
    spp = n_light + n_cos + n_ggx
    out = np.zeros((n, 12))
    vis = np.zeros((n, (spp + 31) // 32), np.uint32)
    recs = np.zeros((n, spp), REC_DTYPE) if want_records else None
    H, W = env.shape[:2]
    prm = _Params(n_light, n_cos, n_ggx, stream, int(seed), float(tau), float(ray_eps), int(want_margin))
    load().orc_shade_fwd(_p(verts), _p(tris), len(tris), _p(env), W, H, _p(cond32), _p(marg32), float(total),
                         _p(gb_rows), _p(cam), _p(ctr), n, prm, _p(out), _p(vis),
                         _p(recs) if recs is not None else None)
    return out, vis, recs


def edge_table(tris):
    """(E, 4) int32 edge records (a, b, c1, c2) in first-half-edge order."""
    tris = _i32(tris).reshape(-1, 3)
    out = np.zeros((max(3 * len(tris), 1), 4), np.int32)
    n = load().orc_edge_table(_p(tris), len(tris), _p(out))
    return out[:n].copy()


def shadow_edge_grad(verts, tris, edges, env, gb_rows, cam_pos_rows, ctr_rows, gcd, gcs, *, n_samples, seed,
                     stream=2, tau=1.0, ray_eps=1e-4, eta=1e-4, want_records=True):
    """Edge-sampling estimate of the shadow-visibility gradient with respect to
    the vertex positions.  Returns (g_verts (V, 3), rec (n, M, 4) or None);
    rec holds per sample (weight, decision margin, edge index, s)."""
    verts, tris, env = _f32(verts).reshape(-1, 3), _i32(tris).reshape(-1, 3), _f32(env)
    edges = _i32(edges).reshape(-1, 4)
    gb_rows = _f32(gb_rows).reshape(-1, 16)
    n = gb_rows.shape[0]
    cam = _f64(cam_pos_rows).reshape(n, 3)
    ctr = np.ascontiguousarray(ctr_rows, dtype=np.uint32).reshape(n, 2)
    gcd, gcs = _f64(gcd).reshape(n, 3), _f64(gcs).reshape(n, 3)
    g = np.zeros((len(verts), 3))
    rec = np.zeros((n, n_samples, 4)) if want_records else None
    H, W = env.shape[:2]
    prm = _EdgeParams(int(seed), int(stream), int(n_samples), float(tau), float(ray_eps), float(eta))
    load().orc_shadow_edge_grad(_p(verts), _p(tris), len(tris), _p(edges), len(edges), _p(env), W, H, _p(gb_rows),
                                _p(cam), _p(ctr), n, _p(gcd), _p(gcs), prm, _p(g),
                                _p(rec) if rec is not None else None)
    return g, rec


def param_rows(gb_rows):
    """Frozen-estimator parameter rows (n, 12): N, k_d, (o,r,m), pos from G-buffer rows."""
    g = np.asarray(gb_rows, dtype=np.float64).reshape(-1, 16)
    return np.concatenate([g[:, 4:7], g[:, 8:11], g[:, 12:15], g[:, 0:3]], axis=1).copy()


def frozen_eval(recs, prow, cam_pos_rows, spec_on, env3):
    recs = np.ascontiguousarray(recs)
    n, spp = recs.shape
    prow = _f64(prow).reshape(n, 12)
    out = np.zeros((n, 9))
    load().orc_frozen_eval(_p(recs), spp, n, _p(prow), _p(_f64(cam_pos_rows)), _p(_i32(spec_on)),
                           _p(_f64(env3)), _p(out))
    return out


def frozen_adjoint(recs, prow, cam_pos_rows, spec_on, env3, g, with_scale=False):
    """Adjoint of frozen_eval.  Returns (grad (n, 9), genv (texels, 3)); with
    with_scale also the per-component sums of |per-sample contribution|."""
    recs = np.ascontiguousarray(recs)
    n, spp = recs.shape
    prow = _f64(prow).reshape(n, 12)
    env3 = _f64(env3)
    grad = np.zeros((n, 9))
    genv = np.zeros_like(env3)
    scale = np.zeros((n, 9)) if with_scale else None
    genv_scale = np.zeros_like(env3) if with_scale else None
    load().orc_frozen_adjoint(_p(recs), spp, n, _p(prow), _p(_f64(cam_pos_rows)), _p(_i32(spec_on)), _p(env3),
                              _p(_f64(g)), _p(grad), _p(genv), _p(scale) if with_scale else None,
                              _p(genv_scale) if with_scale else None)
    return (grad, genv, scale, genv_scale) if with_scale else (grad, genv)


# ---------------------------------------------------------------- batch forms (tests)
def pdf_light_n(cond32, marg32, total, dirs):
    cond32, marg32 = _f32(cond32), _f32(marg32)
    dirs = _f64(dirs).reshape(-1, 3)
    out = np.zeros(len(dirs))
    load().orc_pdf_light_n(_p(cond32), _p(marg32), cond32.shape[1] - 1, cond32.shape[0], float(total), _p(dirs),
                           len(dirs), _p(out))
    return out


def sample_light_n(cond32, marg32, total, u):
    cond32, marg32 = _f32(cond32), _f32(marg32)
    u = _f64(u).reshape(-1, 2)
    n = len(u)
    dirs, tex, pdf = np.zeros((n, 3)), np.zeros(n, np.int32), np.zeros(n)
    load().orc_sample_light_n(_p(cond32), _p(marg32), cond32.shape[1] - 1, cond32.shape[0], float(total), _p(u), n,
                              _p(dirs), _p(tex), _p(pdf))
    return dirs, tex, pdf


def sample_cosine_n(nrm, u):
    u = _f64(u).reshape(-1, 2)
    dirs = np.zeros((len(u), 3))
    load().orc_sample_cosine_n(_p(_f64(nrm)), _p(u), len(u), _p(dirs))
    return dirs


def pdf_cosine_n(nrm, dirs):
    dirs = _f64(dirs).reshape(-1, 3)
    out = np.zeros(len(dirs))
    load().orc_pdf_cosine_n(_p(_f64(nrm)), _p(dirs), len(dirs), _p(out))
    return out


def sample_ggx_n(nrm, wo, alpha, u):
    u = _f64(u).reshape(-1, 2)
    dirs = np.zeros((len(u), 3))
    load().orc_sample_ggx_n(_p(_f64(nrm)), _p(_f64(wo)), float(alpha), _p(u), len(u), _p(dirs))
    return dirs


def pdf_ggx_n(nrm, wo, alpha, dirs):
    dirs = _f64(dirs).reshape(-1, 3)
    out = np.zeros(len(dirs))
    load().orc_pdf_ggx_n(_p(_f64(nrm)), _p(_f64(wo)), float(alpha), _p(dirs), len(dirs), _p(out))
    return out


def ggx_D_n(nh, alpha):
    nh = _f64(nh).ravel()
    out = np.zeros(len(nh))
    load().orc_ggx_D_n(_p(nh), len(nh), float(alpha), _p(out))
    return out


def ggx_G2_n(ci, co, alpha):
    ci, co = _f64(ci).ravel(), _f64(co).ravel()
    out = np.zeros(len(ci))
    load().orc_ggx_G2_n(_p(ci), _p(co), len(ci), float(alpha), _p(out))
    return out
