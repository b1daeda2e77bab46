"""Pins for the oracle's ray/triangle visibility (Sec. 3.1 shadow rays) and its
G-buffer ray cast (stands in for the paper's rasterised primary visibility).

Independent facts used: a ray/plane hit solves a 3x3 linear system (checked
with numpy.linalg.solve); a closed convex mesh blocks every ray from inside and
no ray leaving its surface outward; a line meets a sphere-like mesh exactly
when its distance to the centre is below the inscribed radius; the projected
disk of a sphere fixes the covered pixel count; bilinear filtering reproduces
linear functions and agrees with scipy.ndimage.map_coordinates.
"""
import numpy as np
import pytest
from scipy import ndimage

from paper_2206_03380_gb300 import scenes


def test_ray_triangle_matches_linear_solve(orc):
    rng = np.random.default_rng(20)
    checked = 0
    for _ in range(3000):
        v0, v1, v2 = rng.normal(size=(3, 3))
        o = rng.normal(size=3) * 2
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        hit, t, u, v = orc.ray_triangle(o, d, v0, v1, v2)
        A = np.stack([-d, v1 - v0, v2 - v0], axis=1)
        tt, uu, vv = np.linalg.solve(A, o - v0)
        margin = min(uu, vv, 1 - uu - vv)
        if abs(margin) < 1e-9 or abs(tt) < 1e-9:
            continue
        expect = (margin > 0) and (tt > 0)
        assert hit == expect
        np.testing.assert_allclose([t, u, v], [tt, uu, vv], rtol=1e-8, atol=1e-10)
        checked += 1
    assert checked > 2900


def test_any_hit_convex_closed_mesh(orc):
    verts, _, tris = scenes.icosphere(2, radius=1.0)
    # inscribed radius: smallest distance from the centre to a face plane
    a, b, c = verts[tris[:, 0]], verts[tris[:, 1]], verts[tris[:, 2]]
    nrm = np.cross(b - a, c - a)
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    r_in = np.abs((nrm * a).sum(1)).min()
    rng = np.random.default_rng(21)
    for _ in range(200):
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        o = rng.normal(size=3)
        o *= rng.uniform(0.0, 0.9 * r_in) / np.linalg.norm(o)
        assert orc.any_hit(verts, tris, o, d)  # from inside: always blocked
        p = rng.normal(size=3)
        p = p / np.linalg.norm(p) * 1.0001
        w = rng.normal(size=3)
        w -= min(0.0, w @ p) * p / (p @ p) * 2.0  # reflect into the outward half-space
        w /= np.linalg.norm(w)
        if w @ p > 1e-3:
            assert not orc.any_hit(verts, tris, p, w)  # leaving a convex body outward
    for _ in range(300):
        o = rng.normal(size=3)
        o = o / np.linalg.norm(o) * 3.0
        target = rng.normal(size=3) * 0.7
        d = target - o
        d /= np.linalg.norm(d)
        dist = np.linalg.norm(np.cross(-o, d))
        if dist < r_in - 1e-6:
            assert orc.any_hit(verts, tris, o, d)
        elif dist > 1.0 + 1e-6:
            assert not orc.any_hit(verts, tris, o, d)


def test_any_hit_margin_reports_edge_distance(orc):
    v = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0]], np.float32)
    t = np.array([[0, 1, 2]], np.int32)
    hit, em, tm = orc.any_hit(v, t, [0.25, 0.5, -1.0], [0, 0, 1.0], want_margin=True)
    assert hit and abs(em - 0.25) < 1e-12 and abs(tm - 1.0) < 1e-12
    hit, em, _ = orc.any_hit(v, t, [0.6, 0.6, -1.0], [0, 0, 1.0], want_margin=True)
    assert not hit and abs(em - 0.2) < 1e-7
    assert not orc.any_hit(v, t, [0.25, 0.25, 1.0], [0, 0, 1.0])  # behind the origin: t < 0


def test_closest_hit_is_nearest_solution(orc):
    rng = np.random.default_rng(22)
    verts = rng.normal(size=(60, 3)).astype(np.float32)
    tris = rng.integers(0, 60, size=(40, 3)).astype(np.int32)
    tris = tris[(tris[:, 0] != tris[:, 1]) & (tris[:, 1] != tris[:, 2]) & (tris[:, 0] != tris[:, 2])]
    for _ in range(200):
        o = rng.normal(size=3) * 3
        d = -o / np.linalg.norm(o) + rng.normal(size=3) * 0.2
        d /= np.linalg.norm(d)
        best, bt = -1, np.inf
        for k, (a, b, c) in enumerate(verts[tris].astype(np.float64)):
            A = np.stack([-d, b - a, c - a], axis=1)
            if abs(np.linalg.det(A)) < 1e-12:
                continue
            tt, uu, vv = np.linalg.solve(A, o - a)
            if uu >= 0 and vv >= 0 and uu + vv <= 1 and 0 < tt < bt:
                best, bt = k, tt
        k, t, u, v = orc.closest_hit(verts, tris, o, d)
        assert k == best
        if k >= 0:
            assert abs(t - bt) < 1e-9 * max(1, bt)


def test_camera_rays_geometry(orc):
    cam = scenes.look_at((0, 0, 3), (0, 0, 0), (0, 1, 0), 45.0, 1.5)
    W, H = 96, 64
    # mirror-symmetric about the forward axis
    for x, y in [(0, 0), (10, 40), (95, 63)]:
        d1 = orc.camera_ray(cam, W, H, x, y)
        d2 = orc.camera_ray(cam, W, H, W - 1 - x, H - 1 - y)
        f = np.array([0, 0, -1.0])
        np.testing.assert_allclose(d1 + d2, 2 * (d1 @ f) * f, atol=1e-14)
    # vertical extent: pixel-centre rays of the top and bottom rows span the fov less one pixel
    top = orc.camera_ray(cam, W, 1, W // 2, 0)
    assert abs(np.arctan2(top[1], -top[2]) - 0.0) < 1e-14
    t = orc.camera_ray(cam, 1, H, 0, 0)
    b = orc.camera_ray(cam, 1, H, 0, H - 1)
    ang = np.arccos(np.clip(t @ b, -1, 1))
    assert abs(ang - 2 * np.arctan((1 - 1 / H) * np.tan(np.deg2rad(22.5)))) < 1e-6  # float32 camera
    # y grows downward, x to the right
    assert orc.camera_ray(cam, W, H, 0, 0)[1] > 0 and orc.camera_ray(cam, W, H, 0, 0)[0] < 0


def test_primary_cast_sphere_coverage_and_surface(orc):
    verts, vn, tris = scenes.icosphere(3)
    cam = scenes.look_at((0, 0, 3), (0, 0, 0), (0, 1, 0), 45.0, 1.0)
    W = H = 64
    tex_kd = scenes.constant_texture([0.7, 0.5, 0.3])
    tex_korm = scenes.constant_texture([0.0, 0.4, 0.0])
    gb = orc.primary_cast(verts, vn, tris, cam, W, H, np.arange(W * H), tex_kd, tex_korm, [-1, -1, 0.5])
    cov = gb[:, 3] > 0
    # disk radius in pixels: tan(asin(1/3)) / (2 tan(22.5deg) / 64)
    rpix = np.tan(np.arcsin(1 / 3)) / (2 * np.tan(np.deg2rad(22.5)) / W)
    assert abs(cov.sum() / (np.pi * rpix ** 2) - 1.0) < 0.03
    r = np.linalg.norm(gb[cov, :3], axis=1)
    assert r.max() <= 1.0 + 1e-9 and r.min() > 0.99
    assert np.all(gb[cov, 2] > 0)  # the visible hemisphere faces the camera
    np.testing.assert_allclose(gb[cov][:, 8:11], np.tile([0.7, 0.5, 0.3], (cov.sum(), 1)), atol=1e-7)
    np.testing.assert_allclose(gb[cov][:, 13], 0.4, atol=1e-7)
    nrm = gb[cov, 4:7] / np.linalg.norm(gb[cov, 4:7], axis=1, keepdims=True)
    assert np.all((nrm * gb[cov, :3] / r[:, None]).sum(1) > 0.999)
    assert np.all(gb[~cov] == 0)


def test_bilinear_texture(orc):
    rng = np.random.default_rng(23)
    S = 16
    tex = rng.uniform(size=(S, S, 4)).astype(np.float32)
    for _ in range(200):
        u, v = rng.uniform(-0.1, 1.1, size=2)
        got = orc.texture_bilinear(tex, u, v)
        x, y = u * S - 0.5, v * S - 0.5
        ref = [ndimage.map_coordinates(tex[..., c].astype(np.float64), [[y], [x]], order=1, mode="nearest")[0]
               for c in range(4)]
        np.testing.assert_allclose(got, ref, atol=1e-12)
    # a linear ramp is reproduced exactly between texel centres
    ramp = np.zeros((S, S, 4), np.float32)
    ramp[..., 0] = (np.arange(S) + 0.5)[None, :] / S
    ramp[..., 1] = (np.arange(S) + 0.5)[:, None] / S
    for u, v in [(0.2, 0.7), (0.5, 0.5), (0.9, 0.1)]:
        got = orc.texture_bilinear(ramp, u, v)
        assert abs(got[0] - u) < 1e-6 and abs(got[1] - v) < 1e-6


def test_primary_cast_interpolates_vertex_attributes(orc):
    # one triangle with distinct vertex normals; the hit's barycentrics come from a linear solve
    verts = np.array([[-1, -1, 0], [2, -1, 0], [-1, 2, 0]], np.float32)
    vn = np.array([[1, 0, 0], [0, 1, 0], [0, 0, 1]], np.float32)
    tris = np.array([[0, 1, 2]], np.int32)
    cam = scenes.look_at((0.1, 0.2, 4), (0.1, 0.2, 0), (0, 1, 0), 30.0, 1.0)
    W = H = 16
    pix = np.arange(W * H)
    kd = np.zeros((2, 2, 4), np.float32)
    kd[..., 0] = [[0.0, 1.0], [0.0, 1.0]]  # ramp in u
    gb = orc.primary_cast(verts, vn, tris, cam, W, H, pix, kd, kd, [-1.0, -1.0, 0.5])
    hits = np.nonzero(gb[:, 3] > 0)[0]
    assert len(hits) > 50
    for q in hits[::7]:
        d = orc.camera_ray(cam, W, H, q % W, q // W)
        A = np.stack([-d, verts[1] - verts[0], verts[2] - verts[0]], axis=1).astype(np.float64)
        t, u, v = np.linalg.solve(A, cam[:3].astype(np.float64) - verts[0])
        w = 1 - u - v
        np.testing.assert_allclose(gb[q, 4:7], w * vn[0] + u * vn[1] + v * vn[2], atol=1e-9)
        np.testing.assert_allclose(gb[q, 0:3], w * verts[0] + u * verts[1] + v * verts[2], atol=1e-9)
        # planar map: x in [-1, 1] -> tu in [0, 1]; the texture is the ramp 0 -> 1 across two texels
        tu = (gb[q, 0] + 1.0) * 0.5
        exp = np.clip(tu * 2 - 0.5, 0.0, 1.0)
        assert abs(gb[q, 8] - exp) < 1e-9
