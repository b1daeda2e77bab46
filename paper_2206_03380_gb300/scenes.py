"""Seeded synthetic inputs shaped like the paper's workloads.

This module is the one thing the CUDA path and the CPU oracle share: it makes
meshes, light probes, material textures and cameras from a seed with numpy's
PCG64 generator, and holds none of the estimator's arithmetic (no sampling,
no BSDF, no visibility).  The paper's datasets (NeRF / NeRFactor synthetic
scenes, its own Apollo, Porsche and Roller scenes, Poly Haven probes) are not
available here; these scenes stand in for them with the same shapes: meshes of
1e3..1e6 triangles extracted from an SDF on a grid with marching tetrahedra
(the paper extracts its mesh from an SDF grid each iteration, Sec. 3), lat-long
HDR probes with strong sun lobes (Sec. 4, "strong directional sunlight"),
spatially varying PBR textures (Sec. 3) and orbiting pinhole cameras.

Layouts (all float32, C-contiguous):
  verts (V, 3), vnrm (V, 3) unit vertex normals, tris (T, 3) int32
  env (H, W, 4) lat-long probe, row j = polar band, column i = azimuth, w = 0
  textures (S, S, 4): k_d -> (r, g, b, 0), k_orm -> (o, r, m, 0)
  camera: 14 floats = origin, right, up, forward, tan(fovy/2), aspect
  uvmap: 3 floats (ox, oz, s): planar texture coordinate ((x-ox) s, (z-oz) s)
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

BASE_SEED = 2206033800


@dataclass
class Scene:
    name: str
    verts: np.ndarray
    vnrm: np.ndarray
    tris: np.ndarray
    env: np.ndarray
    tex_kd: np.ndarray
    tex_korm: np.ndarray
    uvmap: np.ndarray
    cams: np.ndarray  # (N, 14)
    width: int
    height: int
    n_light: int
    n_cos: int
    n_ggx: int
    seed: int
    info: dict = field(default_factory=dict)

    @property
    def spp(self) -> int:
        return self.n_light + self.n_cos + self.n_ggx

    @property
    def n_views(self) -> int:
        return int(self.cams.shape[0])


# ------------------------------------------------------------------ geometry
def icosphere(level: int, radius: float = 1.0, center=(0.0, 0.0, 0.0)):
    """Icosahedron subdivided ``level`` times (20 * 4**level triangles) on a sphere."""
    t = (1.0 + 5.0 ** 0.5) / 2.0
    v = [(-1, t, 0), (1, t, 0), (-1, -t, 0), (1, -t, 0), (0, -1, t), (0, 1, t), (0, -1, -t), (0, 1, -t),
         (t, 0, -1), (t, 0, 1), (-t, 0, -1), (-t, 0, 1)]
    f = [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11), (1, 5, 9), (5, 11, 4), (11, 10, 2),
         (10, 7, 6), (7, 1, 8), (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8), (3, 8, 9), (4, 9, 5), (2, 4, 11),
         (6, 2, 10), (8, 6, 7), (9, 8, 1)]
    verts = [np.array(p, dtype=np.float64) / np.linalg.norm(p) for p in v]
    faces = list(f)
    for _ in range(level):
        mid = {}

        def midpoint(a, b):
            key = (min(a, b), max(a, b))
            if key not in mid:
                p = verts[a] + verts[b]
                verts.append(p / np.linalg.norm(p))
                mid[key] = len(verts) - 1
            return mid[key]

        nf = []
        for a, b, c in faces:
            ab, bc, ca = midpoint(a, b), midpoint(b, c), midpoint(c, a)
            nf += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        faces = nf
    unit = np.array(verts)
    pos = unit * radius + np.asarray(center)
    return pos.astype(np.float32), unit.astype(np.float32), np.array(faces, dtype=np.int32)


def ground_grid(nx: int, nz: int, x0: float, x1: float, z0: float, z1: float, y: float):
    """Flat grid of nx * nz quads (2 triangles each) at height y, normals +y."""
    xs = np.linspace(x0, x1, nx + 1)
    zs = np.linspace(z0, z1, nz + 1)
    X, Z = np.meshgrid(xs, zs, indexing="xy")  # (nz+1, nx+1)
    verts = np.stack([X.ravel(), np.full(X.size, y), Z.ravel()], axis=1)
    idx = np.arange((nx + 1) * (nz + 1)).reshape(nz + 1, nx + 1)
    a = idx[:-1, :-1].ravel()
    b = idx[:-1, 1:].ravel()
    c = idx[1:, :-1].ravel()
    d = idx[1:, 1:].ravel()
    tris = np.concatenate([np.stack([a, b, d], 1), np.stack([a, d, c], 1)], axis=0)
    nrm = np.tile(np.array([0.0, 1.0, 0.0]), (verts.shape[0], 1))
    return verts.astype(np.float32), nrm.astype(np.float32), tris.astype(np.int32)


def merge_meshes(*meshes):
    vs, ns, ts, off = [], [], [], 0
    for v, n, t in meshes:
        vs.append(v)
        ns.append(n)
        ts.append(t + off)
        off += v.shape[0]
    return (np.concatenate(vs).astype(np.float32), np.concatenate(ns).astype(np.float32),
            np.concatenate(ts).astype(np.int32))


# The six tetrahedra of the Kuhn split of a cube along its 0-7 diagonal; cube
# corner c = dx + 2 dy + 4 dz.  Neighbouring cubes split their shared faces the
# same way, so the extracted surface is watertight.
_KUHN = np.array([[0, 1, 3, 7], [0, 1, 5, 7], [0, 2, 3, 7], [0, 2, 6, 7], [0, 4, 5, 7], [0, 4, 6, 7]])


def _tet_cases():
    """Per inside-mask (bit k = vertex k inside): up to two triangles as edge pairs."""
    cases = []
    for mask in range(16):
        ins = [k for k in range(4) if mask >> k & 1]
        out = [k for k in range(4) if not mask >> k & 1]
        if len(ins) in (0, 4):
            cases.append([])
        elif len(ins) == 1 or len(out) == 1:
            a = ins[0] if len(ins) == 1 else out[0]
            others = [k for k in range(4) if k != a]
            cases.append([[(a, others[0]), (a, others[1]), (a, others[2])]])
        else:
            a, b = ins
            c, d = out
            cases.append([[(a, c), (a, d), (b, d)], [(a, c), (b, d), (b, c)]])
    return cases


def marching_tetrahedra(sdf: np.ndarray, lo, hi, normal_fn):
    """Zero level set of ``sdf`` sampled on an n^3 vertex grid spanning [lo, hi]^3.

    Returns float32 verts, unit normals from ``normal_fn(points)``, int32 tris.
    Vertices on shared grid edges are welded.
    """
    n = sdf.shape[0]
    assert sdf.shape == (n, n, n)
    step = (hi - lo) / (n - 1)
    inside = sdf < 0.0  # indexed [z, y, x]
    # cubes that straddle the surface
    cube_any = np.zeros((n - 1,) * 3, dtype=np.int8)
    cube_all = np.ones((n - 1,) * 3, dtype=bool)
    for c in range(8):
        dx, dy, dz = c & 1, c >> 1 & 1, c >> 2 & 1
        sl = inside[dz:dz + n - 1, dy:dy + n - 1, dx:dx + n - 1]
        cube_any |= sl
        cube_all &= sl
    cz, cy, cx = np.nonzero(cube_any.astype(bool) & ~cube_all)
    corner_gid = np.empty((cz.size, 8), dtype=np.int64)
    for c in range(8):
        dx, dy, dz = c & 1, c >> 1 & 1, c >> 2 & 1
        corner_gid[:, c] = (cx + dx) + n * ((cy + dy) + n * (cz + dz))
    flat_sdf = sdf.ravel()
    cases = _tet_cases()
    edge_keys = []
    for tet in _KUHN:
        gid = corner_gid[:, tet]  # (m, 4)
        f = flat_sdf[gid]
        mask = ((f < 0).astype(np.int64) * np.array([1, 2, 4, 8])).sum(1)
        for m in range(1, 15):
            sel = np.nonzero(mask == m)[0]
            if sel.size == 0:
                continue
            g = gid[sel]
            for tri in cases[m]:
                keys = []
                for a, b in tri:
                    ga, gb = g[:, a], g[:, b]
                    keys.append(np.minimum(ga, gb) * (n ** 3) + np.maximum(ga, gb))
                edge_keys.append(np.stack(keys, axis=1))
    tri_keys = np.concatenate(edge_keys, axis=0)
    uniq, inv = np.unique(tri_keys.ravel(), return_inverse=True)
    ga, gb = uniq // (n ** 3), uniq % (n ** 3)
    fa, fb = flat_sdf[ga], flat_sdf[gb]
    t = fa / (fa - fb)

    def coords(g):
        x = g % n
        y = (g // n) % n
        z = g // (n * n)
        return lo + step * np.stack([x, y, z], axis=1).astype(np.float64)

    pa, pb = coords(ga), coords(gb)
    verts = pa + t[:, None] * (pb - pa)
    tris = inv.reshape(-1, 3).astype(np.int32)
    nrm = normal_fn(verts)
    return verts.astype(np.float32), nrm.astype(np.float32), tris


def sphere_union_sdf(centers: np.ndarray, radii: np.ndarray):
    def sdf(p):
        d = np.full(p.shape[:-1], np.inf)
        for c, r in zip(centers, radii):
            d = np.minimum(d, np.linalg.norm(p - c, axis=-1) - r)
        return d

    def normal(p):
        best = np.full(p.shape[0], np.inf)
        nrm = np.zeros_like(p)
        for c, r in zip(centers, radii):
            v = p - c
            l = np.linalg.norm(v, axis=1)
            d = l - r
            take = d < best
            best = np.where(take, d, best)
            nrm[take] = v[take] / np.maximum(l[take], 1e-12)[:, None]
        return nrm

    return sdf, normal


def sdf_spheres_mesh(grid: int, n_spheres: int, rng, r_range=(0.05, 0.3), extent=1.35, spread=0.62):
    centers = rng.uniform(-spread, spread, size=(n_spheres, 3))
    radii = rng.uniform(*r_range, size=n_spheres)
    sdf_fn, nrm_fn = sphere_union_sdf(centers, radii)
    lin = np.linspace(-extent, extent, grid)
    Z, Y, X = np.meshgrid(lin, lin, lin, indexing="ij")
    pts = np.stack([X, Y, Z], axis=-1)
    field_ = np.empty((grid, grid, grid))
    for z in range(grid):  # slab-wise to bound memory
        field_[z] = sdf_fn(pts[z])
    return marching_tetrahedra(field_, -extent, extent, nrm_fn)


def box_sdf(center, half):
    def f(p):
        q = np.abs(p - center) - half
        return np.linalg.norm(np.maximum(q, 0.0), axis=-1) + np.minimum(q.max(axis=-1), 0.0)
    return f


def _box_normal(p, center, half):
    """Gradient of the box distance: toward the nearest point outside, the face
    axis of the largest q inside."""
    v = p - center
    q = np.abs(v) - half
    out = np.maximum(q, 0.0)
    lo = np.linalg.norm(out, axis=1)
    n_out = np.sign(v) * out / np.maximum(lo, 1e-12)[:, None]
    ax = np.argmax(q, axis=1)
    n_in = np.zeros_like(p)
    n_in[np.arange(p.shape[0]), ax] = np.sign(v[np.arange(p.shape[0]), ax])
    return np.where((lo > 0)[:, None], n_out, n_in)


def sdf_union_mesh(grid: int, n_spheres: int, n_boxes: int, rng, extent=1.35, spread=0.62):
    """Marching-tetrahedra mesh of the union of seeded spheres (radii 0.05-0.3) and
    axis-aligned boxes (half extents 0.04-0.22) on a grid^3 lattice; vertex normals
    from the gradient of the nearest primitive."""
    centers = rng.uniform(-spread, spread, size=(n_spheres, 3))
    radii = rng.uniform(0.05, 0.3, size=n_spheres)
    bc = rng.uniform(-spread, spread, size=(n_boxes, 3))
    bh = rng.uniform(0.04, 0.22, size=(n_boxes, 3))
    boxes = [box_sdf(c, h) for c, h in zip(bc, bh)]

    def normal(p):
        best = np.full(p.shape[0], np.inf)
        nrm = np.zeros_like(p)
        for c, r in zip(centers, radii):
            v = p - c
            l = np.linalg.norm(v, axis=1)
            d = l - r
            take = d < best
            best = np.where(take, d, best)
            nrm[take] = v[take] / np.maximum(l[take], 1e-12)[:, None]
        for f, c, h in zip(boxes, bc, bh):
            d = f(p)
            take = d < best
            best = np.where(take, d, best)
            if take.any():
                nrm[take] = _box_normal(p[take], c, h)
        return nrm

    # Each primitive is evaluated only inside its bounding box grown by two cells;
    # elsewhere the field keeps a large positive value.  Marching tetrahedra reads
    # values only for its sign and, on edges where the sign changes, both corners
    # lie within a cell of the surface, inside some primitive's window.
    lin = np.linspace(-extent, extent, grid)
    cell = lin[1] - lin[0]
    field_ = np.full((grid, grid, grid), 1e3)
    prims = [(lambda p, c=c, r=r: np.linalg.norm(p - c, axis=-1) - r, c - r, c + r) for c, r in zip(centers, radii)]
    prims += [(f, c - h, c + h) for f, c, h in zip(boxes, bc, bh)]
    idx = lambda v: int(np.clip(np.floor((v + extent) / cell), 0, grid - 1))
    for f, lo, hi in prims:
        (x0, y0, z0), (x1, y1, z1) = [[idx(v - 2 * cell) for v in lo], [idx(v + 2 * cell) + 1 for v in hi]]
        Z, Y, X = np.meshgrid(lin[z0:z1], lin[y0:y1], lin[x0:x1], indexing="ij")
        sub = f(np.stack([X, Y, Z], axis=-1))
        field_[z0:z1, y0:y1, x0:x1] = np.minimum(field_[z0:z1, y0:y1, x0:x1], sub)
    return marching_tetrahedra(field_, -extent, extent, normal)


# ------------------------------------------------------------------ probes
def _dirs_of_texels(W: int, H: int):
    phi = 2.0 * np.pi * (np.arange(W) + 0.5) / W
    theta = np.pi * (np.arange(H) + 0.5) / H
    T, P = np.meshgrid(theta, phi, indexing="ij")
    return np.stack([np.sin(T) * np.cos(P), np.cos(T), np.sin(T) * np.sin(P)], axis=-1)


def env_lognormal(W: int, H: int, rng, sigma: float = 1.0):
    env = np.zeros((H, W, 4), np.float32)
    env[..., :3] = np.exp(rng.normal(0.0, sigma, size=(H, W, 3)))
    return env


def env_with_sun_texel(W: int, H: int, rng, gain: float = 1000.0):
    env = env_lognormal(W, H, rng)
    j = int(rng.integers(0, H // 2))
    i = int(rng.integers(0, W))
    env[j, i, :3] *= gain
    return env, (i, j)


def env_with_lobes(W: int, H: int, rng, n_lobes: int = 3, peak: float = 1e3, sigma_deg=(1.0, 4.0)):
    env = env_lognormal(W, H, rng)
    dirs = _dirs_of_texels(W, H)
    lobes = []
    for _ in range(n_lobes):
        z = rng.uniform(0.15, 0.95)  # upper hemisphere (y up)
        ph = rng.uniform(0.0, 2.0 * np.pi)
        s = np.sqrt(1.0 - z * z)
        d = np.array([s * np.cos(ph), z, s * np.sin(ph)])
        sig = np.deg2rad(rng.uniform(*sigma_deg))
        ang = np.arccos(np.clip(dirs @ d, -1.0, 1.0))
        tint = rng.uniform(0.8, 1.0, size=3)
        env[..., :3] += (peak * np.exp(-0.5 * (ang / sig) ** 2))[..., None] * tint
        lobes.append((d, sig))
    return env.astype(np.float32), lobes


# ------------------------------------------------------------------ textures
def value_noise(S: int, rng, octaves=(4, 8, 16, 32)):
    """Smooth value noise in [0, 1] on an S x S image (periodic lattice, smoothstep blend)."""
    acc = np.zeros((S, S))
    amp_sum = 0.0
    for k, L in enumerate(octaves):
        lat = rng.uniform(0.0, 1.0, size=(L, L))
        u = (np.arange(S) + 0.5) / S * L
        i0 = np.floor(u).astype(int)
        f = u - i0
        s = f * f * (3.0 - 2.0 * f)
        i0 %= L
        i1 = (i0 + 1) % L
        rows0 = lat[i0][:, i0] * (1 - s)[None, :] + lat[i0][:, i1] * s[None, :]
        rows1 = lat[i1][:, i0] * (1 - s)[None, :] + lat[i1][:, i1] * s[None, :]
        val = rows0 * (1 - s)[:, None] + rows1 * s[:, None]
        amp = 0.5 ** k
        acc += amp * val
        amp_sum += amp
    acc /= amp_sum
    lo, hi = acc.min(), acc.max()
    return (acc - lo) / max(hi - lo, 1e-12)


def pbr_textures(S: int, rng):
    kd = np.zeros((S, S, 4), np.float32)
    for c in range(3):
        kd[..., c] = value_noise(S, rng)
    korm = np.zeros((S, S, 4), np.float32)
    korm[..., 0] = value_noise(S, rng)  # occlusion channel: carried, unused by shading
    korm[..., 1] = 0.08 + 0.92 * value_noise(S, rng)
    m = value_noise(S, rng)
    x = np.clip((m - 0.42) / 0.16, 0.0, 1.0)
    korm[..., 2] = x * x * (3.0 - 2.0 * x)  # metallic blended toward {0, 1}
    return kd, korm


def constant_texture(values):
    t = np.zeros((1, 1, 4), np.float32)
    t[0, 0, :len(values)] = values
    return t


# ------------------------------------------------------------------ cameras
def look_at(eye, target, up, fovy_deg: float, aspect: float):
    eye = np.asarray(eye, np.float64)
    fwd = np.asarray(target, np.float64) - eye
    fwd /= np.linalg.norm(fwd)
    right = np.cross(fwd, np.asarray(up, np.float64))
    right /= np.linalg.norm(right)
    upv = np.cross(right, fwd)
    return np.concatenate([eye, right, upv, fwd, [np.tan(np.deg2rad(fovy_deg) / 2.0), aspect]]).astype(np.float32)


def orbit_cameras(n_total: int, pick, radius: float, fovy_deg: float, aspect: float, rng):
    """``n_total`` seeded viewpoints on a sphere around the origin; returns the rows ``pick``."""
    z = rng.uniform(-0.2, 0.9, size=n_total)
    ph = rng.uniform(0.0, 2.0 * np.pi, size=n_total)
    s = np.sqrt(1.0 - z * z)
    eyes = radius * np.stack([s * np.cos(ph), z, s * np.sin(ph)], axis=1)
    return np.stack([look_at(eyes[k], (0, 0, 0), (0, 1, 0), fovy_deg, aspect) for k in pick])


# ------------------------------------------------------------------ denoiser weights
UNET_SHAPES = [("enc1a", 9, 32), ("enc1b", 32, 32), ("enc2a", 32, 48), ("enc2b", 48, 48), ("enc3a", 48, 64),
               ("enc3b", 64, 64), ("bot_a", 64, 96), ("bot_b", 96, 96), ("dec3a", 160, 64), ("dec3b", 64, 64),
               ("dec2a", 112, 48), ("dec2b", 48, 48), ("dec1a", 80, 32), ("dec1b", 32, 32), ("out", 32, 3)]


def unet_xavier_weights(seed: int):
    """Random denoiser weights (the live-trained denoiser of App. B starts from
    Xavier initialisation): W ~ U(-a, a), a = sqrt(6 / (9 c_in + 9 c_out)), and
    small uniform biases; {name: (W (co, ci, 3, 3), b (co,))} float32."""
    rng = np.random.default_rng(seed)
    out = {}
    for name, ci, co in UNET_SHAPES:
        a = np.sqrt(6.0 / (9 * ci + 9 * co))
        W = rng.uniform(-a, a, size=(co, ci, 3, 3)).astype(np.float32)
        b = rng.uniform(-0.05, 0.05, size=co).astype(np.float32)
        out[name] = (W, b)
    return out


# ------------------------------------------------------------------ workloads
def parity_scene(seed: int = BASE_SEED + 1) -> Scene:
    """64 x 64, one view, 8 spp (4 light, 2 cosine, 2 GGX); icosphere (1,280 tris, r = 1)
    above a 25 x 40 quad ground grid (2,000 tris) at y = -1; camera at (0, 0, 3)
    looking down -z with a 45 degree vertical field of view; uniform k_d = (0.7,
    0.5, 0.3), k_orm = (0, 0.4, 0); 32 x 16 log-normal probe with one sun texel x1000."""
    rng = np.random.default_rng(seed)
    sph = icosphere(3)
    gnd = ground_grid(25, 40, -5.0, 5.0, -8.0, 8.0, -1.0)
    verts, vnrm, tris = merge_meshes(sph, gnd)
    env, sun = env_with_sun_texel(32, 16, rng)
    cam = look_at((0, 0, 3), (0, 0, 0), (0, 1, 0), 45.0, 1.0)[None]
    return Scene("icosphere-ground-64x64-8spp", verts, vnrm, tris, env, constant_texture([0.7, 0.5, 0.3]),
                 constant_texture([0.0, 0.4, 0.0]), np.array([-1.0, -1.0, 0.5], np.float32), cam, 64, 64, 4, 2,
                 2, seed, {"sun_texel": sun})


def sphere_union_scene(seed: int = BASE_SEED + 2, res: int = 512, spp=(8, 4, 4), grid: int = 128,
                       n_spheres: int = 32, tex: int = 1024, env_wh=(512, 256), n_views: int = 1) -> Scene:
    """Marching-tetrahedra mesh of the union of 32 seeded spheres (radii 0.05-0.3) on a
    128^3 grid, 1024^2 value-noise k_d / k_orm textures (roughness 0.08-1, metallic
    blended toward 0/1), a 512 x 256 log-normal probe with three Gaussian sun lobes of
    peak 1e3 (1-4 degrees), a 512^2 view at 16 spp split 8 light / 4 cosine / 4 GGX."""
    rng = np.random.default_rng(seed)
    verts, vnrm, tris = sdf_spheres_mesh(grid, n_spheres, rng)
    kd, korm = pbr_textures(tex, rng)
    env, lobes = env_with_lobes(env_wh[0], env_wh[1], rng)
    cams = orbit_cameras(200, list(range(n_views)), 2.4, 45.0, 1.0, rng)
    return Scene(f"sphere-union-{tris.shape[0]}tris-{res}x{res}-{sum(spp)}spp", verts, vnrm, tris, env, kd, korm,
                 np.array([-1.0, -1.0, 0.5], np.float32), cams, res, res, spp[0], spp[1], spp[2], seed,
                 {"lobes": lobes})


def union_step_scene(seed: int = BASE_SEED + 4, res: int = 800, spp=(16, 8, 8), grid: int = 256,
                     n_spheres: int = 32, n_boxes: int = 32, tex: int = 2048, env_wh=(1024, 512),
                     n_views: int = 8) -> Scene:
    """Optimisation-step batch: 8 of 200 orbit views at 800^2 and 32 spp (16 light,
    8 cosine, 8 GGX) of the union of 32 seeded spheres and 32 boxes extracted on a
    256^3 grid (about a million triangles), 2048^2 value-noise textures and a
    1024 x 512 probe with sun lobes."""
    rng = np.random.default_rng(seed)
    verts, vnrm, tris = sdf_union_mesh(grid, n_spheres, n_boxes, rng)
    kd, korm = pbr_textures(tex, rng)
    env, lobes = env_with_lobes(env_wh[0], env_wh[1], rng)
    pick = sorted(rng.choice(200, size=n_views, replace=False).tolist())
    cams = orbit_cameras(200, pick, 2.4, 45.0, 1.0, rng)
    return Scene(f"union-{tris.shape[0]}tris-{n_views}x{res}x{res}-{sum(spp)}spp", verts, vnrm, tris, env, kd, korm,
                 np.array([-1.0, -1.0, 0.5], np.float32), cams, res, res, spp[0], spp[1], spp[2], seed,
                 {"lobes": lobes, "views": pick})


# ------------------------------------------------------------------ serving stream
@dataclass
class RenderRequest:
    rid: int
    arrival: float  # seconds after the start of the stream
    scene: int
    probe: int
    res: int        # square image side
    spp: int
    view: int       # index into the scene's orbit cameras
    seed: int


def split_spp(spp: int):
    """Light / cosine / GGX sample counts: half probe samples, a quarter each lobe."""
    n_l = spp // 2
    n_c = (spp - n_l) // 2
    return n_l, n_c, spp - n_l - n_c


def poisson_requests(n: int, rate: float, n_scenes: int, n_probes: int, seed: int, res_range=(128, 1024),
                     spp_choices=(4, 8, 16, 32, 64), n_views: int = 200):
    """Poisson arrivals at ``rate`` per second; side uniform over multiples of 32
    in ``res_range``; spp uniform over ``spp_choices``; scene, probe and view uniform."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate, size=n))
    sides = np.arange(res_range[0], res_range[1] + 1, 32)
    out = []
    for k in range(n):
        out.append(RenderRequest(k, float(t[k]), int(rng.integers(n_scenes)), int(rng.integers(n_probes)),
                                 int(rng.choice(sides)), int(rng.choice(spp_choices)), int(rng.integers(n_views)),
                                 int(rng.integers(1, 2 ** 62))))
    return out


def serving_scenes(n_scenes: int = 16, grids=(64, 128, 192, 300), seed: int = BASE_SEED + 5, tex: int = 512):
    """Resident scene set: meshes of the sphere-union family on several grid sizes
    (about 50k to 1M triangles), each scene with its own textures and 200 orbit
    cameras."""
    rng = np.random.default_rng(seed)
    meshes = [sdf_spheres_mesh(g, 32, np.random.default_rng(seed + g)) for g in grids]
    out = []
    for k in range(n_scenes):
        v, n, t = meshes[k % len(meshes)]
        kd, korm = pbr_textures(tex, rng)
        cams = orbit_cameras(200, list(range(200)), 2.4, 45.0, 1.0, rng)
        out.append(dict(verts=v, vnrm=n, tris=t, tex_kd=kd, tex_korm=korm, cams=cams,
                        uvmap=np.array([-1.0, -1.0, 0.5], np.float32)))
    return out


def serving_probes(n_probes: int = 16, seed: int = BASE_SEED + 6):
    """Probes from 256 x 128 to 1024 x 512 with sun lobes."""
    rng = np.random.default_rng(seed)
    sizes = [(256, 128), (512, 256), (1024, 512)]
    return [env_with_lobes(*sizes[k % len(sizes)], rng)[0] for k in range(n_probes)]
