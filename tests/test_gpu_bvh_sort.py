"""The BVH build's leaf order is the stable sort of the triangles' 30-bit
Morton codes (equal codes in triangle order), whichever sort the build runs:
one kernel per radix pass over tiles of 2,048 positions, each pass's digit
counts made by the kernel before it (meshes of up to 262,144 triangles), or
three passes of three kernels (larger meshes).  The codes are recomputed here in float32 with the build's
arithmetic (Karras 2012's Morton-ordered LBVH): centroid ((a + b) + c) times
float32(1/3); bounds over all centroids; per axis t = (p - lo) / (hi - lo)
clamped to [0, 1] (0.5 for an empty extent), q = min(1023, trunc(1024 t));
bit i of q_x, q_y, q_z at bits 3i + 2, 3i + 1, 3i.  Meshes: triangle soups
with repeated triangles (ties), at sizes of one partial tile, several tiles
with a ragged last one, exactly the limit, and one above it."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

TILE_SORT_MAX = 262_144


def morton_codes(verts, tris):
    v = verts.astype(np.float32)
    a, b, c = v[tris[:, 0]], v[tris[:, 1]], v[tris[:, 2]]
    cen = ((a + b) + c) * np.float32(1.0 / 3.0)
    lo, hi = cen.min(0), cen.max(0)
    ext = hi - lo
    code = np.zeros(len(tris), np.uint32)
    for ax in range(3):
        if ext[ax] > 0:
            t = (cen[:, ax] - lo[ax]) / ext[ax]
        else:
            t = np.full(len(tris), np.float32(0.5))
        t = np.clip(t.astype(np.float32), np.float32(0), np.float32(1))
        q = np.minimum(np.uint32(1023), (t * np.float32(1024)).astype(np.uint32))
        for i in range(10):
            code |= ((q >> i) & 1).astype(np.uint32) << np.uint32(3 * i + 2 - ax)
    return code


def soup(n, seed):
    """n triangles over a clustered point set; every 5th triangle repeats an earlier one."""
    rng = np.random.default_rng(seed)
    n_verts = max(3, n // 2)
    centres = rng.uniform(-1, 1, size=(64, 3))
    verts = (centres[rng.integers(0, 64, n_verts)] + 0.05 * rng.normal(size=(n_verts, 3))).astype(np.float32)
    tris = rng.integers(0, n_verts, size=(n, 3)).astype(np.int32)
    rep = np.arange(5, n, 5)
    tris[rep] = tris[rng.integers(0, 5, len(rep))]
    return verts, tris


@pytest.mark.parametrize("n", [1, 2, 37, 5000, 8192, 100_003, 198_164, TILE_SORT_MAX, TILE_SORT_MAX + 1])
def test_leaf_order_is_the_stable_morton_sort(cuda_lib, n):
    mcdi = cuda_lib
    verts, tris = soup(n, seed=n)
    dev = torch.device("cuda")
    bvh = mcdi.Bvh.allocate(n, dev).build(torch.from_numpy(verts).to(dev), torch.from_numpy(tris).to(dev))
    torch.cuda.synchronize()
    order = bvh.tri_records.cpu().numpy()[: n * 48].view(np.float32).reshape(n, 12)[:, 3].view(np.int32)
    expect = np.argsort(morton_codes(verts, tris), kind="stable")
    np.testing.assert_array_equal(order, expect)
    launches = mcdi.bvh_build_launches(n)
    if n <= TILE_SORT_MAX:
        assert launches == 3 + 3 + 2 + 1  # one kernel per pass
    else:
        assert launches == 3 + 9 + 2 + 1
