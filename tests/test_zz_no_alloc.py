"""mcdi_build_bvh_noalloc: the BVH build for callers that cannot allocate device
memory (a plugin inside an application that owns all device allocations, or a
loop whose memory budget is fixed at start-up).  It keeps its scratch in one
fixed array inside the library instead of taking a scratch buffer.

Checked through the C ABI against mcdi_build_bvh with caller-provided scratch
on two calls in a row with different meshes (the second call reuses the array
the first one left behind): nodes and triangle records must match, which is
within any tolerance the other tests use since the build is deterministic.
A mesh of exactly the limit is accepted and matches too.  The entry point's
defining property is checked directly: after a warm-up call, a further call
changes neither the bytes the caching allocator holds nor the device's free
memory.  Sizes above the limit, an empty mesh and a misaligned node buffer are
rejected before anything runs.  This file is collected last so that a
stop-at-first-failure run has run everything else."""
import numpy as np
import pytest
import torch

from paper_2206_03380_gb300 import scenes

pytestmark = pytest.mark.gpu


def _build_both(mcdi, verts_np, tris_np):
    dev = torch.device("cuda")
    verts = torch.from_numpy(np.ascontiguousarray(verts_np, np.float32)).to(dev)
    tris = torch.from_numpy(np.ascontiguousarray(tris_np, np.int32)).to(dev)
    n = tris.shape[0]
    ref = mcdi.Bvh.allocate(n, dev).build(verts, tris)
    nb, tb, _ = mcdi.bvh_sizes(n)
    nodes = torch.full((ref.nodes.numel(),), 0xAB, dtype=torch.uint8, device=dev)
    recs = torch.full((ref.tri_records.numel(),), 0xCD, dtype=torch.uint8, device=dev)
    mcdi.build_bvh_noalloc(verts, tris, nodes, recs)
    torch.cuda.synchronize()
    return (ref.nodes[:nb].cpu().numpy(), ref.tri_records[:tb].cpu().numpy(), nodes[:nb].cpu().numpy(),
            recs[:tb].cpu().numpy())


def test_noalloc_bvh_matches_allocating_build_twice(cuda_lib):
    mcdi = cuda_lib
    sc = scenes.parity_scene()
    big_v, _, big_t = scenes.icosphere(5, radius=0.7, center=(0.2, 0.1, -0.3))  # 20,480 triangles
    for verts, tris in [(big_v, big_t), (sc.verts, sc.tris)]:  # larger mesh first, then a smaller one
        rn, rr, nn, nr = _build_both(mcdi, verts, tris)
        np.testing.assert_array_equal(nn, rn)
        np.testing.assert_array_equal(nr, rr)


def test_noalloc_rejects_meshes_above_the_limit(cuda_lib):
    mcdi = cuda_lib
    n = mcdi.NOALLOC_MAX_TRIS + 1
    dev = torch.device("cuda")
    verts = torch.zeros(3, 3, device=dev)
    tris = torch.zeros(n, 3, dtype=torch.int32, device=dev)
    nodes = torch.empty(64 * n, dtype=torch.uint8, device=dev)
    recs = torch.empty(48 * n, dtype=torch.uint8, device=dev)
    with pytest.raises(mcdi.McdiError) as e:
        mcdi.build_bvh_noalloc(verts, tris, nodes, recs)
    assert e.value.status == mcdi.INVALID_ARG and "65536" in str(e.value)


def test_noalloc_accepts_a_mesh_of_exactly_the_limit(cuda_lib):
    mcdi = cuda_lib
    v, _, t = scenes.icosphere(6, radius=0.9)  # 81,920 triangles; keep the first MCDI_NOALLOC_MAX_TRIS
    t = np.ascontiguousarray(t[: mcdi.NOALLOC_MAX_TRIS])
    rn, rr, nn, nr = _build_both(mcdi, v, t)
    np.testing.assert_array_equal(nn, rn)
    np.testing.assert_array_equal(nr, rr)


def test_noalloc_call_allocates_no_device_memory(cuda_lib):
    mcdi = cuda_lib
    dev = torch.device("cuda")
    v, _, t = scenes.icosphere(4, radius=0.8)
    verts = torch.from_numpy(np.ascontiguousarray(v, np.float32)).to(dev)
    tris = torch.from_numpy(np.ascontiguousarray(t, np.int32)).to(dev)
    nb, tb, _ = mcdi.bvh_sizes(tris.shape[0])
    nodes = torch.empty(nb, dtype=torch.uint8, device=dev)
    recs = torch.empty(tb, dtype=torch.uint8, device=dev)
    mcdi.build_bvh_noalloc(verts, tris, nodes, recs)  # warm-up: context set-up and module loading
    torch.cuda.synchronize()
    held, (free, _) = torch.cuda.memory_allocated(), torch.cuda.mem_get_info()
    mcdi.build_bvh_noalloc(verts, tris, nodes, recs)
    torch.cuda.synchronize()
    assert torch.cuda.memory_allocated() == held
    assert torch.cuda.mem_get_info()[0] == free


@pytest.mark.parametrize("case", ["no_triangles", "misaligned_nodes"])
def test_noalloc_rejects_bad_arguments(cuda_lib, case):
    mcdi = cuda_lib
    dev = torch.device("cuda")
    v, _, t = scenes.icosphere(2)
    verts = torch.from_numpy(np.ascontiguousarray(v, np.float32)).to(dev)
    tris = torch.from_numpy(np.ascontiguousarray(t, np.int32)).to(dev)
    nb, tb, _ = mcdi.bvh_sizes(tris.shape[0])
    nodes = torch.empty(nb + 256, dtype=torch.uint8, device=dev)
    recs = torch.empty(tb, dtype=torch.uint8, device=dev)
    if case == "no_triangles":
        tris = tris[:0]
    else:
        nodes = nodes[16:]  # 16-byte offset from a 256-byte aligned allocation
    with pytest.raises(mcdi.McdiError) as e:
        mcdi.build_bvh_noalloc(verts, tris, nodes, recs)
    assert e.value.status == mcdi.INVALID_ARG
