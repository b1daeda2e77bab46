"""The C-ABI library loads and exports every entry point that include/*.h
declares, and rejects bad arguments on the host (no GPU needed: argument checks
run before anything is enqueued)."""
import ctypes as C
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        names |= set(re.findall(r"MCDI_API\s+[\w\s\*]+?\b(mcdi_\w+)\s*\(", open(h).read()))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_2206_03380_gb300 import build, mcdi

    if not os.path.exists(mcdi.LIB_PATH):
        build.build()
    return mcdi.load()


def test_header_declares_entry_points():
    names = declared_symbols()
    for must in ["mcdi_build_envmap_cdf", "mcdi_build_bvh", "mcdi_shade_mc_fwd", "mcdi_shade_mc_bwd",
                 "mcdi_primary_cast", "mcdi_bvh_sizes", "mcdi_last_error"]:
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    from paper_2206_03380_gb300 import mcdi

    for name in declared_symbols():
        assert hasattr(lib, name), name
    assert set(mcdi.EXPORTS) <= set(declared_symbols())


def test_argument_checks_without_gpu(lib):
    from paper_2206_03380_gb300 import mcdi

    assert lib.mcdi_version() >= 100
    # NULL / misaligned / out-of-range arguments fail on the host with INVALID_ARG
    assert lib.mcdi_build_envmap_cdf(None, 32, 16, None, None, None, None, None) == mcdi.INVALID_ARG
    assert b"env" in lib.mcdi_last_error()
    assert lib.mcdi_build_envmap_cdf(C.c_void_p(16), 0, 16, C.c_void_p(16), C.c_void_p(16), C.c_void_p(16),
                                     C.c_void_p(16), None) == mcdi.INVALID_ARG
    a, b, s = C.c_size_t(), C.c_size_t(), C.c_size_t()
    assert lib.mcdi_bvh_sizes(0, C.byref(a), C.byref(b), C.byref(s)) == mcdi.INVALID_ARG
    assert lib.mcdi_bvh_sizes(1000, C.byref(a), C.byref(b), C.byref(s)) == mcdi.OK
    # 999 two-child nodes of 64 B (256-aligned), then 1999 depth-first nodes of 32 B
    # two-child nodes, depth-first copy, four-wide nodes, each at a 256-byte aligned offset
    r256 = lambda x: (x + 255) // 256 * 256
    assert a.value == r256(r256(999 * 64) + 1999 * 32) + 999 * 64 and b.value == 1000 * 48 and s.value > 0
    # scratch smaller than the query -> rejected before any launch
    assert lib.mcdi_build_bvh(C.c_void_p(256), 3, C.c_void_p(256), 1000, C.c_void_p(256), C.c_void_p(256),
                              C.c_void_p(256), s.value - 1, None) == mcdi.INVALID_ARG
    assert b"scratch" in lib.mcdi_last_error()
    bvh = mcdi.BvhView(None, None, 0)
    prm = mcdi.make_params(4, 2, 2, 1)
    bad = mcdi.make_params(0, 0, 0, 1)
    p16 = C.c_void_p(4096)
    args = [C.byref(bvh), p16, 32, 16, p16, p16, p16, p16, p16, p16, p16, p16, 1, 8, 8]
    outs = [p16, p16, p16, None, None, 0, None]
    assert lib.mcdi_shade_mc_fwd(*args, C.byref(bad), *outs) == mcdi.INVALID_ARG
    assert b"spp" in lib.mcdi_last_error()
    mis = C.c_void_p(4100)  # not 16-byte aligned
    args_mis = list(args)
    args_mis[7] = mis
    assert lib.mcdi_shade_mc_fwd(*args_mis, C.byref(prm), *outs) == mcdi.INVALID_ARG
    assert b"gb_pos" in lib.mcdi_last_error()
    tau_bad = mcdi.make_params(4, 2, 2, 1, tau=1.5)
    assert lib.mcdi_shade_mc_fwd(*args, C.byref(tau_bad), *outs) == mcdi.INVALID_ARG


def test_edge_gradient_argument_checks_without_gpu(lib):
    from paper_2206_03380_gb300 import mcdi

    n = C.c_size_t()
    assert lib.mcdi_edge_table_workspace_size(0, C.byref(n)) == mcdi.INVALID_ARG
    assert lib.mcdi_edge_table_workspace_size(1000, C.byref(n)) == mcdi.OK
    # hash table of 8192 slots (>= 2 x 3000 half-edges) of 16 bytes, then per-half-edge slots
    assert n.value >= 8192 * 16 + 3000 * 4
    p = C.c_void_p(4096)
    assert lib.mcdi_build_edge_table(p, 1000, p, p, p, n.value - 1, None) == mcdi.INVALID_ARG
    assert b"workspace" in lib.mcdi_last_error()
    bvh = mcdi.BvhView(None, None, 0)
    prm = mcdi.make_params(4, 2, 2, 1, tau=1.0)
    args = [C.byref(bvh), p, 10, p, p, 30, p, 32, 16, p, p, p, p, p, 1, 8, 8, C.byref(prm)]
    assert lib.mcdi_shadow_edge_grad(*args, 4, C.c_float(0.0), p, p, p, None, None) == mcdi.INVALID_ARG
    assert b"eta" in lib.mcdi_last_error()
    assert lib.mcdi_shadow_edge_grad(*args, -1, C.c_float(1e-4), p, p, p, None, None) == mcdi.INVALID_ARG
    assert lib.mcdi_shadow_edge_grad(*args, 4, C.c_float(1e-4), p, C.c_void_p(4100), p, None,
                                     None) == mcdi.INVALID_ARG
    assert b"g_cs" in lib.mcdi_last_error()


def test_raster_argument_checks_without_gpu(lib):
    from paper_2206_03380_gb300 import mcdi

    n = C.c_size_t()
    assert lib.mcdi_raster_workspace_size(1, 0, 8, C.byref(n)) == mcdi.INVALID_ARG
    assert lib.mcdi_raster_workspace_size(2, 8, 16, C.byref(n)) == mcdi.OK and n.value >= 2 * 8 * 16 * 8
    p = C.c_void_p(4096)
    uv = (C.c_float * 3)(0.0, 0.0, 1.0)
    args = [p, p, p, 10, 4, p, 2, 8, 16, p, p, 64, uv, p, p, p, p, p]
    assert lib.mcdi_raster_gbuffer(*args, n.value - 1, None) == mcdi.INVALID_ARG
    assert b"workspace" in lib.mcdi_last_error()
    bad = list(args)
    bad[13] = C.c_void_p(4100)  # gb_pos not 16-byte aligned
    assert lib.mcdi_raster_gbuffer(*bad, n.value, None) == mcdi.INVALID_ARG
    assert b"gb_pos" in lib.mcdi_last_error()
    pargs = args[:12] + [4] + args[12:]  # tex_channels after tex_size
    assert lib.mcdi_raster_gbuffer_part(*pargs, n.value, 3, None) == mcdi.INVALID_ARG
    assert b"part" in lib.mcdi_last_error()
    assert lib.mcdi_raster_gbuffer_part(*pargs, n.value - 1, 1, None) == mcdi.INVALID_ARG
    assert b"workspace" in lib.mcdi_last_error()
    bad = list(pargs)
    bad[12] = 2
    assert lib.mcdi_raster_gbuffer_part(*bad, n.value, 2, None) == mcdi.INVALID_ARG
    assert b"tex_channels" in lib.mcdi_last_error()
    bad[12], bad[9] = 4, C.c_void_p(4100)  # float4 textures must be 16-byte aligned
    assert lib.mcdi_raster_gbuffer_part(*bad, n.value, 2, None) == mcdi.INVALID_ARG
    bad[12] = 3  # packed RGB: 4-byte alignment suffices
    bad[9] = C.c_void_p(4098)
    assert lib.mcdi_raster_gbuffer_part(*bad, n.value, 2, None) == mcdi.INVALID_ARG


def test_graph_entry_points_check_arguments_without_gpu(lib):
    from paper_2206_03380_gb300 import mcdi

    out = C.c_void_p(1234)
    assert lib.mcdi_graph_instantiate(None, C.byref(out)) == mcdi.INVALID_ARG
    assert lib.mcdi_graph_instantiate(C.c_void_p(4096), None) == mcdi.INVALID_ARG
    assert lib.mcdi_graph_launch(None, None) == mcdi.INVALID_ARG
    assert b"graph_exec" in lib.mcdi_last_error()
    assert lib.mcdi_graph_destroy(None) == mcdi.OK


def test_bvh_build_launch_count_without_gpu(lib):
    from paper_2206_03380_gb300 import mcdi

    out = C.c_int()
    counts = {}
    for n in (1, 2, 198_164, 262_144, 262_145, 1_289_216):
        assert lib.mcdi_bvh_build_launches(n, C.byref(out)) == mcdi.OK
        counts[n] = out.value
    # bounds (2) + Morton + 3 passes (one kernel each up to 262,144 triangles, else three) + leaf records with
    # the hierarchy + boxes (a single triangle: leaf record + root) + depth-first copy
    assert counts == {1: 9, 2: 9, 198_164: 9, 262_144: 9, 262_145: 15, 1_289_216: 15}
    assert lib.mcdi_bvh_build_launches(0, C.byref(out)) == mcdi.INVALID_ARG
    assert lib.mcdi_bvh_build_launches(5, None) == mcdi.INVALID_ARG


def test_graph_dependent_launch_switch_without_gpu(lib):
    from paper_2206_03380_gb300 import mcdi

    assert lib.mcdi_set_graph_dependent_launch(0) == mcdi.OK
    assert lib.mcdi_set_graph_dependent_launch(1) == mcdi.OK
