"""Traversal statistics and the tracer timed alone (measurement aids of the
shadow-ray visibility term): the counting re-trace agrees with the forward
pass's hit flags, counts one shadow ray per active sample of the FP64 oracle,
and on a one-triangle mesh visits exactly one node per ray; re-running the
tracer leaves the forward's results valid; the L2 read sweep runs."""
import numpy as np
import pytest
import torch

from paper_2206_03380_gb300 import scenes
from tests import parity_util as PU

pytestmark = pytest.mark.gpu


def _pipe(sc):
    from paper_2206_03380_gb300.pipeline import ShadingPipeline

    return ShadingPipeline(sc)


def _upload(pipe, rows):
    g = torch.from_numpy(rows.astype(np.float32)).cuda().reshape(pipe.N, pipe.H, pipe.W, 16)
    for k, t in enumerate((pipe.gb.pos, pipe.gb.nrm, pipe.gb.kd, pipe.gb.korm)):
        t.copy_(g[..., 4 * k:4 * k + 4])


def _stats(mcdi, pipe):
    st = torch.zeros(5, dtype=torch.int64, device="cuda")
    mcdi.shadow_ray_stats(pipe.bvh, pipe.N, pipe.H, pipe.W, pipe.params, pipe.workspace, st)
    torch.cuda.synchronize()
    return [int(v) for v in st.cpu()]


def _forward(pipe, rows):
    _upload(pipe, rows)
    pipe.build_probe()
    pipe.build_bvh()
    pipe.forward()
    torch.cuda.synchronize()
    return pipe.mask.cpu().numpy().reshape(pipe.N * pipe.H * pipe.W, -1)


def test_stats_match_forward_and_oracle(cuda_lib, orc):
    sc = scenes.parity_scene()
    W, H = sc.width, sc.height
    rows = orc.primary_cast(sc.verts, sc.vnrm, sc.tris, sc.cams[0], W, H, np.arange(W * H), sc.tex_kd, sc.tex_korm,
                            sc.uvmap)
    pipe = _pipe(sc)
    mask = _forward(pipe, rows)
    rays, visits, tests, blocked, differ = _stats(cuda_lib, pipe)
    assert differ == 0
    gbits = PU.mask_bits(mask, sc.spp)
    assert blocked == int(gbits.sum())
    # one shadow ray per sample the oracle marks active (decisions within the FP32/FP64 margin may flip)
    _, _, recs = PU.oracle_shade(orc, sc, rows.astype(np.float32), np.arange(W * H), 0)
    n_act = int(recs["active"].astype(bool).sum())
    n_marg = int((recs["margin"] < PU.MARGIN).sum())
    assert abs(rays - n_act) <= max(2, n_marg), (rays, n_act, n_marg)
    n = sc.tris.shape[0]
    assert rays <= visits <= rays * (2 * n - 1)
    assert blocked <= tests <= 4 * visits  # up to four leaf children per four-wide node
    # the tracer alone, again over the same rays: the flags it sets agree with the forward's
    c_d0 = pipe.c_d.clone()
    cuda_lib.shadow_ray_retrace(pipe.bvh, pipe.N, pipe.H, pipe.W, pipe.params, pipe.workspace)
    assert _stats(cuda_lib, pipe) == [rays, visits, tests, blocked, 0]
    pipe.forward()
    torch.cuda.synchronize()
    assert torch.equal(c_d0, pipe.c_d)


def test_one_triangle_visits_one_node_per_ray(cuda_lib, orc):
    base = scenes.parity_scene(seed=scenes.BASE_SEED + 13)
    verts = np.array([[-3, -1, -3], [3, -1, -3], [0, -1, 4]], np.float32)
    tris = np.array([[0, 1, 2]], np.int32)
    vn = np.tile(np.array([[0, 1, 0]], np.float32), (3, 1))
    cam = scenes.look_at((0, 2.0, 3.0), (0, -1, 0), (0, 1, 0), 45.0, 1.0)[None]
    sc = scenes.Scene(**{**base.__dict__, "verts": verts, "vnrm": vn, "tris": tris, "cams": cam})
    rows = orc.primary_cast(verts, vn, tris, cam[0], 64, 64, np.arange(4096), sc.tex_kd, sc.tex_korm, sc.uvmap)
    pipe = _pipe(sc)
    _forward(pipe, rows)
    rays, visits, tests, blocked, differ = _stats(cuda_lib, pipe)
    assert rays > 1000 and visits == rays and blocked == 0 and differ == 0 and tests <= rays


def test_read_sweep_runs_and_leaves_sink(cuda_lib):
    buf = torch.zeros(1 << 18, dtype=torch.int32, device="cuda")  # 1 MiB
    sink = torch.full((1,), 7, dtype=torch.int32, device="cuda")
    cuda_lib.read_sweep(buf, 3, sink)
    torch.cuda.synchronize()
    assert int(sink.item()) == 7
    with pytest.raises(cuda_lib.McdiError):
        cuda_lib.read_sweep(buf[:3], 1, sink)  # 12 bytes: not a multiple of 16
