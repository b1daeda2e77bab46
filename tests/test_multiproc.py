"""The N > 1 host path of the benchmark on CPU: two gloo ranks (127.0.0.1)
rendezvous, reduce the step time with MAX and the sample count with SUM, give
each replica its own workload seed, and run the reference arm on rank 0 only
(the other rank exits without work)."""
import contextlib
import io
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench

    r, w = bench.init_dist("gloo")
    out = {"rank": r, "world": w,
           "max": bench.max_over_ranks(1.5 + r, "cpu"), "sum": bench.sum_over_ranks(10.0 * (r + 1), "cpu"),
           "seed": bench.replica_seed(100, r, w)}
    bench.barrier()
    import torch.distributed as dist

    dist.destroy_process_group()
    # the reference arm: rank 0 times the oracle and prints one line; the other rank returns at once
    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        bench.main(["--impl", "reference", "--gpus", str(world), "--steps", "1", "--warmup", "3",
                    "--ref-pixels", "8"])
    out["printed"] = buf.getvalue()
    q.put(out)


def test_two_gloo_ranks_reduce_and_split_work():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted([q.get(timeout=600) for _ in procs], key=lambda d: d["rank"])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [d["world"] for d in res] == [2, 2]
    assert all(d["max"] == 2.5 and d["sum"] == 30.0 for d in res)
    assert res[0]["seed"] != res[1]["seed"]
    import json

    line = json.loads(res[0]["printed"].strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["e2e"]["h2d_bytes_per_step"] == 0
    assert res[1]["printed"] == ""
