"""The N > 1 path of bench.py on CPU with two gloo ranks.

The product has no exchange step, so N GPUs run independent replicas: each rank
draws its own cloud and right-hand sides, the job time is the slowest rank's
(all_reduce MAX), rank 0 alone prints, and the reference arm runs on rank 0 only.
"""
import json
import os
import socket
import sys

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    import contextlib
    import io
    import types

    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        seeds = bench.replica_seeds(rank, 3)
        ms = bench.max_over_ranks(10.0 + 5.0 * rank, dist, "cpu")
        a = types.SimpleNamespace(N=3000, nrhs=1, seed=3, steps=1, warmup=1, gpus=world, leaf=128, tol=1e-7,
                                  points="uniform")
        buf = io.StringIO()
        with contextlib.redirect_stdout(buf):
            bench.run_reference(a)
        with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
            json.dump({"seeds": seeds, "ms": ms, "out": buf.getvalue()}, f)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks(tmp_path):
    mp = pytest.importorskip("torch.multiprocessing")
    mp.spawn(_worker, args=(2, _free_port(), str(tmp_path)), nprocs=2, join=True)
    r0 = json.load(open(tmp_path / "rank0.json"))
    r1 = json.load(open(tmp_path / "rank1.json"))
    assert r0["seeds"] != r1["seeds"]                    # independent replicas
    assert r0["ms"] == r1["ms"] == 15.0                  # the slowest rank's time on every rank
    assert r1["out"] == ""                               # only rank 0 runs and prints the reference arm
    line = json.loads(r0["out"].strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["unit"] == "ms"
    assert line["cpu_baseline"]["kind"] == "oracle" and line["value"] > 0
