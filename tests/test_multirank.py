"""The N > 1 host path of bench.py with two gloo ranks on the CPU (no GPU).

With N GPUs every rank evaluates its own polynomial of the bench shape (weak
scaling, no collective on the data path); the ranks meet only at the barriers
around the timed region and in the max over ranks of its duration, and rank 0
alone prints.  These tests run that logic as two processes: the rendezvous,
the barrier, the max over ranks, per-rank workloads of one shape with
different data, the whole-job throughput, and the reference arm, which only
rank 0 runs.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def rank_main(rank, world, port, out_dir):
    import contextlib
    import io
    import json
    import sys

    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench

    args = bench.parse_args(["--workload", "p1", "--d", "8", "--k", "2", "--steps", "1", "--warmup", "0",
                             "--gpus", str(world), "--cpu-sample-vars", "3"])
    w, r, local = bench.dist_setup(args, backend="gloo")
    assert (w, r, local) == (world, rank, rank)
    bench.barrier(w)
    mx = bench.max_over_ranks(1.5 + rank, w)
    prob = bench.make_workload(args, r)
    shapes = [None] * w
    dist.all_gather_object(shapes, (prob.n, prob.N, prob.d, prob.k, prob.coeff.shape, float(prob.coeff.sum())))
    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        rc = bench.reference_arm(args, w, r)
    bench.barrier(w)
    res = {"rank": r, "max": mx, "shapes": [list(map(str, s)) for s in shapes], "rc": rc,
           "printed": buf.getvalue()}
    with open(os.path.join(out_dir, f"rank{r}.json"), "w") as f:
        json.dump(res, f)
    dist.destroy_process_group()


@pytest.fixture(scope="module")
def results(tmp_path_factory):
    import json

    out = tmp_path_factory.mktemp("ranks")
    world = 2
    mp.start_processes(rank_main, args=(world, free_port(), str(out)), nprocs=world, join=True,
                       start_method="spawn")
    return [json.load(open(out / f"rank{r}.json")) for r in range(world)]


def test_max_over_ranks_and_barrier(results):
    assert [r["max"] for r in results] == [2.5, 2.5]


def test_weak_scaling_workloads(results):
    """Every rank builds a workload of the same shape from its own seed."""
    s0, s1 = results[0]["shapes"]
    assert s0[:5] == s1[:5]       # n, N, d, k, coefficient array shape
    assert s0[5] != s1[5]         # different data


def test_reference_arm_rank0_only(results):
    r0, r1 = results
    assert r0["rc"] == 0 and r1["rc"] == 0
    assert r1["printed"] == ""
    import json
    line = json.loads(r0["printed"].strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0


def test_whole_job_throughput():
    import sys

    sys.path.insert(0, ROOT)
    import bench

    # two ranks, 1e12 operations per step each, 4 steps, slowest rank 2 s: 4 TFLOP/s for the whole job
    assert bench.whole_job_tflops(2, 1e12, 4, 2000.0) == pytest.approx(4.0)
    assert bench.whole_job_tflops(1, 5e11, 2, 100.0) == pytest.approx(10.0)
    assert np.isclose(bench.whole_job_tflops(8, 1e12, 1, 1000.0), 8.0)
