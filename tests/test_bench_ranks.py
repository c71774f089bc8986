"""The multi-rank path of the benchmark on the CPU (gloo, world size 2): the whole-job figures take the
slowest rank's time and the units of all ranks, and the reference arm runs on rank 0 only."""
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, port, q):
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=2)
    import bench

    q.put((rank,) + bench.aggregate_over_ranks([10.0, 25.0][rank], [3, 5][rank], device="cpu"))
    dist.destroy_process_group()


def test_aggregate_takes_the_slowest_rank_and_all_units():
    pytest.importorskip("torch")
    import multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert out == [(0, 25.0, 8.0), (1, 25.0, 8.0)]


def test_single_process_aggregate_is_identity():
    pytest.importorskip("torch")
    sys.path.insert(0, ROOT)
    import bench

    assert bench.aggregate_over_ranks(12.5, 7, device="cpu") == (12.5, 7.0)


def test_reference_arm_runs_on_rank_zero_only():
    """Under torchrun the reference arm's other ranks exit 0 without work or output."""
    env = dict(os.environ, RANK="1", LOCAL_RANK="1", WORLD_SIZE="2", MASTER_ADDR="127.0.0.1")
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--gpus", "2", "--steps", "1",
                        "--warmup", "3"], cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    assert r.stdout.strip() == ""


def test_cpu_baseline_runs_the_oracle_on_a_spawned_pool():
    """The CPU baseline runs one unmodified oracle evaluation per core in spawned processes (safe after
    a CUDA context exists) and scales the sample's rate to 256^3 by voxel count."""
    sys.path.insert(0, ROOT)
    import bench

    cb = bench.cpu_baseline(n=16, cores=2)
    assert cb["cores"] == 2 and cb["kind"] == "oracle"
    assert cb["value"] > 0 and cb["s_per_grad_1core_256"] > 0 and cb["s_per_obj_1core_256"] > 0
    # rate of 2 cores = 2 / (seconds per gradient at 256^3)
    assert abs(cb["value"] * cb["s_per_grad_1core_256"] - 2.0) < 1e-9
