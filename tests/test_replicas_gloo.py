"""The multi-rank path of bench.py (replicas only: no data-path collective)
with two gloo ranks on the CPU: the slowest rank's step time is what every
rank reports, and the whole-job grind time counts every rank's cells."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, ws, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    ms = 10.0 + 5.0 * rank  # rank 1 is the slow replica
    got = bench.max_over_ranks(ms, ws, "cpu")
    dist.barrier()
    q.put((rank, got, bench.grind_ns(got, ws, 1000, 7)))
    dist.destroy_process_group()


def test_max_over_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[1] for o in out] == [15.0, 15.0]
    # 15 ms for 2 replicas x 1000 cells x 7 equations x 3 RHS
    assert out[0][2] == pytest.approx(15e-3 / (2 * 1000 * 7 * 3) * 1e9)


def test_single_rank_is_a_no_op():
    import bench
    assert bench.max_over_ranks(3.5, 1) == 3.5


def test_one_core_oracle_sample_runs_in_a_child_with_one_thread():
    """bench.py's single-core CPU figure: the oracle's RHS timed in a child
    process with OMP_NUM_THREADS=1 on a small slab of the shock-bubble."""
    import bench
    out = bench.cpu_one_core_sample(16, min_seconds=0.2)
    assert "error" not in out, out
    assert out["cores"] == 1 and out["value"] > 0 and out["unit"] == bench.UNIT
