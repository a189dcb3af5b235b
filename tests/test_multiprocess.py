"""The N > 1 host logic of bench.py on CPU: two ranks over gloo (replicas
only, so the process group only carries the barrier and the scalar
reductions of the timings).  Checks the rank bookkeeping, the max-over-ranks
time, the whole-job rate (units summed over ranks / slowest rank's time) and
that only rank 0 runs the reference arm."""
import multiprocessing as mp
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, port, q):
    os.environ.update(RANK=str(rank), WORLD_SIZE="2", LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port),
                      CUDA_VISIBLE_DEVICES="")
    sys.path.insert(0, ROOT)
    sys.argv = ["bench.py"]
    import torch.distributed as dist

    import bench
    ws, r, local = bench.dist_init(None)
    backend = dist.get_backend()
    mx = bench.allreduce_max(1.5 + r, ws)
    sm = bench.allreduce_sum(1.0 + r, ws)
    # rank r processed 100 (r + 1) units in 10 (r + 1) ms
    rate, ms = bench.job_rate(100.0 * (r + 1), 10.0 * (r + 1), ws)
    bench.barrier(ws)
    ref = bench.run_reference(None, ws, r) if r != 0 else "rank 0 runs it"
    q.put((r, ws, local, backend, mx, sm, rate, ms, ref))
    dist.destroy_process_group()


def test_two_ranks_over_gloo():
    pytest.importorskip("torch")
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r, (rank, ws, local, backend, mx, sm, rate, ms, ref) in enumerate(out):
        assert (rank, ws, local, backend) == (r, 2, r, "gloo")
        assert mx == 2.5 and sm == 3.0
        assert ms == 20.0 and rate == pytest.approx(300.0 / 0.020)
    assert out[1][8] is None   # rank 1 leaves the reference arm without work
