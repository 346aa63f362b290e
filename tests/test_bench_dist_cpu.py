"""The bench's multi-rank logic on CPU with gloo, world size 2: each rank
runs its own seed (independent runs, weak scaling, no data-path
collective); timings are max-reduced over ranks; the whole-job rate counts
every rank's sparks over the slowest rank's time; the reference arm prints
only on rank 0."""
import io
import json
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    ms = [12.5, 20.0][rank]
    mx = bench.max_over_ranks(ms, dist, "cpu")
    w, r, _ = bench._dist()

    class Args:
        gpus, steps, warmup = world, 1, 0
    out = ""
    if rank == 1:
        buf = io.StringIO()
        with redirect_stdout(buf):
            rc = bench.reference_arm(Args())
        out = buf.getvalue()
        assert rc == 0
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, mx, bench.run_seed(r), w, out))


def test_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [20.0, 20.0]
    assert res[0][2] != res[1][2]
    assert all(r[3] == 2 for r in res)
    assert res[1][4] == ""  # rank 1 does no reference work and prints nothing
    import bench
    assert bench.whole_job_rate(2, 1040 * 20, 20.0 / 1e3) == pytest.approx(2 * 1040 * 20 / 0.02)
