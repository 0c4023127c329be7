"""The bench's multi-rank host logic on CPU with two gloo ranks: job time is the
maximum over ranks, whole-job throughput counts every rank's bytes, and the
reference arm runs on rank 0 only (the other ranks exit without work)."""
import io
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


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "MASTER_ADDR": "127.0.0.1",
                       "MASTER_PORT": str(port)})
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local = 10.0 + 5.0 * rank  # rank 1 is the slow one
        total = bench.job_ms(local, world)
        value = bench.job_gbps(world, 24 * 1000, 3, total)
        args = type("A", (), {"n": 1 << 12, "steps": 1, "warmup": 1, "gpus": world, "impl": "reference"})()
        buf = io.StringIO()
        with redirect_stdout(buf):
            bench.run_reference(args)
        dist.barrier()
        out.put((rank, total, value, buf.getvalue()))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_max_time_and_rank0_reference():
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    results = [out.get(timeout=240) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res = {r: (t, v, txt) for r, t, v, txt in results}
    assert res[0][0] == res[1][0] == 15.0             # the slowest rank's time on every rank
    assert res[0][1] == pytest.approx(2 * 24 * 1000 * 3 / 15e-3 / 1e9)  # both ranks' bytes
    assert '"impl": "reference"' in res[0][2] and '"n_gpus": 2' in res[0][2]
    assert res[1][2] == ""                            # rank 1: no work, no line
