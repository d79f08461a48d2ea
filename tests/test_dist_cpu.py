"""Multi-process host logic of bench.py on CPU (gloo, world size 2).

Each rank works on its own problem with no data exchange; the only
collectives are the timing reductions: the whole-job throughput is the sum
of the units all ranks processed divided by the SLOWEST rank's time, and
the reference arm runs on rank 0 alone.
"""
import io
import json
import os
import socket
import sys
import contextlib

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        bench.set_group(dist.group.WORLD)
        bench._barrier()
        # rank r: (r+1)*100 ms over 4 steps, 1000*(r+1) units per step
        v, ms = bench.whole_job(100.0 * (rank + 1), 1000 * (rank + 1), 4)
        # the reference arm: rank 0 prints one line, the others return at once
        out = io.StringIO()

        class A:
            steps, warmup = 1, 0
        with contextlib.redirect_stdout(out):
            rc = bench.run_reference(A, "c1", dict(bench.WORKLOADS["c1"]))
        q.put((rank, v, ms, rc, out.getvalue()))
    finally:
        dist.destroy_process_group()


def test_whole_job_and_reference_arm_two_ranks():
    pytest.importorskip("torch")
    ws = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, ws, port, q)) for r in range(ws)]
    for p in procs:
        p.start()
    res = {}
    for _ in range(ws):
        r = q.get(timeout=300)
        res[r[0]] = r[1:]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank in range(ws):
        v, ms, rc, out = res[rank]
        assert rc == 0
        assert ms == pytest.approx(200.0 / 4)               # slowest rank
        assert v == pytest.approx((1000 + 2000) / 0.050)    # all ranks' units
    line = json.loads(res[0][3].strip())
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
    assert res[1][3] == ""
