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


# --------------------------------------------------------------------------
# a batch of independent matrices split across ranks (the graph-batch
# workload under torchrun): every matrix is built by exactly one rank, keyed
# by its index in the whole batch, so the union of the shards equals the
# single-process build bit for bit.  The per-rank builds here are the FP64
# oracle's (no GPU on this machine); the GPU side of the keying is tested in
# test_gpu_parity.py::test_batch_shard_keys.
def _batch():
    sys.path.insert(0, ROOT)
    from paper_1106_5990_gb300 import inputs
    sizes = [300, 1200, 450, 800, 999, 620, 150]
    return [inputs.graph_laplacian(s, 4.0, 4, b) for b, s in enumerate(sizes)]


def _shard_worker(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    import oracle
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        mats = _batch()
        ids = bench.shard_batch([len(m[1]) for m in mats], ws, rank)
        mine = {}
        for b in ids:
            rp, col, val = mats[b]
            out = oracle.build(rp, col, val, 8, 6, 3, 2.0 / 3.0, 0.5, stream=b)
            mine[b] = (out["s_rp"].tolist(), out["s_col"].tolist())
        gathered = [None] * ws
        dist.all_gather_object(gathered, mine)
        q.put((rank, ids, gathered if rank == 0 else None))
    finally:
        dist.destroy_process_group()


def test_batch_sharded_across_two_ranks_equals_one_build():
    pytest.importorskip("torch")
    sys.path.insert(0, ROOT)
    import bench
    import oracle
    ws = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_shard_worker, args=(r, ws, port, q)) for r in range(ws)]
    for p in procs:
        p.start()
    res = {}
    for _ in range(ws):
        r = q.get(timeout=300)
        res[r[0]] = r[1:]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    mats = _batch()
    owned = sorted(res[0][0] + res[1][0])
    assert owned == list(range(len(mats)))                  # every matrix exactly once
    loads = [sum(len(mats[b][1]) for b in res[r][0]) for r in range(ws)]
    assert max(loads) <= 1.5 * min(loads)                   # balanced by stored entries
    merged = {}
    for part in res[0][1]:
        merged.update(part)
    for b, (rp, col, val) in enumerate(mats):
        want = oracle.build(rp, col, val, 8, 6, 3, 2.0 / 3.0, 0.5, stream=b)
        assert merged[b][0] == want["s_rp"].tolist() and merged[b][1] == want["s_col"].tolist()


def test_shard_batch_is_a_partition():
    sys.path.insert(0, ROOT)
    import bench
    nnz = [5, 9, 9, 1, 7, 3, 3, 8]
    for ws in (1, 2, 3, 4, 8, 11):
        parts = [bench.shard_batch(nnz, ws, r) for r in range(ws)]
        assert sorted(sum(parts, [])) == list(range(len(nnz)))
        assert all(p == sorted(p) for p in parts)
