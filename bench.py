"""Throughput of the algebraic-distance strength build on GB300.

One step = one whole build on one synthetic matrix already resident in HBM:
Philox start of the K test vectors, nu relaxation sweeps, the fused
distance/threshold pass, and the strength CSR -- replayed as one CUDA graph.
The metric is edges/s = E (stored off-diagonals) / step time.

Default workload (rotated anisotropic diffusion, 9-point stencil on a
1024 x 1024 grid, eps = 1e-3, alpha = pi/6; K = 16 vectors, nu = 8
red-black Gauss-Seidel sweeps, theta = 0.5): the headline is the mixed path
that meets the accuracy contract against the FP64 oracle (FP32 vector
storage, FP32 arithmetic: distances within 1e-3, strength set identical
outside +-1e-2 of theta); the FP64 path and the BF16-storage path (faster,
but outside the distance bar end to end) are measured beside it on the same
matrix, each with its own accuracy against the oracle.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--config c1..c7]
                  [--precision bf16|fp32|fp64] [--impl ours|reference]

Under torchrun (N > 1) a single-matrix workload runs as an independent
replica per rank (its own start-vector seed; weak scaling); the 64-matrix
graph batch is split across the ranks -- every matrix keeps its key in the
whole batch, so the union of the shards is the one-GPU build -- with no data
exchange (strong scaling).  Rank 0 prints the aggregate.  ``--impl
reference`` times the FP64 CPU oracle on the host cores instead (rank 0
only).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_1106_5990_gb300 import inputs  # noqa: E402

METRIC = "edges/s of algebraic-distance strength build, mixed vs FP64 on GPU; %HBM roof"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "traffic.json")
FALLBACK_HBM_GBS = 6800.0

# --------------------------------------------------------------------------
# workloads
# --------------------------------------------------------------------------
WORKLOADS = {
    "c1": dict(name="2D Poisson 5-point, 64x64 grid (n=4096), K=8, nu=4 Jacobi omega=2/3",
               K=8, seed=0, nu=4, omega=2.0 / 3.0, sweep="jacobi", theta=0.5,
               precision="fp64"),
    "c2": dict(name="rotated anisotropic diffusion 9-point, 1024x1024 grid, eps=1e-3, "
                    "alpha=pi/6; K=16, nu=8 red-black Gauss-Seidel, theta=0.5",
               K=16, seed=1, nu=8, omega=1.0, sweep="mcgs", theta=0.5, precision="fp32"),
    "c3": dict(name="3D jump-coefficient diffusion 7-point, 128^3 cells, lognormal(0,2) "
                    "coefficients, harmonic faces; K=32, nu=6 Jacobi omega=0.8",
               K=32, seed=3, nu=6, omega=0.8, sweep="jacobi", theta=0.5, precision="fp32"),
    "c4": dict(name="batch of 64 graph Laplacians, n ~ U[10k,500k], Poisson(8) neighbours "
                    "symmetrised, lognormal(0,1) weights; K=16, nu=4 Jacobi omega=2/3",
               K=16, seed=6, nu=4, omega=2.0 / 3.0, sweep="jacobi", theta=0.5,
               precision="bf16"),
    "c5": dict(name="anisotropic diffusion 5-point (eps=1e-2), 512x512 grid; K=16, nu=10 "
                    "Jacobi omega=2/3; forward + reverse pass of sum r^2 over strong edges, "
                    "checkpoints every 2 sweeps",
               K=16, seed=7, nu=10, omega=2.0 / 3.0, sweep="jacobi", theta=0.5,
               precision="fp32", adjoint=2),
    "c6": dict(name="rotated anisotropic diffusion 9-point, 1024x1024 grid, eps=1e-3, "
                    "alpha=pi/6; K=16, nu=8 red-black Gauss-Seidel, theta=0.5; search depth "
                    "d=2 (fits, threshold and strength graph over the graph of A^2, "
                    "25-point pattern)",
               K=16, seed=1, nu=8, omega=1.0, sweep="mcgs", theta=0.5, precision="bf16",
               depth=2),
    "c7": dict(name="compatible-relaxation coarsening (Algorithm 1: 5 red-black F-relaxation "
                    "sweeps per stage, theta=0.5, delta=0.6, tol=0.5, at most 12 sets) and "
                    "least-squares interpolation (caliber 2, gamma=1.5, neighbourhood of A) "
                    "of the rotated anisotropic 9-point operator, 1024x1024 grid, eps=1e-3, "
                    "alpha=pi/6; LS from K=16, nu=8 red-black Gauss-Seidel (BF16 build, "
                    "untimed)",
               K=16, seed=1, nu=8, omega=1.0, sweep="mcgs", theta=0.5, precision="bf16",
               coarsen=dict(nu=5, omega=1.0, delta=0.6, tol=0.5, max_sets=12, seed=5,
                            caliber=2, gamma=1.5)),
}


def make_matrix(cfg: str, scale: int | None = None):
    """(list of CSR matrices, coloring or None).  ``scale`` shrinks the grid
    (used for the bounded CPU samples)."""
    if cfg == "c1":
        return [inputs.poisson2d_5pt(64)], None
    if cfg in ("c2", "c6", "c7"):
        N = scale or 1024
        return [inputs.aniso2d_9pt(N, 1e-3, math.pi / 6)], inputs.red_black(N)
    if cfg == "c3":
        N = scale or 128
        return [inputs.jump3d_7pt(N, 2.0, 2)], None
    if cfg == "c4":
        if scale:
            sizes = inputs.batch_sizes(64, 10_000, 500_000, 5)[:scale]
            return [inputs.graph_laplacian(int(s), 8.0, 4, b) for b, s in enumerate(sizes)], None
        return inputs.graph_laplacian_batch(64, 10_000, 500_000, 8.0, 4, 5), None
    if cfg == "c5":
        N = scale or 512
        return [inputs.aniso2d_5pt(N, 1e-2)], None
    raise ValueError(cfg)


# --------------------------------------------------------------------------
# algorithmic bytes (what the method must move; each vector row read once
# per pass, every stored entry of A read once per pass)
# --------------------------------------------------------------------------
SIZES = {"fp64": 8, "fp32": 4, "bf16": 2}


def algorithmic_bytes(n, nnz, E, E_s, K, nu, ncolors, precision, permuted, nnz_p=None):
    """nnz_p: stored entries of the fit pattern (the graph G_d of A^d for
    search depth d > 1; None: A's own pattern)."""
    s_x = SIZES[precision]
    s_a = 8 if precision == "fp64" else 4
    s_c = 8 if precision == "fp64" else 4
    csr = nnz * (4 + s_a) + 4 * (n + 1)
    reads_per_sweep = ncolors                 # every color phase reads the vectors once
    sweep = csr + (reads_per_sweep + 1) * n * K * s_x
    init = n * K * s_x
    pat = 0 if nnz_p is None else nnz_p * 4 + 4 * (n + 1)     # G_d columns and row starts
    nnz_p = nnz if nnz_p is None else nnz_p
    edge = csr + pat + n * K * s_x + nnz_p * (2 * s_c + 1) + 4 * n + (8 * n if permuted else 0)
    strength = 4 * n * 2 + nnz_p + 4 * E_s * 2 + 8 * (n + 1)
    return dict(init=init, sweep=sweep, relax=nu * sweep, relax_per_launch=sweep / ncolors,
                edge=edge, strength=strength, total=init + nu * sweep + edge + strength)


def adjoint_bytes(n, nnz, K, nu, every, precision):
    """Algorithmic bytes of one forward + reverse step (Jacobi sweeps,
    checkpoints every `every` sweeps, built-in loss): every array the step
    must touch, each once per pass that needs it."""
    s_x = SIZES[precision]
    cs = 8 if precision == "fp64" else 4
    s_a = cs
    X = n * K * s_x                     # one stored iterate
    Xc = n * K * cs                     # one arithmetic-type block (Y, Ybar, Xbar)
    csr = nnz * (4 + s_a) + 4 * (n + 1)
    csr_t = nnz * (4 + 4) + 4 * (n + 1)  # transposed pattern: rows and slots
    sweep = csr + 2 * X
    nck = -(-nu // every)
    fwd = X + 2 * X + nu * sweep                               # start, checkpoint 0, sweeps
    edge = csr + X + nnz * (2 * cs + 1) + 4 * n
    up = 4 * (n + 1) + nnz * (4 + cs + 1 + 8)
    bvals = csr_t + nnz * 8 + 8 * n + nnz * cs
    edge_bwd = csr + X + nnz * (8 + cs) + 2 * Xc + nnz * cs
    xbar_nu = csr_t + nnz * (8 + 2 * cs) + X + 3 * Xc
    recompute = (nu - nck) * sweep
    gram = nnz * 4 + 4 * (n + 1) + X + Xc + nnz * cs * 2
    spmm_t = csr_t - nnz * 4 + nnz * cs + 2 * Xc
    finish = nnz * (4 + 8 + 2 * cs + 8) + n * (4 + 8 + 4)
    bwd = up + bvals + edge_bwd + xbar_nu + recompute + nu * (gram + spmm_t) + finish
    return dict(forward=fwd, edge=edge, backward=bwd, relax_per_launch=sweep,
                total=fwd + edge + bwd)


def _code_only(text):
    """C++ source with comments removed and whitespace collapsed: a note
    edited beside a kernel does not make its recorded counters stale."""
    out, i, n = [], 0, len(text)
    while i < n:
        c = text[i]
        if text.startswith("//", i):
            j = text.find("\n", i)
            i = n if j < 0 else j
        elif text.startswith("/*", i):
            j = text.find("*/", i + 2)
            i = n if j < 0 else j + 2
            out.append(" ")
        elif c in "\"'":
            j = i + 1
            while j < n and text[j] != c:
                j += 2 if text[j] == "\\" else 1
            out.append(text[i:j + 1])
            i = j + 1
        else:
            out.append(c)
            i += 1
    return " ".join("".join(out).split())


def source_sha(*names):
    h = hashlib.sha256()
    for nm in names:
        with open(os.path.join(ROOT, "paper_1106_5990_gb300", "csrc", nm)) as f:
            h.update(_code_only(f.read()).encode())
    return h.hexdigest()[:16]


def recorded_traffic(key, sha):
    """dram bytes per launch from a committed ncu capture, if the kernel
    source is unchanged since."""
    try:
        with open(TRAFFIC_FILE) as f:
            t = json.load(f)
    except (OSError, ValueError):
        return None
    e = t.get(key)
    if not e or e.get("source_sha") != sha:
        return None
    return e.get("dram_bytes_per_launch")


def peaks():
    try:
        with open(PEAKS_FILE) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except (OSError, ValueError, KeyError):
        return FALLBACK_HBM_GBS, "fallback"


# --------------------------------------------------------------------------
# clocks sampled during the timed region
# --------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.p = None
        self.path = os.path.join("/tmp", "amgd_clocks_%d_%d.csv" % (os.getpid(), device_index))

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), "--query-gpu=" + self.FIELDS,
                                       "--format=csv,noheader,nounits", "-lms", "50"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return dict(sm_mhz=None, sm_max_mhz=None, reasons=["nvidia-smi unavailable"], samples=0)
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        return dict(sm_mhz=float(np.median(sm)) if sm else None,
                    sm_max_mhz=float(max(smax)) if smax else None,
                    reasons=sorted(reasons), samples=len(sm))


# --------------------------------------------------------------------------
# our arm
# --------------------------------------------------------------------------
def shard_batch(nnz, world, rank):
    """Global indices of the matrices of a batch that `rank` of `world` builds:
    largest first, each to the rank with the fewest stored entries so far (ties:
    the lower rank), returned ascending.  Deterministic, every matrix exactly
    once."""
    load = [0] * world
    owner = [0] * len(nnz)
    for b in sorted(range(len(nnz)), key=lambda b: (-nnz[b], b)):
        r = min(range(world), key=lambda q: (load[q], q))
        owner[b] = r
        load[r] += nnz[b]
    return [b for b in range(len(nnz)) if owner[b] == rank]


def run_gpu_arm(mats, color, w, precision, steps, warmup, rank, flush, want_clocks=True,
                tune_cache=None, summation="compensated", matrix_ids=None):
    """One step = one captured build (or, for a workload with a checkpoint
    interval, one captured forward + reverse step)."""
    import torch
    from paper_1106_5990_gb300 import amgd

    stream = torch.cuda.current_stream()
    if len(mats) == 1:
        h = amgd.Handle(*mats[0], w["K"], w["seed"])
    else:
        h = amgd.Handle(None, None, None, w["K"], w["seed"], batch=mats)
    if matrix_ids is not None:
        h.set_matrix_ids(matrix_ids)      # this rank's share of a larger batch
    h.set_stream(stream)
    h.set_precision(precision)
    h.set_summation(summation)
    ncolors = 1
    sweep = amgd.AMGD_SWEEP_JACOBI
    if w["sweep"] == "mcgs":
        h.set_coloring(color)
        ncolors = int(color.max()) + 1
        sweep = amgd.AMGD_SWEEP_MCGS
    if w.get("depth", 1) > 1:
        h.set_search_depth(w["depth"])
    shapes = h.autotune(sweep, w["omega"], tune_cache)   # kernel shapes; untimed
    h.init_vectors(w["seed"])
    d_rp = torch.empty(h.n + 1, dtype=torch.int64, device="cuda")
    d_col = torch.empty(max(h.E_p, 1), dtype=torch.int32, device="cuda")
    d_vb = None
    h.enable_phase_timing(True)
    if w.get("adjoint"):
        h.set_checkpointing(w["adjoint"])
        d_vb = torch.empty(max(h.nnz, 1), dtype=torch.float64, device="cuda")
        h.graph_capture_backward(w["seed"], w["nu"], w["omega"], w["theta"], d_vb)
    else:
        h.graph_capture(w["seed"], w["nu"], w["omega"], sweep, w["theta"], d_rp, d_col)
    for _ in range(warmup):
        h.graph_launch()
    torch.cuda.synchronize()

    clocks = ClockSampler(torch.cuda.current_device()) if want_clocks else None
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    phase = np.zeros(4)
    if clocks:
        clocks.start()
        time.sleep(0.15)
    _barrier()
    torch.cuda.synchronize()
    for k in range(steps):
        flush.fill_(k & 0xFF)                     # evict L2 between steps (not timed)
        ev[k][0].record(stream)
        h.graph_launch()
        ev[k][1].record(stream)
        phase += np.array(h.phase_times())        # waits for this step's last event
    torch.cuda.synchronize()
    _barrier()
    clk = clocks.stop() if clocks else None
    step_ms = np.array([a.elapsed_time(b) for a, b in ev])
    E_s = int(d_rp[-1].item()) if d_vb is None else None
    scal = h.backward_scalars() if d_vb is not None else None
    return dict(h=h, step_ms=step_ms, phase_ms=phase / steps, E_s=E_s, ncolors=ncolors,
                sweep=sweep, clocks=clk, d_rp=d_rp, d_col=d_col, shapes=shapes, d_vb=d_vb,
                scalars=scal)


def run_e2e(h, mats, w, sweep, steps, adjoint=None):
    """Through the public API with host buffers.  Per step: the matrix values
    are copied from pinned host memory (amgd_set_values_async: staged,
    checked, written in place), the build captured by run_gpu_arm is replayed
    (amgd_graph_launch) and the strength CSR is copied to pinned host memory
    (amgd_strength_async); the copies of one step overlap the builds of its
    neighbours and amgd_sync after the last step waits for everything.  With
    a reverse pass: amgd_set_values, the eager calls and dL/dvalues written to
    pinned host memory (amgd_backward), step by step."""
    import ctypes
    import torch
    from paper_1106_5990_gb300 import amgd

    vals = np.concatenate([m[2] for m in mats])
    val_h = torch.from_numpy(vals).pin_memory()
    s_rp = torch.empty(h.n + 1, dtype=torch.int64).pin_memory()
    s_col = torch.empty(max(h.E_p, 1), dtype=torch.int32).pin_memory()
    L = amgd.lib()
    nnz_s = ctypes.c_int64()
    vb_h = torch.empty(len(vals), dtype=torch.float64).pin_memory() if adjoint else None
    if adjoint:
        h.set_checkpointing(adjoint)
    times = []
    torch.cuda.synchronize()
    if adjoint:
        for _ in range(steps):
            t0 = time.perf_counter()
            h.set_values(val_h)
            h.init_vectors(w["seed"])
            h.relax(w["nu"], w["omega"], sweep)
            amgd.check(L.amgd_distances(h.h, w["theta"], None, None, None, amgd.AMGD_MEM_DEVICE),
                       h.h)
            h.backward(out=vb_h)                 # dL/dvalues to pinned host memory
            times.append(time.perf_counter() - t0)
        t = float(np.mean(times))
        return dict(seconds=t, h2d=int(vals.nbytes), d2h=int(vals.nbytes) + 16, E_s=None)
    # a stream of builds: each step uploads its values and downloads its strength graph;
    # the stream-ordered calls overlap both copies with the neighbouring builds, and one
    # amgd_sync at the end waits for the last download (all inside the timed region)
    h.set_values_async(val_h)                    # warm-up: allocates the staging buffers
    h.graph_launch()
    h.strength_async(s_rp, s_col)
    h.sync()
    t0 = time.perf_counter()
    for _ in range(steps):
        h.set_values_async(val_h)
        h.graph_launch()
        h.strength_async(s_rp, s_col)
    h.sync()
    t = (time.perf_counter() - t0) / steps
    E_s = int(s_rp[-1].item())
    return dict(seconds=t, h2d=int(vals.nbytes), d2h=int((h.n + 1) * 8 + s_col.numel() * 4),
                E_s=E_s)


def oracle_step(oracle, rp, col, val, w, color, keep=None, stream=0):
    """One step of the workload on the FP64 oracle: the strength build, or
    for a workload with a checkpoint interval the forward path and its
    reverse pass (the oracle keeps every iterate).  keep (a dict) receives
    the build's outputs."""
    if w.get("adjoint"):
        X0 = oracle.tv_init(len(rp) - 1, w["K"], w["seed"])
        oracle.adjoint_jacobi(rp, col, val, X0, w["nu"], w["omega"], w["theta"])
    else:
        b = oracle.build(rp, col, val, w["K"], w["seed"], w["nu"], w["omega"], w["theta"],
                         sweep=oracle.SWEEP_MCGS if w["sweep"] == "mcgs" else oracle.SWEEP_JACOBI,
                         color=color, d=w.get("depth", 1), stream=stream)
        if keep is not None:
            keep.update(b)
        return len(b["pcol"]) - (len(rp) - 1)
    return len(col) - (len(rp) - 1)


def accuracy_vs_oracle(h, mat, ref, theta):
    """End-to-end error of the GPU build (its storage precision) against the
    FP64 oracle's build of the same matrix, seed and sweeps: relative error of
    LS where LS is not a cancellation residue (LS >= 1e-6 S_yy), and the edges
    whose strength flag differs, inside and outside the band |rho - theta| <=
    1e-2 (rho = min_k LS_ik / LS_ij, the oracle's)."""
    rp, col, _ = mat
    n = len(rp) - 1
    got = h.distances(theta, want=("ls",))["ls"]
    s_rp, s_col = h.strength()
    rows = np.repeat(np.arange(n), np.diff(rp))
    off = rows != col
    want = ref["ls"]
    syy = np.einsum("ij,ij->i", ref["Y"], ref["Y"])
    big = off & (want >= 1e-6 * syy[rows])
    rel = np.abs(got[big] - want[big]) / want[big]
    srows = np.repeat(np.arange(n), np.diff(s_rp))
    flag = np.isin(rows.astype(np.int64) * n + col, srows.astype(np.int64) * n + s_col)
    m = np.full(n, np.inf)
    np.minimum.at(m, rows[off], want[off])
    with np.errstate(divide="ignore", invalid="ignore"):
        rho = np.where(want[off] > 0, m[rows[off]] / want[off], 1.0)
    diff = flag[off] != (ref["flag"][off] == 1)
    band = np.abs(rho - theta) <= 1e-2
    outside = int((diff & ~band).sum())
    return {"against": "FP64 oracle build of the same matrix, seed and sweeps",
            "ls_rel_err": {"median": float(np.median(rel)), "p99": float(np.quantile(rel, 0.99)),
                           "max": float(rel.max())},
            "edges": int(off.sum()), "strength_flips": int(diff.sum()),
            "flips_outside_band_1e-2": outside,
            "bars": "LS relative error <= 1e-3, no strength flip outside +-1e-2 of theta",
            "meets_accuracy": bool(rel.max() <= 1e-3 and outside == 0)}


def cpu_oracle_time(cfg, w, sample_s=20.0, keep=None):
    """The FP64 oracle (single thread) on a bounded sample of the workload.
    keep (a dict): receives the first build when the sample is the whole
    single-matrix workload."""
    import oracle
    if cfg in ("c1", "c5"):
        mats, color = make_matrix(cfg)
        sample = "full workload"
    elif cfg == "c2":
        mats, color = make_matrix(cfg)
        sample = "full workload (1024x1024)"
    elif cfg == "c6":
        mats, color = make_matrix(cfg, scale=512)
        sample = "512x512 sub-grid of the same operator"
    elif cfg == "c3":
        mats, color = make_matrix(cfg, scale=64)
        sample = "64^3 sub-problem of the same operator"
    else:
        mats, color = make_matrix(cfg, scale=2)
        sample = "first 2 matrices of the batch"
    edges = 0
    t0 = time.perf_counter()
    reps = 0
    whole = cfg in ("c1", "c2") and len(mats) == 1
    while True:
        for rp, col, val in mats:
            edges += oracle_step(oracle, rp, col, val, w, color,
                                 keep if (whole and reps == 0 and keep is not None) else None)
        reps += 1
        if time.perf_counter() - t0 > sample_s / 3 or reps >= 3:
            break
    dt = time.perf_counter() - t0
    return dict(value=edges / dt, unit="edges/s", cores=1, kind="oracle",
                sample="%s, %d repetition(s), %.1f s" % (sample, reps, dt))


# --------------------------------------------------------------------------
# distributed plumbing (one process per GPU)
# --------------------------------------------------------------------------
_PG = None


def _barrier():
    if _PG is not None:
        import torch.distributed as dist
        dist.barrier()


def _reduce(x: float, op: str) -> float:
    """all-reduce of one number over the ranks ("max" or "sum"); the tensor
    lives where the process group's backend wants it (nccl: GPU, gloo: CPU)."""
    if _PG is None:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend(_PG) == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM, group=_PG)
    return float(t.item())


def whole_job(t_ms_local: float, units_local: float, steps: int):
    """Whole-job throughput over all ranks: the units every rank processed in
    one step, summed, divided by the slowest rank's time per step.
    Returns (units/s, ms per step)."""
    ms_per_step = _reduce(t_ms_local, "max") / steps
    units = _reduce(float(units_local), "sum")
    return units / (ms_per_step * 1e-3), ms_per_step


def set_group(pg):
    """use an already initialised process group (tests: gloo on CPU)"""
    global _PG
    _PG = pg


def init_dist():
    global _PG
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        _PG = dist.group.WORLD
    return ws, rank, local


# --------------------------------------------------------------------------
# reference arm: the oracle on the host cores
# --------------------------------------------------------------------------
# the oracle as it stands (one build per process, single-threaded) on every
# host core: a pool of spawned processes (never forked: the parent may hold a
# CUDA context) each building whole samples of the workload
_OW = None


def _oracle_worker_init(cfg, w, scale):
    global _OW
    sys.path.insert(0, ROOT)
    import oracle
    oracle.build_lib()
    mats, color = make_matrix(cfg, scale=scale)
    _OW = (oracle, mats, color, w)


def _oracle_worker_build(k):
    oracle, mats, color, w = _OW
    if len(mats) > 1:                       # a batch: one of its matrices per build, in turn
        rp, col, val = mats[k % len(mats)]
        ww = dict(w)
        return oracle_step(oracle, rp, col, val, ww, color, stream=k % len(mats))
    return sum(oracle_step(oracle, rp, col, val, w, color) for rp, col, val in mats)


def reference_sample(cfg):
    """(scale, description) of one step of the reference arm: the whole workload
    where one oracle build takes seconds, else a stated part of it."""
    if cfg in ("c1", "c2", "c3", "c5"):
        return None, "full workload per step"
    if cfg == "c6":
        return 512, "512x512 sub-grid of the same operator per step"
    return 8, "one matrix of the batch per step (the first 8 in turn)"


def oracle_all_cores(cfg, w, builds, procs=None, warm=True):
    """Throughput of `builds` oracle builds spread over `procs` spawned processes
    (default: every host core).  Returns (edges/s, seconds, processes)."""
    import multiprocessing as mp
    procs = procs or os.cpu_count() or 1
    procs = max(1, min(procs, builds))
    scale, _ = reference_sample(cfg)
    ctx = mp.get_context("spawn")
    with ctx.Pool(procs, initializer=_oracle_worker_init, initargs=(cfg, w, scale)) as pool:
        if warm:
            pool.map(_oracle_worker_build, range(procs), chunksize=1)     # untimed
        t0 = time.perf_counter()
        edges = sum(pool.map(_oracle_worker_build, range(builds), chunksize=1))
        dt = time.perf_counter() - t0
    return edges / dt, dt, procs


def run_reference(args, cfg, w):
    """Reference arm: the FP64 oracle (the plain CPU implementation written
    from the paper; there is no other implementation) on the host cores.  A
    step is one oracle build of the sample reference_sample() names -- for
    the default 1024 x 1024 workload the whole workload, i.e. the same
    config as the GPU arm; the steps run on every host core at once, one
    single-threaded build per process."""
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle
    oracle.build_lib()
    if w.get("coarsen"):
        return run_reference_coarsen(args, cfg, w, ws)
    scale, sample = reference_sample(cfg)
    v, dt, procs = oracle_all_cores(cfg, w, args.steps, warm=args.warmup > 0)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "edges/s",
            "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w["name"], "config": cfg, "same_config": scale is None},
            "cpu_baseline": {"value": v, "unit": "edges/s", "cores": procs, "kind": "oracle",
                             "sample": "%s; %d steps over %d single-threaded processes (one "
                                       "per host core), warm-up build per process untimed"
                                       % (sample, args.steps, procs)},
            "e2e": {"value": v, "unit": "edges/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_reference_coarsen(args, cfg, w, ws):
    """Reference arm of the coarsening workload: the oracle's CR +
    interpolation on a 256 x 256 sub-grid per step (its build untimed)."""
    import oracle
    mats, color = make_matrix(cfg, scale=256)
    rp, col, val = mats[0]
    b = oracle.build(rp, col, val, w["K"], w["seed"], w["nu"], w["omega"], w["theta"],
                     oracle.SWEEP_MCGS, color)
    for _ in range(args.warmup):
        oracle_coarsen_step(oracle, rp, col, val, w, color, b)
    t0 = time.perf_counter()
    rows = sum(oracle_coarsen_step(oracle, rp, col, val, w, color, b) for _ in range(args.steps))
    dt = time.perf_counter() - t0
    v = rows / dt
    line = {"impl": "reference",
            "metric": "rows/s of compatible-relaxation coarsening + LS interpolation",
            "value": v, "unit": "rows/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": w["name"], "config": cfg},
            "cpu_baseline": {"value": v, "unit": "rows/s", "cores": 1, "kind": "oracle",
                             "sample": "256x256 sub-grid of the same operator per step"},
            "e2e": {"value": v, "unit": "rows/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------------------
# coarsening workload: compatible relaxation + least-squares interpolation
# --------------------------------------------------------------------------
def interp_flops(rp, col, coarse, K, caliber):
    """FP64 operations of the exhaustive LS interpolation as its definition
    states it, per fine row with m coarse candidates: the Gram matrix and
    right-hand side (m(m+1)/2 + m + 1 weighted K-term sums, 3K each), and for
    every subset of s <= caliber candidates the elimination of the s x s
    system (2s^3/3 + 2s^2) and the weighted residual sum over K components
    (K (2s + 3))."""
    n = len(rp) - 1
    rows = np.repeat(np.arange(n), np.diff(rp))
    cand = (coarse[col] != 0) & (col != rows)
    m = np.bincount(rows[cand], minlength=n)[coarse == 0]
    total = np.sum((m * (m + 1) / 2 + m + 1) * 3 * K)
    for s_ in range(1, caliber + 1):
        sub = np.array([math.comb(int(v), s_) for v in range(int(m.max(initial=0)) + 1)],
                       dtype=np.float64)
        total += np.sum(sub[m]) * (2 * s_ ** 3 / 3 + 2 * s_ ** 2 + K * (2 * s_ + 3))
    return float(total)


def cr_sweep_bytes(n, nnz, ncolors):
    """Algorithmic bytes of one F-relaxation sweep (K = 1, FP64 values, rows
    in color order): the CSR, the diagonal and the coarse mask once, u read
    once per color phase and written once."""
    return nnz * 12 + 4 * (n + 1) + 8 * n + n + ncolors * 8 * n + 8 * n


def run_coarsen(args, cfg, w, mats, color, precision, ws, rank, flush):
    """One step = amgd_cr_coarsen (Algorithm 1 from the handle's distances,
    empty C_0) + amgd_ls_interpolation of the resulting coarse set, all
    outputs in device memory.  Unit: rows of the matrix coarsened and
    interpolated per second."""
    import ctypes
    import torch
    from paper_1106_5990_gb300 import amgd

    cw = w["coarsen"]
    rp, col, val = mats[0]
    n, nnz = len(rp) - 1, len(col)
    stream = torch.cuda.current_stream()
    h = amgd.Handle(rp, col, val, w["K"], w["seed"])
    h.set_stream(stream)
    h.set_precision(precision)
    h.set_coloring(color)
    ncolors = int(color.max()) + 1
    h.autotune(amgd.AMGD_SWEEP_MCGS, w["omega"], args.tune_cache)
    h.init_vectors(w["seed"])
    h.relax(w["nu"], w["omega"], amgd.AMGD_SWEEP_MCGS)
    h.distances(w["theta"], want=())
    L = amgd.lib()
    DEV, HOST = amgd.AMGD_MEM_DEVICE, amgd.AMGD_MEM_HOST
    coarse = torch.zeros(n, dtype=torch.uint8, device="cuda")
    cap = n * cw["caliber"]
    p_rp = torch.empty(n + 1, dtype=torch.int64, device="cuda")
    p_col = torch.empty(cap, dtype=torch.int32, device="cuda")
    p_val = torch.empty(cap, dtype=torch.float64, device="cuda")
    p_ls = torch.empty(n, dtype=torch.float64, device="cuda")
    rho = np.empty(cw["max_sets"] + 1)
    nr = ctypes.c_int32()
    nnz_pp = ctypes.c_int64()

    def cr():
        amgd.check(L.amgd_cr_coarsen(h.h, coarse.data_ptr(), DEV, None, HOST,
                                     amgd.AMGD_SWEEP_MCGS, cw["omega"], cw["nu"], w["theta"],
                                     cw["delta"], cw["tol"], cw["max_sets"], cw["seed"],
                                     rho.ctypes.data, ctypes.byref(nr)), h.h)

    def interp():
        amgd.check(L.amgd_ls_interpolation(h.h, coarse.data_ptr(), DEV, cw["caliber"],
                                           cw["gamma"], p_rp.data_ptr(), p_col.data_ptr(),
                                           p_val.data_ptr(), cap, ctypes.byref(nnz_pp),
                                           p_ls.data_ptr(), DEV), h.h)

    for _ in range(args.warmup):
        coarse.zero_()
        cr()
        interp()
    torch.cuda.synchronize()
    steps = args.steps
    clocks = ClockSampler(torch.cuda.current_device())
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(steps)]
    clocks.start()
    time.sleep(0.15)
    _barrier()
    torch.cuda.synchronize()
    launches = 0
    t_wall = time.perf_counter()
    for k in range(steps):
        flush.fill_(k & 0xFF)                     # evict L2 between steps (not timed)
        coarse.zero_()
        ev[k][0].record(stream)
        cr()
        ev[k][1].record(stream)
        interp()
        ev[k][2].record(stream)
        # interpolation: unpermute, classify, list, row and warp kernels, 3 scan, fill
        launches += h.cr_stats()[1] + 9
    torch.cuda.synchronize()
    t_wall = time.perf_counter() - t_wall
    _barrier()
    clk = clocks.stop()
    cr_ms = np.array([a.elapsed_time(b) for a, b, _ in ev])
    ip_ms = np.array([b.elapsed_time(c) for _, b, c in ev])
    value, ms_per_step = whole_job(float((cr_ms + ip_ms).sum()), n, steps)
    rounds, cr_launches = h.cr_stats()
    C = coarse.cpu().numpy()
    stages = nr.value
    peak, peak_kind = peaks()
    # dominant phase: its leading kernel against its bound
    flops = interp_flops(rp, col, C, w["K"], cw["caliber"])
    ip_mean = float(ip_ms.mean())
    cr_mean = float(cr_ms.mean())
    fp64_peak = 1250.0          # GB300 FP64 nominal, GFLOP/s (ALU bound of the fits)
    if ip_mean >= cr_mean:
        achieved = flops / (ip_mean * 1e-3) / 1e9
        roofline = {"bound": "alu", "achieved": achieved, "peak": fp64_peak, "unit": "GFLOP/s",
                    "frac": achieved / fp64_peak, "traffic": None,
                    "kernel": "k_ls_interp (FP64 exhaustive fits; phase incl. scan and fill)",
                    "peak_source": "nominal FP64 rate of the GB300 (1.25 TFLOP/s)",
                    "algorithmic_flops_per_launch": flops, "avg_launch_us": ip_mean * 1e3}
    else:
        sb = cr_sweep_bytes(n, nnz, ncolors)
        sweeps = stages * cw["nu"]
        achieved = sweeps * sb / (cr_mean * 1e-3) / 1e9
        roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                    "frac": achieved / peak, "traffic": None,
                    "kernel": "CR phase as a whole against its F-relaxation sweep bytes",
                    "peak_source": "%s hbm_gbs" % peak_kind,
                    "algorithmic_bytes_per_launch": sb, "avg_launch_us": None}
    line = {"metric": "rows/s of compatible-relaxation coarsening + LS interpolation",
            "value": value, "unit": "rows/s", "n_gpus": ws, "steps": steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w["name"], "config": cfg, "n": n, "nnz": nnz,
                       "storage_of_build": precision, "l2": "flushed between steps (256 MiB "
                       "write)", "coarsen": cw},
            "phase_ms": {"cr": cr_mean, "interp": ip_mean},
            "cr": {"stages": stages, "rho": rho[:stages].tolist(), "coarse": int(C.sum()),
                   "selection_rounds": rounds, "kernels": cr_launches,
                   "interp_entries": int(nnz_pp.value)},
            "host_wall_ms_per_step": 1e3 * t_wall / steps,
            "roofline": roofline, "gpu_launches": launches,
            "clocks": {k: clk[k] for k in ("sm_mhz", "sm_max_mhz", "reasons")}}
    # end to end: the same two calls with host buffers (coarse mask in, P out)
    e2e_steps = max(3, min(steps, 20))
    c_h = torch.zeros(n, dtype=torch.uint8).pin_memory()
    prp_h = torch.empty(n + 1, dtype=torch.int64).pin_memory()
    pcol_h = torch.empty(cap, dtype=torch.int32).pin_memory()
    pval_h = torch.empty(cap, dtype=torch.float64).pin_memory()
    pls_h = torch.empty(n, dtype=torch.float64).pin_memory()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        c_h.zero_()
        amgd.check(L.amgd_cr_coarsen(h.h, c_h.data_ptr(), HOST, None, HOST,
                                     amgd.AMGD_SWEEP_MCGS, cw["omega"], cw["nu"], w["theta"],
                                     cw["delta"], cw["tol"], cw["max_sets"], cw["seed"],
                                     rho.ctypes.data, ctypes.byref(nr)), h.h)
        amgd.check(L.amgd_ls_interpolation(h.h, c_h.data_ptr(), HOST, cw["caliber"],
                                           cw["gamma"], prp_h.data_ptr(), pcol_h.data_ptr(),
                                           pval_h.data_ptr(), cap, ctypes.byref(nnz_pp),
                                           pls_h.data_ptr(), HOST), h.h)
    t_e2e = (time.perf_counter() - t0) / e2e_steps
    v_e2e, _ = whole_job(1e3 * t_e2e, n, 1)
    line["e2e"] = {"value": v_e2e, "unit": "rows/s", "h2d_bytes_per_step": 2 * n,
                   "d2h_bytes_per_step": n + 8 * (n + 1) + 12 * int(nnz_pp.value) + 8 * n,
                   "steps": e2e_steps,
                   "api": "amgd_cr_coarsen(host mask) + amgd_ls_interpolation(host mask, host P)"}
    if rank == 0 and not args.no_cpu:
        line["cpu_baseline"] = cpu_coarsen_time(w)
    h.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def oracle_coarsen_step(oracle, rp, col, val, w, color, b):
    """CR + LS interpolation on the oracle from the oracle's own build b."""
    cw = w["coarsen"]
    C, _ = oracle.cr_coarsen(rp, col, val, rp, col, b["ls"], w["theta"], cw["nu"], cw["omega"],
                             oracle.SWEEP_MCGS, color, cw["delta"], cw["tol"], cw["max_sets"],
                             cw["seed"])
    oracle.ls_interp(b["X"], b["Y"], rp, col, C, cw["caliber"], cw["gamma"])
    return len(rp) - 1


def cpu_coarsen_time(w, sample_s=20.0, N=512):
    """The FP64 oracle (single thread) on CR + interpolation of an N x N
    sub-grid of the same operator (its own build, untimed)."""
    import oracle
    mats, color = make_matrix("c7", scale=N)
    rp, col, val = mats[0]
    b = oracle.build(rp, col, val, w["K"], w["seed"], w["nu"], w["omega"], w["theta"],
                     oracle.SWEEP_MCGS, color)
    rows = 0
    reps = 0
    t0 = time.perf_counter()
    while True:
        rows += oracle_coarsen_step(oracle, rp, col, val, w, color, b)
        reps += 1
        if time.perf_counter() - t0 > sample_s / 3 or reps >= 3:
            break
    dt = time.perf_counter() - t0
    return dict(value=rows / dt, unit="rows/s", cores=1, kind="oracle",
                sample="%dx%d sub-grid of the same operator, %d repetition(s), %.1f s"
                       % (N, N, reps, dt))


# --------------------------------------------------------------------------
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--config", default="c2", choices=sorted(WORKLOADS))
    ap.add_argument("--precision", default=None, choices=["fp64", "fp32", "bf16"])
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-side", action="store_true", help="skip the FP64 side measurement")
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle CPU baseline")
    ap.add_argument("--scale", type=int, default=None,
                    help="shrink the workload for profiling captures (grid side; for the "
                         "graph batch: the first SCALE matrices); never for reported numbers")
    ap.add_argument("--tune-cache", default=None,
                    help="autotuner cache file (a matching entry skips the tuning launches)")
    args = ap.parse_args()
    cfg = args.config
    w = dict(WORKLOADS[cfg])
    if args.warmup < 3:
        raise SystemExit("at least 3 warm-up steps are required")
    if args.impl == "reference":
        return run_reference(args, cfg, w)

    import torch
    ws, rank, local = init_dist()
    torch.cuda.set_device(local)
    from paper_1106_5990_gb300 import amgd
    amgd.lib()
    precision = args.precision or w["precision"]
    mats, color = make_matrix(cfg, scale=args.scale)
    # a batch of independent matrices is split across the ranks (each matrix keeps
    # its key in the whole batch: the union of the shards is the one-GPU build);
    # a single matrix runs as an independent replica per rank with its own seed
    ids = None
    if len(mats) > 1:
        ids = shard_batch([len(m[1]) for m in mats], ws, rank)
        mats = [mats[b] for b in ids]
        scaling = "strong"
    else:
        w["seed"] += rank
        scaling = "weak"
    n = sum(len(m[0]) - 1 for m in mats)
    nnz = sum(len(m[1]) for m in mats)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    if w.get("coarsen"):
        return run_coarsen(args, cfg, w, mats, color, precision, ws, rank, flush)

    r = run_gpu_arm(mats, color, w, precision, args.steps, args.warmup, rank, flush,
                    tune_cache=args.tune_cache, matrix_ids=ids)
    depth = w.get("depth", 1)
    nnz_p = r["h"].nnz_p                       # entries of the fit pattern (A, or G_d)
    E = r["h"].E_p                             # edges whose distance the step computes
    value, ms_per_step = whole_job(float(r["step_ms"].sum()), E, args.steps)

    permuted = w["sweep"] == "mcgs"
    adj = w.get("adjoint")
    mixed = precision != "fp64"

    def step_bytes(rr, prec):
        if adj:
            return adjoint_bytes(n, nnz, w["K"], w["nu"], adj, prec)
        return algorithmic_bytes(n, nnz, E, rr["E_s"], w["K"], w["nu"], rr["ncolors"], prec,
                                 permuted, nnz_p=nnz_p if depth > 1 else None)

    ab = step_bytes(r, precision)
    launches_relax = w["nu"] * r["ncolors"]
    relax_launch_ms = r["phase_ms"][1] / launches_relax
    peak, peak_kind = peaks()
    if depth > 1 and r["phase_ms"][2] > r["phase_ms"][1]:
        # the distance pass over G_d dominates the step: one launch (plus the
        # FP64 row fixup of the mixed paths, inside the same phase)
        edge_ms = r["phase_ms"][2]
        achieved = ab["edge"] / (edge_ms * 1e-3) / 1e9
        tkey = "edge/%s/K%d/%s" % (precision, w["K"], cfg)
        traffic = recorded_traffic(tkey, source_sha("k_edge.cuh", "rowops.cuh",
                                                    "amgd_internal.cuh"))
        roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                    "frac": achieved / peak, "traffic": traffic,
                    "kernel": "distance pass over G_%d (edge kernel + FP64 row fixup)" % depth,
                    "peak_source": "%s hbm_gbs" % peak_kind,
                    "algorithmic_bytes_per_launch": ab["edge"],
                    "avg_launch_us": edge_ms * 1e3}
    else:
        achieved = ab["relax_per_launch"] / (relax_launch_ms * 1e-3) / 1e9
        tkey = "relax/%s/K%d/%s" % (precision, w["K"], cfg)
        traffic = recorded_traffic(tkey, source_sha("k_relax.cu", "rowops.cuh",
                                                    "amgd_internal.cuh"))
        roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                    "frac": achieved / peak, "traffic": traffic,
                    "kernel": "k_relax (one color phase of one sweep)",
                    "peak_source": "%s hbm_gbs" % peak_kind,
                    "algorithmic_bytes_per_launch": ab["relax_per_launch"],
                    "avg_launch_us": relax_launch_ms * 1e3}
    names = ["init", "relax", "distances", "backward" if adj else "strength"]
    phases = dict(zip(names, r["phase_ms"].tolist()))
    whole = ab["total"] / (ms_per_step * 1e-3) / 1e9

    line = {"metric": METRIC, "value": value, "unit": "edges/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
            "higher_is_better": True, "scaling": scaling, "vs_baseline": None,
            "dtype": "f64" if precision == "fp64" else "f32", "data": "synthetic",
            "config": {"workload": w["name"], "config": cfg, "n": n, "nnz": nnz, "E": E,
                       "search_depth": depth, "nnz_pattern": nnz_p,
                       "K": w["K"], "nu": w["nu"], "sweep": w["sweep"], "theta": w["theta"],
                       "storage": precision,
                       "ls_sums": ("compensated FP32 (Kahan-Babuska-Neumaier, TwoSum)"
                                   if mixed else "FP64"),
                       "l2": "flushed between steps (256 MiB write)",
                       "graph": "one CUDA graph per step",
                       "shapes": {"relax": list(r["shapes"][0]), "edge": list(r["shapes"][1]),
                                  "legend": "(lanes per row G, 16-byte vectors per lane NV, "
                                            "nonzeros per gather batch U, kernel: relaxation 0 "
                                            "direct / 1 TMA-staged CSR / 2 cp.async pipelined / "
                                            "3 chunked per SM; distances 0 rows / 1 tiles / "
                                            "2 rows in place / 3 warp-staged in place), "
                                            "autotuned"}},
            "phase_ms": phases,
            "timed_region": ("start vectors (Philox) + nu recorded sweeps + distances + reverse "
                             "pass" if adj else "start vectors (Philox) + nu sweeps + distances, "
                             "threshold + strength CSR, one CUDA graph per step"),
            "whole_step_gbs": whole, "whole_step_hbm_frac": whole / peak,
            "roofline": roofline}
    if args.scale:
        line["config"]["scale"] = args.scale
        line["config"]["workload"] += " -- SHRUNK by --scale for profiling, not the workload"
    if adj:
        line["config"]["checkpoint_every"] = adj
        line["config"]["step"] = ("vector start, nu recorded sweeps, distances, reverse pass "
                                  "of sum r^2 over kept edges (dL/dvalues, dL/domega)")
        line["backward_phase_gbs"] = ab["backward"] / (r["phase_ms"][3] * 1e-3) / 1e9
        line["scalars"] = {"omega_bar": r["scalars"][0], "loss": r["scalars"][1]}

    # kernels of ours per step
    edge_launches = 2 if mixed else 1                     # + FP64 row fixup on mixed paths
    if adj:
        nck = -(-w["nu"] // adj)
        bwd_launches = 4 + (w["nu"] - nck) + 2 * w["nu"] + 2
        launches_per_step = 1 + launches_relax + edge_launches + bwd_launches
    else:
        launches_per_step = 1 + launches_relax + (1 if permuted else 0) + edge_launches + 3
    line["gpu_launches"] = launches_per_step * args.steps

    if not args.no_side and precision != "fp64":
        side_steps = max(3, min(args.steps, 100))
        r64 = run_gpu_arm(mats, color, w, "fp64", side_steps, 3, rank, flush, want_clocks=False,
                          tune_cache=args.tune_cache, matrix_ids=ids)
        v64, t64 = whole_job(float(r64["step_ms"].sum()), E, side_steps)
        ab64 = step_bytes(r64, "fp64")
        rl = r64["phase_ms"][1] / launches_relax
        a64 = ab64["relax_per_launch"] / (rl * 1e-3) / 1e9
        line["fp64"] = {"value": v64, "unit": "edges/s", "ms_per_step": t64,
                        "steps": side_steps, "shapes": {"relax": list(r64["shapes"][0]),
                                                        "edge": list(r64["shapes"][1])},
                        "phase_ms": dict(zip(names, r64["phase_ms"].tolist())),
                        "relax_launch_us": rl * 1e3, "relax_hbm_gbs": a64,
                        "relax_hbm_frac": a64 / peak,
                        "mixed_over_fp64": value / v64}
        r64["h"].close()

    # cost of the compensated LS sums: the same build with plain FP32 sums
    if not args.no_side and mixed and not adj and depth == 1:
        side_steps = max(3, min(args.steps, 100))
        r_p = run_gpu_arm(mats, color, w, precision, side_steps, 3, rank, flush,
                          want_clocks=False, tune_cache=args.tune_cache, summation="plain",
                          matrix_ids=ids)
        v_p, t_p = whole_job(float(r_p["step_ms"].sum()), E, side_steps)
        line["plain_ls_sums"] = {"value": v_p, "unit": "edges/s", "ms_per_step": t_p,
                                 "steps": side_steps,
                                 "distances_ms": float(r_p["phase_ms"][2]),
                                 "edge_shape": list(r_p["shapes"][1]),
                                 "compensation_cost_ms": float(r["phase_ms"][2] -
                                                               r_p["phase_ms"][2])}
        r_p["h"].close()

    # the other mixed storage beside the headline (BF16 beside FP32 and the other way
    # round), timed on the same matrix; its accuracy is taken against the same oracle
    # build below
    other = {"fp32": "bf16", "bf16": "fp32"}.get(precision)
    r_o = None
    if not args.no_side and other is not None and not adj:
        side_steps = max(3, min(args.steps, 100))
        r_o = run_gpu_arm(mats, color, w, other, side_steps, 3, rank, flush, want_clocks=False,
                          tune_cache=args.tune_cache, matrix_ids=ids)
        v_o, t_o = whole_job(float(r_o["step_ms"].sum()), E, side_steps)
        ab_o = step_bytes(r_o, other)
        rl_o = r_o["phase_ms"][1] / launches_relax
        a_o = ab_o["relax_per_launch"] / (rl_o * 1e-3) / 1e9
        line[other] = {"value": v_o, "unit": "edges/s", "ms_per_step": t_o,
                       "steps": side_steps, "shapes": {"relax": list(r_o["shapes"][0]),
                                                       "edge": list(r_o["shapes"][1])},
                       "phase_ms": dict(zip(names, r_o["phase_ms"].tolist())),
                       "relax_launch_us": rl_o * 1e3, "relax_hbm_gbs": a_o,
                       "relax_hbm_frac": a_o / peak}
        if "fp64" in line:
            line[other]["over_fp64"] = v_o / line["fp64"]["value"]

    e2e_steps = max(3, min(args.steps, 50))
    e = run_e2e(r["h"], mats, w, r["sweep"], e2e_steps, adjoint=adj)
    v_e2e, _ = whole_job(1e3 * e["seconds"], E, 1)
    line["e2e"] = {"value": v_e2e, "unit": "edges/s", "h2d_bytes_per_step": e["h2d"],
                   "d2h_bytes_per_step": e["d2h"], "steps": e2e_steps,
                   "api": ("amgd_set_values(host) + init + relax (recorded) + distances + "
                           "amgd_backward(host dL/dvalues)") if adj else
                          "per step amgd_set_values_async(pinned host) + amgd_graph_launch "
                          "(captured build) + amgd_strength_async(pinned host); one amgd_sync "
                          "after the last step"}
    line["clocks"] = {k: r["clocks"][k] for k in ("sm_mhz", "sm_max_mhz", "reasons")} \
        if r["clocks"] else None
    if rank == 0 and not args.no_cpu:
        ref = {}
        line["cpu_baseline"] = cpu_oracle_time(cfg, w, keep=ref)
        # the same oracle on every host core (independent builds, one per process)
        procs = os.cpu_count() or 1
        v_all, dt_all, procs = oracle_all_cores(cfg, w, procs, procs)
        line["cpu_baseline_all_cores"] = {
            "value": v_all, "unit": "edges/s", "cores": procs, "kind": "oracle",
            "sample": "%s; %d builds at once, one single-threaded process per host core, "
                      "%.1f s" % (reference_sample(cfg)[1], procs, dt_all)}
        if ref and not args.scale:
            line["accuracy"] = accuracy_vs_oracle(r["h"], mats[0], ref, w["theta"])
            if r_o is not None:
                line[other]["accuracy"] = accuracy_vs_oracle(r_o["h"], mats[0], ref, w["theta"])
                line[other]["meets_accuracy"] = line[other]["accuracy"]["meets_accuracy"]
    if r_o is not None:
        r_o["h"].close()
    r["h"].close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if _PG is not None:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
