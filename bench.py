"""Benchmark: DA-CSR-16 vs CSR-32 SpMV throughput on GB300.

Workload (the configuration the headline metric is quoted on): the 3-D
7-point Laplacian on a 128^3 grid in natural order (n = 2,097,152 rows,
nnz = 14,581,760, half-bandwidth 16,384), FP64 values, x ~ U[-1, 1).
One step = one DA-CSR-16 SpMV y = A x through the C ABI.  Inputs are
resident in HBM; consecutive steps cycle through 4 copies of the matrix
(4 x 188 MB, larger than the 126 MB L2), so every step streams its matrix
from HBM.  Throughput = algorithmic bytes (Section 4: the three arrays of
Eq. (3), x read once, y written once) / time.

Also reported in the same run: CSR-32 on the same matrix and plan (and the
DA/CSR ratio), FP32 / BF16 value variants, an end-to-end number through the
public API with host buffers (x uploaded and y downloaded every step), the
roofline of the SpMV kernel against the measured HBM copy bandwidth, GPU
clocks sampled during the timed region, and the plain-C oracle (Listing 2)
timed on the host cores as a CPU baseline.

Secondary sections of the same line (each on its own synthetic workload,
none of them inside the headline's timed region):
  * ``conversion`` / ``rcm``: CSR -> DA-CSR-16 throughput; the 128^3 grid
    under a seeded random symmetric permutation (int16 fit rate), RCM on it
    (host ordering + device P A P^T) and SpMV throughput after RCM;
  * ``solvers``: 160^3 27-point stencil, time to a true relative residual of
    1e-10 for FP64 CG and for CG with FP64 refinement around FP32 / BF16
    DA-CSR-16 inner solves;
  * ``solvers_perturbed``: the same with a symmetric N(0, 0.01^2)
    perturbation of the off-diagonals (values no longer exact in FP32 /
    BF16), with the low-precision SpMV error per dtype;
  * ``batched``: 512 random banded matrices, k in {1, 4, 16} right-hand
    sides, FP64 / FP32: one persistent launch (direct and graph replay) vs
    512 per-matrix launches (eager and graph-captured);
  * ``da8``: DA-CSR-8 (int8 offsets) vs DA-CSR-16 vs CSR-32 on a 2-D
    Laplacian whose half-bandwidth (127) fits int8, FP64 and FP32 values;
  * ``dabsr``: DA-BSR-16 vs BSR-32 (diagonal addressing of the block
    pattern) on a 96^3 grid with dense 3 x 3 blocks, FP64 and FP32 values;
  * ``dacoo``: DA-COO-16 vs COO-32 on the 128^3 Laplacian;
  * ``banded``: random banded matrices, n in {1e5, 1e6} x h in {100, 1000,
    30000} and n = 1e7 at h = 1000, DA-CSR-16 vs CSR-32 FP64 (``banded_full``:
    n in {1e5, 3e5, 1e6, 3e6, 1e7, 2e7} x the three h, not run by default);
  * ``small``: the 64x64 5-point Laplacian, SpMV time per call under graph
    replay (launch / latency bound, in L2).

``--impl reference`` times the oracle (the plain-C Listing 2 restatement)
on the host cores instead, for the same metric and workload.

Multi-GPU (torchrun): every rank runs its own copy of the workload (weak
scaling, no collective on the data path); rank 0 prints the line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "DA-CSR16 vs CSR32 SpMV GB/s, % HBM peak; mixed-prec CG time-to-1e-10"
WORKLOAD = "laplace3d_7pt_128^3_natural_dacsr16_f64_spmv"
GRID = 128
NCOPY = 4
FP64_TFMA_NOMINAL = 0.625   # GB300 FP64: 1.25 TFLOP/s nominal, one FMA = 2 flops


def spmv_bytes(n, nnz, idx_bytes, val_bytes, vec_bytes):
    """Section 4 traffic: Eq. (3) with 32-bit row pointers, plus x read once
    and y written once (beta = 0)."""
    return (n + 1) * 4 + nnz * (idx_bytes + val_bytes) + 2 * n * vec_bytes


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def kernel_source_hash():
    """Hash of the SpMV kernel's sources with comments and blank lines
    removed (a comment edit does not invalidate recorded counters)."""
    import re
    h = hashlib.sha256()
    for name in ("spmv_kernel.cuh", "spmv_launch.cuh", "spmv.cu", "damn_common.cuh"):
        with open(os.path.join(ROOT, "paper_2307_06305_gb300", "csrc", name)) as f:
            text = f.read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        code = [re.sub(r"//.*$", "", line).rstrip() for line in text.splitlines()]
        h.update("\n".join(l for l in code if l.strip()).encode())
    return h.hexdigest()[:16]


def recorded_traffic():
    """DRAM bytes per launch from the committed ncu summary, when it was taken
    on the current kernel source (else None)."""
    path = os.path.join(ROOT, "profiles", "spmv_dacsr16_f64_laplace3d_128.json")
    try:
        with open(path) as f:
            rec = json.load(f)
    except OSError:
        return None
    if rec.get("kernel_source_hash") != kernel_source_hash():
        return None
    return rec.get("dram_bytes_per_launch")


class ClockSampler:
    """Samples nvidia-smi SM clocks and throttle reasons every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu_index = gpu_index
        self.rows = []
        self._stop = threading.Event()
        self._t = None

    def _run(self):
        while not self._stop.is_set():
            try:
                out = subprocess.run(["nvidia-smi", "-i", str(self.gpu_index),
                                      f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits"],
                                     capture_output=True, text=True, timeout=5).stdout.strip()
                if out:
                    self.rows.append([c.strip() for c in out.split(",")])
            except Exception:
                pass
            self._stop.wait(0.2)

    def __enter__(self):
        self._t = threading.Thread(target=self._run, daemon=True)
        self._t.start()
        return self

    def __exit__(self, *a):
        self._stop.set()
        self._t.join(timeout=10)

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in self.rows for k in range(4)
                          if len(r) > 5 + k and r[5 + k].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(self.rows)}


def max_over_ranks(t, dist, device):
    """The slowest rank's time: N independent replicas (one per GPU) are timed
    together, and the job takes as long as its slowest rank."""
    if dist is None:
        return t
    import torch
    tt = torch.tensor([t], dtype=torch.float64, device=device)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    return float(tt.item())


def replica_value(world, units_per_step, seconds_per_step):
    """Whole-job throughput of `world` replicas: the units every rank
    processed in one step, over the slowest rank's step time, in 1e9 / s."""
    return world * units_per_step / seconds_per_step / 1e9


def _time_repeated(fn, budget_s):
    """Seconds per call of fn() repeated for about budget_s seconds (one
    untimed warm-up call first), and the number of timed calls."""
    fn()
    reps, t0 = 0, time.perf_counter()
    while True:
        fn()
        reps += 1
        el = time.perf_counter() - t0
        if el >= budget_s:
            return el / reps, reps


def cpu_oracle_baseline(rp, col, off, val, x, budget_s=10.0):
    """The plain-C Listing 2 oracle (FP64) timed on the host: DA-CSR-16 on all
    cores of the affinity mask (the reported baseline, about budget_s
    seconds), then DA-CSR-16 on one core and CSR-32 on all cores (about a
    fifth of budget_s each).  Returns {name: (seconds per SpMV, reps, threads)}."""
    from oracle import c_listing2 as C
    cores = len(os.sched_getaffinity(0))
    n = len(rp) - 1
    y = np.zeros(n)
    out = {}
    out["dacsr16"] = _time_repeated(
        lambda: C.spmv_dacsr16(n, rp, off, val, x, out=y, nthreads=cores), budget_s) + (cores,)
    out["dacsr16_1thread"] = _time_repeated(
        lambda: C.spmv_dacsr16(n, rp, off, val, x, out=y, nthreads=1), budget_s / 5) + (1,)
    out["csr32"] = _time_repeated(
        lambda: C.spmv_csr32(n, rp, col, val, x, out=y, nthreads=cores), budget_s / 5) + (cores,)
    return out


def cpu_oracle_cg_sample(iters=2):
    """The oracle's FP64 CG (numpy) on the 160^3 27-point system, b = A x*
    (x* seeded as in the solvers section): seconds per iteration over `iters`
    iterations after the initial residual, timed as one call."""
    import workloads as W
    from oracle import cg as OC
    from oracle import dacsr as OD
    from oracle import c_listing2 as C
    rp, col, val = W.stencil27(160)
    n = len(rp) - 1
    off = OD.translate(n, rp, col).astype(np.int16)
    del col
    xs = W.uniform_vector(n, W.rng_for(4, 1))
    b = C.spmv_dacsr16(n, rp, off, val, xs, nthreads=len(os.sched_getaffinity(0)))
    t0 = time.perf_counter()
    res = OC.cg(n, rp, off, val, b, rtol=1e-10, max_iter=iters)
    el = time.perf_counter() - t0
    return el / max(res.iterations, 1), res.iterations, n, len(val)


def build_inputs():
    import workloads as W
    rp, col, val = W.laplace3d_7pt(GRID)
    x = W.uniform_vector(GRID ** 3, W.rng_for(2, 0))
    return rp, col, val, x


def run_reference(args, rank, world):
    """--impl reference: the oracle on the host cores (rank 0 only)."""
    if rank != 0:
        return
    rp, col, val, x = build_inputs()
    n, nnz = len(rp) - 1, len(col)
    from oracle import c_listing2 as C
    from oracle import dacsr as OD
    off = OD.translate(n, rp, col).astype(np.int16)
    cores = len(os.sched_getaffinity(0))
    y = np.zeros(n)
    for _ in range(max(args.warmup, 1)):
        C.spmv_dacsr16(n, rp, off, val, x, out=y, nthreads=cores)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        C.spmv_dacsr16(n, rp, off, val, x, out=y, nthreads=cores)
    t = (time.perf_counter() - t0) / args.steps
    b = spmv_bytes(n, nnz, 2, 8, 8)
    v = b / t / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": round(v, 2), "unit": "GB/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(t * 1e3, 4), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n": n, "nnz": nnz},
            "cpu_baseline": {"value": round(v, 2), "unit": "GB/s", "cores": cores,
                             "kind": "oracle",
                             "sample": f"{args.steps} whole DA-CSR-16 SpMVs (plain C Listing 2, "
                                       f"OpenMP static rows) of the full workload"},
            "e2e": {"value": round(v, 2), "unit": "GB/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


PROFILE_CASES = ("stencil27_160_rows_long", "batch512_f64_k1", "laplace3d_128",
                 "laplace3d_128_values", "cg_160_f64", "cg_ir_160_f32", "cg_ir_160_bf16",
                 "laplace3d_128_dacoo16",
                 "banded_<n>_h<h>_<tiling>_<fmt>", "batch512_<f64|f32>_k<k>_<streamed|passes>[_e<E>]")


def profile_case(name):
    """argparse type of --case: a fixed case name, or a random banded case
    banded_<n>_h<h>_<tiling>_<fmt> (n like 1e6, tiling auto / rows /
    rows_long / slices, fmt da16 / csr32)."""
    if name in PROFILE_CASES[:8]:
        return name
    parts = name.split("_")
    if (len(parts) in (4, 5) and parts[0] == "batch512" and parts[1] in ("f64", "f32")
            and parts[2][:1] == "k" and parts[2][1:].isdigit() and 1 <= int(parts[2][1:]) <= 64
            and parts[3] in ("streamed", "passes")
            and (len(parts) == 4 or parts[4] in ("e1", "e2", "e4", "e8"))):
        return name
    tiling = "_".join(parts[3:-1])
    ok = (len(parts) >= 5 and parts[0] == "banded" and parts[2].startswith("h")
          and (tiling == "auto" or tiling in TILING_NAMES) and parts[-1] in ("da16", "csr32"))
    if not ok:
        raise argparse.ArgumentTypeError(f"unknown case {name!r}; one of {PROFILE_CASES}")
    return name


def run_case(args):
    """--case NAME: only the launches of one kernel, for an ncu capture; no
    timing (a number taken under a profiler is not a benchmark value).

    stencil27_160_rows_long: the 160^3 27-point stencil converted to
    DA-CSR-16, a plan pinned to the rows-long tiling, then --steps FP64 SpMVs
    (every k_spmv launch of the run).
    laplace3d_128_dacoo16: the 128^3 grid as DA-COO-16 (int32 rows, int16
    offsets), FP64, --steps SpMVs.
    batch512_f64_k1: the 512 random banded matrices converted to DA-CSR-16,
    k = 1 FP64 right-hand sides, a batch plan without autotuning, then
    --steps direct launches of the batched kernel.
    batch512_<f64|f32>_k<k>_<streamed|passes>[_e<E>]: the same with k
    right-hand sides of that type and the plan pinned to streamed rows (items
    of 1024 rows) or fixed passes (items of 256 rows), E entry lanes per row
    (default: the plan's choice from nnz / nrows)."""
    import torch
    import workloads as W
    from paper_2307_06305_gb300 import damn as D
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0")))
    torch.cuda.set_device(dev)
    if args.case.startswith("banded_"):
        parts = args.case.split("_")
        n, h, fmt = int(float(parts[1])), int(parts[2][1:]), parts[-1]
        tiling = "_".join(parts[3:-1])
        rp, col, val = W.random_banded(n, h, W.rng_for(3, 0))
        nnz = len(col)
        t_rp, t_col = torch.from_numpy(rp).to(dev), torch.from_numpy(col).to(dev)
        off, _ = D.damn_csr_to_dacsr(t_rp, t_col, n, raise_on_nofit=True)
        t_val = torch.from_numpy(val).to(dev)
        x = torch.from_numpy(W.uniform_vector(n, W.rng_for(3, 100))).to(dev)
        y = torch.empty(n, dtype=torch.float64, device=dev)
        plan = D.Plan(t_rp, nnz, n, torch.float64, idx=off)
        if tiling != "auto":
            plan.set_tiling(TILING_NAMES.index(tiling))
        for _ in range(args.steps):
            if fmt == "da16":
                D.damn_spmv_dacsr16(t_rp, off, t_val, x, y, plan=plan)
            else:
                D.damn_spmv_csr32(t_rp, t_col, t_val, x, y, plan=plan)
    elif args.case in ("cg_160_f64", "cg_ir_160_f32", "cg_ir_160_bf16"):
        rp, col, val = W.stencil27(160)
        n, nnz = len(rp) - 1, len(col)
        t_rp, t_col = torch.from_numpy(rp).to(dev), torch.from_numpy(col).to(dev)
        off, _ = D.damn_csr_to_dacsr(t_rp, t_col, n, raise_on_nofit=True)
        t_val = torch.from_numpy(val).to(dev)
        xs = torch.from_numpy(W.uniform_vector(n, W.rng_for(4, 1))).to(dev)
        b = torch.empty(n, dtype=torch.float64, device=dev)
        D.damn_spmv_dacsr16(t_rp, off, t_val, xs, b)
        p64 = D.Plan(t_rp, nnz, n, torch.float64, idx=off)
        x = torch.zeros(n, dtype=torch.float64, device=dev)
        for _ in range(args.steps):
            x.zero_()
            if args.case == "cg_160_f64":
                D.damn_cg(t_rp, off, t_val, b, x, 1e-10, 2000, plan=p64)
            else:
                lowp = torch.float32 if args.case.endswith("f32") else torch.bfloat16
                vl = D.damn_cast_values(t_val, lowp)
                pl = D.Plan(t_rp, nnz, n, lowp, idx=off)
                D.damn_cg_ir(t_rp, off, t_val, vl, b, x, 1e-10,
                             1e-3 if lowp == torch.float32 else 1e-2, 200, 60,
                             plan64=p64, plan_low=pl)
    elif args.case == "laplace3d_128_values":
        rp, col, val, xh = build_inputs()
        n, nnz = len(rp) - 1, len(col)
        t_rp, t_col = torch.from_numpy(rp).to(dev), torch.from_numpy(col).to(dev)
        off, _ = D.damn_csr_to_dacsr(t_rp, t_col, n, raise_on_nofit=True)
        t_val = torch.from_numpy(val).to(dev)
        x = torch.from_numpy(xh).to(dev)
        runs = []
        for dt in (torch.float64, torch.float32, torch.bfloat16, torch.float8_e4m3fn):
            v = t_val if dt == torch.float64 else D.damn_cast_values(t_val, dt)
            xv = x if dt == torch.float64 else x.float()
            y = torch.empty(n, dtype=xv.dtype, device=dev)
            runs.append((v, xv, y, D.Plan(t_rp, nnz, n, dt, idx=off)))
        for _ in range(args.steps):
            for v, xv, y, pl in runs:
                D.damn_spmv_dacsr16(t_rp, off, v, xv, y, plan=pl)
    elif args.case == "laplace3d_128":
        rp, col, val, xh = build_inputs()
        n, nnz = len(rp) - 1, len(col)
        t_rp, t_col = torch.from_numpy(rp).to(dev), torch.from_numpy(col).to(dev)
        off, _ = D.damn_csr_to_dacsr(t_rp, t_col, n, raise_on_nofit=True)
        t_val = torch.from_numpy(val).to(dev)
        x = torch.from_numpy(xh).to(dev)
        y = torch.empty(n, dtype=torch.float64, device=dev)
        plan = D.Plan(t_rp, nnz, n, torch.float64, idx=off)
        for _ in range(args.steps):
            D.damn_spmv_dacsr16(t_rp, off, t_val, x, y, plan=plan)
    elif args.case == "laplace3d_128_dacoo16":
        rp, col, val, xh = build_inputs()
        n = len(rp) - 1
        row = np.repeat(np.arange(n, dtype=np.int32), np.diff(rp))
        t_rp, t_col = torch.from_numpy(rp).to(dev), torch.from_numpy(col).to(dev)
        off, _ = D.damn_csr_to_dacsr(t_rp, t_col, n, raise_on_nofit=True)
        t_row, t_val = torch.from_numpy(row).to(dev), torch.from_numpy(val).to(dev)
        x = torch.from_numpy(xh).to(dev)
        y = torch.empty(n, dtype=torch.float64, device=dev)
        ws = D._workspace(D._fn("damn_coo_workspace_size")(len(col), D._DTYPE_CODE[torch.float64]),
                          dev)
        for _ in range(args.steps):
            D.damn_spmv_dacoo16(n, t_row, off, t_val, x, y, workspace=ws)
    elif args.case == "stencil27_160_rows_long":
        rp, col, val = W.stencil27(160)
        n, nnz = len(rp) - 1, len(col)
        t_rp, t_col = torch.from_numpy(rp).to(dev), torch.from_numpy(col).to(dev)
        off, _ = D.damn_csr_to_dacsr(t_rp, t_col, n, raise_on_nofit=True)
        t_val = torch.from_numpy(val).to(dev)
        x = torch.from_numpy(W.uniform_vector(n, W.rng_for(4, 1))).to(dev)
        y = torch.empty(n, dtype=torch.float64, device=dev)
        plan = D.Plan(t_rp, nnz, n, torch.float64, idx=off)
        plan.set_tiling(D.DAMN_TILING_ROWS_LONG)
        for _ in range(args.steps):
            D.damn_spmv_dacsr16(t_rp, off, t_val, x, y, plan=plan)
    else:
        parts = args.case.split("_")
        dt = torch.float64 if parts[1] == "f64" else torch.float32
        k = int(parts[2][1:])
        gen = torch.Generator(device=dev)
        gen.manual_seed(W.seed_for(5, 1))
        mats = []
        for n, rp, col, val in W.batch_banded(512):
            t_rp, t_col = torch.from_numpy(rp).to(dev), torch.from_numpy(col).to(dev)
            off, _ = D.damn_csr_to_dacsr(t_rp, t_col, n, raise_on_nofit=True)
            X = torch.rand((n, k), generator=gen, device=dev, dtype=dt) * 2 - 1
            Y = torch.empty((n, k), dtype=dt, device=dev)
            mats.append((t_rp, off, torch.from_numpy(val).to(dev).to(dt), X, Y))
        plan = D.BatchPlan(mats, k, dt, autotune=False)
        if len(parts) >= 4:
            E = int(parts[4][1:]) if len(parts) == 5 else plan.describe()["entry_lanes"]
            streamed = parts[3] == "streamed"
            plan.set_shape(streamed, 1024 if streamed else 256, E, 256)
        for _ in range(args.steps):
            plan.launch()
    torch.cuda.synchronize()
    if D.damn_device_status() != 0:
        raise RuntimeError("device status word reports an error")
    print(json.dumps({"case": args.case, "launches": args.steps}), flush=True)


# ----------------------------------------------------------------------------
# secondary sections
# ----------------------------------------------------------------------------

def _event_time(torch, fn, reps, stream=None):
    """Median and min seconds of fn() over reps, CUDA events on the stream."""
    stream = stream or torch.cuda.current_stream()
    ts = []
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        e1.synchronize()
        ts.append(e0.elapsed_time(e1) * 1e-3)
    return statistics.median(ts), min(ts)


def section_conversion_rcm(D, torch, dev, reps):
    """a1 conversion throughput on the natural 128^3 grid; a2 RCM on its
    seeded random symmetric permutation; SpMV after RCM."""
    import workloads as W
    out = {}
    rp, col, val = W.laplace3d_7pt(GRID)
    n, nnz = len(rp) - 1, len(col)
    t_rp, t_col = torch.from_numpy(rp).to(dev), torch.from_numpy(col).to(dev)
    off = torch.empty(nnz, dtype=torch.int16, device=dev)
    D.damn_csr_to_dacsr(t_rp, t_col, n, off_out=off)
    med, mn = _event_time(torch, lambda: D.damn_csr_to_dacsr(t_rp, t_col, n, off_out=off), reps)
    b = (n + 1) * 4 + nnz * (4 + 2)
    out["conversion"] = {"workload": "laplace3d_7pt_128^3_natural", "us": round(med * 1e6, 1),
                         "gbs": round(b / med / 1e9, 1), "bytes": b,
                         "note": "includes the synchronising fit-info read-back"}
    del t_col, off
    rp, col, val = W.laplace3d_7pt(GRID, scrambled=True, rng=W.rng_for(2, 1))
    t_rp, t_col, t_val = (torch.from_numpy(a).to(dev) for a in (rp, col, val))
    _, fi = D.damn_csr_to_dacsr(t_rp, t_col, n)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    perm, rp2, col2, val2, bw = D.damn_rcm_permute(t_rp, t_col, t_val)
    t_rcm = time.perf_counter() - t0
    off2, fi2 = D.damn_csr_to_dacsr(rp2, col2, n, raise_on_nofit=True)
    med_p, _ = _event_time(torch, lambda: D.damn_permute_sym(t_rp, t_col, t_val, perm), reps)
    # SpMV after RCM, NCOPY rotating copies (> L2)
    cp = [(rp2, off2, col2, val2)] + [(rp2.clone(), off2.clone(), col2.clone(), val2.clone())
                                     for _ in range(NCOPY - 1)]
    x = torch.from_numpy(W.uniform_vector(n, W.rng_for(2, 0))).to(dev)
    y = torch.empty(n, dtype=torch.float64, device=dev)
    plans = [D.Plan(c[0], nnz, n, torch.float64, idx=c[1]) for c in cp]
    plans[0].autotune(D.DAMN_FMT_DACSR16, cp[0][1], cp[0][3], x, y)
    for p_ in plans[1:]:
        p_.set_tiling(plans[0].describe()["tiling"])
    it = [0]

    def da():
        c = it[0] % NCOPY
        it[0] += 1
        D.damn_spmv_dacsr16(cp[c][0], cp[c][1], cp[c][3], x, y, plan=plans[c])

    def cs():
        c = it[0] % NCOPY
        it[0] += 1
        D.damn_spmv_csr32(cp[c][0], cp[c][2], cp[c][3], x, y, plan=plans[c])
    for _ in range(8):
        da()
        cs()
    t_da, _ = _event_time(torch, lambda: [da() for _ in range(40)], 5)
    t_cs, _ = _event_time(torch, lambda: [cs() for _ in range(40)], 5)
    t_da, t_cs = t_da / 40, t_cs / 40
    out["rcm"] = {
        "workload": "laplace3d_7pt_128^3_random_symmetric_permutation",
        "fit_rate_scrambled": round(fi.n_fit / nnz, 4), "fits_scrambled": bool(fi.fits),
        "w_scrambled": bw["w_before"], "w_after_rcm": bw["w_after"],
        "fit_rate_after_rcm": round(fi2.n_fit / nnz, 4),
        "rcm_permute_s": round(t_rcm, 3), "permute_sym_ms": round(med_p * 1e3, 3),
        "spmv_after_rcm": {"da16_gbs": round(spmv_bytes(n, nnz, 2, 8, 8) / t_da / 1e9, 1),
                           "csr32_gbs": round(spmv_bytes(n, nnz, 4, 8, 8) / t_cs / 1e9, 1),
                           "da16_us": round(t_da * 1e6, 2), "csr32_us": round(t_cs * 1e6, 2),
                           "speedup_da16_over_csr32": round(t_cs / t_da, 4),
                           "tiling": plans[0].describe()["tiling"]}}
    return out


def section_solvers(D, torch, dev, reps, perturb=False):
    """a5/a6: FP64 CG vs CG-IR (FP32 / BF16 inner values) on the 160^3
    27-point stencil, time to a true relative residual of 1e-10.  With
    perturb, the off-diagonals get a symmetric N(0, 0.01^2) perturbation
    (still SPD), so FP32 / BF16 value quantisation is not exact, and the
    low-precision SpMV error against the FP64 SpMV is reported per dtype."""
    import workloads as W
    m = 160
    rp, col, val = W.stencil27(m)
    n, nnz = len(rp) - 1, len(col)
    if perturb:
        val = W.perturb_symmetric(n, rp, col, val, sigma=0.01)
    t_rp, t_col = torch.from_numpy(rp).to(dev), torch.from_numpy(col).to(dev)
    off, _ = D.damn_csr_to_dacsr(t_rp, t_col, n, raise_on_nofit=True)
    del t_col
    t_val = torch.from_numpy(val).to(dev)
    del rp, col, val
    v32 = D.damn_cast_values(t_val, torch.float32)
    v16 = D.damn_cast_values(t_val, torch.bfloat16)
    xs = torch.from_numpy(W.uniform_vector(n, W.rng_for(4, 1))).to(dev)
    b = torch.empty(n, dtype=torch.float64, device=dev)
    D.damn_spmv_dacsr16(t_rp, off, t_val, xs, b)                 # b = A x*
    p64 = D.Plan(t_rp, nnz, n, torch.float64, idx=off)
    p32 = D.Plan(t_rp, nnz, n, torch.float32, idx=off)
    p16 = D.Plan(t_rp, nnz, n, torch.bfloat16, idx=off)
    y = torch.empty(n, dtype=torch.float64, device=dev)
    p64.autotune(D.DAMN_FMT_DACSR16, off, t_val, xs, y)
    x32, y32 = xs.float(), torch.empty(n, dtype=torch.float32, device=dev)
    p32.autotune(D.DAMN_FMT_DACSR16, off, v32, x32, y32)
    p16.autotune(D.DAMN_FMT_DACSR16, off, v16, x32, y32)
    ws_cg = D._workspace(D._fn("damn_cg_workspace_size")(n), dev)
    ws_ir = D._workspace(D._fn("damn_cg_ir_workspace_size")(n), dev)
    x = torch.zeros(n, dtype=torch.float64, device=dev)
    runs = {
        "cg_f64": lambda: D.damn_cg(t_rp, off, t_val, b, x, 1e-10, 2000, plan=p64, workspace=ws_cg),
        "cg_ir_f32": lambda: D.damn_cg_ir(t_rp, off, t_val, v32, b, x, 1e-10, 1e-3, 200, 60,
                                          plan64=p64, plan_low=p32, workspace=ws_ir),
        "cg_ir_bf16": lambda: D.damn_cg_ir(t_rp, off, t_val, v16, b, x, 1e-10, 1e-2, 200, 60,
                                           plan64=p64, plan_low=p16, workspace=ws_ir),
    }
    out = {"workload": "stencil27_160^3_cg_to_1e-10" + ("_perturbed_0.01" if perturb else ""),
           "n": n, "nnz": nnz}
    for name, pl in (("f64", p64), ("f32", p32), ("bf16", p16)):
        dsc = pl.describe()
        out.setdefault("plans", {})[name] = {"tiling": TILING_NAMES[dsc["tiling"]],
                                             "stages": dsc["stages"],
                                             "x_staging": dsc["x_staging"]}
    # low-precision SpMV error against the FP64 SpMV, per dtype (x = x*)
    y64 = torch.empty(n, dtype=torch.float64, device=dev)
    D.damn_spmv_dacsr16(t_rp, off, t_val, xs, y64, plan=p64)
    for name, vl, pl in (("f32", v32, p32), ("bf16", v16, p16)):
        D.damn_spmv_dacsr16(t_rp, off, vl, x32, y32, plan=pl)
        err = float((y32.double() - y64).abs().max() / y64.abs().max())
        out[f"spmv_{name}_max_rel_err_vs_f64"] = float(f"{err:.3e}")
    stream = torch.cuda.current_stream()
    for name, fn in runs.items():
        ts, res = [], None
        for r in range(reps + 1):
            x.zero_()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            res = fn()
            e1.record(stream)
            e1.synchronize()
            if r > 0:                                            # first run warms up
                ts.append(e0.elapsed_time(e1) * 1e-3)
        err = float(torch.linalg.vector_norm(x - xs) / torch.linalg.vector_norm(xs))
        out[name] = {"ms": round(statistics.median(ts) * 1e3, 2),
                     "ms_min": round(min(ts) * 1e3, 2),
                     "iterations": res["iterations"], "outer": res.get("outer", 0),
                     "converged": bool(res["converged"]),
                     "true_relres": float(f"{res['true_relres']:.3e}"),
                     "rel_err_vs_xstar": float(f"{err:.3e}")}
    for name in ("cg_ir_f32", "cg_ir_bf16"):
        out[name]["speedup_vs_cg_f64"] = round(out["cg_f64"]["ms"] / out[name]["ms"], 3)
    return out


def section_batched(D, torch, dev, reps):
    """a7: 512 independent banded matrices, k in {1, 4, 16}, FP64 / FP32."""
    import workloads as W
    mats_np = W.batch_banded(512)
    out = {"workload": "batch_banded_512", "count": len(mats_np),
           "rows": int(sum(m[0] for m in mats_np)), "nnz": int(sum(len(m[2]) for m in mats_np))}
    base = []
    for n, rp, col, val in mats_np:
        t_rp, t_col = torch.from_numpy(rp).to(dev), torch.from_numpy(col).to(dev)
        off, _ = D.damn_csr_to_dacsr(t_rp, t_col, n, raise_on_nofit=True)
        base.append((n, t_rp, off, torch.from_numpy(val).to(dev)))
    del mats_np
    gen = torch.Generator(device=dev)
    gen.manual_seed(W.seed_for(5, 1))
    stream = torch.cuda.current_stream()
    for dt, s in ((torch.float64, 8), (torch.float32, 4)):
        vals = [v.to(dt) for (_, _, _, v) in base]
        for k in (1, 4, 16):
            mats = []
            for (n, t_rp, off, _), v in zip(base, vals):
                X = torch.rand((n, k), generator=gen, device=dev, dtype=dt) * 2 - 1
                Y = torch.empty((n, k), dtype=dt, device=dev)
                mats.append((t_rp, off, v, X, Y))
            nbytes = sum((m[0].numel()) * 4 + m[1].numel() * (2 + s) + 2 * m[3].numel() * s
                         for m in mats)
            flops = sum(2 * m[1].numel() * k for m in mats)
            plan = D.BatchPlan(mats, k, dt, autotune=True)
            t_b, _ = _event_time(torch, plan.launch, reps)
            t_g, _ = _event_time(torch, plan.graph_launch, reps)

            def per_matrix():
                for (rp_, off_, v_, X_, Y_) in mats:
                    D.damn_spmm_dacsr16(rp_, off_, v_, X_, Y_)
            per_matrix()
            t_e, _ = _event_time(torch, per_matrix, reps)
            g = torch.cuda.CUDAGraph()
            side = torch.cuda.Stream()
            side.wait_stream(stream)
            with torch.cuda.stream(side):
                per_matrix()
            stream.wait_stream(side)
            with torch.cuda.graph(g):
                per_matrix()
            g.replay()
            t_pg, _ = _event_time(torch, g.replay, reps)
            desc = plan.describe()
            key = f"{'f64' if s == 8 else 'f32'}_k{k}"
            out[key] = {"batched_graph_gbs": round(nbytes / t_g / 1e9, 1),
                        "batched_graph_ms": round(t_g * 1e3, 3),
                        "batched_direct_ms": round(t_b * 1e3, 3),
                        "per_matrix_eager_ms": round(t_e * 1e3, 3),
                        "per_matrix_graph_ms": round(t_pg * 1e3, 3),
                        "speedup_vs_per_matrix_graph": round(t_pg / t_g, 3),
                        "gflops": round(flops / t_g / 1e9, 1), "bytes": nbytes,
                        "tuned": {"rows_per_item": desc["tile_items"], "threads": desc["threads"],
                                  "entry_lanes": desc["entry_lanes"],
                                  "streamed": desc["streamed"], "grid": desc["grid"]}}
            plan.close()
            del g, mats, plan
        del vals
    return out


def section_da8(D, torch, dev, reps):
    """DA-CSR-8 vs DA-CSR-16 vs CSR-32 on a matrix whose bandwidth fits int8:
    2-D 5-point Laplacian, 131072 lines of 127 points (w = 127), one copy of
    > 1 GB (larger than L2), FP64 and FP32 values."""
    import workloads as W
    mx, my = 127, 131072
    rp, col, val = W.laplace2d_5pt_rect(mx, my)
    n, nnz = len(rp) - 1, len(col)
    t_rp, t_col = torch.from_numpy(rp).to(dev), torch.from_numpy(col).to(dev)
    del rp, col
    off8, fi8 = D.damn_csr_to_dacsr8(t_rp, t_col, n, raise_on_nofit=True)
    off16, _ = D.damn_csr_to_dacsr(t_rp, t_col, n, raise_on_nofit=True)
    t_val = torch.from_numpy(val).to(dev)
    del val
    gen = torch.Generator(device=dev)
    gen.manual_seed(W.seed_for(3, 8))
    out = {"workload": f"laplace2d_5pt_{mx}x{my}", "n": n, "nnz": nnz, "w": int(fi8.w)}
    for name, dt, vb, xb in (("f64", torch.float64, 8, 8), ("f32", torch.float32, 4, 4)):
        vals = t_val if dt == torch.float64 else D.damn_cast_values(t_val, torch.float32)
        x = torch.rand(n, generator=gen, device=dev, dtype=torch.float64).to(dt) * 2 - 1
        y = torch.empty(n, dtype=dt, device=dev)
        plan = D.Plan(t_rp, nnz, n, dt, idx=off8)
        res = {}
        for fmt, fn, idx, ib in (("da8", D.damn_spmv_dacsr8, off8, 1),
                                 ("da16", D.damn_spmv_dacsr16, off16, 2),
                                 ("csr32", D.damn_spmv_csr32, t_col, 4)):
            for _ in range(3):
                fn(t_rp, idx, vals, x, y, plan=plan)
            t, _ = _event_time(torch, lambda: [fn(t_rp, idx, vals, x, y, plan=plan) for _ in range(10)],
                               max(3, reps // 2))
            t /= 10
            b = spmv_bytes(n, nnz, ib, vb, xb)
            res[fmt] = {"us": round(t * 1e6, 1), "gbs": round(b / t / 1e9, 1), "bytes": b}
        res["speedup_da8_over_da16"] = round(res["da16"]["us"] / res["da8"]["us"], 4)
        res["speedup_da8_over_csr32"] = round(res["csr32"]["us"] / res["da8"]["us"], 4)
        res["model_da8_over_csr32"] = round(res["csr32"]["bytes"] / res["da8"]["bytes"], 4)
        res["tiling"] = plan.describe()["tiling"]
        out[name] = res
        del plan, vals, x, y
    return out


def section_dabsr(D, torch, dev, reps):
    """DA-BSR-16 vs BSR-32: the 3-D 7-point block pattern on a 96^3 grid with
    dense 3 x 3 blocks (3 unknowns per point), FP64 and FP32 values."""
    import workloads as W
    m, b = 96, 3
    nbr, browptr, bcol, bval = W.block_stencil3d(m, b)
    nblk = len(bcol)
    t_bp, t_bc = torch.from_numpy(browptr).to(dev), torch.from_numpy(bcol).to(dev)
    off16, fi = D.damn_csr_to_dacsr(t_bp, t_bc, nbr, raise_on_nofit=True)
    t_val = torch.from_numpy(bval.reshape(-1)).to(dev)
    del bval
    n = nbr * b
    gen = torch.Generator(device=dev)
    gen.manual_seed(W.seed_for(6, 9))
    out = {"workload": f"block_stencil3d_{m}^3_b{b}", "block_rows": nbr, "blocks": nblk,
           "nnz": nblk * b * b, "block_w": int(fi.w)}
    for name, dt, vb in (("f64", torch.float64, 8), ("f32", torch.float32, 4)):
        vals = t_val if dt == torch.float64 else D.damn_cast_values(t_val, torch.float32)
        x = (torch.rand(n, generator=gen, device=dev, dtype=torch.float64) * 2 - 1).to(dt)
        y = torch.empty(n, dtype=dt, device=dev)
        res = {}
        for fmt, fn, idx, ib in (("dabsr16", D.damn_spmv_dabsr16, off16, 2),
                                 ("bsr32", D.damn_spmv_bsr32, t_bc, 4)):
            for _ in range(3):
                fn(t_bp, idx, vals, b, x, y)
            t, _ = _event_time(torch, lambda: [fn(t_bp, idx, vals, b, x, y) for _ in range(10)],
                               max(3, reps // 2))
            t /= 10
            bytes_ = (nbr + 1) * 4 + nblk * (ib + b * b * vb) + 2 * n * vb
            res[fmt] = {"us": round(t * 1e6, 1), "gbs": round(bytes_ / t / 1e9, 1), "bytes": bytes_}
        res["speedup_dabsr16_over_bsr32"] = round(res["bsr32"]["us"] / res["dabsr16"]["us"], 4)
        res["model_speedup"] = round(res["bsr32"]["bytes"] / res["dabsr16"]["bytes"], 4)
        out[name] = res
        del vals, x, y
    return out


def section_dacoo(D, torch, dev, reps):
    """DA-COO-16 vs COO-32 on the 128^3 7-point Laplacian (row vector int32,
    column vector as int16 offsets or int32 columns), FP64 and FP32 values."""
    import workloads as W
    rp, col, val = W.laplace3d_7pt(GRID)
    n, nnz = len(rp) - 1, len(col)
    row = np.repeat(np.arange(n, dtype=np.int32), np.diff(rp))
    t_row, t_col = torch.from_numpy(row).to(dev), torch.from_numpy(col).to(dev)
    t_rp = torch.from_numpy(rp).to(dev)
    off, _ = D.damn_csr_to_dacsr(t_rp, t_col, n, raise_on_nofit=True)
    t_val = torch.from_numpy(val).to(dev)
    out = {"workload": "laplace3d_7pt_128^3_coo", "n": n, "nnz": nnz}
    for name, dt, vb in (("f64", torch.float64, 8), ("f32", torch.float32, 4)):
        vals = t_val if dt == torch.float64 else D.damn_cast_values(t_val, torch.float32)
        x = torch.from_numpy(W.uniform_vector(n, W.rng_for(2, 0))).to(dev).to(dt)
        y = torch.empty(n, dtype=dt, device=dev)
        ws = D._workspace(D._fn("damn_coo_workspace_size")(nnz, D._DTYPE_CODE[dt]), dev)
        res = {}
        for fmt, fn, idx, ib in (("dacoo16", D.damn_spmv_dacoo16, off, 2),
                                 ("coo32", D.damn_spmv_coo32, t_col, 4)):
            for _ in range(3):
                fn(n, t_row, idx, vals, x, y, workspace=ws)
            t, _ = _event_time(torch, lambda: [fn(n, t_row, idx, vals, x, y, workspace=ws)
                                               for _ in range(10)], max(3, reps // 2))
            t /= 10
            b = nnz * (4 + ib + vb) + 2 * n * vb
            res[fmt] = {"us": round(t * 1e6, 1), "gbs": round(b / t / 1e9, 1), "bytes": b}
        res["speedup_dacoo16_over_coo32"] = round(res["coo32"]["us"] / res["dacoo16"]["us"], 4)
        res["model_speedup"] = round(res["coo32"]["bytes"] / res["dacoo16"]["bytes"], 4)
        out[name] = res
        del vals, x, y, ws
    return out


BANDED_POINTS = ((100_000, 100), (100_000, 1000), (100_000, 30000),
                 (1_000_000, 100), (1_000_000, 1000), (1_000_000, 30000),
                 (10_000_000, 1000))
BANDED_POINTS_FULL = tuple((n, h) for n in (100_000, 300_000, 1_000_000, 3_000_000, 10_000_000,
                                            20_000_000) for h in (100, 1000, 30000))
L2_BYTES = 126e6
TILING_NAMES = ("slices", "rows", "rows_long", "band", "lanes4", "lanes8", "lanes16",
                "lanes32", "sorted", "rows_x2")   # DAMN_TILING_* 0 .. 9
BANDED_TILINGS = (0, 2, 3, 8)  # the tilings timed in the banded section
# (tiling, x staging) pairs of the banded section: band also without its ring
BANDED_SHAPES = tuple((t, True) for t in BANDED_TILINGS) + ((3, False),)


def section_banded(D, torch, dev, reps, full=False):
    """Random banded matrices (row lengths LogNormal(ln 12, 0.5), columns
    uniform in [r - h, r + h]), DA-CSR-16 vs CSR-32 FP64 under each of the
    three tilings; the best of each format is reported.  Small matrices are
    replicated and cycled so that every step reads its matrix from HBM; x
    (counted once) may stay in L2."""
    import workloads as W
    peak = measured_peaks()[0]["hbm_gbs"]
    pts = BANDED_POINTS_FULL if full else BANDED_POINTS
    out = {"workload": "random_banded_sweep", "points": []}
    for i, (n, h) in enumerate(pts):
        rp, col, val = W.random_banded(n, h, W.rng_for(3, i))
        nnz = len(col)
        b16, b32 = spmv_bytes(n, nnz, 2, 8, 8), spmv_bytes(n, nnz, 4, 8, 8)
        copies = int(min(16, max(1, -(-3 * L2_BYTES // b16))))
        t_rp = torch.from_numpy(rp).to(dev)
        t_col = torch.from_numpy(col).to(dev)
        t_val = torch.from_numpy(val).to(dev)
        del rp, col, val
        off, fi = D.damn_csr_to_dacsr(t_rp, t_col, n, raise_on_nofit=True)
        mats = [(t_rp, t_col, off, t_val)] + [tuple(t.clone() for t in (t_rp, t_col, off, t_val))
                                             for _ in range(copies - 1)]
        plans = [D.Plan(m[0], nnz, n, torch.float64, idx=m[2]) for m in mats]
        x = torch.from_numpy(W.uniform_vector(n, W.rng_for(3, 100 + i))).to(dev)
        y = torch.empty(n, dtype=torch.float64, device=dev)
        desc = plans[0].describe()
        pt = {"n": n, "h": h, "nnz": nnz, "w": int(fi.w), "copies": copies,
              "heuristic_tiling": TILING_NAMES[desc["tiling"]],
              "row_efficiency": round(desc["row_efficiency"], 3), "max_row": desc["max_row"],
              "tilings": {}}
        for tiling, xstage in BANDED_SHAPES:
            tname = TILING_NAMES[tiling] + ("" if xstage else "_xg")
            for pl in plans:
                pl.set_tiling(tiling)
                pl.set_x_staging(xstage)
            tt = {"x_staged_tiles_frac": round(plans[0].describe()["x_staged_tiles"]
                                               / max(1, plans[0].describe()["ntiles"]), 3)}
            for fmt, fn, k in (("da16", D.damn_spmv_dacsr16, 2), ("csr32", D.damn_spmv_csr32, 1)):
                def step(j):
                    m = mats[j % copies]
                    fn(m[0], m[k], m[3], x, y, plan=plans[j % copies])
                for j in range(3):
                    step(j)
                calls = 10 * copies
                t, _ = _event_time(torch, lambda: [step(j) for j in range(calls)], max(3, reps // 2))
                tt[fmt + "_us"] = round(t / calls * 1e6, 2)
            pt["tilings"][tname] = tt
        best = min(pt["tilings"], key=lambda k: pt["tilings"][k]["da16_us"])
        bc = min(pt["tilings"], key=lambda k: pt["tilings"][k]["csr32_us"])
        pt["best_tiling"] = best
        pt["da16_us"] = pt["tilings"][best]["da16_us"]
        pt["csr32_us"] = pt["tilings"][bc]["csr32_us"]
        pt["da16_gbs"] = round(b16 / pt["da16_us"] / 1e3, 1)
        pt["csr32_gbs"] = round(b32 / pt["csr32_us"] / 1e3, 1)
        pt["da16_frac_hbm"] = round(pt["da16_gbs"] / peak, 3)
        pt["speedup_da16_over_csr32"] = round(pt["csr32_us"] / pt["da16_us"], 4)
        pt["model_speedup"] = round(b32 / b16, 4)
        out["points"].append(pt)
        del mats, plans, x, y, t_rp, t_col, t_val, off
        torch.cuda.empty_cache()
    return out


def section_small(D, torch, dev, reps):
    """Config 1 size (64x64 5-point Laplacian, in L2): time per SpMV under
    graph replay of 1000 calls.  284 KB per SpMV: at any L2 bandwidth of
    several TB/s that is well under 0.1 us, so the time per call is the
    launch / latency floor of one persistent kernel, not a bandwidth."""
    import workloads as W
    rp, col, val = W.laplace2d_5pt(64)
    n, nnz = len(rp) - 1, len(col)
    t_rp, t_col, t_val = (torch.from_numpy(a).to(dev) for a in (rp, col, val))
    off, _ = D.damn_csr_to_dacsr(t_rp, t_col, n, raise_on_nofit=True)
    x = torch.from_numpy(W.uniform_vector(n, W.rng_for(1, 0))).to(dev)
    y = torch.empty(n, dtype=torch.float64, device=dev)
    plan = D.Plan(t_rp, nnz, n, torch.float64, idx=off)
    out = {"workload": "laplace2d_5pt_64^2", "n": n, "nnz": nnz}
    for name, call in (("da16", lambda: D.damn_spmv_dacsr16(t_rp, off, t_val, x, y, plan=plan)),
                       ("csr32", lambda: D.damn_spmv_csr32(t_rp, t_col, t_val, x, y, plan=plan))):
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            call()
        torch.cuda.current_stream().wait_stream(side)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            for _ in range(1000):
                call()
        g.replay()
        t, _ = _event_time(torch, g.replay, reps)
        out[f"{name}_us_per_spmv"] = round(t / 1000 * 1e6, 3)
        # algorithmic bytes per SpMV over its time (the matrix stays in L2)
        b = spmv_bytes(n, nnz, 2 if name == "da16" else 4, 8, 8)
        out[f"{name}_gbs"] = round(b / (t / 1000) / 1e9, 1)
    out["bound"] = "launch / latency: 284 KB per SpMV is under 0.1 us of L2 reads"
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--cpu-budget", type=float, default=10.0)
    ap.add_argument("--sections",
                    default="conversion,solvers,solvers_perturbed,batched,da8,dabsr,dacoo,banded,"
                            "small",
                    help="comma list of secondary sections to run after the headline ('' for none)")
    ap.add_argument("--section-reps", type=int, default=10)
    ap.add_argument("--step-reps", type=int, default=30,
                    help="individually timed steps (event pair each) after the window, >= 30")
    ap.add_argument("--e2e-parts", type=int, default=1,
                    help="parts (streams) each end-to-end upload / download is split into")
    ap.add_argument("--tiling", default="auto", choices=["auto"] + list(TILING_NAMES),
                    help="plan tiling of the headline and mixed-precision plans: autotuned, or fixed")
    ap.add_argument("--case", default=None, type=profile_case,
                    help="run only the launches of one profiled kernel (for ncu), no timing")
    args = ap.parse_args()

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.case:
        run_case(args)
        return

    import torch
    from paper_2307_06305_gb300 import damn as D

    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", init_method="env://")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)

    rp, col, val, x = build_inputs()
    n, nnz = len(rp) - 1, len(col)
    t_rp = [torch.from_numpy(rp).to(dev) for _ in range(NCOPY)]
    t_col = [torch.from_numpy(col).to(dev) for _ in range(NCOPY)]
    t_val = [torch.from_numpy(val).to(dev) for _ in range(NCOPY)]
    t_off = []
    for c in range(NCOPY):
        off, info = D.damn_csr_to_dacsr(t_rp[c], t_col[c], n, raise_on_nofit=True)
        t_off.append(off)
    t_x = torch.from_numpy(x).to(dev)
    y = torch.empty(n, dtype=torch.float64, device=dev)
    plans = [D.Plan(t_rp[c], nnz, n, torch.float64, idx=t_off[c]) for c in range(NCOPY)]
    if args.tiling == "auto":
        plans[0].autotune(D.DAMN_FMT_DACSR16, t_off[0], t_val[0], t_x, y)
        tiling = plans[0].describe()["tiling"]
    else:
        tiling = TILING_NAMES.index(args.tiling)
        plans[0].set_tiling(tiling)
    stages = plans[0].describe()["stages_requested"]
    for c in range(1, NCOPY):
        plans[c].set_tiling(tiling)
        plans[c].set_stages(stages)
    stream = torch.cuda.current_stream()

    def step_da(i):
        c = i % NCOPY
        D.damn_spmv_dacsr16(t_rp[c], t_off[c], t_val[c], t_x, y, plan=plans[c])

    def step_csr(i):
        c = i % NCOPY
        D.damn_spmv_csr32(t_rp[c], t_col[c], t_val[c], t_x, y, plan=plans[c])

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    def timed(fn, steps, warmup):
        for i in range(warmup):
            fn(i)
        barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for i in range(steps):
            fn(i)
        e1.record(stream)
        barrier()
        return max_over_ranks(e0.elapsed_time(e1) * 1e-3, dist, dev)

    def per_step(fn, reps):
        """Each of `reps` steps bracketed by its own event pair on the
        launching stream (median / min / max in us), after the window."""
        ts = []
        for i in range(reps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn(i)
            e1.record(stream)
            ts.append((e0, e1))
        torch.cuda.synchronize()
        us = sorted(a.elapsed_time(b) * 1e3 for a, b in ts)
        return {"reps": reps, "median_us": round(statistics.median(us), 3),
                "min_us": round(us[0], 3), "max_us": round(us[-1], 3)}

    clk = ClockSampler(local).__enter__()  # sampled across every timed phase below
    t_da = timed(step_da, args.steps, args.warmup)
    t_cs = timed(step_csr, args.steps, args.warmup)
    reps = max(30, args.step_reps)
    steps_da = per_step(step_da, reps)
    steps_cs = per_step(step_csr, reps)
    if D.damn_device_status() != 0:
        raise RuntimeError("device status word reports a timed-out wait")

    b_da = spmv_bytes(n, nnz, 2, 8, 8)
    b_cs = spmv_bytes(n, nnz, 4, 8, 8)
    per_step_da = t_da / args.steps
    per_step_cs = t_cs / args.steps
    value = replica_value(world, b_da, per_step_da)

    # reduced-precision values (FP32 / BF16 values, FP32 vectors)
    mixed = {}
    for name, dt, vb in (("f32", torch.float32, 4), ("bf16", torch.bfloat16, 2),
                         ("f8e4m3", torch.float8_e4m3fn, 1)):
        vals = [D.damn_cast_values(t_val[c], dt) for c in range(NCOPY)]
        x32 = t_x.float()
        y32 = torch.empty(n, dtype=torch.float32, device=dev)
        pl = [D.Plan(t_rp[c], nnz, n, dt, idx=t_off[c]) for c in range(NCOPY)]
        if args.tiling == "auto":
            pl[0].autotune(D.DAMN_FMT_DACSR16, t_off[0], vals[0], x32, y32)
        else:  # a pinned tiling also pins these plans (a profiled run stays deterministic)
            pl[0].set_tiling(TILING_NAMES.index(args.tiling))
        dsc = pl[0].describe()
        for c in range(1, NCOPY):
            pl[c].set_tiling(dsc["tiling"])
            pl[c].set_stages(dsc["stages_requested"])

        def step_m(i, vals=vals, pl=pl, x32=x32, y32=y32):
            c = i % NCOPY
            D.damn_spmv_dacsr16(t_rp[c], t_off[c], vals[c], x32, y32, plan=pl[c])
        def step_mc(i, vals=vals, pl=pl, x32=x32, y32=y32):
            c = i % NCOPY
            D.damn_spmv_csr32(t_rp[c], t_col[c], vals[c], x32, y32, plan=pl[c])
        tm = timed(step_m, args.steps, args.warmup) / args.steps
        tc = timed(step_mc, args.steps, args.warmup) / args.steps
        bm = spmv_bytes(n, nnz, 2, vb, 4)
        bc = spmv_bytes(n, nnz, 4, vb, 4)
        mixed[name] = {"gbs": round(bm / tm / 1e9, 1), "us": round(tm * 1e6, 2),
                       "frac_hbm": round(bm / tm / 1e9 / float(measured_peaks()[0]["hbm_gbs"]), 4),
                       "tiling": TILING_NAMES[dsc["tiling"]], "stages": dsc["stages"],
                       "bytes": bm, "csr32_us": round(tc * 1e6, 2),
                       "csr32_gbs": round(bc / tc / 1e9, 1),
                       "speedup_da16_over_csr32": round(tc / tm, 4),
                       "model_speedup": round(bc / bm, 4)}
        del vals, pl

    # end to end through the public API: every step uploads its x from pinned
    # host memory, runs the SpMV and reads its y back.  Steps are pipelined
    # over three streams (upload of step i+1 and download of step i-1 overlap
    # the SpMV of step i), with two x and two y buffers ordered by events.
    hx = [torch.from_numpy(x).pin_memory() for _ in range(2)]
    hy = [torch.empty(n, dtype=torch.float64).pin_memory() for _ in range(2)]
    dx = [torch.empty(n, dtype=torch.float64, device=dev) for _ in range(2)]
    dy = [torch.empty(n, dtype=torch.float64, device=dev) for _ in range(2)]
    # each upload / download is split into NPART parts on their own streams
    # so that several copy engines work on it at once
    NPART = args.e2e_parts
    bounds = [n * q // NPART for q in range(NPART + 1)]
    s_in = [torch.cuda.Stream(device=dev) for _ in range(NPART)]
    s_out = [torch.cuda.Stream(device=dev) for _ in range(NPART)]
    ev_in = [[torch.cuda.Event() for _ in range(NPART)] for _ in range(2)]
    ev_c = [torch.cuda.Event() for _ in range(2)]
    ev_out = [[torch.cuda.Event() for _ in range(NPART)] for _ in range(2)]

    def run_e2e(nsteps):
        for i in range(nsteps):
            b, c = i % 2, i % NCOPY
            for q in range(NPART):
                lo, hi = bounds[q], bounds[q + 1]
                if i >= 2:
                    s_in[q].wait_event(ev_c[b])          # SpMV(i-2) has read dx[b]
                with torch.cuda.stream(s_in[q]):
                    dx[b][lo:hi].copy_(hx[b][lo:hi], non_blocking=True)
                ev_in[b][q].record(s_in[q])
                stream.wait_event(ev_in[b][q])
                if i >= 2:
                    stream.wait_event(ev_out[b][q])      # download(i-2) has read dy[b]
            D.damn_spmv_dacsr16(t_rp[c], t_off[c], t_val[c], dx[b], dy[b], plan=plans[c],
                                stream=stream)
            ev_c[b].record(stream)
            for q in range(NPART):
                lo, hi = bounds[q], bounds[q + 1]
                s_out[q].wait_event(ev_c[b])
                with torch.cuda.stream(s_out[q]):
                    hy[b][lo:hi].copy_(dy[b][lo:hi], non_blocking=True)
                ev_out[b][q].record(s_out[q])
        for q in range(NPART):
            stream.wait_stream(s_in[q])
            stream.wait_stream(s_out[q])

    e2e_steps = max(10, args.steps // 4)
    run_e2e(min(args.warmup, 5))
    barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for q in range(NPART):
        s_in[q].wait_stream(stream)
        s_out[q].wait_stream(stream)
    run_e2e(e2e_steps)
    e1.record(stream)
    barrier()
    t_e2e = max_over_ranks(e0.elapsed_time(e1) * 1e-3 / e2e_steps, dist, dev)
    if not torch.equal(torch.from_numpy(hy[(e2e_steps - 1) % 2].numpy()).to(dev), dy[(e2e_steps - 1) % 2]):
        raise RuntimeError("e2e: downloaded y differs from the device result")
    e2e_value = replica_value(world, b_da, t_e2e)
    # the host link that bounds the end-to-end leg: one pinned copy of the
    # step's x up and of its y down, each alone (best of 5, CUDA events)
    def copy_gbs(dst, src):
        best = 1e30
        for _ in range(5):
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            dst.copy_(src, non_blocking=True)
            b.record(stream)
            b.synchronize()
            best = min(best, a.elapsed_time(b) * 1e-3)
        return src.numel() * src.element_size() / best / 1e9
    h2d_gbs = copy_gbs(dx[0], hx[0])
    d2h_gbs = copy_gbs(hy[0], dy[0])
    clk.__exit__(None, None, None)

    peaks, peak_kind = measured_peaks()
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    achieved = b_da / per_step_da / 1e9
    traffic = recorded_traffic()
    desc = plans[0].describe()

    line = {
        "metric": METRIC, "value": round(value, 2), "unit": "GB/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(per_step_da * 1e3, 5),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": n, "nnz": nnz, "half_bandwidth": GRID * GRID,
                   "l2": f"steps cycle over {NCOPY} matrix copies "
                         f"({NCOPY * b_da / 1e6:.0f} MB > 126 MB L2)",
                   "parallelism": f"replicas{world}",
                   "plan": {k: desc[k] for k in ("tiling", "ntiles", "grid", "stages", "threads",
                                                 "x_staged_tiles")}},
        "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": hbm,
                     "unit": "GB/s", "frac": round(achieved / hbm, 4), "traffic": traffic,
                     "peak_kind": f"{peak_kind} hbm_gbs (copy)",
                     "algorithmic_bytes_per_launch": b_da,
                     "da16_us": round(per_step_da * 1e6, 3),
                     "csr32_us": round(per_step_cs * 1e6, 3),
                     "speedup_da16_over_csr32": round(per_step_cs / per_step_da, 4),
                     "model_speedup": round(b_cs / b_da, 4),
                     "per_step_da16": steps_da, "per_step_csr32": steps_cs,
                     # the second bound of FP64 SpMV on this part: one FMA per entry
                     "fp64": {"achieved_tfma_per_s": round(nnz / per_step_da / 1e12, 4),
                              "peak_tfma_per_s": FP64_TFMA_NOMINAL,
                              "frac": round(nnz / per_step_da / 1e12 / FP64_TFMA_NOMINAL, 4),
                              "peak_kind": "nominal 1.25 TFLOP/s FP64 = 0.625 TFMA/s"}},
        "csr32": {"gbs": round(b_cs / per_step_cs / 1e9, 1), "us": round(per_step_cs * 1e6, 2),
                  "gflops": round((2 * nnz + 2 * n) / per_step_cs / 1e9, 2),
                  "speedup_da16_over_csr32": round(per_step_cs / per_step_da, 4),
                  "model_speedup": round(b_cs / b_da, 4)},
        "da16_us": round(per_step_da * 1e6, 2),
        # Section 4's work W = 2 nnz + 2 n per SpMV, over the same step time
        "gflops": round((2 * nnz + 2 * n) / per_step_da / 1e9, 2),
        "mixed_precision_spmv": mixed,
        "e2e": {"value": round(e2e_value, 2), "unit": "GB/s", "h2d_bytes_per_step": 8 * n,
                "d2h_bytes_per_step": 8 * n, "us_per_step": round(t_e2e * 1e6, 2),
                "pipelined": f"upload / SpMV / download of consecutive steps overlap; each copy "
                             f"split into {args.e2e_parts} parts on their own streams",
                "link_h2d_gbs": round(h2d_gbs, 1), "link_d2h_gbs": round(d2h_gbs, 1),
                "link_bound_us_per_step": round(max(8 * n / h2d_gbs, 8 * n / d2h_gbs) / 1e3, 2)},
        "gpu_launches": args.steps,
        "timing": f"one CUDA-event window over the {args.steps} steps (value, ms_per_step); "
                  f"then {reps} steps each timed by its own event pair (roofline.per_step_*)",
        "clocks": clk.summary(),
    }
    secs = [t for t in args.sections.split(",") if t]
    fns = {"conversion": section_conversion_rcm, "solvers": section_solvers,
           "solvers_perturbed": lambda *a: section_solvers(*a, perturb=True),
           "batched": section_batched, "da8": section_da8, "dabsr": section_dabsr,
           "dacoo": section_dacoo, "banded": section_banded,
           "banded_full": lambda *a: section_banded(*a, full=True),
           "small": section_small}
    for name in secs:
        t0 = time.perf_counter()
        res = fns[name](D, torch, dev, args.section_reps)
        line.setdefault("sections", {}).update(res if name == "conversion" else {name: res})
        line["sections"].setdefault("_seconds", {})[name] = round(time.perf_counter() - t0, 1)
        torch.cuda.empty_cache()
    if D.damn_device_status() != 0:
        raise RuntimeError("device status word reports an error after the sections")
    if rank == 0:
        from oracle import dacsr as OD
        cb = cpu_oracle_baseline(rp, col, OD.translate(n, rp, col).astype(np.int16), val, x,
                                 args.cpu_budget)
        t_cpu, reps, cores = cb["dacsr16"]
        b_csr = spmv_bytes(n, nnz, 4, 8, 8)
        line["cpu_baseline"] = {
            "value": round(b_da / t_cpu / 1e9, 2), "unit": "GB/s", "cores": cores,
            "kind": "oracle",
            "sample": f"{reps} whole DA-CSR-16 SpMVs of the full workload "
                      f"(plain C Listing 2, OpenMP static rows), {t_cpu * reps:.1f} s",
            "dacsr16_1thread": {"gbs": round(b_da / cb["dacsr16_1thread"][0] / 1e9, 2),
                                "us": round(cb["dacsr16_1thread"][0] * 1e6, 1),
                                "reps": cb["dacsr16_1thread"][1], "cores": 1},
            "csr32": {"gbs": round(b_csr / cb["csr32"][0] / 1e9, 2),
                      "us": round(cb["csr32"][0] * 1e6, 1), "reps": cb["csr32"][1],
                      "cores": cores}}
        if args.cpu_budget >= 5:
            s_it, its, n_cg, nnz_cg = cpu_oracle_cg_sample()
            gpu_its = line.get("sections", {}).get("solvers", {}).get("cg_f64", {}).get("iterations")
            cg = {"s_per_iteration": round(s_it, 3), "iterations_timed": its,
                  "sample": f"the oracle's FP64 CG (numpy, Listing 2 order per row) on the "
                            f"160^3 27-point system (n={n_cg}, nnz={nnz_cg}), {its} iterations "
                            f"after the initial residual, timed as one call"}
            if gpu_its:
                cg["projected_s_to_1e-10"] = round(s_it * gpu_its, 1)
                cg["projected_iterations"] = gpu_its
            line["cpu_baseline"]["cg_f64"] = cg
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
