"""Benchmark: arrowhead tile Cholesky + log-determinant + solves on one B300.

Headline (default): the largest configuration, the spatio-temporal INLA-like
precision -- Q_t (x) Q_s with an AR(1) temporal precision (n_t = 100,
rho = 0.9) and the spatial (kappa^2 I + L)^2 of a 45 x 45 5-point grid
(kappa^2 = 1), time-major, plus 20 dense fixed-effect arrow rows/columns
(N(0, 0.1^2), diagonal dominance +1): n = 202,520, one N(0,1) right-hand
side, seed 0.  FP64, tile 16, one level of the adaptable nested dissection.

One step = factorize (value copy, CTSF scatter, persistent factorization
kernel with the forward sweep folded in) + log-determinant + backward sweep,
all through the C ABI.  The symbolic analysis is done once per pattern and
timed separately (the paper excludes preprocessing).  Inputs are larger than
L2 (factor tiles > 1 GB vs 126 MB of L2), so no explicit flush is needed.

value  = tile-level factorization task flops / device time per step [TFLOP/s]
e2e    = the same through host buffers (H2D of values and RHS, D2H of x and
         the log-determinant inside the timed region)

Nested in the same line (``config``), each with its own timing:
  mixed_precision   the same matrix with FP16 updates on the tensor cores and
                    FP64 refinement: step time, refined residual, log-det
                    error against the FP64 step
  batched_sweep     256 matrices of a hyperparameter sweep in one persistent
                    launch (mixed precision, sliced and FP64 arms)
  batched_sweep_8   the same with 8 matrices (chain-bound)
  serving           a Poisson stream (500 req/s) through the continuous-
                    batching loop: solves/s, requests/s, p50/p99 (both arms)
  large_band        the 200,000-row variable band + 100 arrow rows (FP64, T=16)
                    and its tile-size sweep (T = 32 .. 512)
  marginal_variances  diag(A^-1) of the headline matrix by selected inversion

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                       [--workload full|spatiotemporal|large|sweep|serve|servebatch] [--no-nested]
For N > 1 launch with torch.distributed.run; each rank factorizes its own
replica (weak scaling, no collective on the data path).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

# The oracle's CPU baseline runs one process per core, each single-threaded:
# pin BLAS to one thread before numpy loads (the GPU path does not use numpy's
# BLAS).  Spawned workers inherit this.
for _v in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

import numpy as np  # noqa: E402

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2501_02483_b300 import inputs  # noqa: E402

METRIC = "arrowhead Cholesky TFLOP/s, %peak; served solves/s, p50/p99 at set residual"
ST_NAME = ("spatio-temporal Q_t (x) Q_s: AR(1) n_t=100 rho=0.9, (kappa^2 I + L)^2 on a 45x45 grid (kappa^2=1), "
           "time-major, + 20 fixed-effect arrow rows, n=202520, nrhs 1")
LARGE_NAME = "band200000_hw100-500_d0.2_arrow100_nrhs4 (variable band + arrow, n=200100)"

# Source files whose contents decide the FP64 factorization kernel's memory
# traffic; the DRAM bytes measured by an ncu capture stay valid only while
# their digest is the one the capture was taken with.
KERNEL_SOURCES = ("factor_f64.cuh", "device_common.cuh", "plan.h", "analyze.cpp")


def kernel_digest():
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2501_02483_b300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


# DRAM bytes (read + write) per launch of factor_f64_kernel, keyed by (kernel
# digest, workload, tile, block): one capture of a smaller case of the same
# structure, scaled to the full launch by the number of sub-tiles.
TRAFFIC = {("4481f1c3dac5fd48", "spatiotemporal", 16, 16): 1.717e10}  # 20 time steps: 3.246e9 B x 5.289 sub-tiles


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=["full", "spatiotemporal", "large", "sweep", "serve", "servebatch"],
                    default="full",
                    help="full: the spatio-temporal headline with every nested measurement")
    ap.add_argument("--no-nested", action="store_true", help="full: the headline step only")
    ap.add_argument("--tile", type=int, default=16)
    ap.add_argument("--block", type=int, default=0)
    ap.add_argument("--ordering", choices=["none", "rcm", "auto", "nd"], default="nd")
    ap.add_argument("--precision", choices=["f64", "bf16", "f16", "sliced"], default="f64",
                    help="spatiotemporal/large: update precision (bf16/f16 need tile 64, FP64 refinement; "
                         "sliced: FP64-accurate tensor-core updates, tile a multiple of 32)")
    ap.add_argument("--nested-steps", type=int, default=5, help="timed steps of each nested measurement")
    ap.add_argument("--sweep", default="32,64,128,256,512", help="large band: tile sizes timed briefly; '' to skip")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--marginal-variances", action="store_true",
                    help="spatiotemporal/large (FP64): also time diag(A^-1) by selected inversion")
    ap.add_argument("--cpu-workers", type=int, default=0, help="oracle processes (0 = every core of the host)")
    ap.add_argument("--rows", type=int, default=200_000,
                    help="large: body rows (profiling runs only; the benchmarked workload is 200,000)")
    ap.add_argument("--time-steps", type=int, default=100,
                    help="spatiotemporal: AR(1) time steps (profiling runs only; the benchmarked workload is 100)")
    ap.add_argument("--batch", type=int, default=256, help="sweep: matrices per batch")
    ap.add_argument("--lp-tile", type=int, default=64, help="mixed-precision arms: tile")
    ap.add_argument("--lp-precision", choices=["bf16", "f16"], default="f16",
                    help="mixed-precision arms: 16-bit type of the updates")
    ap.add_argument("--f64-tile", type=int, default=16, help="sweep/serve: tile of the FP64 arm")
    ap.add_argument("--requests", type=int, default=1500, help="serve: requests in the stream")
    ap.add_argument("--rate", type=float, default=500.0, help="serve: mean arrivals per second")
    ap.add_argument("--max-batch", type=int, default=256, help="serve: matrices per batched launch")
    ap.add_argument("--gpu-workers", type=int, default=2, help="serve: GPU jobs in flight (one stream each)")
    ap.add_argument("--sweep-ordering", choices=["none", "rcm", "auto", "nd"], default="nd",
                    help="sweep: ordering of every plan (nd halves the chains of the large matrices)")
    ap.add_argument("--serve-ordering", choices=["none", "rcm", "auto", "nd"], default="nd",
                    help="serve: ordering of every plan (nd halves the chains of the large matrices)")
    return ap.parse_args()


def _order(st, name):
    return {"none": st.ORDER_NONE, "rcm": st.ORDER_RCM, "auto": st.ORDER_AUTO, "nd": st.ORDER_ND}[name]


def _prec(st, name):
    return {"f64": st.PREC_F64, "bf16": st.PREC_BF16, "f16": st.PREC_F16, "sliced": st.PREC_SLICED}[name]


def spatiotemporal(time_steps=100, seed=0):
    if time_steps == 100:
        return inputs.config_spatiotemporal(seed)
    return inputs.kronecker_spatiotemporal(time_steps, 0.9, 45, 1.0, 20, 0.1, seed, nrhs=1)


FLOPS_RULE = ("tile-level task flops of Algorithm 1 at tile T (POTRF b(b+1)(2b+1)/6, SYRK kb(b+1), GEMM 2mnk, "
              "TRSM mb^2)")
STEP_RULE = ("factorize + logdet + solve (analysis once per pattern, timed separately); FP64: the forward sweep "
             "inside the factorization launch (stiles_factorize_solve), then the backward sweep; mixed precision: "
             "factorize, then the solve refined in FP64 to residual 1e-10")


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.result = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        self.result = None
        if self.proc is None:
            return False
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        rows = []
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 8:
                rows.append(parts)
        if not rows:
            return False
        sm = [float(r[0]) for r in rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[4 + i].lower() == "active"})
        self.result = {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                       "reasons": reasons, "samples": len(rows)}
        return False


# ---------------------------------------------------------------------------
# CPU baseline: the oracle, as it stands, on bounded samples, one process per core
# ---------------------------------------------------------------------------
def _oracle_job(spec):
    """One oracle factorize + logdet + solve of a bounded sample; returns
    (seconds, tile flops).  Runs in a spawned worker (no CUDA)."""
    from oracle import analyze as oan
    from oracle import cholesky as och
    from oracle import tiles as otiles

    kind, size, T, seed = spec
    if kind == "spatiotemporal":
        m = inputs.kronecker_spatiotemporal(size, 0.9, 45, 1.0, 20, 0.1, seed, nrhs=1)
    else:
        m = inputs.config_large(seed, n_body=size, n_arrow=100, nrhs=4)
    p = oan.analyze(m, T, oan.ORDER_NONE)
    fl = otiles.task_flops(m["n"], T, p["tcolptr"], p["trowidx"])["total"]
    t0 = time.perf_counter()
    L = och.factorize(m, p["perm"], T, p["tcolptr"], p["trowidx"])
    och.logdet(L, p["nt"])
    och.solve(L, p["perm"], T, p["tcolptr"], p["trowidx"], m["rhs"])
    return time.perf_counter() - t0, fl


def _noop(_):
    return os.getpid()


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


class OraclePool:
    """``workers`` spawned processes (spawn: safe after CUDA is initialised),
    each running whole oracle samples single-threaded.  The oracle has no
    parallelism inside one factorization, so the host's cores work on
    independent samples of the workload at once (throughput)."""

    def __init__(self, workers):
        import multiprocessing as mp

        self.workers = workers
        self.pool = mp.get_context("spawn").Pool(workers)
        self.pool.map(_noop, range(4 * workers))  # every worker started and numpy imported

    def run(self, specs):
        t0 = time.perf_counter()
        res = self.pool.map(_oracle_job, specs, chunksize=1)
        return time.perf_counter() - t0, res

    def close(self):
        self.pool.close()
        self.pool.join()


def _sample_spec(workload):
    if workload in ("full", "spatiotemporal"):
        return ("spatiotemporal", 8, 64), "the same Kronecker construction with 8 time steps (16,220 rows), T=64"
    return ("large", 40_000, 16), "the same generator with 40,000 body rows + 100 arrow rows, T=16"


def cpu_baseline(args):
    """The oracle on the host: one sample on one core (threads_1), then one
    sample per core on every core at once (value = total flops / wall time)."""
    (kind, size, T), what = _sample_spec(args.workload)
    s1, fl1 = _oracle_job((kind, size, T, 0))
    cores = args.cpu_workers or host_cores()
    pool = OraclePool(cores)
    wall, res = pool.run([(kind, size, T, i) for i in range(cores)])
    pool.close()
    fl = sum(r[1] for r in res)
    return {"value": fl / wall / 1e12, "unit": "TFLOP/s", "cores": cores, "kind": "oracle",
            "sample": f"{what}, ordering none, FP64 factorize+logdet+solve: {cores} independent samples (seeds "
                      f"0..{cores - 1}) in {cores} single-threaded Python/numpy processes ({wall:.1f} s wall); "
                      f"one process alone {s1:.1f} s",
            "threads_1": {"value": fl1 / s1 / 1e12, "seconds": round(s1, 2), "flops": fl1},
            "host_cores": host_cores()}


def run_reference(args):
    """The oracle as the reference arm: each step is one sample per host core,
    all cores at once."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    (kind, _, T), what = _sample_spec(args.workload)
    size = 4 if kind == "spatiotemporal" else 20_000
    what = what.replace("8 time steps (16,220 rows)", "4 time steps (8,120 rows)").replace("40,000", "20,000")
    cores = args.cpu_workers or host_cores()
    pool = OraclePool(cores)
    walls, fl = [], 0
    for i in range(args.warmup + args.steps):
        wall, res = pool.run([(kind, size, T, c) for c in range(cores)])
        if i >= args.warmup:
            walls.append(wall)
            fl = sum(r[1] for r in res)
    pool.close()
    v = fl / statistics.mean(walls) / 1e12
    sample = (f"{what}, FP64 factorize+logdet+solve: one sample per core on {cores} single-threaded Python/numpy "
              "processes per step")
    cfg = {"workload": ST_NAME if kind == "spatiotemporal" else LARGE_NAME, "tile": T, "ordering": "none",
           "step": STEP_RULE, "flops": FLOPS_RULE, "sample": sample}
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "TFLOP/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(walls),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": cfg,
            "cpu_baseline": {"value": v, "unit": "TFLOP/s", "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# our arm: one matrix
# ---------------------------------------------------------------------------
def _selinv_flops(plan):
    """Useful flops of the selected inverse at the plan's sub-tile size B: per
    sub-column with s sub-rows below the diagonal, s^2 + s operand pairs of
    2 B^3 (Sigma_mj U_jk, Sigma_jk^T U_jk), s products L_jk L_kk^{-1} and one
    L_kk^{-T} L_kk^{-1} of B^3 each."""
    inf = plan.info()
    T, B, n = inf["tile"], inf["block"], inf["n"]
    R = T // B
    nsb = -(-n // B)
    tc, tr = plan.tilemap()
    total = 0
    for K in range(tc.size - 1):
        below_tiles = int(tc[K + 1] - tc[K] - 1)
        for q in range(R):
            jj = K * R + q
            if jj >= nsb:
                break
            s = below_tiles * R + (R - 1 - q)
            total += (s * s + s) * 2 * B ** 3 + (s + 1) * B ** 3
    return total


def _setup_rank():
    import torch

    from paper_2501_02483_b300 import build

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    build.build_library()
    return torch, world, rank, local, dist


def _max_over_ranks(torch, dist, dev, v):
    from paper_2501_02483_b300 import replicas

    return replicas.max_over_ranks(dist, v, dev)


def single_matrix(st, torch, dev, m, *, tile, order, prec, steps, warmup, block=0, e2e=True, dist=None,
                  keep=False):
    """W + K steps of factorize + logdet + solve of one matrix through the C
    ABI (device-resident inputs), then K end-to-end steps through pinned host
    buffers.  Returns the measurements (and the plan/factor when ``keep``)."""
    stream = torch.cuda.current_stream(dev)
    t0 = time.perf_counter()
    plan = st.Plan.from_matrix(m, tile=tile, block=block, ordering=order, precision=prec)
    analyze_s = time.perf_counter() - t0
    info = plan.info()
    flops = info["flops_total"]
    nrhs = m["rhs"].shape[1]
    vals_d = torch.from_numpy(m["values"]).to(dev)
    b_d = torch.from_numpy(np.asfortranarray(m["rhs"])).to(dev)
    f = st.Factor(plan)
    # FP64: the forward sweep runs inside the factorization launch
    # (stiles_factorize_solve); mixed precision: factorize, then the refined solve
    fused = prec == st.PREC_F64 and nrhs <= min(info["block"], 16)
    x_d = torch.empty((nrhs, m["n"]), dtype=torch.float64, device=dev).t()  # n x nrhs, column-major

    def step_device():
        if fused:
            x = f.factorize_solve(vals_d, b_d, x=x_d, stream=stream)
            return f.logdet(), x
        f.factorize(vals_d, stream=stream)
        ld = f.logdet()
        return ld, f.solve(b_d, x=x_d, stream=stream)

    t1 = time.perf_counter()
    step_device()  # first call: uploads the plan's device arrays (and builds the folded graph)
    torch.cuda.synchronize()
    first_call_s = time.perf_counter() - t1
    for _ in range(max(warmup - 1, 0)):
        step_device()
    torch.cuda.synchronize()
    kernel_ms = []
    n0 = st.kernel_launches()
    with ClockSampler(dev.index) as clk:
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            ld, x = step_device()
            kernel_ms.append(f.timing()[1])
        e1.record(stream)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
    launches = st.kernel_launches() - n0
    ms = _max_over_ranks(torch, dist, dev, e0.elapsed_time(e1) / steps)
    out = {"ms_per_step": ms, "flops": flops, "tflops": flops / (ms * 1e-3) / 1e12,
           "kernel_ms": statistics.mean(kernel_ms), "gpu_launches": launches, "clocks": clk.result,
           "analyze_s": round(analyze_s, 3), "first_call_s": round(first_call_s, 3), "logdet": ld,
           "refine_iters": f.refine_iters(), "tile": tile, "block": info["block"], "nnzt": info["nnzt"],
           "ntasks": info["ntasks"], "fused_forward_sweep": fused}
    out["kernel_tflops"] = flops / (out["kernel_ms"] * 1e-3) / 1e12
    if prec == st.PREC_SLICED:
        # tensor work issued: per tile pair (and per diagonal-chain SYRK term) four
        # M = 128, N = 32, K = 32 BF16 MMAs (the 16 slice products)
        nchain = int(np.sum(plan.tasks(0)[:, 0] == 4))
        out["tensor_flops"] = (info["npairs"] + nchain) * 4 * 2 * 128 * 32 * 32
        out["tensor_tflops"] = out["tensor_flops"] / (out["kernel_ms"] * 1e-3) / 1e12

    if e2e:
        # end to end through pinned host buffers: H2D values + RHS, D2H x + logdet
        vals_pin = torch.from_numpy(m["values"]).pin_memory()
        bt = torch.from_numpy(np.ascontiguousarray(m["rhs"].T)).pin_memory()
        xt = torch.empty_like(bt).pin_memory()
        vals_stage = torch.empty_like(vals_d)
        b_stage = torch.empty((nrhs, m["n"]), dtype=torch.float64, device=dev)

        def step_e2e():
            vals_stage.copy_(vals_pin, non_blocking=True)
            b_stage.copy_(bt, non_blocking=True)
            if fused:
                f.factorize_solve(vals_stage, b_stage.t(), x=x_d, stream=stream)
                f.logdet()
            else:
                f.factorize(vals_stage, stream=stream)
                f.logdet()
                f.solve(b_stage.t(), x=x_d, stream=stream)
            xt.copy_(x_d.t())  # synchronous D2H of the solution

        step_e2e()
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        t0 = time.perf_counter()
        for _ in range(steps):
            step_e2e()
        torch.cuda.synchronize()
        e2e_ms = _max_over_ranks(torch, dist, dev, (time.perf_counter() - t0) * 1e3 / steps)
        out["e2e"] = {"ms_per_step": e2e_ms, "h2d_bytes_per_step": int(m["values"].nbytes + bt.numel() * 8),
                      "d2h_bytes_per_step": int(xt.numel() * 8 + 8)}

    # correctness of what was timed
    _, relres = f.solve(b_d, stream=stream, relres=True)
    out["relres"] = relres
    if keep:
        out["_plan"], out["_factor"], out["_vals"] = plan, f, vals_d
    else:
        f.close()
        plan.close()
    return out


def _public(d):
    return {k: v for k, v in d.items() if not k.startswith("_")}


def _fp64_roofline(st, res, peak, workload, fused):
    achieved = res["kernel_tflops"]
    key = (kernel_digest(), workload, res["tile"], res["block"])
    return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "traffic": TRAFFIC.get(key), "kernel_ms": res["kernel_ms"],
            "kernel": f"factor_f64_kernel<{res['block']}>" + (" (forward sweep folded in; achieved counts the "
                                                              "factorization's flops only)" if fused else ""),
            "kernel_digest": key[0],
            "peak_source": "FP64 DFMA probe of libstiles.so measured in this run (MEASURED_PEAKS.json has no "
                           "FP64 entry)"}


def _tensor_peak():
    """The sustained bf16 tensor peak of MEASURED_PEAKS.json (f16 runs at the same rate)."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            v = json.load(fh).get("bf16_tflops_sustained")
        if v:
            return float(v), "MEASURED_PEAKS.json bf16_tflops_sustained (of measured; f16 has the same nominal rate)"
    except OSError:
        pass
    return 1400.0, "fallback sustained bf16 (of fallback)"


def marginal_variances(st, torch, dev, kept, peak):
    """diag(A^{-1}) by selected inversion on a kept FP64 factor: the first call
    builds and uploads its task graph; a new factorization invalidates Sigma,
    so the timed call recomputes all of it."""
    stream = torch.cuda.current_stream(dev)
    plan, f, vals = kept["_plan"], kept["_factor"], kept["_vals"]
    t0 = time.perf_counter()
    f.marginal_variances(stream=stream)
    first = time.perf_counter() - t0
    f.factorize(vals, stream=stream)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    var = f.marginal_variances(stream=stream)
    ms = (time.perf_counter() - t0) * 1e3
    sfl = _selinv_flops(plan)
    return {"ms": round(ms, 2), "first_call_s": round(first, 2), "flops": sfl, "tflops": round(sfl / ms / 1e9, 4),
            "frac_of_fp64_peak": round(sfl / ms / 1e9 / peak, 4), "min_variance": float(var.min()),
            "max_variance": float(var.max()),
            "flops_rule": "2 B^3 per operand pair, B^3 per L_jk L_kk^{-1} and per L_kk^{-T} L_kk^{-1}"}


def tile_sweep(st, torch, dev, m, tiles, order, prec):
    """Kernel time of two factorizations after one warm-up per tile size."""
    vals_d = torch.from_numpy(m["values"]).to(dev)
    out = {}
    for T in tiles:
        if prec != st.PREC_F64 and T % 64:
            continue
        pl = st.Plan.from_matrix(m, tile=T, ordering=order, precision=prec)
        ff = st.Factor(pl)
        ff.factorize(vals_d)
        ks = []
        for _ in range(2):
            ff.factorize(vals_d)
            ks.append(ff.timing()[1])
        fl = pl.info()["flops_total"]
        out[str(T)] = {"kernel_ms": round(min(ks), 3), "tflops": round(fl / min(ks) / 1e9, 4), "flops": fl,
                       "block": pl.info()["block"]}
        ff.close()
        pl.close()
    return out


def run_single(args):
    """One matrix: the headline (spatio-temporal, FP64) with every nested
    measurement (--workload full), or one workload alone."""
    torch, world, rank, local, dist = _setup_rank()
    from paper_2501_02483_b300 import stiles as st

    dev = torch.device("cuda", local)
    order = _order(st, args.ordering)
    prec = _prec(st, args.precision)
    if args.workload == "large":
        m, name = inputs.config_large(rank, n_body=args.rows), LARGE_NAME
        if args.rows != 200_000:
            name = name.replace("band200000", f"band{args.rows}")
    else:
        m, name = spatiotemporal(args.time_steps, seed=rank), ST_NAME
        if args.time_steps != 100:
            name = name.replace("n_t=100", f"n_t={args.time_steps}")
    wl = "spatiotemporal" if args.workload in ("full", "spatiotemporal") else "large"
    peak = st.probe_fp64_peak()
    nested = args.workload == "full" and not args.no_nested and world == 1
    keep = (nested or args.marginal_variances) and prec == st.PREC_F64
    res = single_matrix(st, torch, dev, m, tile=args.tile, block=args.block, order=order, prec=prec,
                        steps=args.steps, warmup=args.warmup, dist=dist, keep=keep)
    value = world * res["flops"] / (res["ms_per_step"] * 1e-3) / 1e12
    e2e = {"value": world * res["flops"] / (res["e2e"]["ms_per_step"] * 1e-3) / 1e12, "unit": "TFLOP/s",
           **res["e2e"]}
    if prec == st.PREC_F64:
        roof = _fp64_roofline(st, res, peak, wl, res["fused_forward_sweep"])
    elif prec == st.PREC_SLICED:
        tpeak, src = _tensor_peak()
        roof = {"bound": "tensor", "achieved": res["tensor_tflops"], "peak": tpeak, "unit": "TFLOP/s",
                "frac": res["tensor_tflops"] / tpeak, "traffic": None, "kernel": "factor_oz_kernel",
                "kernel_ms": res["kernel_ms"], "peak_source": src,
                "achieved_fp64_equivalent": res["kernel_tflops"],
                "note": "achieved counts the BF16 slice products issued (16 per tile pair); the FP64-equivalent "
                        "rate counts Algorithm 1's tile flops"}
    else:
        tpeak, src = _tensor_peak()
        roof = {"bound": "tensor", "achieved": res["kernel_tflops"], "peak": tpeak, "unit": "TFLOP/s",
                "frac": res["kernel_tflops"] / tpeak, "traffic": None, "kernel": "factor_lp_kernel",
                "kernel_ms": res["kernel_ms"], "peak_source": src}
    cfg = {"workload": f"{name} ({args.precision})", "n": m["n"], "n_arrow": m["n_arrow"],
           "nrhs": int(m["rhs"].shape[1]), "tile": args.tile, "ordering": args.ordering,
           "l2": "inputs larger than L2 (factor tiles > 1 GB vs 126 MB L2); no flush", "step": STEP_RULE,
           "flops": FLOPS_RULE, "block": res["block"], "nnzt": res["nnzt"], "ntasks": res["ntasks"],
           "flops_factor": res["flops"], "analyze_s": res["analyze_s"], "first_call_s": res["first_call_s"],
           "logdet": res["logdet"], "relres": res["relres"], "refine_iters": res["refine_iters"],
           "percent_of_fp64_peak": round(100 * value / world / peak, 2), "fp64_peak_tflops": peak}
    line = {"metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": res["ms_per_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": args.precision, "data": "synthetic", "config": cfg, "roofline": roof,
            "e2e": e2e, "gpu_launches": res["gpu_launches"], "clocks": res["clocks"]}

    if keep:
        cfg["marginal_variances"] = marginal_variances(st, torch, dev, res, peak)
        res["_factor"].close()
        res["_plan"].close()
    if nested:
        K, W = args.nested_steps, 2
        # the same matrix with 16-bit updates on the tensor cores + FP64 refinement
        lp = single_matrix(st, torch, dev, m, tile=args.lp_tile, order=order, prec=_prec(st, args.lp_precision),
                           steps=K, warmup=W, e2e=False)
        tpeak, src = _tensor_peak()
        lp.update({"precision": args.lp_precision, "steps": K, "warmup": W,
                   "logdet_rel_err_vs_fp64": abs(lp["logdet"] - res["logdet"]) / abs(res["logdet"]),
                   "speedup_vs_fp64_step": res["ms_per_step"] / lp["ms_per_step"],
                   "tensor_frac": lp["kernel_tflops"] / tpeak, "tensor_peak_source": src})
        cfg["mixed_precision"] = lp
        # the same matrix with FP64-accurate updates from BF16 digit slices on the tensor cores
        sl = single_matrix(st, torch, dev, m, tile=32, order=order, prec=st.PREC_SLICED, steps=K, warmup=W,
                           e2e=False)
        sl.update({"precision": "sliced", "steps": K, "warmup": W,
                   "logdet_rel_err_vs_fp64": abs(sl["logdet"] - res["logdet"]) / abs(res["logdet"]),
                   "speedup_vs_fp64_step": res["ms_per_step"] / sl["ms_per_step"],
                   "kernel_frac_of_fp64_peak": sl["kernel_tflops"] / peak,
                   "tensor_frac": sl["tensor_tflops"] / tpeak, "tensor_peak_source": src})
        cfg["sliced_fp64_accurate"] = sl
        cfg["batched_sweep"] = sweep_measure(args, st, torch, dev, None, steps=K, warmup=W)
        # a small batch of the same generator: chain-bound, each arm's step is the dependency
        # chain of its largest matrix
        a8 = argparse.Namespace(**vars(args))
        a8.batch = 8
        cfg["batched_sweep_8"] = sweep_measure(a8, st, torch, dev, None, steps=K, warmup=W)
        cfg["serving"] = serve_measure(args, st, torch, dev, seed=0)
        # the large variable band: FP64 step at T = 16 and the tile-size sweep
        ml = inputs.config_large(0)
        lg = single_matrix(st, torch, dev, ml, tile=16, order=order, prec=st.PREC_F64, steps=K, warmup=W,
                           e2e=False)
        lg.update({"workload": LARGE_NAME, "steps": K, "warmup": W,
                   "kernel_frac_of_fp64_peak": lg["kernel_tflops"] / peak,
                   "tile_sweep": tile_sweep(st, torch, dev, ml, [int(t) for t in args.sweep.split(",") if t],
                                            order, st.PREC_F64) if args.sweep else {}})
        cfg["large_band"] = lg
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args)
    if rank == 0:
        print(json.dumps(line, default=_jsonable), flush=True)
    if dist:
        dist.destroy_process_group()


def _jsonable(o):
    if isinstance(o, np.generic):
        return o.item()
    raise TypeError(type(o))


# ---------------------------------------------------------------------------
# batched sweep and serving workloads
# ---------------------------------------------------------------------------
def _sweep_arm(st, torch, mats, prec, T, dev, dist, steps, warmup, order):
    """One precision arm of the batched sweep: analysis, then W + K steps of
    batched factorize + logdets + batched solve."""
    stream = torch.cuda.current_stream(dev)
    t0 = time.perf_counter()
    plans = [st.Plan.from_matrix(m, tile=T, ordering=order, precision=prec) for m in mats]
    analyze_s = time.perf_counter() - t0
    infos = [p.info() for p in plans]
    flops = sum(i["flops_total"] for i in infos)
    batch = st.Batch(plans)
    vals_d = [torch.from_numpy(m["values"]).to(dev) for m in mats]
    rhs_d = [torch.from_numpy(np.asfortranarray(m["rhs"])).to(dev) for m in mats]
    nsolve = sum(m["rhs"].shape[1] for m in mats)

    def step(vals, rhs):
        statuses, _ = batch.factorize(vals, stream=stream)
        lds = batch.logdets(stream=stream)
        xs, rel, its, status = batch.solve(rhs, stream=stream, raise_on_error=False)
        return statuses, lds, rel, its, batch.timing()

    for _ in range(warmup):
        step(vals_d, rhs_d)
    torch.cuda.synchronize()
    n0 = st.kernel_launches()
    kms = []
    with ClockSampler(dev.index) as clk:
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            statuses, lds, rel, its, km = step(vals_d, rhs_d)
            kms.append(km)
        e1.record(stream)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
    launches = st.kernel_launches() - n0
    ms = _max_over_ranks(torch, dist, dev, e0.elapsed_time(e1) / steps)
    ok = int(np.sum((statuses == 0) & (rel <= 1e-10)))
    # end to end from pinned host buffers: H2D values + right-hand sides, D2H solutions + logdets
    vals_h = [torch.from_numpy(m["values"]).pin_memory().numpy() for m in mats]
    rhs_h = [torch.from_numpy(np.asfortranarray(m["rhs"])).pin_memory().numpy() for m in mats]
    step(vals_h, rhs_h)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        step(vals_h, rhs_h)
    torch.cuda.synchronize()
    e2e_ms = _max_over_ranks(torch, dist, dev, (time.perf_counter() - t0) * 1e3 / steps)
    out = {"tile": T, "block": infos[0]["block"], "ms_per_step": ms, "tflops": flops / (ms * 1e-3) / 1e12,
           "matrices_per_s": len(mats) / (ms * 1e-3), "solves_per_s": ok * (nsolve / len(mats)) / (ms * 1e-3),
           "solved_at_1e-10": ok, "max_relres": float(np.max(rel)), "max_refine_iters": int(np.max(its)),
           "kernel_ms": statistics.mean(kms), "flops": flops, "analyze_s": round(analyze_s, 2),
           "gpu_launches": launches, "clocks": clk.result,
           "e2e_ms": e2e_ms, "e2e_h2d": int(sum(v.nbytes for v in vals_h) + sum(r.nbytes for r in rhs_h)),
           "e2e_d2h": int(sum(r.nbytes for r in rhs_h) + 8 * len(mats)), "logdets": lds}
    batch.close()
    for p in plans:
        p.close()
    return out


def sweep_measure(args, st, torch, dev, dist, steps, warmup, seed=0):
    """Both arms of the batched sweep on the same matrices."""
    mats = inputs.batch_sweep(args.batch, seed=seed)
    prec = _prec(st, args.lp_precision)
    order = _order(st, args.sweep_ordering)
    lp = _sweep_arm(st, torch, mats, prec, args.lp_tile, dev, dist, steps, warmup, order)
    sl = _sweep_arm(st, torch, mats, st.PREC_SLICED, 32, dev, dist, steps, warmup, order)
    f64 = _sweep_arm(st, torch, mats, st.PREC_F64, args.f64_tile, dev, dist, steps, warmup, order)
    ld_err = float(np.max(np.abs(lp["logdets"] - f64["logdets"]) / np.abs(f64["logdets"])))
    sl["logdet_rel_diff_vs_fp64"] = float(np.max(np.abs(sl["logdets"] - f64["logdets"]) / np.abs(f64["logdets"])))
    sl["solves_per_s_over_fp64"] = sl["solves_per_s"] / max(f64["solves_per_s"], 1e-30)
    for a in (lp, sl, f64):
        a.pop("logdets")
    peak, peak_src = _tensor_peak()
    lp["tensor_frac"] = lp["flops"] / (lp["kernel_ms"] * 1e-3) / 1e12 / peak
    return {"workload": f"batched sweep: {args.batch} matrices, n log-uniform [5000, 50000], hw {{64,128,256}}, "
                        "arrow 0..50, theta ~ U(0.5, 2), 1 RHS each; refined to 1e-10",
            "step": "batched factorize (one persistent launch) + all logdets + batched solve with FP64 "
                    "refinement (analysis once per pattern, timed separately)",
            "ordering": args.sweep_ordering,
            "steps": steps, "warmup": warmup, "precision": args.lp_precision,
            "mixed_precision": lp, "sliced_fp64_accurate": sl, "fp64": f64, "logdet_rel_diff_lp_vs_fp64": ld_err,
            "solves_per_s_lp_over_fp64": lp["solves_per_s"] / max(f64["solves_per_s"], 1e-30),
            "tensor_peak_source": peak_src}


def run_sweep(args):
    torch, world, rank, local, dist = _setup_rank()
    from paper_2501_02483_b300 import stiles as st

    dev = torch.device("cuda", local)
    res = sweep_measure(args, st, torch, dev, dist, args.steps, args.warmup, seed=rank)
    lp = res["mixed_precision"]
    peak, peak_src = _tensor_peak()
    achieved = lp["flops"] / (lp["kernel_ms"] * 1e-3) / 1e12
    line = {
        "metric": METRIC, "value": world * lp["tflops"], "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": lp["ms_per_step"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": args.lp_precision, "data": "synthetic",
        "config": dict(res, l2="inputs larger than L2 (factor tiles of the batch > 1 GB); no flush"),
        "roofline": {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": None, "kernel": "factor_lp_kernel (batched)",
                     "kernel_ms": lp["kernel_ms"], "peak_source": peak_src},
        "e2e": {"value": world * lp["flops"] / (lp["e2e_ms"] * 1e-3) / 1e12, "unit": "TFLOP/s",
                "h2d_bytes_per_step": lp["e2e_h2d"], "d2h_bytes_per_step": lp["e2e_d2h"],
                "ms_per_step": lp["e2e_ms"]},
        "gpu_launches": lp["gpu_launches"], "clocks": lp["clocks"],
    }
    if rank == 0:
        print(json.dumps(line, default=_jsonable), flush=True)
    if dist:
        dist.destroy_process_group()


def _pin_requests(torch, reqs):
    """Client-side buffers in page-locked host memory (as a server receiving
    requests would hold them): values arrays shared between requests stay
    shared; right-hand sides keep their column-major layout."""
    pinned = {}
    for r in reqs:
        if r["matrix"] is not None:
            v = r["matrix"]["values"]
            if id(v) not in pinned:
                pinned[id(v)] = (v, torch.from_numpy(v).pin_memory().numpy())
            r["matrix"] = dict(r["matrix"], values=pinned[id(v)][1])
        r["rhs"] = torch.from_numpy(np.ascontiguousarray(r["rhs"].T)).pin_memory().numpy().T


def _serve_arm(args, st, sv, torch, work, prec, T, stream):
    reqs, arrivals = work
    # warm-up on a throw-away server: a few requests of another stream load the kernels
    order = _order(st, args.serve_ordering)
    warm = sv.Server(precision=prec, tile=T, ordering=order, max_batch=args.max_batch, hbm_budget=150e9,
                     gpu_workers=args.gpu_workers)
    wr, wa = inputs.serving_workload(12, rate=args.rate, seed=99, n_hi=20_000, pool=4)
    warm.run([sv.Request(r["id"], r["kind"], r["key"], r["matrix"], r["rhs"], r["target"]) for r in wr], wa,
             stream=stream, realtime=False)
    warm.close()
    srv = sv.Server(precision=prec, tile=T, ordering=order, max_batch=args.max_batch, hbm_budget=150e9,
                    gpu_workers=args.gpu_workers)
    objs = [sv.Request(r["id"], r["kind"], r["key"], r["matrix"], r["rhs"], r["target"]) for r in reqs]
    n0 = st.kernel_launches()
    with ClockSampler(stream.device.index) as clk:
        done = srv.run(objs, arrivals, stream=stream, realtime=True)
        torch.cuda.synchronize()
    launches = st.kernel_launches() - n0
    lat = np.array([(r.t_done - r.t_arrival) * 1e3 for r in done])
    ok = [r for r in done if r.status == 0 and r.relres is not None and r.relres <= 1e-10]
    cols = sum(r.rhs.shape[1] for r in ok)
    out = {"tile": T, "wall_s": srv.wall, "solves_per_s": cols / srv.wall, "requests_per_s": len(done) / srv.wall,
           "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
           "mean_batch": float(np.mean([r.batch_size for r in done if r.batch_size])),
           "requests_at_1e-10": len(ok), "requests": len(done), "stats": dict(srv.stats),
           "seconds_by_phase": {k: round(v, 3) for k, v in srv.times.items()},
           "gpu_launches": launches, "clocks": clk.result}
    both, busy, peak = srv.overlap()
    kboth, kbusy, kpeak = srv.overlap(kernels=True)
    out["device_overlap"] = {"jobs_ms_two_or_more": round(both, 1), "jobs_ms_busy": round(busy, 1),
                             "jobs_peak_in_flight": peak, "factor_kernels_ms_two_or_more": round(kboth, 1),
                             "factor_kernels_ms_busy": round(kbusy, 1), "factor_kernels_peak": kpeak,
                             "how": "CUDA events per GPU job on its stream and around each batched persistent "
                                    "factorization kernel, on one device clock"}
    srv.close()
    return out


def serve_measure(args, st, torch, dev, seed=0):
    from paper_2501_02483_b300 import serve as sv

    stream = torch.cuda.current_stream(dev)
    work = inputs.serving_workload(args.requests, rate=args.rate, seed=seed, variants=2)
    _pin_requests(torch, work[0])
    lp = _serve_arm(args, st, sv, torch, work, _prec(st, args.lp_precision), args.lp_tile, stream)
    sl = _serve_arm(args, st, sv, torch, work, st.PREC_SLICED, 32, stream)
    sl["solves_per_s_over_fp64"] = None
    f64 = _serve_arm(args, st, sv, torch, work, st.PREC_F64, args.f64_tile, stream)
    sl["solves_per_s_over_fp64"] = sl["solves_per_s"] / max(f64["solves_per_s"], 1e-30)
    return {"workload": f"serving: Poisson {args.rate:g} req/s, {args.requests} requests, n log-uniform "
                        "[1000, 200000], hw 32..512, arrow 0..100, nrhs 1..16, 30% re-solves, HBM budget 150 GB; "
                        "48 patterns x 2 value scales (theta in {0.875, 1.625}); client buffers in pinned host "
                        "memory; ordering " + args.serve_ordering,
            "step": "the whole request stream through the continuous-batching loop (arrivals in real time)",
            "precision": args.lp_precision, "mixed_precision": lp, "sliced_fp64_accurate": sl, "fp64": f64,
            "solves_per_s_lp_over_fp64": lp["solves_per_s"] / max(f64["solves_per_s"], 1e-30)}


def run_serve(args):
    torch, world, rank, local, dist = _setup_rank()
    from paper_2501_02483_b300 import stiles as st

    dev = torch.device("cuda", local)
    res = serve_measure(args, st, torch, dev, seed=rank)
    lp = res["mixed_precision"]
    value = -_max_over_ranks(torch, dist, dev, -lp["solves_per_s"])
    line = {
        "metric": METRIC, "value": value * world, "unit": "solves/s", "n_gpus": world, "steps": 1,
        "warmup": 1, "ms_per_step": 1e3 * lp["wall_s"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": args.lp_precision, "data": "synthetic", "config": res,
        "e2e": {"value": value * world, "unit": "solves/s", "h2d_bytes_per_step": None,
                "d2h_bytes_per_step": None,
                "note": "requests enter as host arrays; every value and right-hand side crosses H2D"},
        "gpu_launches": lp["gpu_launches"], "clocks": lp["clocks"],
    }
    if rank == 0:
        print(json.dumps(line, default=_jsonable), flush=True)
    if dist:
        dist.destroy_process_group()


def run_servebatch(args):
    """The batched refined solve of serving requests, for profiling the solve
    phase of a served job: the first --batch new requests of the serving
    generator (n up to 200,000, 1..16 right-hand sides each; the mixed-precision
    arm's precision and tile), factorized once; then W + K timed batched solves
    with FP64 refinement to 1e-10 (device-resident right-hand sides)."""
    torch, world, rank, local, dist = _setup_rank()
    from paper_2501_02483_b300 import stiles as st

    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    reqs, _ = inputs.serving_workload(int(args.batch * 1.6) + 16, rate=args.rate, seed=rank, variants=2)
    new = [r for r in reqs if r["kind"] == "new"][:args.batch]
    prec = _prec(st, args.lp_precision)
    t0 = time.perf_counter()
    plans = [st.Plan.from_matrix(r["matrix"], tile=args.lp_tile, ordering=_order(st, args.serve_ordering),
                                 precision=prec) for r in new]
    analyze_s = time.perf_counter() - t0
    batch = st.Batch(plans)
    statuses, _ = batch.factorize([torch.from_numpy(r["matrix"]["values"]).to(dev) for r in new], stream=stream)
    rhs = [torch.from_numpy(np.asfortranarray(r["rhs"])).to(dev) for r in new]
    ncol = sum(r["rhs"].shape[1] for r in new)
    for _ in range(args.warmup):
        batch.solve(rhs, stream=stream, raise_on_error=False)
    torch.cuda.synchronize()
    n0 = st.kernel_launches()
    with ClockSampler(dev.index) as clk:
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            xs, rel, its, status = batch.solve(rhs, stream=stream, raise_on_error=False)
        e1.record(stream)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
    launches = st.kernel_launches() - n0
    ms = _max_over_ranks(torch, dist, dev, e0.elapsed_time(e1) / args.steps)
    ok = int(np.sum((statuses == 0) & (rel <= 1e-10)))
    line = {
        "metric": METRIC, "value": world * ncol / (ms * 1e-3), "unit": "solves/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": args.lp_precision, "data": "synthetic",
        "config": {"workload": f"served batch solve: the first {len(new)} new requests of the serving generator "
                               "(n log-uniform [1000, 200000], hw 32..512, arrow 0..100, nrhs 1..16), "
                               f"{args.lp_precision} factors at T = {args.lp_tile}, ordering {args.serve_ordering}",
                   "step": "one batched solve of every request's right-hand sides, refined in FP64 to 1e-10",
                   "matrices": len(new), "columns": ncol, "n_max": max(r["matrix"]["n"] for r in new),
                   "solved_at_1e-10": ok, "max_relres": float(np.max(rel)), "max_refine_iters": int(np.max(its)),
                   "status": status, "analyze_s": round(analyze_s, 2),
                   "l2": "inputs larger than L2 (factors of the batch > 10 GB); no flush"},
        "roofline": None, "e2e": None, "gpu_launches": launches, "clocks": clk.result,
    }
    if rank == 0:
        print(json.dumps(line, default=_jsonable), flush=True)
    if dist:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "sweep":
        run_sweep(args)
    elif args.workload == "serve":
        run_serve(args)
    elif args.workload == "servebatch":
        run_servebatch(args)
    else:
        run_single(args)


if __name__ == "__main__":
    main()
