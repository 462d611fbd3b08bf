"""Benchmark: FP64 arrowhead tile Cholesky + log-determinant + solve on one B300.

Workload (default): the large single matrix -- a 200,000-row band whose lower
half-width is drawn uniformly from 100..500 per 2,000-row segment (in-band
density 0.2, U(-1,1)), plus 100 dense N(0,1) arrow rows, diagonal = row |sum|
+ 1, four N(0,1) right-hand sides, seed 0.  Synthetic data of the paper's
spatial/INLA arrowhead shape.

One step = factorize (value copy, CTSF scatter, persistent factorization
kernel) + log-determinant + 4-RHS solve, all through the C ABI.  The
symbolic analysis is done once per pattern and timed separately (the paper
excludes preprocessing).  Inputs are larger than L2 (values 0.26 GB, factor
tiles >= 0.7 GB vs 126 MB of L2), so no explicit flush is needed.

value  = tile-level factorization task flops / device time per step [TFLOP/s]
e2e    = the same through host buffers (H2D of values and RHS, D2H of x and
         the log-determinant inside the timed region)

Other workloads (--workload):
  sweep  256 matrices of a hyperparameter sweep (n log-uniform in [5,000,
         50,000], half-width in {64,128,256}, arrow 0..50, values scaled by
         theta ~ U(0.5, 2)); one step = batched factorization in one persistent
         launch + all log-determinants + batched solves refined to residual
         1e-10; mixed precision (BF16 updates) timed beside FP64.
  serve  Poisson request stream (500 req/s) of factorize+logdet+solve and
         re-solve requests through the continuous-batching loop; p50/p99
         latency and solves/s at residual 1e-10, BF16 beside FP64.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                       [--workload large|sweep|serve]
For N > 1 launch with torch.distributed.run; each rank factorizes its own
replica (weak scaling, no collective on the data path).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

# The oracle's CPU baseline runs single-threaded: pin BLAS to one thread
# before numpy loads (the GPU path does not use numpy's BLAS).
for _v in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

import numpy as np  # noqa: E402

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2501_02483_b300 import inputs  # noqa: E402

METRIC = "arrowhead Cholesky TFLOP/s, %peak; served solves/s, p50/p99 at set residual"

# DRAM bytes per launch of the factorization kernel, from an ncu capture (see
# profiles/); keyed by (kernel build tag, tile, block).  None when the kernel
# changed after the capture.
TRAFFIC = {("factor_f64_v9_fwd", "large", 16, 16): 1.415e9}  # profiles/factor_f64_b16_band50000.md, scaled by tiles
KERNEL_TAG = "factor_f64_v9_fwd"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--tile", type=int, default=16)
    ap.add_argument("--block", type=int, default=0)
    ap.add_argument("--ordering", choices=["none", "rcm", "auto", "nd"], default="nd")
    ap.add_argument("--sweep", default="32,64,128,256,512", help="tile sizes timed briefly; '' to skip")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-largest", action="store_true", help="large: skip the largest-configuration FP64 line")
    ap.add_argument("--cpu-sample-rows", type=int, default=60_000)
    ap.add_argument("--rows", type=int, default=200_000,
                    help="body rows (profiling runs only; the benchmarked workload is 200,000)")
    ap.add_argument("--workload", choices=["large", "spatiotemporal", "sweep", "serve"], default="large")
    ap.add_argument("--precision", choices=["f64", "bf16", "f16"], default="f64",
                    help="large/spatiotemporal: update precision (bf16/f16 need tile 64; FP64 refinement)")
    ap.add_argument("--batch", type=int, default=256, help="sweep: matrices per batch")
    ap.add_argument("--lp-tile", type=int, default=64, help="sweep/serve: tile of the mixed-precision arm")
    ap.add_argument("--lp-precision", choices=["bf16", "f16"], default="f16",
                    help="sweep/serve: 16-bit type of the mixed-precision updates")
    ap.add_argument("--f64-tile", type=int, default=16, help="sweep/serve: tile of the FP64 arm")
    ap.add_argument("--requests", type=int, default=1500, help="serve: requests in the stream")
    ap.add_argument("--rate", type=float, default=500.0, help="serve: mean arrivals per second")
    ap.add_argument("--max-batch", type=int, default=256, help="serve: matrices per batched launch")
    ap.add_argument("--gpu-workers", type=int, default=2, help="serve: GPU jobs in flight (one stream each)")
    ap.add_argument("--serve-ordering", choices=["none", "rcm", "auto", "nd"], default="nd",
                    help="serve: ordering of every plan (nd halves the chains of the large matrices)")
    return ap.parse_args()


def workload(args, seed=0):
    if args.workload == "spatiotemporal":
        return inputs.config_spatiotemporal(seed)
    return inputs.config_large(seed, n_body=args.rows)


def workload_config(args, info=None):
    if args.workload == "spatiotemporal":
        cfg = {"workload": "spatio-temporal Q_t (x) Q_s: AR(1) n_t=100 rho=0.9, (kappa^2 I + L)^2 on a 45x45 grid "
                           f"(kappa^2=1), time-major, + 20 fixed-effect arrow rows, nrhs 1 ({args.precision})",
               "n": 202520, "n_arrow": 20, "nrhs": 1, "tile": args.tile, "ordering": args.ordering,
               "l2": "inputs larger than L2 (factor tiles > 1 GB vs 126 MB L2); no flush"}
    else:
        cfg = {"workload": f"band{args.rows}_hw100-500_d0.2_arrow100_nrhs4 (large single matrix, {args.precision})",
               "n": args.rows + 100, "n_arrow": 100, "nrhs": 4, "tile": args.tile, "ordering": args.ordering,
               "l2": "inputs larger than L2 (values 0.26 GB, factor tiles > 0.7 GB vs 126 MB L2); no flush"}
    cfg.update({
           "step": ("factorize + logdet + solve (analysis once per pattern, timed separately); FP64: the "
                    "forward sweep inside the factorization launch (stiles_factorize_solve), then the "
                    "backward sweep"),
           "flops": "tile-level task flops of Algorithm 1 at tile T (POTRF b(b+1)(2b+1)/6, SYRK kb(b+1), "
                    "GEMM 2mnk, TRSM mb^2)"})
    if info:
        cfg.update({"block": info["block"], "nnzt": info["nnzt"], "ntasks": info["ntasks"],
                    "flops_factor": info["flops_total"]})
    return cfg


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
# CPU baseline: the oracle, as it stands, on a bounded sample
# ---------------------------------------------------------------------------
def cpu_baseline(args, T):
    from oracle import analyze as oan
    from oracle import cholesky as och
    from oracle import tiles as otiles

    rows = args.cpu_sample_rows
    if args.workload == "spatiotemporal":
        # 4 time steps of the same Kronecker structure (8,120 rows), tile 64
        m = inputs.kronecker_spatiotemporal(4, 0.9, 45, 1.0, 20, 0.1, 0, nrhs=1)
        T = 64
        rows = m["n"]
    else:
        m = inputs.config_large(0, n_body=rows, n_arrow=100, nrhs=4)
    p = oan.analyze(m, T, oan.ORDER_NONE)
    fl = otiles.task_flops(m["n"], T, p["tcolptr"], p["trowidx"])["total"]
    t0 = time.perf_counter()
    L = och.factorize(m, p["perm"], T, p["tcolptr"], p["trowidx"])
    och.logdet(L, p["nt"])
    och.solve(L, p["perm"], T, p["tcolptr"], p["trowidx"], m["rhs"])
    dt = time.perf_counter() - t0
    what = (f"the same generator with {rows} body rows + 100-row arrow" if args.workload != "spatiotemporal"
            else f"the same Kronecker structure with 4 time steps ({rows} rows)")
    return {"value": fl / dt / 1e12, "unit": "TFLOP/s", "cores": 1, "kind": "oracle",
            "sample": f"{what}, T={T}, one factorize+logdet+solve ({dt:.1f} s, one thread: Python/numpy, BLAS "
                      f"pinned to 1 thread)", "seconds": dt, "flops": fl}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    T = args.tile
    vals = []
    base = None
    for i in range(args.warmup + args.steps):
        base = cpu_baseline(args, T)
        if i >= args.warmup:
            vals.append(base["seconds"])
    v = base["flops"] / statistics.mean(vals) / 1e12
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "TFLOP/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(vals),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": dict(workload_config(args), sample=base["sample"]),
            "cpu_baseline": {"value": v, "unit": "TFLOP/s", "cores": 1, "kind": "oracle", "sample": base["sample"]},
            "e2e": {"value": v, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# our arm
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


def run_ours(args):
    import torch

    from paper_2501_02483_b300 import build
    from paper_2501_02483_b300 import stiles as st

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    build.build_library()
    order = {"none": st.ORDER_NONE, "rcm": st.ORDER_RCM, "auto": st.ORDER_AUTO, "nd": st.ORDER_ND}[args.ordering]

    m = workload(args, seed=rank)
    prec = {"f64": st.PREC_F64, "bf16": st.PREC_BF16, "f16": st.PREC_F16}[args.precision]
    t0 = time.perf_counter()
    plan = st.Plan.from_matrix(m, tile=args.tile, block=args.block, ordering=order, precision=prec)
    analyze_s = time.perf_counter() - t0
    info = plan.info()
    flops = info["flops_total"]
    nrhs = m["rhs"].shape[1]
    dev = torch.device("cuda", local)
    vals_d = torch.from_numpy(m["values"]).to(dev)
    b_d = torch.from_numpy(np.asfortranarray(m["rhs"])).to(dev)
    # pinned host buffers for the end-to-end measurement (b, x: n x nrhs column-major views)
    vals_host = torch.from_numpy(m["values"]).pin_memory().numpy()
    bt = torch.from_numpy(np.ascontiguousarray(m["rhs"].T)).pin_memory()
    xt = torch.empty_like(bt).pin_memory()
    b_host, x_host = bt.numpy().T, xt.numpy().T
    peak = st.probe_fp64_peak()

    f = st.Factor(plan)
    stream = torch.cuda.current_stream(dev)
    # FP64: the forward sweep runs inside the factorization launch
    # (stiles_factorize_solve); mixed precision: factorize, then the refined solve
    fused = prec == st.PREC_F64 and nrhs <= min(info["block"], 16)
    x_d = torch.empty((nrhs, m["n"]), dtype=torch.float64, device=dev).t()  # n x nrhs, column-major

    def step_device():
        if fused:
            x = f.factorize_solve(vals_d, b_d, x=x_d, stream=stream)
            ld = f.logdet()
            return ld, x
        f.factorize(vals_d, stream=stream)
        ld = f.logdet()
        x = f.solve(b_d, stream=stream)
        return ld, x

    for _ in range(args.warmup):
        step_device()
    torch.cuda.synchronize()
    kernel_ms = []
    n0 = st.kernel_launches()
    with ClockSampler(local) as clk:
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            ld, x = step_device()
            kernel_ms.append(f.timing()[1])
        e1.record(stream)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
    launches = st.kernel_launches() - n0
    ms = e0.elapsed_time(e1) / args.steps
    if dist:
        t = torch.tensor([ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    value = world * flops / (ms * 1e-3) / 1e12

    # end to end through host buffers (pinned): H2D values + RHS, D2H x + logdet
    vals_pin = torch.from_numpy(vals_host)
    vals_stage = torch.empty_like(vals_d)
    b_stage = torch.empty((nrhs, m["n"]), dtype=torch.float64, device=dev)

    def step_e2e():
        if fused:  # explicit copies: the folded call takes device arrays
            vals_stage.copy_(vals_pin, non_blocking=True)
            b_stage.copy_(bt, non_blocking=True)
            f.factorize_solve(vals_stage, b_stage.t(), x=x_d, stream=stream)
            f.logdet()
            xt.copy_(x_d.t())
        else:
            f.factorize(vals_host)
            f.logdet()
            f.solve(b_host, x=x_host)

    step_e2e()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step_e2e()
    torch.cuda.synchronize()
    e2e_ms = (time.perf_counter() - t0) * 1e3 / args.steps
    if dist:
        t = torch.tensor([e2e_ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_ms = float(t.item())
    e2e = {"value": world * flops / (e2e_ms * 1e-3) / 1e12, "unit": "TFLOP/s",
           "h2d_bytes_per_step": int(m["values"].nbytes + b_host.nbytes),
           "d2h_bytes_per_step": int(x_host.nbytes + 8), "ms_per_step": e2e_ms}

    # correctness of what was timed
    _, relres = f.solve(b_d, stream=stream, relres=True)

    # marginal variances diag(A^{-1}) through the selected inverse (FP64 factors):
    # the first call builds and uploads its task graph; a new factorization
    # invalidates Sigma, so the timed call recomputes all of it
    sinv = None
    if prec == st.PREC_F64 and rank == 0:
        f.marginal_variances(stream=stream)
        f.factorize(vals_d, stream=stream)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        var = f.marginal_variances(stream=stream)
        ms_sinv = (time.perf_counter() - t0) * 1e3
        sfl = _selinv_flops(plan)
        sinv = {"ms": round(ms_sinv, 2), "flops": sfl, "tflops": round(sfl / ms_sinv / 1e9, 4),
                "frac_of_fp64_peak": round(sfl / ms_sinv / 1e9 / peak, 4),
                "min_variance": float(var.min()), "max_variance": float(var.max()),
                "flops_rule": "2 B^3 per operand pair, B^3 per L_jk L_kk^{-1} and per L_kk^{-T} L_kk^{-1}"}

    # tile-size sweep (the workload names 128/256/512; 32/64 added)
    sweep = {}
    if rank == 0 and args.sweep:
        for T in [int(t) for t in args.sweep.split(",") if t]:
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
            sweep[str(T)] = {"kernel_ms": round(min(ks), 3), "tflops": round(fl / min(ks) / 1e9, 4),
                             "flops": fl, "block": pl.info()["block"]}
            ff.close()
            pl.close()

    kms = statistics.mean(kernel_ms)
    achieved = flops / (kms * 1e-3) / 1e12
    if prec == st.PREC_F64:
        traffic = TRAFFIC.get((KERNEL_TAG, args.workload, args.tile, info["block"]))
        roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": traffic, "kernel_ms": kms,
                "kernel": f"factor_f64_kernel<{info['block']}>" + (" (forward sweep folded in; achieved counts the "
                                                                    "factorization's flops only)" if fused else ""),
                "peak_source": "FP64 DFMA probe of libstiles.so measured in this run (MEASURED_PEAKS.json "
                               "has no FP64 entry)"}
    else:
        tpeak, src = _tensor_peak()
        roof = {"bound": "tensor", "achieved": achieved, "peak": tpeak, "unit": "TFLOP/s", "frac": achieved / tpeak,
                "traffic": None, "kernel": "factor_lp_kernel", "kernel_ms": kms, "peak_source": src}
    line = {
        "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": args.precision, "data": "synthetic",
        "config": dict(workload_config(args, info), analyze_s=round(analyze_s, 3), logdet=ld,
                       relres=relres, tile_sweep=sweep, percent_of_fp64_peak=round(100 * value / peak, 2),
                       refine_iters=f.refine_iters(), marginal_variances=sinv),
        "roofline": roof,
        "e2e": e2e, "gpu_launches": launches, "clocks": clk.result,
    }
    f.close()
    plan.close()
    if rank == 0 and args.workload == "large" and not args.no_largest:
        line["config"]["largest_config_fp64"] = _largest_config_fp64(st, torch, dev, stream, peak)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = {k: v for k, v in cpu_baseline(args, args.tile).items() if k not in ("seconds", "flops")}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


# ---------------------------------------------------------------------------
# batched sweep and serving workloads
# ---------------------------------------------------------------------------
def _largest_config_fp64(st, torch, dev, stream, peak):
    """FP64 factorization of the largest configuration (the spatio-temporal
    matrix, n = 202,520, tile 16, nested dissection): kernel time of 2 timed
    factorizations after one warm-up, as a fraction of the measured FP64 peak."""
    m = inputs.config_spatiotemporal(0)
    pl = st.Plan.from_matrix(m, tile=16, ordering=st.ORDER_ND)
    ff = st.Factor(pl)
    vd = torch.from_numpy(m["values"]).to(dev)
    ff.factorize(vd, stream=stream)
    ks = []
    for _ in range(2):
        ff.factorize(vd, stream=stream)
        ks.append(ff.timing()[1])
    fl = pl.info()["flops_total"]
    ms = statistics.mean(ks)
    out = {"workload": "spatio-temporal Q_t (x) Q_s + 20 arrow rows, n = 202,520, T = 16, ND",
           "factor_kernel_ms": round(ms, 2), "flops": fl, "tflops": round(fl / ms / 1e9, 4),
           "frac_of_fp64_peak": round(fl / ms / 1e9 / peak, 4)}
    ff.close()
    pl.close()
    return out


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
    if not dist:
        return v
    t = torch.tensor([v], device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _sweep_arm(args, st, torch, mats, prec, T, dev, stream, dist):
    """One precision arm of the batched sweep: analysis, then W + K steps of
    batched factorize + logdets + batched solve."""
    t0 = time.perf_counter()
    plans = [st.Plan.from_matrix(m, tile=T, ordering=st.ORDER_NONE, precision=prec) for m in mats]
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

    for _ in range(args.warmup):
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
        for _ in range(args.steps):
            statuses, lds, rel, its, km = step(vals_d, rhs_d)
            kms.append(km)
        e1.record(stream)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
    launches = st.kernel_launches() - n0
    ms = _max_over_ranks(torch, dist, dev, e0.elapsed_time(e1) / args.steps)
    ok = int(np.sum((statuses == 0) & (rel <= 1e-10)))
    # end to end from pinned host buffers: H2D values + right-hand sides, D2H solutions + logdets
    vals_h = [torch.from_numpy(m["values"]).pin_memory().numpy() for m in mats]
    rhs_h = [torch.from_numpy(np.asfortranarray(m["rhs"])).pin_memory().numpy() for m in mats]
    step(vals_h, rhs_h)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step(vals_h, rhs_h)
    torch.cuda.synchronize()
    e2e_ms = _max_over_ranks(torch, dist, dev, (time.perf_counter() - t0) * 1e3 / args.steps)
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


def run_sweep(args):
    torch, world, rank, local, dist = _setup_rank()
    from paper_2501_02483_b300 import stiles as st

    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    mats = inputs.batch_sweep(args.batch, seed=rank)
    prec = st.PREC_BF16 if args.lp_precision == "bf16" else st.PREC_F16
    lp = _sweep_arm(args, st, torch, mats, prec, args.lp_tile, dev, stream, dist)
    f64 = _sweep_arm(args, st, torch, mats, st.PREC_F64, args.f64_tile, dev, stream, dist)
    ld_err = float(np.max(np.abs(lp["logdets"] - f64["logdets"]) / np.abs(f64["logdets"])))
    for a in (lp, f64):
        a.pop("logdets")
    peak, peak_src = _tensor_peak()
    achieved = lp["flops"] / (lp["kernel_ms"] * 1e-3) / 1e12
    line = {
        "metric": METRIC, "value": world * lp["tflops"], "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": lp["ms_per_step"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": args.lp_precision, "data": "synthetic",
        "config": {"workload": f"batched sweep: {args.batch} matrices, n log-uniform [5000, 50000], hw {{64,128,256}}, "
                               "arrow 0..50, theta ~ U(0.5, 2), 1 RHS each; refined to 1e-10",
                   "step": "batched factorize (one persistent launch) + all logdets + batched solve with FP64 "
                           "refinement (analysis once per pattern, timed separately)",
                   "l2": "inputs larger than L2 (factor tiles of the batch > 1 GB); no flush",
                   "mixed_precision": lp, "fp64": f64, "logdet_rel_diff_lp_vs_fp64": ld_err,
                   "solves_per_s_lp_over_fp64": lp["solves_per_s"] / max(f64["solves_per_s"], 1e-30)},
        "roofline": {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": None, "kernel": "factor_lp_kernel (batched)",
                     "kernel_ms": lp["kernel_ms"], "peak_source": peak_src},
        "e2e": {"value": world * lp["flops"] / (lp["e2e_ms"] * 1e-3) / 1e12, "unit": "TFLOP/s",
                "h2d_bytes_per_step": lp["e2e_h2d"], "d2h_bytes_per_step": lp["e2e_d2h"],
                "ms_per_step": lp["e2e_ms"]},
        "gpu_launches": lp["gpu_launches"], "clocks": lp["clocks"],
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = sweep_cpu_baseline(args)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def sweep_cpu_baseline(args, count=4):
    """The oracle (FP64) on the first ``count`` matrices of the sweep."""
    from oracle import analyze as oan
    from oracle import cholesky as och
    from oracle import tiles as otiles

    mats = inputs.batch_sweep(args.batch, seed=0)[:count]
    fl, t0 = 0, time.perf_counter()
    for m in mats:
        p = oan.analyze(m, args.lp_tile, oan.ORDER_NONE)
        fl += otiles.task_flops(m["n"], args.lp_tile, p["tcolptr"], p["trowidx"])["total"]
        L = och.factorize(m, p["perm"], args.lp_tile, p["tcolptr"], p["trowidx"])
        och.logdet(L, p["nt"])
        och.solve(L, p["perm"], args.lp_tile, p["tcolptr"], p["trowidx"], m["rhs"])
    dt = time.perf_counter() - t0
    return {"value": fl / dt / 1e12, "unit": "TFLOP/s", "cores": 1, "kind": "oracle",
            "sample": f"the first {count} matrices of the sweep, T={args.lp_tile}, FP64 factorize+logdet+solve "
                      f"({dt:.1f} s, one thread)", "seconds": dt, "flops": fl}


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
    order = {"none": st.ORDER_NONE, "rcm": st.ORDER_RCM, "auto": st.ORDER_AUTO, "nd": st.ORDER_ND}[args.serve_ordering]
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
    srv.close()
    return out


def run_serve(args):
    torch, world, rank, local, dist = _setup_rank()
    from paper_2501_02483_b300 import serve as sv
    from paper_2501_02483_b300 import stiles as st

    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    work = inputs.serving_workload(args.requests, rate=args.rate, seed=rank, variants=2)
    _pin_requests(torch, work[0])
    lp_prec = st.PREC_BF16 if args.lp_precision == "bf16" else st.PREC_F16
    lp = _serve_arm(args, st, sv, torch, work, lp_prec, args.lp_tile, stream)
    f64 = _serve_arm(args, st, sv, torch, work, st.PREC_F64, args.f64_tile, stream)
    value = _max_over_ranks(torch, dist, dev, -lp["solves_per_s"])
    line = {
        "metric": METRIC, "value": -value * world, "unit": "solves/s", "n_gpus": world, "steps": 1,
        "warmup": 1, "ms_per_step": 1e3 * lp["wall_s"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": args.lp_precision, "data": "synthetic",
        "config": {"workload": f"serving: Poisson {args.rate:g} req/s, {args.requests} requests, n log-uniform "
                               "[1000, 200000], hw 32..512, arrow 0..100, nrhs 1..16, 30% re-solves, "
                               "HBM budget 150 GB; 48 patterns x 2 value scales (theta in {0.875, 1.625}); client "
                               "buffers in pinned host memory; ordering " + args.serve_ordering,
                   "step": "the whole request stream through the continuous-batching loop (arrivals in real time)",
                   "mixed_precision": lp, "fp64": f64,
                   "solves_per_s_lp_over_fp64": lp["solves_per_s"] / max(f64["solves_per_s"], 1e-30)},
        "e2e": {"value": -value * world, "unit": "solves/s", "h2d_bytes_per_step": None,
                "d2h_bytes_per_step": None,
                "note": "requests enter as host arrays; every value and right-hand side crosses H2D"},
        "gpu_launches": lp["gpu_launches"], "clocks": lp["clocks"],
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
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
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
