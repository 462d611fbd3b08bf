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

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
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
TRAFFIC = {("factor_f64_v2", 16, 16): 1.285e9}  # profiles/factor_f64_b16_band50000.md, scaled by tiles
KERNEL_TAG = "factor_f64_v4"


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
    ap.add_argument("--cpu-sample-rows", type=int, default=60_000)
    ap.add_argument("--rows", type=int, default=200_000,
                    help="body rows (profiling runs only; the benchmarked workload is 200,000)")
    return ap.parse_args()


def workload(args, seed=0):
    return inputs.config_large(seed, n_body=args.rows)


def workload_config(args, info=None):
    cfg = {"workload": f"band{args.rows}_hw100-500_d0.2_arrow100_nrhs4 (large single matrix, FP64)",
           "n": args.rows + 100, "n_arrow": 100, "nrhs": 4, "tile": args.tile, "ordering": args.ordering,
           "l2": "inputs larger than L2 (values 0.26 GB, factor tiles > 0.7 GB vs 126 MB L2); no flush",
           "step": "factorize + logdet + 4-RHS solve (analysis once per pattern, timed separately)",
           "flops": "tile-level task flops of Algorithm 1 at tile T (POTRF b(b+1)(2b+1)/6, SYRK kb(b+1), "
                    "GEMM 2mnk, TRSM mb^2)"}
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
    m = inputs.config_large(0, n_body=rows, n_arrow=100, nrhs=4)
    p = oan.analyze(m, T, oan.ORDER_NONE)
    fl = otiles.task_flops(m["n"], T, p["tcolptr"], p["trowidx"])["total"]
    t0 = time.perf_counter()
    L = och.factorize(m, p["perm"], T, p["tcolptr"], p["trowidx"])
    och.logdet(L, p["nt"])
    och.solve(L, p["perm"], T, p["tcolptr"], p["trowidx"], m["rhs"])
    dt = time.perf_counter() - t0
    return {"value": fl / dt / 1e12, "unit": "TFLOP/s", "cores": 1, "kind": "oracle",
            "sample": f"the same generator with {rows} body rows + 100-row arrow, T={T}, one "
                      f"factorize+logdet+4-RHS solve ({dt:.1f} s, one thread: Python/numpy, BLAS pinned to 1 "
                      f"thread)", "seconds": dt, "flops": fl}


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
    t0 = time.perf_counter()
    plan = st.Plan.from_matrix(m, tile=args.tile, block=args.block, ordering=order)
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

    def step_device():
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
    for _ in range(1):
        f.factorize(vals_host)
        f.solve(b_host, x=x_host)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        f.factorize(vals_host)
        f.logdet()
        f.solve(b_host, x=x_host)
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

    # tile-size sweep (the workload names 128/256/512; 32/64 added)
    sweep = {}
    if rank == 0 and args.sweep:
        for T in [int(t) for t in args.sweep.split(",") if t]:
            pl = st.Plan.from_matrix(m, tile=T, ordering=order)
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
    traffic = TRAFFIC.get((KERNEL_TAG, args.tile, info["block"]))
    line = {
        "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": dict(workload_config(args, info), analyze_s=round(analyze_s, 3), logdet=ld,
                       relres=relres, tile_sweep=sweep, percent_of_fp64_peak=round(100 * value / peak, 2)),
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": traffic, "kernel": f"factor_f64_kernel<{info['block']}>",
                     "kernel_ms": kms,
                     "peak_source": "FP64 DFMA probe of libstiles.so measured in this run (MEASURED_PEAKS.json "
                                    "has no FP64 entry)"},
        "e2e": e2e, "gpu_launches": launches, "clocks": clk.result,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = {k: v for k, v in cpu_baseline(args, args.tile).items() if k not in ("seconds", "flops")}
    if rank == 0:
        print(json.dumps(line), flush=True)
    f.close()
    plan.close()
    if dist:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
