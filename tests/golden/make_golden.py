"""Write the stored expected values of tests/golden/ from the oracle alone.

Each value is computed by oracle/ on inputs from the seeded generator module
(paper_2501_02483_b300/inputs.py, which holds none of the method's
arithmetic); nothing here calls the CUDA library.

    python tests/golden/make_golden.py          # rewrite large_workload.json
    python tests/golden/make_golden.py --check  # recompute and compare

large_workload.json: the 200,000-row variable band + 100 dense arrow rows
(seed 0), natural order, tile 32:
  - flops_total: the tile-level task flops of Algorithm 1 (POTRF b(b+1)(2b+1)/6,
    SYRK k b(b+1), GEMM 2mnk, TRSM m b^2) over the closed tile map;
  - logdet: 2 sum log L_ii of the oracle's factor.
"""
from __future__ import annotations

import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

PATH = os.path.join(HERE, "large_workload.json")


def large_workload_values(with_logdet=True):
    from oracle import analyze as oan
    from oracle import cholesky as och
    from oracle import tiles as otiles
    from paper_2501_02483_b300 import inputs

    m = inputs.config_large(0)
    T = 32
    p = oan.analyze(m, T, oan.ORDER_NONE)
    out = {"workload": "inputs.config_large(0): 200,000 band rows (half-width 100..500 per 2,000-row segment, "
                       "density 0.2) + 100 arrow rows, seed 0",
           "tile": T, "ordering": "none",
           "flops_total": int(otiles.task_flops(m["n"], T, p["tcolptr"], p["trowidx"])["total"])}
    if with_logdet:
        L = och.factorize(m, p["perm"], T, p["tcolptr"], p["trowidx"])
        out["logdet"] = och.logdet(L, p["nt"])
    return out


def load():
    with open(PATH) as fh:
        return json.load(fh)


if __name__ == "__main__":
    vals = large_workload_values()
    if "--check" in sys.argv:
        ref = load()
        ok = vals["flops_total"] == ref["flops_total"] and abs(vals["logdet"] - ref["logdet"]) <= 1e-13 * abs(
            ref["logdet"])
        print("match" if ok else f"MISMATCH: {vals} vs {ref}")
        sys.exit(0 if ok else 1)
    vals["written_by"] = "tests/golden/make_golden.py (oracle only)"
    with open(PATH, "w") as fh:
        json.dump(vals, fh, indent=1)
        fh.write("\n")
    print(vals)
