"""Exact FP64 operation counts of one particle-substep of the oracle's
propagation (Steps 2 and 4 of Algorithm 1), from the op-counting build of the
oracle (opcount.cpp): the algorithmic work the benchmark's roofline divides by
time for the problems whose Newton system the oracle solves the way the
method states it (a dense LU of I - gamma J for d <= 3: linear2, Robertson
and M1 with each LMM).

A count is the sum of additions/subtractions, multiplications, divisions and
square roots (a multiply-add is 2; the oracle has no fused operations);
elementary functions (M1's input exp) are reported apart.  The substep is a
steady-state one of the family (BDF2, BDF3, AM_q or AB_q at full order, after
the cold start) with Step 4's Milne sums.

    python oracle/count_flops.py          # prints the table bench.py stores
"""
from __future__ import annotations

import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from paper_1411_1702_gb300 import workloads as W  # noqa: E402

# the bench workloads whose substeps are counted here
NAMES = ["linear2", "robertson"] + ["michaelis" + n for n in W.LMM_NAMES] + ["michaelis"]


def substep_counts(w, K=None, with_error=True):
    """Counts of one steady-state substep of workload w (its second interval,
    a substep after the order ramp) at the reference state."""
    K = w.newton_iters if K is None else K
    cfg = oracle.make_config(w)
    t0, t1, t2 = w.t0, w.t_obs[0], w.t_obs[1]
    tab0, S0, d0 = oracle.build_substeps(cfg, t0, t1, 0, 0.0, 0.0)
    tab, S, _ = oracle.build_substeps(cfg, t1, t2, d0, tab0[S0 - 1].h,
                                      tab0[S0 - 2].h if S0 >= 2 else 0.0)
    one = (oracle.Substep * 1)()
    one[0] = tab[S // 2]
    x = np.array(w.x_true[0], dtype=np.float64)
    c = oracle.count_propagate(w.ode, K, w.theta_true, one, 1, x, x, x, with_error)
    del c["x"]
    c["flops"] = c["add"] + c["mul"] + c["div"] + c["sqrt"]
    c["kind"] = int(one[0].kind)
    return c


def table():
    out = {}
    for name in NAMES:
        w = W.get(name, N=4, T=3)
        c = substep_counts(w)
        out[name] = {"K": w.newton_iters, "flops": c["flops"], "add": c["add"], "mul": c["mul"],
                     "div": c["div"], "sqrt": c["sqrt"], "elem": c["elem"], "kind": c["kind"]}
    return out


if __name__ == "__main__":
    print(json.dumps(table(), indent=1, sort_keys=True))
