"""The op-counting build of the oracle (oracle/opcount.cpp) and the table of
exact substep counts the benchmark stores (bench.ORACLE_SUBSTEP_FLOPS).

The counts are pinned to facts about the oracle's algorithm that do not come
from the counter: every Newton iteration costs the same, so a substep's count
is affine in K; Step 4's Milne sums cost exactly 4 operations a component
(difference, scaling, square, sum); a Newton iteration of the dense 3x3 solve
divides 6 times (3 multipliers of the elimination, 3 back-substitution rows);
and the counted run computes the oracle's own state to the bit.  The stored
table must equal what oracle/count_flops.py prints."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

import bench
import oracle
from paper_1411_1702_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _one_substep(w):
    cfg = oracle.make_config(w)
    tab0, S0, d0 = oracle.build_substeps(cfg, w.t0, w.t_obs[0], 0, 0.0, 0.0)
    tab, S, _ = oracle.build_substeps(cfg, w.t_obs[0], w.t_obs[1], d0, tab0[S0 - 1].h, tab0[S0 - 2].h)
    one = (oracle.Substep * 1)()
    one[0] = tab[S // 2]
    return one


@pytest.mark.parametrize("name", ["linear2", "robertson", "michaelis"])
def test_counts_affine_in_newton_iterations(oracle_lib, name):
    w = W.get(name, N=4, T=3)
    one = _one_substep(w)
    x = np.array(w.x_true[0])
    tot = []
    for K in (1, 2, 3, 4):
        c = oracle.count_propagate(w.ode, K, w.theta_true, one, 1, x, x, x, True)
        tot.append(c["add"] + c["mul"] + c["div"])
    d = np.diff(tot)
    assert np.all(d == d[0]) and d[0] > 0


@pytest.mark.parametrize("name", ["linear2", "robertson", "michaelis"])
def test_milne_sums_cost_four_operations_a_component(oracle_lib, name):
    w = W.get(name, N=4, T=3)
    one = _one_substep(w)
    x = np.array(w.x_true[0])
    with_e = oracle.count_propagate(w.ode, 2, w.theta_true, one, 1, x, x, x, True)
    without = oracle.count_propagate(w.ode, 2, w.theta_true, one, 1, x, x, x, False)
    assert (with_e["add"] - without["add"], with_e["mul"] - without["mul"]) == (2 * w.d, 2 * w.d)
    assert with_e["div"] == without["div"]


def test_dense_solve_divisions(oracle_lib):
    # one Newton iteration of the 3-state Robertson system: the LU of the 3x3
    # matrix divides for its 2 + 1 multipliers and the back substitution for its
    # 3 rows -- 6 divisions, none elsewhere in the iteration
    w = W.robertson(N=4, T=3)
    one = _one_substep(w)
    x = np.array(w.x_true[0])
    c1 = oracle.count_propagate(w.ode, 1, w.theta_true, one, 1, x, x, x, True)
    c2 = oracle.count_propagate(w.ode, 2, w.theta_true, one, 1, x, x, x, True)
    assert c2["div"] - c1["div"] == 6


@pytest.mark.parametrize("name", ["linear2", "robertson", "michaelisAM3", "michaelisBDF3"])
def test_counted_run_gives_the_oracles_state(oracle_lib, name):
    w = W.get(name, N=4, T=3)
    one = _one_substep(w)
    x = np.array(w.x_true[0])
    ref, _, _, _ = oracle.propagate(w.ode, w.newton_iters, w.theta_true, one, 1, x, x, x)
    c = oracle.count_propagate(w.ode, w.newton_iters, w.theta_true, one, 1, x, x, x, True)
    assert np.array_equal(c["x"], ref)


def test_bench_table_is_the_scripts_output(oracle_lib):
    out = json.loads(subprocess.check_output([sys.executable, os.path.join(ROOT, "oracle", "count_flops.py")]))
    stored = bench.ORACLE_SUBSTEP_FLOPS
    assert set(stored) == set(out)
    for k, v in out.items():
        assert stored[k] == {"K": v["K"], "flops": v["flops"]}, k
    assert all(v["sqrt"] == 0 for v in out.values())
