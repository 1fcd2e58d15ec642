"""bench.py's CPU baseline: the oracle's complete solve with the shifted
solves spread over worker processes gives exactly the serial oracle's result
(same arithmetic, same node order of the sums).  No GPU."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def test_parallel_node_solvers_match_serial_oracle():
    import bench
    from oracle import feast_nh as OF
    from oracle.contour import contour_nodes
    from paper_1506_04463_gb300 import workloads as wl
    wk = wl.config2(N=20, m0=48, ne=16)
    ser = OF.feast_nh(wk.A, None, wk.contour, wk.m0, wk.Y0, wk.Yh0, dense=False)
    pool = bench.ParallelNodeSolvers(wk.A, None, contour_nodes(wk.contour)[0], wk.m0, workers=3)
    try:
        par, ph = bench.oracle_full_solve(wk, pool)
    finally:
        pool.close()
    assert par["m"] == ser["m"] == 30 and par["iterations"] == ser["iterations"]
    assert np.array_equal(par["lam"], ser["lam"])
    assert ph["total_s"] > 0 and ph["factor_s"] > 0
    e = bench.per_pair_errors(par["lam"], par["res"], ser)
    assert e["max_rel_err"] == 0.0 and len(e["rel_err"]) == 30


def test_reference_arm_line():
    # bench.py --impl reference on a small grid: complete oracle solves, the
    # base contract's keys, and the cpu_baseline / e2e objects of this arm
    import argparse
    import bench
    args = argparse.Namespace(N=20, steps=1, warmup=0, impl="reference")
    line = bench.run_reference(args, 0, 1)
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "cpu_baseline", "e2e", "config"):
        assert k in line, k
    assert line["impl"] == "reference" and line["value"] > 0 and line["steps_timed"] == 1
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"]
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["value"] == line["value"]
    assert line["cpu_baseline"]["per_phase_s"]["total_s"] > 0
