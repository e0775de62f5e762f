"""The oracle's operation counter (its point physics on an op-counting number
type), pinned by hand counts of two formulas, and the per-item counts the
benchmark's algorithmic roofline uses.

WENO5 face value (one call): three candidate values 3 x (3 mul + 2 add) = 15;
indicators b0 = k (x0 - 2x1 + x2)^2 + 1/4 (x0 - 4x1 + 3x2)^2 -> 3 + 1 + 1 +
4 + 1 + 1 + 1 = 12, b1 = 9 (the second difference is x1 - x3), b2 = 12;
weights d_k / (eps + b_k)^2 -> 3 x 3 = 9; their sum 3; the weighted sum
3 x (div + mul + add) = 9: 15 + 33 + 9 + 3 + 9 = 69.
MC cell (monotone stencil): two differences and their product 3, the
candidates 2 dm, 2 dp, (dm + dp)/2 -> 4, the face values q -/+ s/2 -> 4: 11."""
import numpy as np

from paper_2408_01361_gb300 import inputs


def test_hand_counts_and_value_independence(orc):
    P = np.array([0.5, 0.1, 0.2, -0.01, 0.3, 0.05, 0.02, -0.01])
    a = orc.count_ops(inputs.torus_cfg(48, 32, 8), 2.0, 0.45, P)
    b = orc.count_ops(inputs.linear_mode_cfg(8, ndim=3), 0.5, 0.5, 3.0 * P)
    assert a["weno5"] == 69 and a["mc"] == 11
    assert a == b  # the formulas' operation counts do not depend on the metric or the state


def test_bench_constants_are_the_oracle_counts(orc):
    import importlib.util
    import os
    spec = importlib.util.spec_from_file_location(
        "bench_mod", os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    P = np.array([0.5, 0.1, 0.2, -0.01, 0.3, 0.05, 0.02, -0.01])
    assert orc.count_ops(inputs.torus_cfg(48, 32, 8), 2.0, 0.45, P) == bench.ALG_OPS
