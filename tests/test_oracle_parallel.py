"""The oracle's angle-parallel formal solution (the all-core CPU baseline).

With one thread it must be the serial formal solution bit for bit; with
several threads the angle sum is associated per thread, so it agrees to
rounding and is reproducible for a fixed thread count.
"""
import numpy as np

from oracle import oracle as O
from paper_0903_1949_gb300 import inputs as I


def test_parallel_formal_solution_equals_serial():
    p = I.make_problem("sph17")
    g = O.OracleGrid(p["coord"], p["edges"], p["dirs"], p["weights"], p["inner_bc"])
    S = p["B"] * np.random.default_rng(4).uniform(0.8, 1.2, p["B"].size)
    J, L, F, miss = g.formal_solution(S, p["chi"], p["B"])
    J1, L1, F1, m1, used = g.formal_solution_par(S, p["chi"], p["B"], threads=1)
    assert miss == 0 and m1 == 0 and used == 1
    assert np.array_equal(J, J1) and np.array_equal(L, L1) and np.array_equal(F, F1)
    J4, L4, F4, m4, used4 = g.formal_solution_par(S, p["chi"], p["B"], threads=4)
    J4b, _, _, _, _ = g.formal_solution_par(S, p["chi"], p["B"], threads=4)
    assert m4 == 0 and used4 >= 1
    assert np.array_equal(J4, J4b)
    assert np.max(np.abs(J4 - J) / J) < 1e-14
    assert np.max(np.abs(L4 - L) / L) < 1e-14
    assert np.max(np.abs(F4 - F)) < 1e-14 * np.max(np.abs(F))
