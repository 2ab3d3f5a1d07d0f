"""rt_set_opacity rejects out-of-range input with nothing changed.

chi must be > 0 and finite, eps in (0, 1], B >= 0 and finite (the opacity,
thermalisation parameter and Planck function of Sect. 3.1).  A rejected call
returns RT_EINVAL naming the first bad voxel and leaves chi, eps, B and S as
they were, for host arrays and for device arrays alike.
"""
import numpy as np
import pytest

from paper_0903_1949_gb300 import build as Bld
from paper_0903_1949_gb300 import rt
from tests.helpers import tiny_problem
from paper_0903_1949_gb300 import inputs as I

pytestmark = pytest.mark.gpu

BAD = [("chi", np.nan, "chi"), ("chi", 0.0, "chi"), ("chi", -1.0, "chi"), ("chi", np.inf, "chi"),
       ("eps", 0.0, "eps"), ("eps", 1.5, "eps"), ("eps", np.nan, "eps"),
       ("B", -0.1, "B"), ("B", np.inf, "B"), ("B", np.nan, "B")]


@pytest.mark.parametrize("on_device", [False, True])
def test_bad_opacity_is_rejected_without_state_change(on_device):
    torch = pytest.importorskip("torch")
    Bld.build()
    rt.load()
    p = tiny_problem(I.SPHERICAL, (6, 5, 7), 4, 4, I.CORE_B)
    g = rt.Grid(p["coord"], p["edges"], p["dirs"], p["weights"], inner_bc=p["inner_bc"])
    try:
        g.set_opacity(p["chi"], p["eps"], p["B"])
        S = p["B"] * np.random.default_rng(5).uniform(0.8, 1.2, p["nvox"])
        g.set_S(S)
        g.formal_solution(rt.RT_FP64)
        J_ref = g.J()
        for name, value, word in BAD:
            arrs = {"chi": p["chi"].copy(), "eps": p["eps"].copy(), "B": p["B"].copy()}
            arrs[name][37] = value
            if on_device:
                arrs = {k: torch.tensor(v, dtype=torch.float64, device="cuda:0") for k, v in arrs.items()}
            with pytest.raises(rt.RtError) as ei:
                g.set_opacity(arrs["chi"], arrs["eps"], arrs["B"])
            assert ei.value.code == rt.RT_EINVAL
            assert ("%s[37]" % word) in str(ei.value), str(ei.value)
            # nothing changed: S is the one set before, the formal solution is the same
            assert np.array_equal(g.S(), S)
            g.formal_solution(rt.RT_FP64)
            assert np.array_equal(g.J(), J_ref), (name, value)
        # a valid device call still works and resets S := B
        if on_device:
            d = {k: torch.tensor(p[k], dtype=torch.float64, device="cuda:0") for k in ("chi", "eps", "B")}
            g.set_opacity(d["chi"], d["eps"], d["B"])
            torch.cuda.synchronize()
            assert np.array_equal(g.S(), p["B"])
    finally:
        g.close()
