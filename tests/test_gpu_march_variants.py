"""The FP32 J-only march of the ALI iteration in all its launch configurations
(rt_tune): streamed weights on/off, segments per lane, bundle size, list-order
output (scatter), overlapped gather, shared-memory rings fed by cp.async or
bulk copies.  Configurations that only move data differently give bit-identical
iterates; the others agree to FP32 rounding; all stay within the mixed-precision
bar of the FP64 oracle."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_0903_1949_gb300 import build as Bd
from paper_0903_1949_gb300 import inputs as I
from paper_0903_1949_gb300 import rt
from tests.helpers import tiny_problem

pytestmark = pytest.mark.gpu

STEPS = 6


@pytest.fixture(scope="module", autouse=True)
def _built():
    Bd.build()
    rt.load()


def _problems():
    p1 = I.make_problem("sph17")
    p1["nvox"] = p1["chi"].size
    p2 = tiny_problem(I.CYLINDRICAL, (9, 8, 7), 6, 6, I.TRANSPARENT, eps=0.05, seed=21)  # hole: restarts
    p3 = tiny_problem(I.SPHERICAL, (11, 6, 10), 6, 6, I.CORE_B, eps=0.1, seed=22)
    return {"sph17": (p1, rt.RT_PARABOLIC), "cyl_hole": (p2, rt.RT_PARABOLIC), "sph_linear": (p3, rt.RT_LINEAR)}


def _iterate(p, interp, knobs, precision=rt.RT_MIXED, angle_block=0):
    g = rt.Grid(p["coord"], p["edges"], p["dirs"], p["weights"], inner_bc=p["inner_bc"], interp=interp,
                precision=precision, ng=False, angle_block=angle_block)
    for k, v in knobs.items():
        g.tune(k, v)
    g.set_opacity(p["chi"], p["eps"], p["B"])
    for _ in range(STEPS):
        g.ali_step()
    S = g.S()
    g.close()
    return S


T = rt
# the unfolded march (the staged rings support only that one); the folded default is checked in FOLDED
BASE = {T.RT_TUNE_STREAMED_WEIGHTS: 1, T.RT_TUNE_MARCH_COARSEN: 2, T.RT_TUNE_MARCH_CHUNK: 512, T.RT_TUNE_SCATTER: 1,
        T.RT_TUNE_OVERLAP: 1, T.RT_TUNE_MARCH_STAGES: 0, T.RT_TUNE_MARCH_BULK: 0, T.RT_TUNE_MARCH_LOOKAHEAD: 1,
        T.RT_TUNE_S_BLOCKED: 1, T.RT_TUNE_MARCH_STREAMS: 3, T.RT_TUNE_GRAPH: 1, T.RT_TUNE_FOLD_WEIGHT: 0}
# the library's defaults (gather weight folded into the streamed weights, one segment per lane) and,
# bit-identical to them, the same arithmetic with the data moved differently
FOLDED = {**BASE, T.RT_TUNE_FOLD_WEIGHT: 1, T.RT_TUNE_MARCH_COARSEN: 1}
FOLDED_SAME = [{T.RT_TUNE_SCATTER: 0}, {T.RT_TUNE_OVERLAP: 0}, {T.RT_TUNE_S_BLOCKED: 0}, {T.RT_TUNE_GRAPH: 0},
               {T.RT_TUNE_MARCH_STREAMS: 1}, {T.RT_TUNE_MARCH_LOOKAHEAD: 0}]
# same arithmetic in the same order, data moved differently: bit-identical
SAME = [
    {T.RT_TUNE_S_BLOCKED: 0},
    {T.RT_TUNE_S_BLOCKED: 0, T.RT_TUNE_MARCH_STAGES: 3},
    {T.RT_TUNE_MARCH_LOOKAHEAD: 0},
    {T.RT_TUNE_MARCH_LOOKAHEAD: 0, T.RT_TUNE_SCATTER: 0},
    {T.RT_TUNE_SCATTER: 0},
    {T.RT_TUNE_OVERLAP: 0},
    {T.RT_TUNE_SCATTER: 0, T.RT_TUNE_OVERLAP: 0},
    {T.RT_TUNE_MARCH_STAGES: 2},
    {T.RT_TUNE_MARCH_STAGES: 3},
    {T.RT_TUNE_MARCH_STAGES: 4, T.RT_TUNE_SCATTER: 0},
    {T.RT_TUNE_MARCH_STAGES: 3, T.RT_TUNE_MARCH_BULK: 1},
    {T.RT_TUNE_MARCH_STAGES: 2, T.RT_TUNE_MARCH_BULK: 1, T.RT_TUNE_OVERLAP: 0},
]
# another association of the FP32 scan, or the on-the-fly weights: FP32 rounding
CLOSE = [
    {T.RT_TUNE_MARCH_COARSEN: 1},
    {T.RT_TUNE_MARCH_COARSEN: 4},
    {T.RT_TUNE_MARCH_CHUNK: 64},
    {T.RT_TUNE_MARCH_CHUNK: 4096, T.RT_TUNE_MARCH_COARSEN: 1, T.RT_TUNE_MARCH_STAGES: 3},
    {T.RT_TUNE_STREAMED_WEIGHTS: 0},
    {T.RT_TUNE_FOLD_WEIGHT: 1},
    {T.RT_TUNE_FOLD_WEIGHT: 1, T.RT_TUNE_MARCH_COARSEN: 1},
    {T.RT_TUNE_FOLD_WEIGHT: 1, T.RT_TUNE_MARCH_STREAMS: 1, T.RT_TUNE_GRAPH: 0},
]


@pytest.mark.parametrize("name", ["sph17", "cyl_hole", "sph_linear"])
def test_march_configurations(name):
    p, interp = _problems()[name]
    S0 = _iterate(p, interp, BASE)
    for var in SAME:
        S = _iterate(p, interp, {**BASE, **var})
        assert np.array_equal(S, S0), (name, var, float(np.max(np.abs(S - S0) / np.abs(S0))))
    for var in CLOSE:
        S = _iterate(p, interp, {**BASE, **var})
        assert np.max(np.abs(S - S0) / np.abs(S0)) < 2e-6, (name, var)
    S1 = _iterate(p, interp, FOLDED)
    assert np.array_equal(S1, _iterate(p, interp, {}))  # FOLDED is what the library does by default
    for var in FOLDED_SAME:
        S = _iterate(p, interp, {**FOLDED, **var})
        assert np.array_equal(S, S1), (name, var, float(np.max(np.abs(S - S1) / np.abs(S1))))
    o = O.OracleGrid(p["coord"], p["edges"], p["dirs"], p["weights"], p["inner_bc"], interp=interp)
    S_o, _, _ = o.solve(p["chi"], p["eps"], p["B"], tol=0.0, max_iter=STEPS, ng=False)
    assert np.max(np.abs(S0 - S_o) / np.abs(S_o)) < 1e-5


@pytest.mark.parametrize("name", ["sph17", "cyl_hole", "sph_linear"])
def test_fp64_march_configurations(name):
    """The FP64 streamed-weight march against the FP64 march that evaluates its
    weights itself, and against the oracle's iterates at the FP64 bar."""
    p, interp = _problems()[name]
    S0 = _iterate(p, interp, BASE, rt.RT_FP64)
    for var in ({T.RT_TUNE_SCATTER: 0}, {T.RT_TUNE_OVERLAP: 0}, {T.RT_TUNE_SCATTER: 0, T.RT_TUNE_OVERLAP: 0}):
        assert np.array_equal(_iterate(p, interp, {**BASE, **var}, rt.RT_FP64), S0), var
    S_plain = _iterate(p, interp, {**BASE, T.RT_TUNE_STREAMED_WEIGHTS: 0}, rt.RT_FP64)
    assert np.max(np.abs(S_plain - S0) / np.abs(S0)) < 1e-13
    o = O.OracleGrid(p["coord"], p["edges"], p["dirs"], p["weights"], p["inner_bc"], interp=interp)
    S_o, _, _ = o.solve(p["chi"], p["eps"], p["B"], tol=0.0, max_iter=STEPS, ng=False)
    assert np.max(np.abs(S0 - S_o) / np.abs(S_o)) < 1e-11


@pytest.mark.parametrize("precision", [rt.RT_MIXED, rt.RT_FP64])
def test_march_streams_give_identical_iterates(precision):
    """Angle blocks of 5 solid angles (13 blocks of sph17): the marches on one
    stream or alternating between two or three, replayed as a CUDA graph or
    launched one by one, and without overlap, give the same bits."""
    p, interp = _problems()["sph17"]
    S0 = _iterate(p, interp, BASE, precision, angle_block=5)
    for var in ({T.RT_TUNE_MARCH_STREAMS: 1}, {T.RT_TUNE_MARCH_STREAMS: 1, T.RT_TUNE_SCATTER: 0},
                {T.RT_TUNE_MARCH_STREAMS: 2}, {T.RT_TUNE_MARCH_STREAMS: 2, T.RT_TUNE_SCATTER: 0},
                {T.RT_TUNE_GRAPH: 0}, {T.RT_TUNE_GRAPH: 0, T.RT_TUNE_MARCH_STREAMS: 1},
                {T.RT_TUNE_SCATTER: 0},
                {T.RT_TUNE_OVERLAP: 0}):
        assert np.array_equal(_iterate(p, interp, {**BASE, **var}, precision, angle_block=5), S0), var
    S_one = _iterate(p, interp, BASE, precision)  # one block: the same sums in another association
    tol = 2e-6 if precision == rt.RT_MIXED else 1e-13
    assert np.max(np.abs(S_one - S0) / np.abs(S0)) < tol


def test_tune_rejects_bad_values():
    p, interp = _problems()["sph17"]
    g = rt.Grid(p["coord"], p["edges"], p["dirs"], p["weights"], inner_bc=p["inner_bc"], precision=rt.RT_MIXED)
    for knob, bad in ((T.RT_TUNE_MARCH_CHUNK, 32), (T.RT_TUNE_MARCH_COARSEN, 3), (T.RT_TUNE_MARCH_STAGES, 1),
                      (T.RT_TUNE_MARCH_STAGES, 5), (T.RT_TUNE_MARCH_BULK, 2), (T.RT_TUNE_SCATTER, -1),
                      (T.RT_TUNE_OVERLAP, 7), (T.RT_TUNE_STREAMED_WEIGHTS, 3), (T.RT_TUNE_MARCH_LOOKAHEAD, 2),
                      (T.RT_TUNE_S_BLOCKED, 2), (T.RT_TUNE_MARCH_STREAMS, 0), (T.RT_TUNE_MARCH_STREAMS, 4), (T.RT_TUNE_GRAPH, 2), (T.RT_TUNE_FOLD_WEIGHT, 2),
                      (99, 1)):
        with pytest.raises(rt.RtError) as ei:
            g.tune(knob, bad)
        assert ei.value.code == rt.RT_EINVAL
    g.close()
