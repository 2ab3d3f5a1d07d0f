"""Two-level-atom line transfer on the GPU (rt_line_*) against the oracle's
frequency-averaged line ALI (Sect. 3.1, 3.2.2): Lbar*, the iterates and the
converged line source function at the mixed-precision bar, the single-frequency
reduction to the continuum ALI, the thermal limit at the paper's full grid
size, and the argument checks."""
import numpy as np
import pytest

from oracle import line as OL
from oracle import oracle as O
from paper_0903_1949_gb300 import build as Bd
from paper_0903_1949_gb300 import inputs as I
from paper_0903_1949_gb300 import rt
from tests.helpers import tiny_problem

pytestmark = pytest.mark.gpu

MIXED = 1e-5  # FP32 formal solutions against the FP64 oracle


@pytest.fixture(scope="module", autouse=True)
def _built():
    Bd.build()
    rt.load()


def _grid(p, **kw):
    return rt.Grid(p["coord"], p["edges"], p["dirs"], p["weights"], inner_bc=p["inner_bc"], precision=rt.RT_MIXED,
                   **kw)


def _oracle(p):
    return O.OracleGrid(p["coord"], p["edges"], p["dirs"], p["weights"], p["inner_bc"])


def _case(name):
    if name == "sph_core":
        p = tiny_problem(I.SPHERICAL, (9, 6, 8), 6, 6, I.CORE_B, seed=51)
    elif name == "cyl_hole":
        p = tiny_problem(I.CYLINDRICAL, (8, 7, 6), 6, 6, I.TRANSPARENT, seed=52)
    else:
        p = I.line_problem("sph17", n_freq=8, ratio=300.0, eps_l=0.1)
        p["nvox"] = p["chi_c"].size
        return p
    n = p["nvox"]
    phi, w = I.line_profile(5, span=2.5)
    chi_c = 0.2 * p["chi"]
    p.update(chi_c=chi_c, chi_l=40.0 * chi_c, eps_l=np.full(n, 0.1), phi=phi, wq=w)
    return p


def _line(p, g, use_lstar=rt.RT_LSTAR_DIAG, ng=False):
    ln = rt.Line(g, p["phi"], p["wq"], use_lstar, ng)
    ln.set(p["chi_c"], p["chi_l"], p["eps_l"], p["B"])
    return ln


@pytest.mark.parametrize("name", ["sph_core", "cyl_hole", "sph17"])
def test_line_iterates_match_oracle(name):
    p = _case(name)
    o = _oracle(p)
    g = _grid(p)
    ln = _line(p, g)
    Lbar_o = OL.line_lbar(o, p["chi_c"], p["chi_l"], p["B"], p["phi"], p["wq"])
    assert np.max(np.abs(ln.Lbar() - Lbar_o) / np.abs(Lbar_o)) < MIXED
    steps = 6
    rel = [ln.step() for _ in range(steps)]
    S_o, _, h_o = OL.line_solve(o, p["chi_c"], p["chi_l"], p["eps_l"], p["B"], p["phi"], p["wq"], tol=0.0,
                                max_iter=steps)
    assert np.max(np.abs(ln.S_l() - S_o) / np.abs(S_o)) < MIXED
    # Jbar of the last iteration is that of the previous iterate
    S_prev, _, _ = OL.line_solve(o, p["chi_c"], p["chi_l"], p["eps_l"], p["B"], p["phi"], p["wq"], tol=0.0,
                                 max_iter=steps - 1)
    Jb_o = OL.line_jbar(o, S_prev, p["chi_c"], p["chi_l"], p["B"], p["phi"], p["wq"])
    assert np.max(np.abs(ln.Jbar() - Jb_o) / np.abs(Jb_o)) < MIXED
    assert np.allclose(rel[:3], h_o[:3], rtol=1e-3, atol=0)
    # member k of the batch is frequency k: its S_k follows from S_l of the step before
    chik = OL.frequency_opacity(p["chi_c"], p["chi_l"], p["phi"])
    k = len(p["phi"]) // 2
    Sk = (p["chi_c"] * p["B"] + p["chi_l"] * p["phi"][k] * S_prev) / chik[k]
    assert np.max(np.abs(ln.S(k) - Sk) / np.abs(Sk)) < MIXED
    ln.close()
    g.close()


def test_line_converges_to_oracle_fixed_point():
    p = _case("sph17")
    o = _oracle(p)
    S_o, it_o, h_o = OL.line_solve(o, p["chi_c"], p["chi_l"], p["eps_l"], p["B"], p["phi"], p["wq"], tol=1e-11,
                                   max_iter=400)
    assert it_o > 0
    tol = 1e-7  # above the FP32 formal solutions' noise
    g = _grid(p)
    ln = _line(p, g)
    it, ok = ln.solve(tol, 400)
    assert ok and it > 1
    # the converged iterate: the FP32 formal solutions' error, amplified by at most 1 / eps_l
    assert np.max(np.abs(ln.S_l() - S_o) / np.abs(S_o)) < 2e-5
    it_o7 = int(np.argmax(h_o < tol)) + 1
    assert abs(it - it_o7) <= max(3, 0.15 * it_o7), (it, it_o7)
    ln.close()
    g.close()


def test_single_frequency_pure_line_is_the_batch_continuum_ali():
    """n_freq = 1, phi = 1 and no continuum: S_k = S_l, chi_k = chi_l and Lbar* is
    the member's Lambda*, so the line iteration is the batch's continuum ALI."""
    p = tiny_problem(I.SPHERICAL, (9, 6, 8), 6, 6, I.CORE_B, seed=53)
    n = p["nvox"]
    eps = np.full(n, 0.05)
    g = _grid(p)
    ln = rt.Line(g, np.ones(1), np.ones(1))
    ln.set(np.zeros(n), p["chi"], eps, p["B"])
    b = rt.Batch([g], [0])
    b.set_member(0, p["chi"], eps, p["B"])
    assert np.array_equal(ln.Lbar(), b.Lstar(0))
    for _ in range(5):
        r_line = ln.step()
        r_batch = b.ali_step()[0]
    assert np.max(np.abs(ln.S_l() - b.S(0)) / np.abs(b.S(0))) < 1e-6
    assert abs(r_line - r_batch) <= 1e-3 * r_batch
    S_o, _, _ = _oracle(p).solve(p["chi"], eps, p["B"], tol=0.0, max_iter=5, ng=False)
    assert np.max(np.abs(ln.S_l() - S_o) / np.abs(S_o)) < MIXED
    b.close()
    ln.close()
    g.close()


def test_full_size_grid_line_iterates_with_few_angles():
    """The paper's 65 x 33 x 65 grid and 32 wavelength points with 2 x 2 solid
    angles (small enough for the oracle): iterates of the line source function."""
    p = I.line_problem("sph65", n_freq=32, ratio=1e3, eps_l=0.05, n_mu=2, n_phi=2)
    o = _oracle(p)
    g = _grid(p)
    ln = _line(p, g)
    for _ in range(3):
        ln.step()
    S_o, _, _ = OL.line_solve(o, p["chi_c"], p["chi_l"], p["eps_l"], p["B"], p["phi"], p["wq"], tol=0.0,
                              max_iter=3)
    assert np.max(np.abs(ln.S_l() - S_o) / np.abs(S_o)) < MIXED
    ln.close()
    g.close()


def test_full_size_thermal_line_is_planck():
    """eps_l = 1: one iteration sets S_l = B whatever Jbar is (one rounding), with
    all 32 x 32 solid angles and 32 frequencies of the paper's line test."""
    p = I.line_problem("sph65", n_freq=32, ratio=1e6, eps_l=1.0)
    g = _grid(p)
    ln = _line(p, g)
    ln.step()
    assert np.max(np.abs(ln.S_l() - p["B"]) / p["B"]) <= 2.3e-16
    Jb = ln.Jbar()
    assert np.all(np.isfinite(Jb)) and np.all(Jb >= 0)
    Lb = ln.Lbar()
    assert np.all(Lb >= 0) and np.all(Lb < 1.0 + 1e-6)
    ln.close()
    g.close()


def test_autotune_restores_the_line_source():
    p = _case("sph_core")
    g = _grid(p)
    ln = _line(p, g)
    for _ in range(2):
        ln.step()
    S_before = ln.S_l()
    ln.autotune()
    assert np.array_equal(ln.S_l(), S_before)
    ln.step()
    ref = _line(p, g)
    for _ in range(3):
        ref.step()
    assert np.max(np.abs(ln.S_l() - ref.S_l()) / np.abs(ref.S_l())) < 1e-6
    ref.close()
    ln.close()
    g.close()


@pytest.mark.parametrize("name", ["sph_core", "cyl_hole", "sph17"])
def test_nn_line_operator_and_iterates_match_oracle(name):
    """Nearest-neighbour line operator (exact, FP64) entry by entry, and the
    iterates of the NN line ALI at the mixed-precision bar."""
    p = _case(name)
    p["eps_l"] = np.full(p["nvox"], 0.05)
    o = _oracle(p)
    g = _grid(p)
    ln = _line(p, g, rt.RT_LSTAR_NN)
    L_o = OL.line_lbar_nn(o, p["chi_c"], p["chi_l"], p["phi"], p["wq"])
    scale = np.max(np.abs(L_o))
    assert np.max(np.abs(ln.Lbar_nn() - L_o)) <= 1e-13 * scale, float(np.max(np.abs(ln.Lbar_nn() - L_o)) / scale)
    steps = 5
    rel = [ln.step() for _ in range(steps)]
    S_o, _, h_o = OL.line_solve(o, p["chi_c"], p["chi_l"], p["eps_l"], p["B"], p["phi"], p["wq"], tol=0.0,
                                max_iter=steps, use_lstar=2)
    assert np.max(np.abs(ln.S_l() - S_o) / np.abs(S_o)) < MIXED
    assert np.allclose(rel[:3], h_o[:3], rtol=1e-3, atol=0)
    ln.close()
    g.close()


def test_nn_line_converges_faster_to_the_same_fixed_point():
    """eps_l = 1e-2 with the line centre at tau ~ 3e2: the NN line operator needs
    a fraction of the diagonal one's iterations (the oracle: 28 against 97 to
    1e-5), to the oracle's fixed point."""
    p = I.line_problem("sph17", n_freq=8, ratio=3e4, eps_l=1e-2)
    o = _oracle(p)
    S_o, it_o, h_o = OL.line_solve(o, p["chi_c"], p["chi_l"], p["eps_l"], p["B"], p["phi"], p["wq"], tol=1e-8,
                                   max_iter=400, use_lstar=2)
    assert it_o > 0
    tol = 1e-5
    it_o5 = int(np.argmax(h_o < tol)) + 1
    g = _grid(p)
    ln = _line(p, g, rt.RT_LSTAR_NN)
    it_nn, ok_nn = ln.solve(tol, 150)
    S_nn = ln.S_l()
    ln.close()
    assert ok_nn, it_nn
    assert abs(it_nn - it_o5) <= max(3, 0.15 * it_o5), (it_nn, it_o5)
    ln = _line(p, g, rt.RT_LSTAR_DIAG)
    it_d, ok_d = ln.solve(tol, 2 * it_nn)
    ln.close()
    assert not ok_d, (it_nn, it_d)
    # within tol of convergence, plus the FP32 formal solutions' error amplified by the OS operator
    assert np.max(np.abs(S_nn - S_o) / np.abs(S_o)) < 2e-4
    g.close()


@pytest.mark.parametrize("lstar", [rt.RT_LSTAR_DIAG, rt.RT_LSTAR_NN])
def test_line_with_ng_matches_oracle(lstar):
    """Ng on S_l (every fourth iterate) step by step against the oracle's."""
    p = _case("sph_core")
    p["eps_l"] = np.full(p["nvox"], 0.02)
    o = _oracle(p)
    g = _grid(p)
    ln = _line(p, g, lstar, ng=True)
    steps = 10
    rel = [ln.step() for _ in range(steps)]
    S_o, _, h_o = OL.line_solve(o, p["chi_c"], p["chi_l"], p["eps_l"], p["B"], p["phi"], p["wq"], tol=0.0,
                                max_iter=steps, use_lstar=2 if lstar == rt.RT_LSTAR_NN else 1, ng=True)
    assert np.max(np.abs(ln.S_l() - S_o) / np.abs(S_o)) < 2e-5
    assert np.allclose(rel[:4], h_o[:4], rtol=1e-3, atol=0)
    ln.close()
    g.close()


def test_line_argument_checks():
    p = _case("sph_core")
    n = p["nvox"]
    g = _grid(p)
    with pytest.raises(rt.RtError) as ei:
        rt.Line(g, p["phi"], 2.0 * p["wq"])  # sum w phi = 2
    assert ei.value.code == rt.RT_EINVAL
    with pytest.raises(rt.RtError):
        rt.Line(g, -p["phi"], p["wq"])
    ln = rt.Line(g, p["phi"], p["wq"])
    with pytest.raises(rt.RtError):
        ln.step()  # not set yet
    with pytest.raises(rt.RtError):
        ln.set(p["chi_c"], p["chi_l"], np.zeros(n), p["B"])  # eps_l = 0
    z = rt.Line(g, np.array([0.0, 1.0]), np.ones(2))  # a frequency outside the line
    with pytest.raises(rt.RtError):
        z.set(np.zeros(n), p["chi_l"], p["eps_l"], p["B"])  # chi_c + chi_l phi_0 = 0
    z.close()
    ln.set(p["chi_c"], p["chi_l"], p["eps_l"], p["B"])
    for call in (lambda: ln.ali_step(), lambda: ln.set_member(0, p["chi"], p["eps"], p["B"]),
                 lambda: rt.rt_line_get(ln.h, 3, 27 * n), lambda: rt.rt_line_get(ln.h, 4, n)):
        with pytest.raises(rt.RtError) as ei:
            call()
        assert ei.value.code == rt.RT_EINVAL
    ln.close()
    with pytest.raises(rt.RtError) as ei:
        rt.Line(g, p["phi"], p["wq"], use_lstar=rt.RT_LSTAR_NONE)
    assert ei.value.code == rt.RT_EINVAL
    with pytest.raises(rt.RtError) as ei:
        rt.rt_line_create(g.h, p["phi"], p["wq"], rt.RT_LSTAR_DIAG, 2)
    assert ei.value.code == rt.RT_EINVAL
    g.close()
