"""Pins of the oracle's two-level-atom line transfer (oracle/line.py): the
frequency-averaged line ALI against the continuum ALI it reduces to, the
thermal limit, and the dense solve of its linear fixed point."""
import numpy as np
import pytest

from oracle import line as OL
from oracle import oracle as O
from paper_0903_1949_gb300 import inputs as I
from tests.helpers import tiny_problem


def grid(p):
    return O.OracleGrid(p["coord"], p["edges"], p["dirs"], p["weights"], p["inner_bc"])


def test_single_frequency_pure_line_is_the_continuum_ali():
    """n_freq = 1, phi = 1, no continuum: S_k = S_l and chi_k = chi_l, so the line ALI
    is the continuum ALI of chi_l with eps = eps_l, iterate by iterate."""
    p = tiny_problem(I.SPHERICAL, (5, 4, 6), 4, 4, I.CORE_B, seed=41)
    o = grid(p)
    n = p["nvox"]
    eps = np.full(n, 0.05)
    S_line, it, h_line = OL.line_solve(o, np.zeros(n), p["chi"], eps, p["B"], np.ones(1), np.ones(1), tol=0.0,
                                       max_iter=5)
    S_cont, _, h_cont = o.solve(p["chi"], eps, p["B"], tol=0.0, max_iter=5, ng=False)
    assert np.max(np.abs(S_line - S_cont) / np.abs(S_cont)) < 1e-14
    assert np.allclose(h_line, h_cont, rtol=1e-12, atol=0)


def test_thermal_line_is_planck_after_one_step():
    p = tiny_problem(I.SPHERICAL, (5, 4, 6), 4, 4, I.CORE_B, seed=42)
    o = grid(p)
    n = p["nvox"]
    phi, w = I.line_profile(5)
    chi_c = 0.1 * p["chi"]
    S0 = p["B"] * np.random.default_rng(1).uniform(0.5, 1.5, n)
    S, it, _ = OL.line_solve(o, chi_c, 1e3 * chi_c, np.ones(n), p["B"], phi, w, tol=0.0, max_iter=1, S0=S0)
    assert np.max(np.abs(S - p["B"]) / p["B"]) <= 1e-15  # S + (B - S): one rounding at most


@pytest.mark.parametrize("coord,bc", [(I.SPHERICAL, I.CORE_B), (I.CYLINDRICAL, I.TRANSPARENT)])
def test_converged_line_equals_dense_solve(coord, bc):
    """Jbar is affine in S_l: Jbar = M S_l + c with M = sum_k w_k phi_k Lambda_k
    diag(chi_l phi_k / chi_k), c from the continuum part and the boundaries; the
    converged S_l solves (I - (1 - eps_l) M) S_l = eps_l B + (1 - eps_l) c."""
    n3 = (5, 4, 6) if coord == I.SPHERICAL else (4, 5, 3)
    p = tiny_problem(coord, n3, 4, 4, bc, seed=43)
    o = grid(p)
    n = p["nvox"]
    phi, w = I.line_profile(3, span=2.0)
    chi_c = 0.2 * p["chi"]
    chi_l = 30.0 * chi_c
    eps = np.full(n, 0.1)
    B = p["B"]
    chik = OL.frequency_opacity(chi_c, chi_l, phi)
    M = np.zeros((n, n))
    c = np.zeros(n)
    for k in range(len(phi)):
        Lam = np.empty((n, n))
        for u in range(n):
            e = np.zeros(n)
            e[u] = 1.0
            Lam[:, u] = o.formal_solution(e, chik[k], B, homog=True)[0]
        b = chi_l * phi[k] / chik[k]
        M += w[k] * phi[k] * Lam * b[None, :]
        a = chi_c / chik[k]
        Jbc = o.formal_solution(np.zeros(n), chik[k], B)[0]
        c += w[k] * phi[k] * (Lam @ (a * B) + Jbc)
    S_direct = np.linalg.solve(np.eye(n) - (1.0 - eps)[:, None] * M, eps * B + (1.0 - eps) * c)
    S, it, _ = OL.line_solve(o, chi_c, chi_l, eps, B, phi, w, tol=1e-14, max_iter=3000)
    assert it > 0
    assert np.max(np.abs(S - S_direct) / np.abs(S_direct)) < 1e-11


def test_profile_quadrature_is_normalised():
    for nf in (1, 3, 32):
        phi, w = I.line_profile(nf)
        assert abs(np.sum(w * phi) - 1.0) < 1e-14


def _line_matrix(o, chi_c, chi_l, B, phi, w):
    """The exact line operator dJbar / dS_l (dense, from unit-vector formal solutions)."""
    n = o.nvox
    chik = OL.frequency_opacity(chi_c, chi_l, phi)
    M = np.zeros((n, n))
    for k in range(len(phi)):
        Lam = np.empty((n, n))
        for u in range(n):
            e = np.zeros(n)
            e[u] = 1.0
            Lam[:, u] = o.formal_solution(e, chik[k], B, homog=True)[0]
        M += w[k] * phi[k] * Lam * (chi_l * phi[k] / chik[k])[None, :]
    return M


@pytest.mark.parametrize("coord,bc", [(I.SPHERICAL, I.CORE_B), (I.CYLINDRICAL, I.TRANSPARENT)])
def test_nn_line_operator_is_the_exact_operator_on_the_neighbourhood(coord, bc):
    """Lbar*_NN[v, q] is dJbar_v / dS_l,u for the voxel u in slot q, with the
    chi_l phi_k / chi_k factor of u (a factor taken at v fails where chi varies)."""
    n3 = (5, 4, 6) if coord == I.SPHERICAL else (4, 5, 3)
    p = tiny_problem(coord, n3, 4, 4, bc, seed=44)
    o = grid(p)
    phi, w = I.line_profile(3, span=2.0)
    chi_c = 0.2 * p["chi"]
    chi_l = 30.0 * chi_c * np.random.default_rng(5).uniform(0.5, 2.0, p["nvox"])
    M = _line_matrix(o, chi_c, chi_l, p["B"], phi, w)
    L27 = OL.line_lbar_nn(o, chi_c, chi_l, phi, w)
    nb = OL.nn_neighbours(o)
    exp = np.where(nb >= 0, M[np.arange(o.nvox)[:, None], np.maximum(nb, 0)], 0.0)
    assert np.max(np.abs(L27 - exp)) <= 1e-13 * np.max(np.abs(M))
    # every entry of M outside the neighbourhoods is left out, none inside is
    inside = np.zeros_like(M, dtype=bool)
    inside[np.arange(o.nvox)[:, None].repeat(27, 1)[nb >= 0], nb[nb >= 0]] = True
    assert np.isclose(np.abs(M[inside]).sum(), np.abs(L27).sum(), rtol=1e-12)


def test_nn_line_reaches_the_dense_fixed_point_faster():
    p = tiny_problem(I.SPHERICAL, (5, 4, 6), 4, 4, I.CORE_B, seed=45)
    o = grid(p)
    n = p["nvox"]
    phi, w = I.line_profile(3, span=2.0)
    chi_c = 0.05 * p["chi"]
    chi_l = 400.0 * chi_c
    eps = np.full(n, 1e-3)
    B = p["B"]
    S_d, it_d, _ = OL.line_solve(o, chi_c, chi_l, eps, B, phi, w, tol=1e-12, max_iter=5000, use_lstar=1)
    S_n, it_n, _ = OL.line_solve(o, chi_c, chi_l, eps, B, phi, w, tol=1e-12, max_iter=5000, use_lstar=2)
    assert it_d > 0 and 0 < it_n < it_d / 2, (it_n, it_d)
    assert np.max(np.abs(S_n - S_d) / np.abs(S_d)) < 1e-9


def test_single_frequency_nn_line_is_the_continuum_nn_ali():
    p = tiny_problem(I.CYLINDRICAL, (4, 5, 3), 4, 4, I.TRANSPARENT, seed=46)
    o = grid(p)
    n = p["nvox"]
    eps = np.full(n, 0.01)
    S_line, _, h_line = OL.line_solve(o, np.zeros(n), p["chi"], eps, p["B"], np.ones(1), np.ones(1), tol=0.0,
                                      max_iter=4, use_lstar=2)
    S_cont, _, h_cont = o.solve(p["chi"], eps, p["B"], tol=0.0, max_iter=4, use_lstar=2, ng=False)
    assert np.max(np.abs(S_line - S_cont) / np.abs(S_cont)) < 1e-14
    assert np.allclose(h_line, h_cont, rtol=1e-12, atol=0)


def test_single_frequency_line_with_ng_is_the_continuum_ali_with_ng():
    """Ng on S_l follows the continuum solve's Ng step for step (n_freq = 1, no continuum)."""
    p = tiny_problem(I.SPHERICAL, (5, 4, 6), 4, 4, I.CORE_B, seed=47)
    o = grid(p)
    n = p["nvox"]
    eps = np.full(n, 0.01)
    for lstar in (1, 2):
        S_line, _, h_line = OL.line_solve(o, np.zeros(n), p["chi"], eps, p["B"], np.ones(1), np.ones(1), tol=0.0,
                                          max_iter=10, use_lstar=lstar, ng=True)
        S_cont, _, h_cont = o.solve(p["chi"], eps, p["B"], tol=0.0, max_iter=10, use_lstar=lstar, ng=True)
        assert np.max(np.abs(S_line - S_cont) / np.abs(S_cont)) < 1e-13, lstar
        assert np.allclose(h_line, h_cont, rtol=1e-6, atol=0)  # late dS: differences of near-equal S


def test_ng_line_reaches_the_same_fixed_point_in_fewer_iterations():
    p = tiny_problem(I.CYLINDRICAL, (4, 5, 3), 4, 4, I.TRANSPARENT, seed=48)
    o = grid(p)
    n = p["nvox"]
    phi, w = I.line_profile(3, span=2.0)
    chi_c = 0.05 * p["chi"]
    chi_l = 400.0 * chi_c
    eps = np.full(n, 1e-3)
    S0, it0, _ = OL.line_solve(o, chi_c, chi_l, eps, p["B"], phi, w, tol=1e-12, max_iter=5000, use_lstar=1)
    S1, it1, _ = OL.line_solve(o, chi_c, chi_l, eps, p["B"], phi, w, tol=1e-12, max_iter=5000, use_lstar=1, ng=True)
    assert 0 < it1 < it0 / 2, (it1, it0)
    assert np.max(np.abs(S1 - S0) / np.abs(S0)) < 1e-9
