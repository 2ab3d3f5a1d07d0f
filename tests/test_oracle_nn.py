"""Pins of the oracle's nearest-neighbour Lambda* (3^3 neighbour voxels built
exactly, Sect. 2 and 3.2.1) and of its operator-splitting step.

The reference is the Lambda matrix itself, column by column: column u is J of
a homogeneous formal solution (no incoming intensity) with S = e_u, so the
pins need nothing of the NN construction (which tracks derivatives along the
characteristics instead)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_0903_1949_gb300 import inputs as I
from tests.helpers import tiny_problem

CASES = {
    "sph_core": lambda: (tiny_problem(I.SPHERICAL, (5, 4, 6), 4, 4, I.CORE_B, seed=31), O.PARABOLIC),
    "sph_hole": lambda: (tiny_problem(I.SPHERICAL, (4, 5, 5), 4, 4, I.TRANSPARENT, seed=32), O.PARABOLIC),
    "cyl_hole": lambda: (tiny_problem(I.CYLINDRICAL, (5, 6, 4), 4, 4, I.TRANSPARENT, seed=33), O.PARABOLIC),
    "sph_linear": lambda: (tiny_problem(I.SPHERICAL, (5, 4, 6), 4, 4, I.CORE_B, seed=34), O.LINEAR),
}


def grid(p, interp):
    return O.OracleGrid(p["coord"], p["edges"], p["dirs"], p["weights"], p["inner_bc"], interp=interp)


def lambda_matrix(o, p):
    n = p["nvox"]
    Lam = np.empty((n, n))
    for u in range(n):
        e = np.zeros(n)
        e[u] = 1.0
        J, _, _, miss = o.formal_solution(e, p["chi"], p["B"], homog=True)
        assert miss == 0
        Lam[:, u] = J
    return Lam


def neighbour(p, v, q):
    """Voxel at offset (q // 9 - 1, (q // 3) % 3 - 1, q % 3 - 1) of v, phi periodic; None outside."""
    n1, n2, n3 = p["n"]
    i, j, k = v // (n2 * n3), (v // n3) % n2, v % n3
    i, j, k = i + q // 9 - 1, j + (q // 3) % 3 - 1, k + q % 3 - 1
    if p["coord"] == I.SPHERICAL:
        k %= n3
    else:
        j %= n2
    if not (0 <= i < n1 and 0 <= j < n2 and 0 <= k < n3):
        return None
    return (i * n2 + j) * n3 + k


@pytest.mark.parametrize("name", sorted(CASES))
def test_nn_lstar_equals_lambda_matrix_on_neighbours(name):
    p, interp = CASES[name]()
    o = grid(p, interp)
    L27 = o.nn_lstar(p["chi"])
    Lam = lambda_matrix(o, p)
    scale = np.max(np.abs(Lam))
    for v in range(p["nvox"]):
        for q in range(27):
            u = neighbour(p, v, q)
            if u is None:
                assert L27[v, q] == 0.0
            else:
                assert abs(L27[v, q] - Lam[v, u]) <= 1e-13 * scale, (v, q, L27[v, q], Lam[v, u])
    # the neighbourhood carries most of every row, never more than all of it
    rows = Lam.sum(axis=1)
    assert np.all(L27.sum(axis=1) <= rows + 1e-13)


@pytest.mark.parametrize("name", ["sph_core", "cyl_hole"])
def test_nn_ali_converges_to_direct_solution(name):
    p, interp = CASES[name]()
    o = grid(p, interp)
    eps = np.full(p["nvox"], 1e-3)
    Lam = lambda_matrix(o, p)
    Jbc, _, _, _ = o.formal_solution(np.zeros(p["nvox"]), p["chi"], p["B"])
    A = np.eye(p["nvox"]) - (1.0 - eps)[:, None] * Lam
    S_direct = np.linalg.solve(A, eps * p["B"] + (1.0 - eps) * Jbc)
    S, it, hist = o.solve(p["chi"], eps, p["B"], tol=1e-14, max_iter=500, use_lstar=2, ng=False)
    assert it > 0
    assert np.max(np.abs(S - S_direct) / np.abs(S_direct)) < 1e-11


def test_nn_update_solves_its_banded_system():
    p, interp = CASES["sph_core"]()
    o = grid(p, interp)
    n = p["nvox"]
    eps = np.full(n, 0.05)
    L27 = o.nn_lstar(p["chi"])
    S = p["B"] * np.random.default_rng(5).uniform(0.5, 1.5, n)
    J, _, _, _ = o.formal_solution(S, p["chi"], p["B"])
    S_new, rel, sweeps = o.nn_ali_update(S, J, L27, eps, p["B"])
    assert sweeps > 1
    M = np.zeros((n, n))
    for v in range(n):
        for q in range(27):
            u = neighbour(p, v, q)
            if u is not None:
                M[v, u] = L27[v, q]
    dS = np.linalg.solve(np.eye(n) - (1.0 - eps)[:, None] * M, (1.0 - eps) * J + eps * p["B"] - S)
    assert np.max(np.abs(S_new - (S + dS)) / np.abs(S + dS)) < 1e-12
    assert abs(rel - np.max(np.abs(dS) / np.abs(S + dS))) < 1e-12


def test_nn_update_reports_sweeps_that_do_not_contract():
    """The OS step is defined by its linear system (Sect. 3.2.1); Jacobi sweeps only
    reach it when they contract.  With the off-diagonal weights scaled up until the
    sweep matrix has spectral radius > 1 (the system stays regular) the sweeps blow
    up: the update must say so (NaN) and leave S alone, not stop on a test that an
    infinite max |dS| passes."""
    p, interp = CASES["sph_core"]()
    o = grid(p, interp)
    n = p["nvox"]
    eps = np.full(n, 0.05)
    L27 = o.nn_lstar(p["chi"])
    L27[:, [q for q in range(27) if q != 13]] *= 40.0
    S = p["B"] * np.random.default_rng(6).uniform(0.5, 1.5, n)
    J, _, _, _ = o.formal_solution(S, p["chi"], p["B"])
    M = np.zeros((n, n))
    for v in range(n):
        for q in range(27):
            u = neighbour(p, v, q)
            if u is not None and q != 13:
                M[v, u] = L27[v, q]
    d = 1.0 - (1.0 - eps) * L27[:, 13]
    G = ((1.0 - eps) / d)[:, None] * M
    assert np.max(np.abs(np.linalg.eigvals(G))) > 1.0
    A = np.eye(n) - (1.0 - eps)[:, None] * (M + np.diag(L27[:, 13]))
    assert np.linalg.cond(A) < 1e12
    S_new, rel, sweeps = o.nn_ali_update(S, J, L27, eps, p["B"])
    assert np.isnan(rel) and sweeps > 1
    assert np.array_equal(S_new, S)


def test_nn_without_ng_beats_diagonal_with_ng():
    """The paper's convergence statement for the 3D case (Sect. 3.2.1): the local
    (diagonal) Lambda* with Ng converges more slowly than the nearest-neighbour one
    without Ng."""
    p = I.make_problem("sph17", eps=1e-3, tau=10.0)
    o = O.OracleGrid(p["coord"], p["edges"], p["dirs"], p["weights"], p["inner_bc"])
    _, it_nn, _ = o.solve(p["chi"], p["eps"], p["B"], tol=1e-6, max_iter=2000, use_lstar=2, ng=False)
    _, it_dg, _ = o.solve(p["chi"], p["eps"], p["B"], tol=1e-6, max_iter=2000, use_lstar=1, ng=True)
    assert 0 < it_nn < it_dg, (it_nn, it_dg)
