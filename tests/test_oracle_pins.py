"""Pins of the FP64 CPU oracle against facts that do not come from the oracle.

P1 interpolation weights vs. high-precision quadrature of polynomial source
   functions; P2 homogeneous sphere / cylinder closed forms; P3 geometry
   (chord lengths, adjacency, coverage, brute-force point location);
P4 angle quadrature moments; P5 constant-S invariance; P6 linearity and the
   exact diagonal of the dense Lambda matrix; P7 converged ALI equals the direct
   solve; P8 Ng on a linear iteration with a known fixed point.
"""
import json
import math
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_0903_1949_gb300 import inputs as I
from tests.helpers import centre, domain_intervals, locate_points, runs, tiny_problem

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def og(p, I_outer=0.0, interp=O.PARABOLIC):
    return O.OracleGrid(p["coord"], p["edges"], p["dirs"], p["weights"], p["inner_bc"], I_outer, interp)


# ---------------------------------------------------------------- P1 -------

def _exact_integral(mp, dm, poly):
    """int_0^dm S(u) exp(-(dm-u)) du at 40 digits for S(u) = sum poly[n] u^n."""
    dm = mp.mpf(dm)
    f = lambda u: (poly[0] + poly[1] * u + poly[2] * u * u) * mp.exp(u - dm)
    a = dm - 90 if dm > 90 else mp.mpf(0)
    return mp.quad(f, [a, dm]) if a > 0 else mp.quad(f, [0, dm])


def test_p1_parabolic_weights_exact_for_quadratics():
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    rng = np.random.default_rng(11)
    for _ in range(60):
        dm = 10.0 ** rng.uniform(-8, 4)
        dp = dm * rng.uniform(0.5, 20.0)
        D = dm + dp
        c = rng.uniform(0.1, 1.0, 3)
        poly = [mp.mpf(c[0]), mp.mpf(c[1]) / D, mp.mpf(c[2]) / (D * D)]
        S = [float(poly[0] + poly[1] * u + poly[2] * u * u) for u in (mp.mpf(0), mp.mpf(dm), mp.mpf(dm) + mp.mpf(dp))]
        a, b, g = O.coeffs(dm, dp, True)
        got = a * S[0] + b * S[1] + g * S[2]
        ref = float(_exact_integral(mp, dm, poly))
        assert abs(got - ref) <= 2e-13 * abs(ref), (dm, dp, got, ref)
        # weights sum to 1 - exp(-dm) (constant S is integrated exactly)
        assert abs((a + b + g) - (-math.expm1(-dm))) <= 1e-14 * (-math.expm1(-dm))


def test_p1_linear_weights_exact_for_lines():
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    rng = np.random.default_rng(12)
    for _ in range(40):
        dm = 10.0 ** rng.uniform(-8, 4)
        c = rng.uniform(0.1, 1.0, 2)
        poly = [mp.mpf(c[0]), mp.mpf(c[1]) / dm, mp.mpf(0)]
        a, b, g = O.coeffs(dm, 0.0, False)
        assert g == 0.0
        got = a * float(poly[0]) + b * float(poly[0] + poly[1] * dm)
        ref = float(_exact_integral(mp, dm, poly))
        assert abs(got - ref) <= 2e-13 * abs(ref)


# ---------------------------------------------------------------- P3 -------

def _check_geometry(p, angles, n_brute=0, seed=0):
    g = og(p)
    nv = p["nvox"]
    n1, n2, n3 = p["n"]
    rng = np.random.default_rng(seed)
    core_b = p["inner_bc"] == I.CORE_B
    for w in angles:
        A = g.angle(w)
        d = p["dirs"][w]
        assert A["n_lost"] == 0
        # every voxel is hit at least once per solid angle (Sect. 2)
        assert np.all(np.bincount(A["vox"], minlength=nv) >= 1)
        assert np.all(A["len"] > 0)
        off = A["ray_off"]
        for r in range(len(A["ray_origin"])):
            s0, s1 = off[r], off[r + 1]
            vox = A["vox"][s0:s1]
            # consecutive voxels are neighbours (face, or edge/corner on exact ties)
            ii, jj, kk = vox // (n2 * n3), (vox // n3) % n2, vox % n3
            rs = A["restart"][s0 + 1:s1].astype(bool)
            di = np.abs(np.diff(ii))
            if p["coord"] == I.SPHERICAL:
                dj = np.abs(np.diff(jj))
                dk = np.minimum(np.abs(np.diff(kk)), n3 - np.abs(np.diff(kk)))
            else:
                dj = np.minimum(np.abs(np.diff(jj)), n2 - np.abs(np.diff(jj)))
                dk = np.abs(np.diff(kk))
            step = np.maximum(np.maximum(di, dj), dk)
            assert np.all(step[~rs] == 1), (w, r)
            # total path length equals the analytic chord through the domain
            x0 = centre(p["coord"], p["edges"], A["ray_origin"][r])
            lo, hi, hole = domain_intervals(p["coord"], p["edges"], x0, d, core_b)
            L = A["len"][s0:s1].sum()
            scale = p["edges"][0][-1]
            assert abs(L - (hi - lo - hole)) <= 1e-12 * scale, (w, r, L, hi - lo - hole)
        # brute force: sample the line densely and locate each sample directly
        for r in rng.choice(len(A["ray_origin"]), size=min(n_brute, len(A["ray_origin"])), replace=False):
            s0, s1 = off[r], off[r + 1]
            x0 = centre(p["coord"], p["edges"], A["ray_origin"][r])
            lo, hi, _ = domain_intervals(p["coord"], p["edges"], x0, d, core_b)
            N = 40000
            h = (hi - lo) / N
            t = lo + h * (np.arange(N) + 0.5)
            ids = locate_points(p["coord"], p["edges"], x0[None, :] + t[:, None] * d[None, :])
            # a segment of length l holds floor(l/h) or ceil(l/h) samples: pick a cut T
            # with no segment length within 2h of it so both sides drop the same slivers
            lens = A["len"][s0:s1]
            T = 4.0 * h
            while np.any(np.abs(lens - T) <= 2.0 * h):
                T *= 1.37
            ref = runs(ids, np.full(N, h), T)
            got = runs(A["vox"][s0:s1], lens, T)
            assert got == ref, (w, r)


def test_p3_geometry_spherical_core():
    p = tiny_problem(I.SPHERICAL, (7, 5, 9), 4, 4, I.CORE_B)
    _check_geometry(p, range(p["n_ang"]), n_brute=6)


def test_p3_geometry_spherical_transparent():
    p = tiny_problem(I.SPHERICAL, (6, 7, 5), 4, 4, I.TRANSPARENT)
    _check_geometry(p, range(p["n_ang"]), n_brute=6, seed=1)


def test_p3_geometry_cylindrical_hole():
    p = tiny_problem(I.CYLINDRICAL, (6, 7, 5), 4, 4, I.TRANSPARENT)
    _check_geometry(p, range(p["n_ang"]), n_brute=6, seed=2)


def test_p3_geometry_cylindrical_core_and_axis():
    p = tiny_problem(I.CYLINDRICAL, (5, 9, 6), 4, 6, I.CORE_B)
    _check_geometry(p, range(p["n_ang"]), n_brute=4, seed=3)
    q = tiny_problem(I.CYLINDRICAL, (5, 7, 4), 4, 4, I.TRANSPARENT, R_min=0.0)
    _check_geometry(q, range(q["n_ang"]), n_brute=4, seed=4)


def test_p3_geometry_paper_grid_sampled_angles():
    p = I.make_problem("sph17")
    p["nvox"] = int(np.prod(p["n"]))
    _check_geometry(p, [0, 13, 37, 63], n_brute=4, seed=5)


# ---------------------------------------------------------------- P2 -------

@pytest.mark.parametrize("coord,bc", [(I.SPHERICAL, I.CORE_B), (I.SPHERICAL, I.TRANSPARENT),
                                      (I.CYLINDRICAL, I.TRANSPARENT), (I.CYLINDRICAL, I.CORE_B)])
def test_p2_homogeneous_closed_form(coord, bc):
    chi, Sc, Bc = 0.7, 2.0, 1.0
    p = tiny_problem(coord, (6, 5, 7), 4, 4, bc, chi=chi, B=Bc)
    g = og(p)
    S = np.full(p["nvox"], Sc)
    for w in range(p["n_ang"]):
        A = g.angle(w)
        _, _, Iex, miss = g.fs_angle(w, S, p["chi"], p["B"])
        assert miss == 0
        d = p["dirs"][w]
        for r in range(len(A["ray_origin"])):
            x0 = centre(coord, p["edges"], A["ray_origin"][r])
            lo, hi, hole = domain_intervals(coord, p["edges"], x0, d, bc == I.CORE_B)
            tau = chi * (hi - lo - hole)
            I_in = Bc if A["ray_core"][r] else 0.0
            ref = I_in * math.exp(-tau) - Sc * math.expm1(-tau)
            assert abs(Iex[r] - ref) <= 1e-13 * ref, (w, r, Iex[r], ref)


# ---------------------------------------------------------------- P4 -------

def test_p4_angle_moments():
    for n in (2, 4, 8, 32, 64):
        dirs, w = I.angle_set(n, n)
        assert abs(w.sum() - 1.0) < 1e-15
        assert abs((w * dirs[:, 2] ** 2).sum() - 1.0 / 3.0) < 1e-15
        assert np.all(np.abs(w @ dirs) < 1e-15)
        assert np.max(np.abs((dirs ** 2).sum(1) - 1.0)) <= 8.9e-16


def test_paper_grid_facts():
    fx = json.load(open(os.path.join(GOLDEN, "paper_grid_facts.json")))
    e = I.sph_edges(*fx["n_voxels"])
    assert [len(a) - 1 for a in e] == fx["n_voxels"]
    dth, dph = np.degrees(np.diff(e[1])), np.degrees(np.diff(e[2]))
    assert np.allclose(dth, dth[0]) and np.allclose(dph, dph[0])
    assert abs(dth[0] - fx["angular_resolution_deg"]) < 0.1
    assert abs(dph[0] - fx["angular_resolution_deg"]) < 0.1
    per_shell = fx["n_voxels"][1] * fx["n_voxels"][2]
    europe = per_shell * fx["europe_area_km2"] / fx["earth_area_km2"]
    assert round(europe) == fx["europe_voxels"]


# ---------------------------------------------------------------- P5 -------

@pytest.mark.parametrize("coord,bc", [(I.SPHERICAL, I.CORE_B), (I.CYLINDRICAL, I.TRANSPARENT),
                                      (I.SPHERICAL, I.TRANSPARENT)])
def test_p5_constant_source_is_invariant(coord, bc):
    Sc = 1.7
    p = tiny_problem(coord, (6, 5, 7), 4, 4, bc, B=Sc)
    g = og(p, I_outer=Sc)
    S = np.full(p["nvox"], Sc)
    J, L, F, miss = g.formal_solution(S, p["chi"], p["B"])
    assert miss == 0
    assert np.max(np.abs(J - Sc)) <= 1e-14 * Sc * 4
    # no net flux in an isotropic radiation field (quadrature is symmetric)
    assert np.max(np.abs(F)) <= 1e-13 * Sc


def test_p5_thick_interior_J_equals_S():
    p = I.make_problem("sph17", tau=1e5)
    g = og(p)
    rng = np.random.default_rng(3)
    S = 1.0 + 0.0 * rng.uniform(size=p["chi"].size)
    J, _, _, _ = g.formal_solution(S, p["chi"], p["B"])
    n1, n2, n3 = p["n"]
    J = J.reshape(n1, n2, n3)
    # innermost shells are optically very deep (tau ~ 1e5): J -> S
    assert np.max(np.abs(J[:6] - 1.0)) < 1e-6


# ---------------------------------------------------------------- P6/P7 ----

def _dense_lambda(g, p):
    nv = p["nvox"]
    Lam = np.zeros((nv, nv))
    zero = np.zeros(nv)
    for v in range(nv):
        e = np.zeros(nv)
        e[v] = 1.0
        J, _, _, _ = g.formal_solution(e, p["chi"], zero, homog=True)
        Lam[:, v] = J
    Jbc, _, _, _ = g.formal_solution(zero, p["chi"], p["B"])
    return Lam, Jbc


def _reentered(g, p):
    """Voxels visited twice by the same characteristic in some solid angle."""
    bad = np.zeros(p["nvox"], bool)
    for w in range(p["n_ang"]):
        A = g.angle(w)
        off = A["ray_off"]
        for r in range(len(A["ray_origin"])):
            vv = A["vox"][off[r]:off[r + 1]]
            u, c = np.unique(vv, return_counts=True)
            bad[u[c > 1]] = True
    return bad


@pytest.mark.parametrize("coord,bc,interp", [(I.SPHERICAL, I.CORE_B, O.PARABOLIC),
                                             (I.CYLINDRICAL, I.TRANSPARENT, O.PARABOLIC),
                                             (I.SPHERICAL, I.CORE_B, O.LINEAR)])
def test_p6_linearity_and_exact_diagonal(coord, bc, interp):
    p = tiny_problem(coord, (4, 3, 5), 2, 4, bc)
    g = og(p, interp=interp)
    Lam, Jbc = _dense_lambda(g, p)
    rng = np.random.default_rng(5)
    S = rng.uniform(0.5, 2.0, p["nvox"])
    J, Lst, _, _ = g.formal_solution(S, p["chi"], p["B"])
    assert np.max(np.abs(J - (Lam @ S + Jbc))) <= 1e-13 * np.max(np.abs(J))
    bad = _reentered(g, p)
    assert (~bad).sum() > p["nvox"] // 2
    diag = np.diag(Lam)
    assert np.max(np.abs(Lst[~bad] - diag[~bad])) <= 1e-14
    # Lambda* never exceeds the true diagonal by more than rounding where voxels are re-entered
    assert np.all(Lst[bad] <= diag[bad] + 1e-14)


@pytest.mark.parametrize("coord,bc", [(I.SPHERICAL, I.CORE_B), (I.CYLINDRICAL, I.TRANSPARENT)])
def test_p7_converged_ali_equals_direct_solve(coord, bc):
    p = tiny_problem(coord, (4, 3, 5), 2, 4, bc, eps=0.05)
    g = og(p)
    Lam, Jbc = _dense_lambda(g, p)
    e = p["eps"]
    A = np.eye(p["nvox"]) - (1.0 - e)[:, None] * Lam
    S_direct = np.linalg.solve(A, e * p["B"] + (1.0 - e) * Jbc)
    for use_lstar, ng in ((True, True), (True, False), (False, True)):
        S, it, hist = g.solve(p["chi"], p["eps"], p["B"], tol=1e-14, max_iter=3000, use_lstar=use_lstar, ng=ng)
        assert it > 0, (use_lstar, ng, hist[-3:])
        assert np.max(np.abs(S - S_direct) / S_direct) < 1e-10, (use_lstar, ng)


# ---------------------------------------------------------------- P8 -------

def test_p8_ng_exact_on_two_mode_linear_iteration():
    rng = np.random.default_rng(9)
    n = 50
    xstar = rng.uniform(1.0, 2.0, n)
    u, v = rng.standard_normal(n), rng.standard_normal(n)
    it = [xstar + 0.3 * (0.9 ** k) * u + 0.2 * (0.5 ** k) * v for k in range(4)]
    out = O.ng(it[3], it[2], it[1], it[0])
    assert out is not None
    assert np.max(np.abs(out - xstar)) < 1e-9
    # and it beats the newest iterate by orders of magnitude
    assert np.max(np.abs(out - xstar)) < 1e-6 * np.max(np.abs(it[3] - xstar))


def test_p8_ng_reduces_iterations():
    p = tiny_problem(I.SPHERICAL, (6, 5, 7), 4, 4, I.CORE_B, eps=1e-3, chi=3.0)
    g = og(p)
    _, it_ng, _ = g.solve(p["chi"], p["eps"], p["B"], tol=1e-10, max_iter=4000, ng=True)
    _, it_plain, _ = g.solve(p["chi"], p["eps"], p["B"], tol=1e-10, max_iter=4000, ng=False)
    assert 0 < it_ng < it_plain
