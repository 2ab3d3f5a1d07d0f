"""Physics pins of the oracle that hold only up to discretisation error.

P9  spherically symmetric input: the (theta_c, phi_c) scatter of J per shell
    falls as the solid-angle set is refined (Sect. 3.2.1, solid-angle tests).
P10 shell-mean J of the 3D formal solution converges to an exact 1D p-z
    integration of the same shell-constant S and chi as the grid and the
    solid-angle set are refined together (Sect. 3.2.1, 1D comparison).
P11 pure scattering: r^2 F_r becomes constant across shells and the
    tangential flux components fall relative to F_r as the resolution grows
    (Sect. 3.2.2, flux vectors of the outermost voxels).
"""
import numpy as np

from oracle import oracle as O
from paper_0903_1949_gb300 import inputs as I


def _shell_problem(nr, nth, nph):
    edges = I.sph_edges(nr, nth, nph, 1.0, 10.0)
    rm = 0.5 * (edges[0][:-1] + edges[0][1:])
    return edges, rm


def _j1d(edges, Sh, chih, r, B_core):
    """Exact 1D mean intensity at radius r: Gauss-Legendre in mu split at the tangent kinks."""
    mu, wm = np.polynomial.legendre.leggauss(200)
    kinks = [-1.0, 1.0]
    for e in edges[0]:
        if e < r:
            s = np.sqrt(1.0 - (e / r) ** 2)
            kinks += [-s, s]
    kinks = sorted(set(kinks))
    tot = 0.0
    for a, b in zip(kinks[:-1], kinks[1:]):
        m = 0.5 * (b - a) * mu + 0.5 * (a + b)
        tot += 0.5 * (b - a) * sum(wi * O.pz_intensity(edges[0], Sh, chih, r, mi, True, B_core)
                                   for wi, mi in zip(wm, m))
    return 0.5 * tot


def _p10_error(nr, nth, nph, nang):
    edges, rm = _shell_problem(nr, nth, nph)
    dirs, w = I.angle_set(nang, nang)
    g = O.OracleGrid(I.SPHERICAL, edges, dirs, w, I.CORE_B)
    Sh = 1.0 + 0.5 * np.sin(rm)
    chih = 0.5 / rm
    per = nth * nph
    J, _, _, miss = g.formal_solution(np.repeat(Sh, per), np.repeat(chih, per), np.full(nr * per, 2.0))
    assert miss == 0
    J = J.reshape(nr, per)
    J1 = np.array([_j1d(edges, Sh, chih, r, 2.0) for r in rm])
    return np.max(np.abs(J.mean(1) / J1 - 1.0)), np.max(J.std(1) / J.mean(1))


def test_p10_converges_to_1d_pz_solution():
    e1, s1 = _p10_error(8, 5, 9, 4)
    e2, s2 = _p10_error(16, 9, 17, 8)
    # first-order convergence of the voxel-node discretisation
    assert e2 < 0.6 * e1
    assert e2 < 0.15


def test_p9_angular_scatter_falls_with_solid_angles():
    edges, rm = _shell_problem(8, 9, 17)
    per = 9 * 17
    Sh = np.repeat(1.0 + 0.5 * np.sin(rm), per)
    chi = np.repeat(0.5 / rm, per)
    B = np.full(8 * per, 2.0)
    scat = []
    for n in (2, 4, 8):
        dirs, w = I.angle_set(n, n)
        g = O.OracleGrid(I.SPHERICAL, edges, dirs, w, I.CORE_B)
        J, _, _, _ = g.formal_solution(Sh, chi, B)
        J = J.reshape(8, per)
        scat.append(np.max(J.std(1) / J.mean(1)))
    assert scat[0] > scat[1] > scat[2]


def _p11(nr, nth, nph, na):
    edges, rm = _shell_problem(nr, nth, nph)
    dirs, w = I.angle_set(na, na)
    g = O.OracleGrid(I.SPHERICAL, edges, dirs, w, I.CORE_B)
    per = nth * nph
    chi = np.repeat(2.0 / rm ** 2, per)
    eps = np.full(nr * per, 1e-8)
    B = np.ones(nr * per)
    S, it, _ = g.solve(chi, eps, B, tol=1e-10, max_iter=2000)
    assert it > 0
    _, _, F, _ = g.formal_solution(S, chi, B)
    F = F.reshape(nr, per, 3)
    r2F = rm ** 2 * F[:, :, 0].mean(1)
    Fr = F[-1, :, 0].mean()
    return r2F.max() / r2F.min() - 1.0, np.abs(F[-1, :, 1]).max() / Fr, np.abs(F[-1, :, 2]).max() / Fr


def test_p11_flux_conservation_improves_with_resolution():
    s1, t1, p1 = _p11(8, 5, 9, 4)
    s2, t2, p2 = _p11(16, 9, 17, 8)
    assert s2 < 0.5 * s1
    assert t2 < 0.5 * t1 and p2 < 0.5 * p1


def test_p12_outer_flux_vectors_become_radial_with_solid_angles():
    """Sect. 3.2.2 (flux vectors of the outermost voxels): in spherical symmetry
    only F_r is non-zero; on a fixed grid the scatter of F_r over the outermost
    shell and F_phi fall as the solid-angle set is refined; F_theta falls until the
    9 theta cells of the grid, not the solid angles, set its error."""
    edges, rm = _shell_problem(8, 9, 17)
    per = 9 * 17
    chi = np.repeat(2.0 / rm ** 2, per)
    S = np.ones(8 * per)
    scat, fth, fph = [], [], []
    for n in (2, 4, 8, 16):
        dirs, w = I.angle_set(n, n)
        g = O.OracleGrid(I.SPHERICAL, edges, dirs, w, I.CORE_B)
        _, _, F, _ = g.formal_solution(S, chi, S)
        out = F.reshape(8, per, 3)[-1]
        Fr = out[:, 0].mean()
        scat.append(out[:, 0].max() / out[:, 0].min() - 1.0)
        fth.append(np.abs(out[:, 1]).max() / Fr)
        fph.append(np.abs(out[:, 2]).max() / Fr)
    assert scat[0] > scat[1] > scat[2] > scat[3]
    assert fph[0] > fph[1] > fph[2] > fph[3]
    assert fth[0] > fth[1] and max(fth[2], fth[3]) < 0.6 * fth[1]
