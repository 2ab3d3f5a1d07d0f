"""Seeded synthetic inputs: voxel-grid edges, solid-angle sets and per-voxel fields.

This module builds problem descriptions only (no part of the formal solution,
ALI or Ng arithmetic).  It is the one module that both the CUDA path and the
CPU oracle receive their inputs from, so both see bit-identical edges,
directions, weights and fields.

Grids follow the paper's test setups (Sect. 3.1: spherical (r, theta_c, phi_c)
grid, regular in theta_c and phi_c, radial grid of highly variable spacing;
Sect. 4: cylindrical (R, phi_c, z) grid, regular in phi_c and z, linear in R).
Solid angles: Gauss-Legendre in mu = cos(theta) times a uniform phi offset by
half a step (the paper prescribes (theta, phi) pairs with n_theta = n_phi but
no rule; Sect. 3.1).
"""
import math

import numpy as np

SPHERICAL, CYLINDRICAL = 0, 1
CORE_B, TRANSPARENT = 0, 1

SEED = 0x09031949


def sph_edges(n_r, n_th, n_ph, r_min=1.0, r_max=100.0):
    """Edges of a spherical voxel grid: r log-spaced, theta_c and phi_c regular."""
    i = np.arange(n_r + 1, dtype=np.float64)
    r = r_min * (r_max / r_min) ** (i / n_r)
    r[0], r[-1] = r_min, r_max
    th = np.pi * np.arange(n_th + 1, dtype=np.float64) / n_th
    ph = 2.0 * np.pi * np.arange(n_ph + 1, dtype=np.float64) / n_ph
    return [r, th, ph]


def cyl_edges(n_R, n_ph, n_z, R_min=0.1, R_max=10.0, z_max=2.0):
    """Edges of a cylindrical voxel grid: R linear, phi_c and z regular."""
    R = np.linspace(R_min, R_max, n_R + 1)
    ph = 2.0 * np.pi * np.arange(n_ph + 1, dtype=np.float64) / n_ph
    z = np.linspace(-z_max, z_max, n_z + 1)
    return [R, ph, z]


def angle_set(n_mu, n_phi):
    """Unit directions (N,3) and weights (N,) summing to 1; mu Gauss-Legendre, phi uniform."""
    mu, wmu = np.polynomial.legendre.leggauss(n_mu)
    phi = 2.0 * np.pi * (np.arange(n_phi) + 0.5) / n_phi
    M, P = np.meshgrid(mu, phi, indexing="ij")
    W = np.repeat(wmu[:, None] / (2.0 * n_phi), n_phi, axis=1)
    s = np.sqrt(1.0 - M * M)
    dirs = np.stack([s * np.cos(P), s * np.sin(P), M], axis=-1).reshape(-1, 3)
    return np.ascontiguousarray(dirs), np.ascontiguousarray(W.reshape(-1))


def voxel_centres(coord, edges):
    """Centres (mid-points of the edges) as three broadcast arrays of shape n1 x n2 x n3."""
    m = [0.5 * (e[:-1] + e[1:]) for e in edges]
    return np.meshgrid(m[0], m[1], m[2], indexing="ij")


def lognormal(shape, sigma, seed):
    """Mean-preserving lognormal factors exp(sigma Z - sigma^2/2)."""
    z = np.random.default_rng(seed).standard_normal(shape)
    return np.exp(sigma * z - 0.5 * sigma * sigma)


def make_problem(name, **over):
    """A named synthetic workload: dict(coord, edges, dirs, weights, chi, eps, B, inner_bc, ...).

    Keyword overrides replace sizes (n, n_mu, n_phi) for scaled-down variants.
    """
    cfg = dict(PROBLEMS[name])
    cfg.update(over)
    coord = cfg["coord"]
    n1, n2, n3 = cfg["n"]
    if coord == SPHERICAL:
        edges = sph_edges(n1, n2, n3, cfg.get("r_min", 1.0), cfg.get("r_max", 100.0))
    else:
        edges = cyl_edges(n1, n2, n3, cfg.get("R_min", 0.1), cfg.get("R_max", 10.0), cfg.get("z_max", 2.0))
    dirs, wts = angle_set(cfg["n_mu"], cfg["n_phi"])
    c1, c2, c3 = voxel_centres(coord, edges)
    shape = (n1, n2, n3)
    kind = cfg["fields"]
    if kind == "r2":
        # chi = chi0 r^-2 with radial optical depth tau over [r_min, r_max]
        rmin, rmax = edges[0][0], edges[0][-1]
        chi0 = cfg["tau"] / (1.0 / rmin - 1.0 / rmax)
        chi = chi0 / (c1 * c1)
        B = np.full(shape, cfg.get("B", 1.0))
        if cfg.get("noise", 0.0) > 0.0:
            chi = chi * lognormal(shape, cfg["noise"], cfg.get("seed", SEED))
            B = B * lognormal(shape, cfg["noise"], cfg.get("seed", SEED) + 1)
    elif kind == "disc":
        # chi = chi0 (R/R0)^-1.5 exp(-z^2 / 2H^2), H = 0.1 R, midplane tau over [R_min, R_max]
        Rmin, Rmax = edges[0][0], edges[0][-1]
        chi0 = cfg["tau"] / (2.0 * (Rmin ** -0.5 - Rmax ** -0.5))
        H = 0.1 * c1
        chi = chi0 * c1 ** -1.5 * np.exp(-(c3 * c3) / (2.0 * H * H))
        chi = np.maximum(chi, cfg.get("chi_floor", 1e-10) * chi0)
        B = c1 ** -0.75
    elif kind == "const":
        chi = np.full(shape, cfg.get("chi", 1.0))
        B = np.full(shape, cfg.get("B", 1.0))
    else:
        raise ValueError(kind)
    eps = np.full(shape, cfg["eps"])
    return dict(name=name, coord=coord, edges=edges, dirs=dirs, weights=wts,
                chi=np.ascontiguousarray(chi.reshape(-1)), eps=np.ascontiguousarray(eps.reshape(-1)),
                B=np.ascontiguousarray(B.reshape(-1)), inner_bc=cfg["inner_bc"], n=(n1, n2, n3),
                n_ang=len(wts), tol=cfg.get("tol", 1e-8))


# Workloads shaped like the paper's tests (Sect. 3.1, 3.2, 4).
PROBLEMS = {
    # small spherical ALI: 17x9x17 voxels, 8x8 angles, tau 4, eps 1e-2
    "sph17": dict(coord=SPHERICAL, n=(17, 9, 17), n_mu=8, n_phi=8, fields="r2", tau=4.0, eps=1e-2,
                  inner_bc=CORE_B, tol=1e-8),
    # the paper's spherical grid 65x33x65, 32x32 angles, tau 1e2, eps 1e-4, 20% lognormal noise
    "sph65": dict(coord=SPHERICAL, n=(65, 33, 65), n_mu=32, n_phi=32, fields="r2", tau=1e2, eps=1e-4,
                  noise=0.2, inner_bc=CORE_B),
    # the same spherical grid with 8x8 solid angles (small case for profiling)
    "sph65a64": dict(coord=SPHERICAL, n=(65, 33, 65), n_mu=8, n_phi=8, fields="r2", tau=1e2, eps=1e-4,
                     noise=0.2, inner_bc=CORE_B),
    # cylindrical disc 65^3, R 0.1..10, |z| <= 2, 64x64 angles, midplane tau 1e3, eps 1e-6
    "cyl65": dict(coord=CYLINDRICAL, n=(65, 65, 65), n_mu=64, n_phi=64, fields="disc", tau=1e3, eps=1e-6,
                  inner_bc=TRANSPARENT),
    # deep adjoint case 129x65x129, 64x64 angles, tau 1e4, eps 1e-8
    "sph129": dict(coord=SPHERICAL, n=(129, 65, 129), n_mu=64, n_phi=64, fields="r2", tau=1e4, eps=1e-8,
                   inner_bc=CORE_B),
}


def make_batch_problem(n_members=256, n_angle=16, shapes=((33, 17, 33), (65, 33, 65), (97, 49, 97)), seed=SEED + 2,
                       tau=1.0):
    """Many wavelengths on spherical grids of uneven size (round-robin by member index).

    Each member m has chi = s_m chi0 r^-2 (radial tau of the base law `tau`), eps_m and
    B = 1, with s_m log-uniform in [1e-2, 1e2] and eps_m log-uniform in [1e-6, 1e-2].
    Returns (grids: list of dict(coord, edges, dirs, weights, inner_bc, n), member_grid,
    members: list of (chi, eps, B)).
    """
    rng = np.random.default_rng(seed)
    grids = []
    dirs, wts = angle_set(n_angle, n_angle)
    for n in shapes:
        edges = sph_edges(*n)
        grids.append(dict(coord=SPHERICAL, edges=edges, dirs=dirs, weights=wts, inner_bc=CORE_B, n=tuple(n)))
    scale = 10.0 ** rng.uniform(-2.0, 2.0, n_members)
    eps = 10.0 ** rng.uniform(-6.0, -2.0, n_members)
    member_grid = [m % len(shapes) for m in range(n_members)]
    base = []
    for g in grids:
        c1, _, _ = voxel_centres(SPHERICAL, g["edges"])
        rmin, rmax = g["edges"][0][0], g["edges"][0][-1]
        base.append(np.ascontiguousarray((tau / (1.0 / rmin - 1.0 / rmax) / (c1 * c1)).reshape(-1)))
    members = []
    for m in range(n_members):
        chi = base[member_grid[m]] * scale[m]
        members.append((chi, np.full(chi.size, eps[m]), np.ones(chi.size)))
    return grids, member_grid, members


def line_profile(n_freq=32, width=1.0, span=4.0):
    """Frequency sampling of a Doppler (Gaussian) line over +-span widths, the outer
    points effectively continuum (the paper's 32 wavelength points, Sect. 3.1):
    (phi, w) with trapezoid weights w and phi normalised to sum_k w_k phi_k = 1."""
    x = np.linspace(-span, span, n_freq)
    w = np.full(n_freq, x[1] - x[0]) if n_freq > 1 else np.ones(1)
    if n_freq > 1:
        w[0] *= 0.5
        w[-1] *= 0.5
    phi = np.exp(-(x / width) ** 2)
    phi /= np.sum(w * phi)
    return phi, w


def line_problem(name="sph17", n_freq=32, ratio=1e6, eps_l=1e-2, **over):
    """The paper's two-level test on a named grid: grey continuum chi_c (the grid's chi
    law scaled to a radial continuum tau of 1e-2, so the line centre reaches 1e4 with
    chi_l / chi_c = ratio), thermal B, line profile of line_profile(n_freq)."""
    p = make_problem(name, **over)
    rmin, rmax = p["edges"][0][0], p["edges"][0][-1]
    c1, _, _ = voxel_centres(p["coord"], p["edges"])
    if p["coord"] == SPHERICAL:
        chi_c = (1e-2 / (1.0 / rmin - 1.0 / rmax)) / (c1 * c1)
    else:
        chi_c = np.full(c1.shape, 1e-2 / (rmax - rmin))
    chi_c = np.ascontiguousarray(chi_c.reshape(-1))
    phi, w = line_profile(n_freq)
    p.update(chi_c=chi_c, chi_l=ratio * chi_c, eps_l=np.full(chi_c.size, eps_l), phi=phi, wq=w)
    return p


def voxel_angle_count(n, n_ang):
    return int(np.prod(n)) * int(n_ang)


def deg(x):
    return x * 180.0 / math.pi
