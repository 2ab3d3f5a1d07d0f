"""Test helpers: tiny problems, analytic chords and brute-force cell location.

Nothing here computes the method itself; these are independent geometric
facts (line/sphere and line/cylinder intersections, point location by
arccos/arctan2) used to pin the oracle.
"""
import numpy as np

from paper_0903_1949_gb300 import inputs as I


def tiny_problem(coord, n, n_mu, n_phi, inner_bc, chi=None, eps=0.1, B=1.0, seed=7, **edge_kw):
    """A small problem dict with seeded lognormal chi unless chi is given."""
    if coord == I.SPHERICAL:
        edges = I.sph_edges(*n, edge_kw.get("r_min", 1.0), edge_kw.get("r_max", 10.0))
    else:
        edges = I.cyl_edges(*n, edge_kw.get("R_min", 0.5), edge_kw.get("R_max", 5.0), edge_kw.get("z_max", 2.0))
    dirs, wts = I.angle_set(n_mu, n_phi)
    nv = int(np.prod(n))
    if chi is None:
        chi = 0.8 * I.lognormal(nv, 0.5, seed)
    chi = np.broadcast_to(np.asarray(chi, dtype=np.float64), (nv,)).copy()
    return dict(coord=coord, edges=edges, dirs=dirs, weights=wts, chi=chi,
                eps=np.full(nv, float(eps)), B=np.broadcast_to(np.asarray(B, np.float64), (nv,)).copy(),
                inner_bc=inner_bc, n=tuple(n), nvox=nv, n_ang=len(wts))


def centre(coord, edges, v):
    n1, n2, n3 = (len(e) - 1 for e in edges)
    k = v % n3
    j = (v // n3) % n2
    i = v // (n3 * n2)
    m = [0.5 * (edges[a][q] + edges[a][q + 1]) for a, q in ((0, i), (1, j), (2, k))]
    if coord == I.SPHERICAL:
        r, th, ph = m
        return np.array([r * np.sin(th) * np.cos(ph), r * np.sin(th) * np.sin(ph), r * np.cos(th)])
    R, ph, z = m
    return np.array([R * np.cos(ph), R * np.sin(ph), z])


def _quad_interval(a, b, c):
    """Interval where a t^2 + 2 b t + c < 0 (a > 0), or None."""
    disc = b * b - a * c
    if disc <= 0:
        return None
    s = np.sqrt(disc)
    return ((-b - s) / a, (-b + s) / a)


def domain_intervals(coord, edges, x0, d, core_b):
    """Parameter intervals (t_lo, t_hi) of the line x0 + t d inside the voxel domain,
    cut at an opaque core (core_b) so that the interval containing t = 0 is returned
    together with the hole chord inside it (for a transparent inner boundary)."""
    if coord == I.SPHERICAL:
        rmin, rmax = edges[0][0], edges[0][-1]
        a, b = d @ d, x0 @ d
        out = _quad_interval(a, b, x0 @ x0 - rmax * rmax)
        hole = _quad_interval(a, b, x0 @ x0 - rmin * rmin)
        lo, hi = out
        hole_len = 0.0
        if hole is not None:
            if core_b:
                if hole[1] <= 0:
                    lo = max(lo, hole[1])
                else:
                    hi = min(hi, hole[0])
            else:
                hole_len = hole[1] - hole[0]
        return lo, hi, hole_len
    Rmin, Rmax = edges[0][0], edges[0][-1]
    zmin, zmax = edges[2][0], edges[2][-1]
    a = d[0] ** 2 + d[1] ** 2
    b = x0[0] * d[0] + x0[1] * d[1]
    p2 = x0[0] ** 2 + x0[1] ** 2
    if a > 0:
        lo, hi = _quad_interval(a, b, p2 - Rmax * Rmax)
    else:
        lo, hi = -np.inf, np.inf
    if d[2] != 0:
        t1, t2 = (zmin - x0[2]) / d[2], (zmax - x0[2]) / d[2]
        lo, hi = max(lo, min(t1, t2)), min(hi, max(t1, t2))
    hole_len = 0.0
    hole = _quad_interval(a, b, p2 - Rmin * Rmin) if a > 0 else None
    if hole is not None:
        h0, h1 = max(hole[0], lo), min(hole[1], hi)
        if core_b:
            if hole[1] <= 0:
                lo = max(lo, hole[1])
            else:
                hi = min(hi, hole[0])
        elif h1 > h0:
            hole_len = h1 - h0
    return lo, hi, hole_len


def locate_points(coord, edges, P):
    """Voxel id of each point (or -1 outside the voxels) by direct coordinates."""
    n1, n2, n3 = (len(e) - 1 for e in edges)
    x, y, z = P[:, 0], P[:, 1], P[:, 2]
    if coord == I.SPHERICAL:
        r = np.sqrt(x * x + y * y + z * z)
        c1 = r
        c2 = np.arccos(np.clip(z / r, -1.0, 1.0))
        c3 = np.mod(np.arctan2(y, x), 2 * np.pi)
    else:
        c1 = np.sqrt(x * x + y * y)
        c2 = np.mod(np.arctan2(y, x), 2 * np.pi)
        c3 = z
    i = np.searchsorted(edges[0], c1, side="right") - 1
    j = np.clip(np.searchsorted(edges[1], c2, side="right") - 1, 0, n2 - 1)
    k = np.clip(np.searchsorted(edges[2], c3, side="right") - 1, 0, n3 - 1)
    if coord == I.CYLINDRICAL:
        k = np.searchsorted(edges[2], c3, side="right") - 1
    ok = (i >= 0) & (i < n1) & (k >= 0) & (k < n3)
    return np.where(ok, (i * n2 + j) * n3 + k, -1)


def runs(seq, weights, min_weight):
    """Collapse a cell sequence into runs, dropping runs lighter than min_weight."""
    out = []
    for c, w in zip(seq, weights):
        if out and out[-1][0] == c:
            out[-1][1] += w
        else:
            out.append([c, w])
    kept = [c for c, w in out if w >= min_weight and c >= 0]
    merged = []
    for c in kept:
        if not merged or merged[-1] != c:
            merged.append(c)
    return merged
