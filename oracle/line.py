"""Two-level-atom line transfer on the oracle (TEST INFRASTRUCTURE: only tests/,
__graft_entry__.smoke() and bench.py's CPU baseline use anything under oracle/).

The line is sampled at n_freq frequencies with profile values phi_k and
quadrature weights w_k (sum_k w_k phi_k = 1).  At frequency k the opacity is
chi_k = chi_c + chi_l phi_k and the source function mixes the continuum
(S_c = B, eps_c = 1) and the line:
    S_k = (chi_c B + chi_l phi_k S_l) / chi_k,
    S_l = (1 - eps_l) Jbar + eps_l B,   Jbar = sum_k w_k phi_k J_k
(Sect. 3.1 and 3.2.2, the 2-level test of the paper, with the grey continuum
and thermal B of its setup).  The ALI step for S_l uses the diagonal
    Lbar* = sum_k w_k phi_k (chi_l phi_k / chi_k) Lambda*_k,
    S_l <- S_l + [(1 - eps_l) Jbar + eps_l B - S_l] / (1 - (1 - eps_l) Lbar*),
the continuum ALI of R10 applied to the frequency-averaged line.  Every formal
solution is the oracle's own (orc_formal_solution).

With the nearest-neighbour operator (Sect. 2, 3.2.1) the line operator is the
exact dJbar_v / dS_l,u restricted to the 3 x 3 x 3 index neighbourhood of v:
S_k depends on S_l at its own voxel with weight chi_l phi_k / chi_k there, so
    Lbar*_vu = sum_k w_k phi_k Lambda*_k,vu (chi_l phi_k / chi_k)_u,
the factor taken at the neighbour u, and the OS step solves
(I - (1 - eps_l) Lbar*) dS_l = (1 - eps_l) Jbar + eps_l B - S_l
(orc_nn_ali_update).
"""
import numpy as np

from oracle import oracle as O
from oracle.oracle import SPH


def frequency_opacity(chi_c, chi_l, phi):
    """chi_k (n_freq, n_vox)."""
    return chi_c[None, :] + np.outer(phi, chi_l)


def line_lbar(o, chi_c, chi_l, B, phi, wq):
    """Lbar* of the line: sum_k w_k phi_k (chi_l phi_k / chi_k) Lambda*_k."""
    chik = frequency_opacity(chi_c, chi_l, phi)
    Lbar = np.zeros(chi_c.size)
    for k in range(len(phi)):
        _, Lk, _, miss = o.formal_solution(B, chik[k], B)
        assert miss == 0
        Lbar += wq[k] * phi[k] * (chi_l * phi[k] / chik[k]) * Lk
    return Lbar


def nn_neighbours(o):
    """(n_vox, 27): the voxel in slot q = 9 (di+1) + 3 (dj+1) + (dk+1) of each voxel's
    index neighbourhood, -1 outside the grid; phi is periodic (the third index of a
    spherical grid, the second of a cylindrical one)."""
    n1, n2, n3 = o.n
    i, j, k = np.unravel_index(np.arange(o.nvox), o.n)
    out = np.full((o.nvox, 27), -1, dtype=np.int64)
    for q in range(27):
        a, b, c = i + q // 9 - 1, j + (q // 3) % 3 - 1, k + q % 3 - 1
        if o.coord == SPH:
            c = c % n3
        else:
            b = b % n2
        ok = (a >= 0) & (a < n1) & (b >= 0) & (b < n2) & (c >= 0) & (c < n3)
        out[ok, q] = np.ravel_multi_index((a[ok], b[ok], c[ok]), o.n)
    return out


def line_lbar_nn(o, chi_c, chi_l, phi, wq):
    """Nearest-neighbour Lbar* (n_vox, 27) of the line, columns as nn_neighbours."""
    chik = frequency_opacity(chi_c, chi_l, phi)
    nb = nn_neighbours(o)
    Lbar = np.zeros((o.nvox, 27))
    for k in range(len(phi)):
        Lk = o.nn_lstar(chik[k])
        f = chi_l * phi[k] / chik[k]
        Lbar += wq[k] * phi[k] * Lk * np.where(nb >= 0, f[np.maximum(nb, 0)], 0.0)
    return Lbar


def line_jbar(o, S_l, chi_c, chi_l, B, phi, wq):
    """Jbar of the line source S_l: frequency-weighted J of the S_k it implies."""
    chik = frequency_opacity(chi_c, chi_l, phi)
    Jbar = np.zeros(chi_c.size)
    for k in range(len(phi)):
        Sk = (chi_c * B + chi_l * phi[k] * S_l) / chik[k]
        Jk, _, _, miss = o.formal_solution(Sk, chik[k], B)
        assert miss == 0
        Jbar += wq[k] * phi[k] * Jk
    return Jbar


def line_solve(o, chi_c, chi_l, eps_l, B, phi, wq, tol=1e-10, max_iter=500, S0=None, use_lstar=1, jtol=1e-14,
               ng=False):
    """Two-level ALI to max rel dS_l < tol from S0 (default B), with the diagonal
    (use_lstar=1) or nearest-neighbour (2) line operator; ng: order-2 Ng
    extrapolation of S_l whenever four iterates have accumulated since the last
    one (R11, as the continuum solve).
    Returns (S_l, iterations (negative: not converged), history of max rel dS_l)."""
    S = np.array(B if S0 is None else S0, dtype=np.float64, copy=True)
    if use_lstar == 2:
        L27 = line_lbar_nn(o, chi_c, chi_l, phi, wq)
    else:
        Lbar = line_lbar(o, chi_c, chi_l, B, phi, wq)
    hist = []
    H = []
    for it in range(1, max_iter + 1):
        Jbar = line_jbar(o, S, chi_c, chi_l, B, phi, wq)
        if use_lstar == 2:
            Sn, rel, _ = o.nn_ali_update(S, Jbar, L27, eps_l, B, jtol=jtol)
        else:
            Sn = S + ((1.0 - eps_l) * Jbar + eps_l * B - S) / (1.0 - (1.0 - eps_l) * Lbar)
            rel = float(np.max(np.abs(Sn - S) / np.abs(Sn)))
        S = Sn
        hist.append(rel)
        if rel < tol:
            return S, it, np.array(hist)
        if ng:
            H = (H + [S.copy()])[-4:]
            if len(H) == 4:
                Sx = O.ng(H[3], H[2], H[1], H[0])
                if Sx is not None:
                    S = Sx
                    H = []
    return S, -max_iter, np.array(hist)
