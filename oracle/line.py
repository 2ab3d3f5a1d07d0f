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
"""
import numpy as np


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


def line_solve(o, chi_c, chi_l, eps_l, B, phi, wq, tol=1e-10, max_iter=500, S0=None):
    """Two-level ALI to max rel dS_l < tol from S0 (default B).
    Returns (S_l, iterations (negative: not converged), history of max rel dS_l)."""
    S = np.array(B if S0 is None else S0, dtype=np.float64, copy=True)
    Lbar = line_lbar(o, chi_c, chi_l, B, phi, wq)
    hist = []
    for it in range(1, max_iter + 1):
        Jbar = line_jbar(o, S, chi_c, chi_l, B, phi, wq)
        Sn = S + ((1.0 - eps_l) * Jbar + eps_l * B - S) / (1.0 - (1.0 - eps_l) * Lbar)
        rel = float(np.max(np.abs(Sn - S) / np.abs(Sn)))
        S = Sn
        hist.append(rel)
        if rel < tol:
            return S, it, np.array(hist)
    return S, -max_iter, np.array(hist)
