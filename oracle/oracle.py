"""ctypes wrapper of the serial FP64 CPU oracle (``rt_oracle.c``).

TEST INFRASTRUCTURE.  The oracle is the slow, plain reference that the CUDA
path is checked against (long-characteristics formal solution, Sect. 2 of
Hauschildt & Baron, "A 3D radiative transfer framework IV"; ALI with the
diagonal Lambda* and Ng acceleration, Sect. 3.2.1).  Only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import it.  It shares no code with the product library.
"""
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rt_oracle.c")
_SO = os.path.join(_HERE, "liboracle.so")

SPH, CYL = 0, 1
CORE_B, TRANSPARENT = 0, 1
PARABOLIC, LINEAR = 0, 1

_c_int_p = ctypes.POINTER(ctypes.c_int)
_c_dbl_p = ctypes.POINTER(ctypes.c_double)
_c_u8_p = ctypes.POINTER(ctypes.c_uint8)


def build(force=False):
    """Compile the oracle with contraction off so every operation is one IEEE rounding."""
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(_SRC):
        return _SO
    tmp = _SO + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math",
           "-o", tmp, _SRC, "-lm"]
    try:  # the angle-parallel formal solution wants OpenMP; without it that call runs on one thread
        subprocess.check_call(cmd[:-1] + ["-fopenmp", "-lm"], stderr=subprocess.DEVNULL)
    except (subprocess.CalledProcessError, OSError):
        subprocess.check_call(cmd)
    os.replace(tmp, _SO)
    return _SO


_lib_handle = None


def _lib():
    global _lib_handle
    if _lib_handle is None:
        build()
        L = ctypes.CDLL(_SO)
        L.orc_create.restype = ctypes.c_void_p
        L.orc_create.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                 _c_dbl_p, _c_dbl_p, _c_dbl_p, ctypes.c_int, _c_dbl_p, _c_dbl_p,
                                 ctypes.c_int, ctypes.c_double, ctypes.c_int]
        L.orc_destroy.argtypes = [ctypes.c_void_p]
        L.orc_angle_geometry.argtypes = [ctypes.c_void_p, ctypes.c_int]
        L.orc_angle_free.argtypes = [ctypes.c_void_p, ctypes.c_int]
        L.orc_angle_counts.argtypes = [ctypes.c_void_p, ctypes.c_int, _c_int_p, _c_int_p, _c_int_p]
        L.orc_angle_copy.argtypes = [ctypes.c_void_p, ctypes.c_int, _c_int_p, _c_int_p, _c_int_p,
                                     _c_int_p, _c_int_p, _c_dbl_p, _c_u8_p]
        L.orc_coeffs.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_int, _c_dbl_p, _c_dbl_p,
                                 _c_dbl_p]
        L.orc_fs_angle.argtypes = [ctypes.c_void_p, ctypes.c_int, _c_dbl_p, _c_dbl_p, _c_dbl_p,
                                   ctypes.c_int, _c_dbl_p, _c_dbl_p, _c_dbl_p]
        L.orc_formal_solution.argtypes = [ctypes.c_void_p, _c_dbl_p, _c_dbl_p, _c_dbl_p, ctypes.c_int,
                                          _c_dbl_p, _c_dbl_p, _c_dbl_p]
        L.orc_formal_solution_par.argtypes = [ctypes.c_void_p, _c_dbl_p, _c_dbl_p, _c_dbl_p, ctypes.c_int,
                                              _c_dbl_p, _c_dbl_p, _c_dbl_p, ctypes.c_int, _c_int_p]
        L.orc_ali_update.restype = ctypes.c_double
        L.orc_ali_update.argtypes = [ctypes.c_int, _c_dbl_p, _c_dbl_p, _c_dbl_p, _c_dbl_p, _c_dbl_p,
                                     ctypes.c_int]
        L.orc_ng.argtypes = [ctypes.c_int, _c_dbl_p, _c_dbl_p, _c_dbl_p, _c_dbl_p, _c_dbl_p]
        L.orc_solve.argtypes = [ctypes.c_void_p, _c_dbl_p, _c_dbl_p, _c_dbl_p, _c_dbl_p, ctypes.c_double,
                                ctypes.c_int, ctypes.c_int, ctypes.c_int, _c_dbl_p, ctypes.c_int]
        L.orc_nn_lstar.argtypes = [ctypes.c_void_p, _c_dbl_p, _c_dbl_p]
        L.orc_nn_ali_update.restype = ctypes.c_double
        L.orc_nn_ali_update.argtypes = [ctypes.c_void_p, _c_dbl_p, _c_dbl_p, _c_dbl_p, _c_dbl_p, _c_dbl_p,
                                        ctypes.c_double, ctypes.c_int, _c_int_p]
        L.orc_pz_intensity.restype = ctypes.c_double
        L.orc_pz_intensity.argtypes = [ctypes.c_int, _c_dbl_p, _c_dbl_p, _c_dbl_p, ctypes.c_int,
                                       ctypes.c_double, ctypes.c_double, ctypes.c_double]
        _lib_handle = L
    return _lib_handle


def _d(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(_c_dbl_p)


def coeffs(dm, dp, parabolic=True):
    """(alpha, beta, gamma) of one segment (see ``orc_coeffs``)."""
    a, b, g = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _lib().orc_coeffs(float(dm), float(dp), 1 if parabolic else 0, ctypes.byref(a), ctypes.byref(b),
                      ctypes.byref(g))
    return a.value, b.value, g.value


def ali_update(S, J, Lstar, eps, B, use_lstar=True):
    """One diagonal-Lambda* operator-splitting update; returns (S_new, max rel dS)."""
    S, pS = _d(np.array(S, dtype=np.float64, copy=True))
    J, pJ = _d(J)
    L, pL = _d(Lstar)
    e, pe = _d(eps)
    Bb, pB = _d(B)
    rel = _lib().orc_ali_update(S.size, pS, pJ, pL, pe, pB, 1 if use_lstar else 0)
    return S, rel


def ng(y0, y1, y2, y3):
    """Order-2 Ng extrapolation from four iterates (newest first); None if singular."""
    arrs = [_d(y) for y in (y0, y1, y2, y3)]
    out = np.empty_like(arrs[0][0])
    ok = _lib().orc_ng(out.size, arrs[0][1], arrs[1][1], arrs[2][1], arrs[3][1],
                       out.ctypes.data_as(_c_dbl_p))
    return out if ok else None


def pz_intensity(rs, S_shell, chi_shell, r, mu, core_b=True, I_core=0.0):
    """Exact 1D spherical intensity at radius r, direction cosine mu (shell-constant S, chi)."""
    rs, prs = _d(rs)
    Sh, pS = _d(S_shell)
    ch, pc = _d(chi_shell)
    return _lib().orc_pz_intensity(len(rs) - 1, prs, pS, pc, 1 if core_b else 0, float(I_core),
                                   float(r), float(mu))


class OracleGrid:
    """One voxel grid + solid-angle set; crossing lists are built per angle on demand."""

    def __init__(self, coord, edges, dirs, weights, inner_bc=CORE_B, I_outer=0.0, interp=PARABOLIC):
        self._keep = [_d(e) for e in edges]
        self.coord = int(coord)
        self.n = tuple(len(e) - 1 for e in edges)
        self.nvox = int(np.prod(self.n))
        dirs, pdir = _d(np.asarray(dirs).reshape(-1, 3))
        wts, pw = _d(weights)
        self.n_ang = wts.size
        self.dirs = dirs.copy()
        self.weights = wts.copy()
        self._h = _lib().orc_create(int(coord), self.n[0], self.n[1], self.n[2], self._keep[0][1],
                                    self._keep[1][1], self._keep[2][1], self.n_ang, pdir, pw,
                                    int(inner_bc), float(I_outer), int(interp))
        if not self._h:
            raise ValueError("oracle rejected the grid description")

    def close(self):
        if self._h:
            _lib().orc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def angle(self, w):
        """Crossing lists of angle w: dict of numpy arrays (segments in propagation order)."""
        nr, ns, nl = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        rc = _lib().orc_angle_counts(self._h, int(w), ctypes.byref(nr), ctypes.byref(ns), ctypes.byref(nl))
        if rc < 0:
            raise ValueError("bad angle index")
        nr, ns = nr.value, ns.value
        out = dict(ray_off=np.empty(nr + 1, np.int32), ray_origin=np.empty(nr, np.int32),
                   ray_kind=np.empty(nr, np.int32), ray_core=np.empty(nr, np.int32),
                   vox=np.empty(ns, np.int32), len=np.empty(ns, np.float64),
                   restart=np.empty(ns, np.uint8))
        _lib().orc_angle_copy(self._h, int(w), *(out[k].ctypes.data_as(_c_int_p) for k in
                                                 ("ray_off", "ray_origin", "ray_kind", "ray_core", "vox")),
                              out["len"].ctypes.data_as(_c_dbl_p), out["restart"].ctypes.data_as(_c_u8_p))
        out["n_lost"] = nl.value
        return out

    def free_angle(self, w):
        _lib().orc_angle_free(self._h, int(w))

    def fs_angle(self, w, S, chi, B, homog=False):
        """(Ibar, Lambda*-bar, per-ray emergent I, n missing voxels) of one angle."""
        S, pS = _d(S)
        c, pc = _d(chi)
        Bb, pB = _d(B)
        A = self.angle(w)
        Ib = np.empty(self.nvox)
        Lb = np.empty(self.nvox)
        Ie = np.empty(len(A["ray_origin"]))
        miss = _lib().orc_fs_angle(self._h, int(w), pS, pc, pB, 1 if homog else 0,
                                   Ib.ctypes.data_as(_c_dbl_p), Lb.ctypes.data_as(_c_dbl_p),
                                   Ie.ctypes.data_as(_c_dbl_p))
        return Ib, Lb, Ie, miss

    def nn_lstar(self, chi):
        """Nearest-neighbour Lambda* (nvox, 27): column q is dJ_v/dS_u for the voxel u at offset
        (q // 9 - 1, (q // 3) % 3 - 1, q % 3 - 1) of v in (i, j, k), phi periodic (see orc_nn_lstar)."""
        c, pc = _d(chi)
        out = np.empty((self.nvox, 27))
        rc = _lib().orc_nn_lstar(self._h, pc, out.ctypes.data_as(_c_dbl_p))
        if rc < 0:
            raise RuntimeError("orc_nn_lstar failed (%d)" % rc)
        return out

    def nn_ali_update(self, S, J, L27, eps, B, jtol=1e-14, jmax=100000):
        """One NN-Lambda* operator-splitting update; returns (S_new, max rel dS, Jacobi sweeps).
        max rel dS is NaN (and S_new the input S) when the Jacobi sweeps leave a
        non-finite iterate."""
        S, pS = _d(np.array(S, dtype=np.float64, copy=True))
        J, pJ = _d(J)
        L, pL = _d(L27)
        e, pe = _d(eps)
        Bb, pB = _d(B)
        sw = ctypes.c_int()
        rel = _lib().orc_nn_ali_update(self._h, pS, pJ, pL, pe, pB, float(jtol), int(jmax), ctypes.byref(sw))
        return S, rel, sw.value

    def formal_solution(self, S, chi, B, homog=False):
        """(J, Lambda*, F[nvox,3] in the local basis, n missing (voxel, angle) pairs)."""
        S, pS = _d(S)
        c, pc = _d(chi)
        Bb, pB = _d(B)
        J = np.empty(self.nvox)
        L = np.empty(self.nvox)
        F = np.empty((self.nvox, 3))
        miss = _lib().orc_formal_solution(self._h, pS, pc, pB, 1 if homog else 0,
                                          J.ctypes.data_as(_c_dbl_p), L.ctypes.data_as(_c_dbl_p),
                                          F.ctypes.data_as(_c_dbl_p))
        return J, L, F, miss

    def formal_solution_par(self, S, chi, B, homog=False, threads=None):
        """formal_solution with the angle loop over host threads (default: all cores);
        returns (J, Lambda*, F, n missing, threads used)."""
        S, pS = _d(S)
        c, pc = _d(chi)
        Bb, pB = _d(B)
        J = np.empty(self.nvox)
        L = np.empty(self.nvox)
        F = np.empty((self.nvox, 3))
        used = ctypes.c_int(1)
        n = int(threads) if threads else (os.cpu_count() or 1)
        miss = _lib().orc_formal_solution_par(self._h, pS, pc, pB, 1 if homog else 0,
                                              J.ctypes.data_as(_c_dbl_p), L.ctypes.data_as(_c_dbl_p),
                                              F.ctypes.data_as(_c_dbl_p), n, ctypes.byref(used))
        return J, L, F, miss, used.value

    def solve(self, chi, eps, B, tol=1e-8, max_iter=500, use_lstar=True, ng=True, S0=None, threads=1):
        """ALI (+Ng) to max rel dS < tol from S0 (default B); returns (S, iterations, history).

        use_lstar: False/0 Lambda iteration, True/1 diagonal Lambda*, 2 nearest-neighbour Lambda*.
        threads > 1: each formal solution with the angle loop over that many host threads."""
        c, pc = _d(chi)
        e, pe = _d(eps)
        Bb, pB = _d(B)
        S, pS = _d(np.array(B if S0 is None else S0, dtype=np.float64, copy=True))
        hist = np.zeros(max_iter)
        mode = int(use_lstar) if not isinstance(use_lstar, bool) else (1 if use_lstar else 0)
        it = _lib().orc_solve(self._h, pS, pc, pe, pB, float(tol), int(max_iter), mode,
                              1 if ng else 0, hist.ctypes.data_as(_c_dbl_p), int(threads))
        n = abs(it)
        return S, it, hist[:n]
