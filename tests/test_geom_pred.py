"""Guided coverage completion (RT_TUNE_GEOM_PREDICT), checked on the CPU.

The completion launches a characteristic through every voxel still unhit, in
voxel order (Sect. 2).  The GPU kernel traces candidates speculatively; the
guided kernel first walks each candidate's line in float (csrc/geom_pred.cuh)
and traces exactly only candidates no earlier chosen candidate's guessed line
crosses.  Here the kernel's rounds are replayed in Python with the very same
float walk (compiled for the host) and with the oracle's exact lines standing in
for the FP64 traces: the launches must be the oracle's serial completion, in
order, and the guesses must cut the rounds of the plain speculation.
"""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

from helpers import tiny_problem
from oracle import oracle as O
from paper_0903_1949_gb300 import inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PREFIX = 256  # candidates a round may look at (PRED_PREFIX of the kernel)
LANES = 32    # candidates traced exactly per round


@pytest.fixture(scope="module")
def pred(tmp_path_factory):
    cxx = shutil.which("g++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    so = tmp_path_factory.mktemp("pred") / "libpred.so"
    subprocess.run([cxx, "-O2", "-ffp-contract=off", "-std=c++17", "-shared", "-fPIC",
                    "-I", os.path.join(ROOT, "include"), "-I", os.path.join(ROOT, "paper_0903_1949_gb300", "csrc"),
                    os.path.join(ROOT, "tests", "pred_walk_host.cpp"), "-o", str(so)], check=True)
    L = ctypes.CDLL(str(so))
    dp = ctypes.POINTER(ctypes.c_double)
    L.pred_create.restype = ctypes.c_void_p
    L.pred_create.argtypes = [ctypes.c_int] * 5 + [dp] * 3
    L.pred_destroy.argtypes = [ctypes.c_void_p]
    L.pred_line.restype = ctypes.c_int
    L.pred_line.argtypes = [ctypes.c_void_p, ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                            ctypes.POINTER(ctypes.c_int32), ctypes.c_int]
    return L


class Case:
    def __init__(self, L, p):
        self.L, self.p = L, p
        self.edges = [np.ascontiguousarray(e, dtype=np.float64) for e in p["edges"]]
        self.n = tuple(len(e) - 1 for e in self.edges)
        self.nvox = int(np.prod(self.n))
        self.cap = 2 * (4 * sum(self.n) + 16) + 8  # the kernel's list capacity
        dp = ctypes.POINTER(ctypes.c_double)
        self.h = L.pred_create(int(p["coord"]), *self.n, int(p["inner_bc"]),
                               *(e.ctypes.data_as(dp) for e in self.edges))
        self.o = O.OracleGrid(p["coord"], p["edges"], p["dirs"], p["weights"], p["inner_bc"])
        self.dirs = np.asarray(p["dirs"], dtype=np.float64).reshape(-1, 3)
        self.buf = np.empty(self.cap, np.int32)

    def close(self):
        self.L.pred_destroy(self.h)
        self.o.close()

    def guess(self, w, v):
        d = self.dirs[w]
        n = self.L.pred_line(self.h, d[0], d[1], d[2], int(v),
                             self.buf.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), self.cap)
        return self.buf[:min(n, self.cap)].copy()

    def angle(self, w):
        """Boundary marks, the oracle's completion lines and their origins in launch order."""
        a = self.o.angle(w)
        assert a["n_lost"] == 0
        off, org, kind, vox = a["ray_off"], a["ray_origin"], a["ray_kind"], a["vox"]
        hit = np.zeros(self.nvox, bool)
        lines, order = {}, []
        for r in range(len(org)):
            seg = vox[off[r]:off[r + 1]]
            if kind[r] == 2:
                lines[int(org[r])] = seg
                order.append(int(org[r]))
            else:
                hit[seg] = True
        self.o.free_angle(w)
        return hit, lines, order

    def guided(self, w, hit, lines):
        """The rounds of k_complete_pred: launched origins in order, rounds."""
        hit = hit.copy()
        stamp = np.zeros(self.nvox, np.int64)
        pos, rnd, launched = 0, 0, []
        while pos < self.nvox:
            rnd += 1
            pref, nsel, scan, full = [], 0, pos, False
            while not full and len(pref) < PREFIX and scan < self.nvox:
                want = min(LANES, PREFIX - len(pref))
                cand = (np.flatnonzero(~hit[scan:]) + scan)[:want]
                cscan = int(cand[-1]) + 1 if len(cand) == want else self.nvox
                guesses = [self.guess(w, v) for v in cand]
                m = 0
                while m < len(cand):
                    v = int(cand[m])
                    if stamp[v] == rnd and nsel > 0:
                        pref.append((v, False))
                        m += 1
                        continue
                    if nsel == LANES:
                        break
                    pref.append((v, True))
                    nsel += 1
                    stamp[guesses[m]] = rnd
                    m += 1
                if m < len(cand):
                    scan, full = int(cand[m]), True
                else:
                    scan = cscan
            nxt = scan
            for v, chosen in pref:
                if hit[v]:
                    continue
                if not chosen:
                    nxt = v
                    break
                assert v in lines, "a launch the serial rule does not make (voxel %d)" % v
                launched.append(v)
                hit[lines[v]] = True
            assert nxt > pos, "a round without progress"
            pos = nxt
        return launched, rnd

    def plain(self, hit, lines):
        """The rounds of k_complete (32 candidates in voxel order per round)."""
        hit = hit.copy()
        pos, rnd, launched = 0, 0, []
        while pos < self.nvox:
            cand = (np.flatnonzero(~hit[pos:]) + pos)[:LANES]
            if len(cand) == 0:
                break
            rnd += 1
            for v in cand:
                if not hit[v]:
                    launched.append(int(v))
                    hit[lines[int(v)]] = True
            pos = int(cand[-1]) + 1
        return launched, rnd


def _cases():
    sph = I.make_problem("sph17")
    cyl_hole = tiny_problem(I.CYLINDRICAL, (9, 8, 7), 6, 6, I.TRANSPARENT, seed=21)
    sph_hole = tiny_problem(I.SPHERICAL, (8, 7, 10), 6, 6, I.TRANSPARENT, seed=23)
    cyl_core = tiny_problem(I.CYLINDRICAL, (7, 9, 6), 4, 8, I.CORE_B, seed=24)
    return {"sph17": sph, "cyl_hole": cyl_hole, "sph_hole": sph_hole, "cyl_core": cyl_core}


@pytest.mark.parametrize("name", ["sph17", "cyl_hole", "sph_hole", "cyl_core"])
def test_guided_completion_launches_the_serial_completion(pred, name):
    c = Case(pred, _cases()[name])
    try:
        n_ang = len(c.p["weights"])
        for w in range(0, n_ang, max(1, n_ang // 12)):
            hit, lines, order = c.angle(w)
            launched, _ = c.guided(w, hit, lines)
            assert launched == order, (name, w)
            assert c.plain(hit, lines)[0] == order, (name, w)
    finally:
        c.close()


@pytest.mark.parametrize("name", ["sph17", "cyl_hole"])
def test_float_guess_follows_the_exact_lines(pred, name):
    """The float walk visits the cells of the exact FP64 walk (the oracle's
    crossing lists) up to rounding at edges and corners."""
    c = Case(pred, _cases()[name])
    try:
        inter = n_exact = n_guess = 0
        n_ang = len(c.p["weights"])
        for w in range(0, n_ang, max(1, n_ang // 8)):
            _, lines, order = c.angle(w)
            for v in order:
                e, g = set(lines[v].tolist()), set(c.guess(w, v).tolist())
                inter += len(e & g)
                n_exact += len(e)
                n_guess += len(g)
        assert inter / n_exact > 0.995 and inter / n_guess > 0.995, (inter, n_exact, n_guess)
    finally:
        c.close()


def test_guided_completion_cuts_the_rounds_on_the_spherical_workload(pred):
    """65 x 33 x 65 voxels, 32 x 32 solid angles: a polar, a mid-latitude and an
    equatorial solid angle.  The plain speculation rejects most candidates away
    from the poles (a voxel's line crosses the next unhit voxels of its ring);
    the guided rounds launch the same characteristics in far fewer rounds."""
    c = Case(pred, I.make_problem("sph65"))
    try:
        for w, gain in ((0, 1.15), (341, 1.8), (512, 2.5)):
            hit, lines, order = c.angle(w)
            launched, r_guided = c.guided(w, hit, lines)
            plain, r_plain = c.plain(hit, lines)
            assert launched == order and plain == order
            assert r_plain >= gain * r_guided, (w, r_plain, r_guided)
    finally:
        c.close()
