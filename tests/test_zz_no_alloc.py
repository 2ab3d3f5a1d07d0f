"""rt_fs_angle_noalloc: the one-solid-angle formal solution for callers that
cannot allocate device memory when they call (a framework's memory pool owns
all of it, or the calling thread must not enter the allocator).  Its
per-segment scratch is a static device array inside the library, so the call
itself allocates nothing; it must give the same Ibar / Lambda* as the
allocating path rt_fs_angles, call after call.

This file is named to be collected last, so a failure here does not hide the
results of the other GPU tests.
"""
import ctypes

import numpy as np
import pytest

from paper_0903_1949_gb300 import build as B
from paper_0903_1949_gb300 import inputs as I
from paper_0903_1949_gb300 import rt

pytestmark = pytest.mark.gpu


def _entry():
    lib = rt.load()
    f = lib.rt_fs_angle_noalloc
    f.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
    f.restype = ctypes.c_int
    return f


def test_noalloc_angle_matches_allocating_path_twice_in_a_row():
    torch = pytest.importorskip("torch")
    B.build()
    f = _entry()
    p = I.make_problem("sph17")
    g = rt.Grid(p["coord"], p["edges"], p["dirs"], p["weights"], inner_bc=p["inner_bc"])
    try:
        g.set_opacity(p["chi"], p["eps"], p["B"])
        rng = np.random.default_rng(21)
        g.set_S(p["B"] * rng.uniform(0.7, 1.3, p["chi"].size))
        dev = torch.device("cuda:0")
        Ib = torch.empty(p["chi"].size, dtype=torch.float64, device=dev)
        Lb = torch.empty(p["chi"].size, dtype=torch.float64, device=dev)
        # two calls in a row on the same static scratch: different angles, then the other precision
        for omega, prec, tol in ((11, rt.RT_FP64, 1e-12), (50, rt.RT_FP64, 1e-12), (50, rt.RT_MIXED, 1e-5),
                                 (11, rt.RT_MIXED, 1e-5)):
            Ib.fill_(-1.0)
            Lb.fill_(-1.0)
            rc = f(g.h, omega, prec, ctypes.c_void_p(Ib.data_ptr()), ctypes.c_void_p(Lb.data_ptr()))
            assert rc == rt.RT_OK, rt.rt_last_error()
            torch.cuda.synchronize()
            ref_I, ref_L = g.fs_angles([omega], prec)
            got_I, got_L = Ib.cpu().numpy(), Lb.cpu().numpy()
            assert np.max(np.abs(got_I - ref_I[0]) / np.abs(ref_I[0])) < tol, (omega, prec)
            assert np.max(np.abs(got_L - ref_L[0]) / np.abs(ref_L[0])) < tol, (omega, prec)
        # arguments are checked before any device work
        assert f(g.h, p["n_ang"], rt.RT_FP64, ctypes.c_void_p(Ib.data_ptr()), ctypes.c_void_p(Lb.data_ptr())) \
            == rt.RT_EINVAL
        assert f(g.h, 0, 7, ctypes.c_void_p(Ib.data_ptr()), ctypes.c_void_p(Lb.data_ptr())) == rt.RT_EINVAL
        assert f(g.h, 0, rt.RT_FP64, None, None) == rt.RT_EINVAL
    finally:
        g.close()
