"""rt_fs_angle_noalloc: the one-solid-angle formal solution for callers that
cannot allocate device memory when they call (a framework's memory pool owns
all of it, or the calling thread must not enter the allocator).  Its
per-segment scratch is a static device array inside the library, placed on
the device by rt_grid_create, so the call itself allocates nothing: the
device's free memory must not move across the calls.  Its Ibar / Lambda*
must equal the oracle's for that angle, and those of the allocating path
rt_fs_angles, call after call.

The two GPU paths run the same kernels, but rt_fs_angles marches the angle's
whole block while this call marches the angle alone, which groups the
characteristics into warp bundles differently: the shuffle scan then
associates each recurrence differently, so they agree to rounding (here
1e-13 in FP64 and 2e-6 in FP32), not bit for bit.  A wrong offset into the
scratch or the lists would put whole segments in the wrong voxels, far
outside those bounds.

This file is named to be collected last, so a failure here does not hide the
results of the other GPU tests.
"""
import ctypes

import numpy as np
import pytest

from oracle import oracle as O
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


def _rel(a, b):
    return float(np.max(np.abs(a - b) / np.abs(b)))


def test_noalloc_angle_matches_allocating_path_twice_in_a_row():
    torch = pytest.importorskip("torch")
    B.build()
    f = _entry()
    p = I.make_problem("sph17")
    g = rt.Grid(p["coord"], p["edges"], p["dirs"], p["weights"], inner_bc=p["inner_bc"])
    try:
        g.set_opacity(p["chi"], p["eps"], p["B"])
        rng = np.random.default_rng(21)
        S = p["B"] * rng.uniform(0.7, 1.3, p["chi"].size)
        g.set_S(S)
        dev = torch.device("cuda:0")
        n = p["chi"].size
        calls = ((11, rt.RT_FP64), (50, rt.RT_FP64), (50, rt.RT_MIXED), (11, rt.RT_MIXED))
        outs = [(torch.full((n,), -1.0, dtype=torch.float64, device=dev),
                 torch.full((n,), -1.0, dtype=torch.float64, device=dev)) for _ in calls]
        torch.cuda.synchronize()
        free0, _ = torch.cuda.mem_get_info()
        # four calls in a row on the one static scratch: different angles, then the other precision
        for (omega, prec), (Ib, Lb) in zip(calls, outs):
            rc = f(g.h, omega, prec, ctypes.c_void_p(Ib.data_ptr()), ctypes.c_void_p(Lb.data_ptr()))
            assert rc == rt.RT_OK, rt.rt_last_error()
        torch.cuda.synchronize()
        free1, _ = torch.cuda.mem_get_info()
        assert free1 == free0, "device free memory moved by %d bytes across the allocation-free calls" % (free0 - free1)
        o = O.OracleGrid(p["coord"], p["edges"], p["dirs"], p["weights"], p["inner_bc"])
        for (omega, prec), (Ib, Lb) in zip(calls, outs):
            got_I, got_L = Ib.cpu().numpy(), Lb.cpu().numpy()
            ref_I, ref_L = g.fs_angles([omega], prec)
            tol = 1e-13 if prec == rt.RT_FP64 else 2e-6
            assert _rel(got_I, ref_I[0]) < tol, (omega, prec, _rel(got_I, ref_I[0]))
            assert _rel(got_L, ref_L[0]) < tol, (omega, prec, _rel(got_L, ref_L[0]))
            oI, oL, _, miss = o.fs_angle(omega, S, p["chi"], p["B"])
            assert miss == 0
            tol_o = 1e-12 if prec == rt.RT_FP64 else 1e-5
            assert _rel(got_I, oI) < tol_o and _rel(got_L, oL) < tol_o, (omega, prec)
        o.close()
        # arguments are checked before any device work
        Ib, Lb = outs[0]
        assert f(g.h, p["n_ang"], rt.RT_FP64, ctypes.c_void_p(Ib.data_ptr()), ctypes.c_void_p(Lb.data_ptr())) \
            == rt.RT_EINVAL
        assert f(g.h, 0, 7, ctypes.c_void_p(Ib.data_ptr()), ctypes.c_void_p(Lb.data_ptr())) == rt.RT_EINVAL
        assert f(g.h, 0, rt.RT_FP64, None, None) == rt.RT_EINVAL
    finally:
        g.close()
