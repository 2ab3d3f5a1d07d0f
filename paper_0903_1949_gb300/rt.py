"""ctypes binding of the C ABI in include/rt.h (argument marshalling only).

Every computation happens in the CUDA library librt3d.so; if it is missing
this module raises instead of falling back to anything else.  Arrays may be
numpy arrays (host memory) or CUDA tensors (device memory, passed by
pointer); results come back as numpy arrays unless a device buffer is given.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "librt3d.so")

RT_OK, RT_EINVAL, RT_ENOMEM, RT_ECUDA, RT_ENOTCONVERGED, RT_ETIMEOUT, RT_EDEVICE = range(7)
RT_SPHERICAL, RT_CYLINDRICAL = 0, 1
RT_CORE_B, RT_TRANSPARENT = 0, 1
RT_FP64, RT_MIXED = 0, 1
RT_PARABOLIC, RT_LINEAR = 0, 1
RT_LSTAR_NONE, RT_LSTAR_DIAG, RT_LSTAR_NN = 0, 1, 2
RT_HOST, RT_DEVICE = 0, 1
RT_TUNE_MARCH_CHUNK, RT_TUNE_STREAMED_WEIGHTS, RT_TUNE_MARCH_COARSEN, RT_TUNE_OVERLAP, RT_TUNE_SCATTER = 1, 2, 3, 4, 5
RT_TUNE_MARCH_STAGES, RT_TUNE_MARCH_BULK, RT_TUNE_NN_JTOL, RT_TUNE_MARCH64_COARSEN = 6, 7, 8, 9
RT_TUNE_MARCH_LOOKAHEAD = 10
RT_TUNE_S_BLOCKED = 11
RT_TUNE_NN_KRYLOV = 12
RT_TUNE_MARCH_STREAMS = 13
RT_TUNE_GRAPH = 15
RT_TUNE_GEOM_PREDICT = 16
RT_TUNE_FOLD_WEIGHT = 17
RT_TUNE_NN_TEST_STALL = 18

_STATUS = {0: "RT_OK", 1: "RT_EINVAL", 2: "RT_ENOMEM", 3: "RT_ECUDA", 4: "RT_ENOTCONVERGED", 5: "RT_ETIMEOUT",
           6: "RT_EDEVICE"}


class RtError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s: %s" % (_STATUS.get(code, code), msg))
        self.code = code


class rt_grid_desc(ctypes.Structure):
    _fields_ = [("coord", ctypes.c_int), ("n", ctypes.c_int * 3), ("edges", ctypes.c_void_p * 3),
                ("n_angles", ctypes.c_int), ("dirs", ctypes.c_void_p), ("weights", ctypes.c_void_p),
                ("inner_bc", ctypes.c_int), ("interp", ctypes.c_int), ("I_outer", ctypes.c_double),
                ("precision", ctypes.c_int), ("use_lstar", ctypes.c_int), ("ng", ctypes.c_int),
                ("refine_every", ctypes.c_int), ("angle_block", ctypes.c_int), ("device", ctypes.c_int),
                ("stream", ctypes.c_void_p)]


class rt_info(ctypes.Structure):
    _fields_ = [("n_vox", ctypes.c_int64), ("n_angles", ctypes.c_int64), ("n_rays", ctypes.c_int64),
                ("n_segments", ctypes.c_int64), ("device_bytes", ctypes.c_int64), ("n_blocks", ctypes.c_int32),
                ("angle_block", ctypes.c_int32), ("lost_rays", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("geometry_ms", ctypes.c_double), ("geometry_trace_ms", ctypes.c_double),
                ("geometry_lists_ms", ctypes.c_double)]


class rt_timing(ctypes.Structure):
    _fields_ = [("march_ms", ctypes.c_double), ("gather_ms", ctypes.c_double), ("march_launches", ctypes.c_int64),
                ("gather_launches", ctypes.c_int64), ("march_segments", ctypes.c_int64),
                ("kernel_launches", ctypes.c_int64), ("march_bytes", ctypes.c_int64), ("os_ms", ctypes.c_double),
                ("os_solves", ctypes.c_int64), ("os_krylov_its", ctypes.c_int64), ("os_sweeps", ctypes.c_int64)]


_lib = None
_P = ctypes.c_void_p
_I = ctypes.c_int


def load():
    """Load librt3d.so (built by paper_0903_1949_gb300.build); raise if it is absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("librt3d.so not found at %s: build it first (paper_0903_1949_gb300.build.build())"
                           % LIB_PATH)
    L = ctypes.CDLL(LIB_PATH)
    L.rt_last_error.restype = ctypes.c_char_p
    L.rt_last_error.argtypes = []
    sig = {
        "rt_grid_create": [ctypes.POINTER(_P), ctypes.POINTER(rt_grid_desc)],
        "rt_grid_destroy": [_P],
        "rt_get_info": [_P, ctypes.POINTER(rt_info)],
        "rt_set_opacity": [_P, _P, _P, _P, _I],
        "rt_set_S": [_P, _P, _I],
        "rt_formal_solution": [_P],
        "rt_formal_solution_ex": [_P, _I, _I],
        "rt_ali_step": [_P, ctypes.POINTER(ctypes.c_double)],
        "rt_solve": [_P, ctypes.c_double, _I, ctypes.POINTER(_I)],
        "rt_get_J": [_P, _P, _I],
        "rt_get_S": [_P, _P, _I],
        "rt_get_Lstar": [_P, _P, _I],
        "rt_get_flux": [_P, _P, _I],
        "rt_get_history": [_P, _P, _I, ctypes.POINTER(_I)],
        "rt_get_crossings": [_P, _I, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64), _P, _P, _P,
                             _P, _P, _P],
        "rt_fs_angles": [_P, _P, _I, _I, _P, _P, _I],
        "rt_set_timing": [_P, _I],
        "rt_set_precision": [_P, _I],
        "rt_tune": [_P, _I, _I],
        "rt_fs_angle_noalloc": [_P, _I, _I, _P, _P],
        "rt_batch_create": [ctypes.POINTER(_P), ctypes.POINTER(_P), _I, _I, _P, _P],
        "rt_batch_destroy": [_P],
        "rt_batch_set_member": [_P, _I, _P, _P, _P, _I],
        "rt_batch_ali_step": [_P, _P],
        "rt_batch_solve": [_P, ctypes.c_double, _I, _P],
        "rt_batch_get": [_P, _I, _I, _P, _I],
        "rt_batch_autotune": [_P, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32),
                              ctypes.POINTER(ctypes.c_double)],
        "rt_get_timing": [_P, ctypes.POINTER(rt_timing)],
        "rt_adjoint": [_P, _P, _P, _P, ctypes.c_double, _I, _P, _P, _P, _I, ctypes.POINTER(_I)],
        "rt_get_Lstar_nn": [_P, _P, _I],
        "rt_line_create": [ctypes.POINTER(_P), _P, _I, _P, _P, _I, _I, _P],
        "rt_line_set": [_P, _P, _P, _P, _P, _I],
        "rt_line_step": [_P, _P],
        "rt_line_solve": [_P, ctypes.c_double, _I, ctypes.POINTER(ctypes.c_int32)],
        "rt_line_get": [_P, _I, _P, _I],
        "rt_fs_sweep": [ctypes.POINTER(rt_grid_desc), _I, _P, _P, _P, _I, _P, _P, _I],
        "rt_measure_fp64_rate": [_I, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)],
    }
    for name, args in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = _I
    _lib = L
    return L


def _check(rc):
    if rc != RT_OK:
        raise RtError(rc, load().rt_last_error().decode())
    return rc


def _ptr(x):
    """(pointer, where, keepalive) of a host numpy array or a CUDA tensor of float64."""
    if hasattr(x, "data_ptr") and getattr(x, "is_cuda", False):
        if str(x.dtype) != "torch.float64" or not x.is_contiguous():
            raise TypeError("device arrays must be contiguous float64 CUDA tensors")
        return ctypes.c_void_p(x.data_ptr()), RT_DEVICE, x
    a = np.ascontiguousarray(x, dtype=np.float64)
    return ctypes.c_void_p(a.ctypes.data), RT_HOST, a


# ---- the C ABI, one function per entry point ----------------------------------

def rt_last_error():
    return load().rt_last_error().decode()


def _desc(coord, edges, dirs, weights, inner_bc=RT_CORE_B, interp=RT_PARABOLIC, I_outer=0.0, precision=RT_FP64,
          use_lstar=True, ng=True, refine_every=0, angle_block=0, device=0, stream=None):
    """(rt_grid_desc, arrays it points to)."""
    keep = [np.ascontiguousarray(e, dtype=np.float64) for e in edges]
    dirs = np.ascontiguousarray(np.asarray(dirs, dtype=np.float64).reshape(-1, 3))
    wts = np.ascontiguousarray(weights, dtype=np.float64)
    d = rt_grid_desc()
    d.coord = int(coord)
    for a in range(3):
        d.n[a] = len(keep[a]) - 1
        d.edges[a] = keep[a].ctypes.data
    d.n_angles = len(wts)
    d.dirs = dirs.ctypes.data
    d.weights = wts.ctypes.data
    d.inner_bc, d.interp, d.I_outer = int(inner_bc), int(interp), float(I_outer)
    lst = (1 if use_lstar else 0) if isinstance(use_lstar, bool) else int(use_lstar)
    d.precision, d.use_lstar, d.ng = int(precision), lst, 1 if ng else 0
    d.refine_every, d.angle_block, d.device = int(refine_every), int(angle_block), int(device)
    d.stream = stream if stream else None
    return d, (keep, dirs, wts)


def rt_grid_create(coord, edges, dirs, weights, inner_bc=RT_CORE_B, interp=RT_PARABOLIC, I_outer=0.0,
                   precision=RT_FP64, use_lstar=True, ng=True, refine_every=0, angle_block=0, device=0, stream=None):
    L = load()
    d, keep = _desc(coord, edges, dirs, weights, inner_bc, interp, I_outer, precision, use_lstar, ng, refine_every,
                    angle_block, device, stream)
    h = ctypes.c_void_p()
    _check(L.rt_grid_create(ctypes.byref(h), ctypes.byref(d)))
    return h


def rt_fs_sweep(coord, edges, dirs, weights, chi, S, B, angles_per_chunk, precision=RT_MIXED, inner_bc=RT_CORE_B,
                interp=RT_PARABOLIC, I_outer=0.0, angle_block=0, device=0, stream=None, J=None, F=None):
    """J (n_vox) and flux (n_vox, 3; local basis) of (chi, S, B) over the whole solid-angle set,
    angles_per_chunk solid angles at a time.  Host arrays in and out, or CUDA float64 tensors
    for chi, S, B with J and F given as CUDA tensors (written in place)."""
    d, keep = _desc(coord, edges, dirs, weights, inner_bc, interp, I_outer, precision, True, False, 0, angle_block,
                    device, stream)
    n = d.n[0] * d.n[1] * d.n[2]
    ins = [_ptr(a) for a in (chi, S, B)]
    where = ins[0][1]
    if any(w != where for _, w, _ in ins):
        raise TypeError("chi, S and B must live in the same memory space")
    if where == RT_HOST:
        for a in (chi, S, B):
            _host(a, n)  # size check
        J, F = np.empty(n), np.empty((n, 3))
    elif J is None or F is None:
        raise TypeError("device inputs need device outputs J (n_vox) and F (n_vox, 3)")
    pj, wj, _ = _ptr(J)
    pf, wf, _ = _ptr(F)
    if wj != where or wf != where:
        raise TypeError("J and F must live where the inputs do")
    _check(load().rt_fs_sweep(ctypes.byref(d), int(angles_per_chunk), ins[0][0], ins[1][0], ins[2][0], int(precision),
                              pj, pf, where))
    return J, F


def _host(x, n):
    a = np.ascontiguousarray(x, dtype=np.float64).reshape(-1)
    if a.size != n:
        raise ValueError("expected %d values, got %d" % (n, a.size))
    return a, ctypes.c_void_p(a.ctypes.data)


def rt_grid_destroy(h):
    return _check(load().rt_grid_destroy(h))


def rt_get_info(h):
    info = rt_info()
    _check(load().rt_get_info(h, ctypes.byref(info)))
    return {k: getattr(info, k) for k, _ in rt_info._fields_}


def rt_set_opacity(h, chi, eps, B):
    pc, wc, k1 = _ptr(chi)
    pe, we, k2 = _ptr(eps)
    pb, wb, k3 = _ptr(B)
    if not (wc == we == wb):
        raise TypeError("chi, eps and B must live in the same memory space")
    return _check(load().rt_set_opacity(h, pc, pe, pb, wc))


def rt_set_S(h, S):
    p, w, k = _ptr(S)
    return _check(load().rt_set_S(h, p, w))


def rt_formal_solution(h):
    return _check(load().rt_formal_solution(h))


def rt_formal_solution_ex(h, precision, homog=False):
    return _check(load().rt_formal_solution_ex(h, int(precision), 1 if homog else 0))


def rt_ali_step(h):
    rel = ctypes.c_double()
    _check(load().rt_ali_step(h, ctypes.byref(rel)))
    return rel.value


def rt_solve(h, tol, max_iter):
    it = ctypes.c_int()
    rc = load().rt_solve(h, float(tol), int(max_iter), ctypes.byref(it))
    if rc not in (RT_OK, RT_ENOTCONVERGED):
        _check(rc)
    return it.value, rc == RT_OK


def _get(fn, h, n, out):
    if out is None:
        out = np.empty(n)
    p, w, k = _ptr(out)
    _check(fn(h, p, w))
    return out


def rt_get_J(h, n_vox, out=None):
    return _get(load().rt_get_J, h, n_vox, out)


def rt_get_S(h, n_vox, out=None):
    return _get(load().rt_get_S, h, n_vox, out)


def rt_get_Lstar(h, n_vox, out=None):
    return _get(load().rt_get_Lstar, h, n_vox, out)


def rt_get_Lstar_nn(h, n_vox, out=None):
    f = _get(load().rt_get_Lstar_nn, h, 27 * n_vox, out)
    return f.reshape(n_vox, 27) if isinstance(f, np.ndarray) else f


def rt_get_flux(h, n_vox, out=None):
    f = _get(load().rt_get_flux, h, 3 * n_vox, out)
    return f.reshape(n_vox, 3) if isinstance(f, np.ndarray) else f


def rt_get_history(h):
    n = ctypes.c_int()
    _check(load().rt_get_history(h, None, 0, ctypes.byref(n)))
    buf = np.empty(max(1, n.value))
    _check(load().rt_get_history(h, ctypes.c_void_p(buf.ctypes.data), n.value, ctypes.byref(n)))
    return buf[:n.value]


def rt_adjoint(h, n_vox, dL_dS=None, dL_dJ=None, dL_dF=None, tol=1e-10, max_iter=10000, device=False):
    """(dchi, deps, dB, iters, converged) of a loss with gradients dL_dS, dL_dJ (n_vox) and
    dL_dF (n_vox x 3, local basis) at the grid's current S.  device=True: CUDA float64
    tensors in and out (then every given gradient must be a CUDA tensor)."""
    keep = []

    def arg(x):
        if x is None:
            return None, None
        p, w, k = _ptr(x)
        keep.append(k)
        return p, w
    ins = [arg(x) for x in (dL_dS, dL_dJ, dL_dF)]
    where = RT_DEVICE if device else RT_HOST
    if any(w is not None and w != where for _, w in ins):
        raise TypeError("gradients and outputs must live in the same memory space")
    if device:
        import torch
        outs = [torch.empty(n_vox, dtype=torch.float64, device="cuda") for _ in range(3)]
    else:
        outs = [np.empty(n_vox) for _ in range(3)]
    po = [_ptr(o)[0] for o in outs]
    it = ctypes.c_int()
    rc = load().rt_adjoint(h, ins[0][0], ins[1][0], ins[2][0], float(tol), int(max_iter), po[0], po[1], po[2], where,
                           ctypes.byref(it))
    if rc not in (RT_OK, RT_ENOTCONVERGED):
        _check(rc)
    return outs[0], outs[1], outs[2], it.value, rc == RT_OK


def rt_get_crossings(h, omega):
    nr, ns = ctypes.c_int64(), ctypes.c_int64()
    L = load()
    _check(L.rt_get_crossings(h, int(omega), ctypes.byref(nr), ctypes.byref(ns), None, None, None, None, None, None))
    nr, ns = nr.value, ns.value
    out = dict(ray_off=np.empty(nr + 1, np.int32), ray_origin=np.empty(nr, np.int32), ray_core=np.empty(nr, np.int32),
               vox=np.empty(ns, np.int32), len=np.empty(ns, np.float64), restart=np.empty(ns, np.uint8))
    a, b = ctypes.c_int64(), ctypes.c_int64()
    _check(L.rt_get_crossings(h, int(omega), ctypes.byref(a), ctypes.byref(b),
                              *(ctypes.c_void_p(out[k].ctypes.data)
                                for k in ("ray_off", "ray_origin", "ray_core", "vox", "len", "restart"))))
    return out


def rt_fs_angles(h, omegas, precision, n_vox):
    om = np.ascontiguousarray(omegas, dtype=np.int32)
    Ib = np.empty((len(om), n_vox))
    Lb = np.empty((len(om), n_vox))
    _check(load().rt_fs_angles(h, ctypes.c_void_p(om.ctypes.data), len(om), int(precision),
                               ctypes.c_void_p(Ib.ctypes.data), ctypes.c_void_p(Lb.ctypes.data), RT_HOST))
    return Ib, Lb


def rt_set_precision(h, precision):
    return _check(load().rt_set_precision(h, int(precision)))


def rt_fs_angle_noalloc(h, omega, precision, Ibar_dev, Lbar_dev):
    """One solid angle's Ibar / Lambda* into caller-owned CUDA tensors; allocates nothing."""
    if not (getattr(Ibar_dev, "is_cuda", False) and getattr(Lbar_dev, "is_cuda", False)):
        raise TypeError("rt_fs_angle_noalloc writes device buffers: pass CUDA tensors")
    return _check(load().rt_fs_angle_noalloc(h, int(omega), int(precision), ctypes.c_void_p(Ibar_dev.data_ptr()),
                                             ctypes.c_void_p(Lbar_dev.data_ptr())))


def rt_tune(h, knob, value):
    return _check(load().rt_tune(h, int(knob), int(value)))


def rt_measure_fp64_rate(device=0):
    """(FP64 flop/s of the device, ms per launch of the FMA-chain kernel)."""
    f, ms = ctypes.c_double(), ctypes.c_double()
    _check(load().rt_measure_fp64_rate(int(device), ctypes.byref(f), ctypes.byref(ms)))
    return f.value, ms.value


def rt_set_timing(h, enable=True):
    """enable: False/0 off, True/1 every march and gather launch, N > 1 every N-th march launch."""
    v = int(enable) if not isinstance(enable, bool) else (1 if enable else 0)
    return _check(load().rt_set_timing(h, v))


def rt_get_timing(h):
    t = rt_timing()
    _check(load().rt_get_timing(h, ctypes.byref(t)))
    return {k: getattr(t, k) for k, _ in rt_timing._fields_}


def rt_batch_create(grid_handles, member_grid, stream=None):
    L = load()
    arr = (ctypes.c_void_p * len(grid_handles))(*[h.value if hasattr(h, "value") else h for h in grid_handles])
    mg = np.ascontiguousarray(member_grid, dtype=np.int32)
    h = ctypes.c_void_p()
    _check(L.rt_batch_create(ctypes.byref(h), ctypes.cast(arr, ctypes.POINTER(ctypes.c_void_p)), len(grid_handles),
                             len(mg), ctypes.c_void_p(mg.ctypes.data), stream if stream else None))
    return h


def rt_batch_destroy(h):
    return _check(load().rt_batch_destroy(h))


def rt_batch_set_member(h, m, chi, eps, B):
    pc, wc, k1 = _ptr(chi)
    pe, we, k2 = _ptr(eps)
    pb, wb, k3 = _ptr(B)
    if not (wc == we == wb):
        raise TypeError("chi, eps and B must live in the same memory space")
    return _check(load().rt_batch_set_member(h, int(m), pc, pe, pb, wc))


def rt_batch_ali_step(h, n_members):
    rel = np.empty(n_members)
    _check(load().rt_batch_ali_step(h, ctypes.c_void_p(rel.ctypes.data)))
    return rel


def rt_batch_solve(h, tol, max_iter, n_members):
    it = np.zeros(n_members, np.int32)
    rc = load().rt_batch_solve(h, float(tol), int(max_iter), ctypes.c_void_p(it.ctypes.data))
    if rc not in (RT_OK, RT_ENOTCONVERGED):
        _check(rc)
    return it, rc == RT_OK


def rt_batch_get(h, m, what, n_vox, out=None):
    return _get(lambda hh, p, w: load().rt_batch_get(hh, int(m), int(what), p, w), h, n_vox, out)


def rt_batch_autotune(h):
    c, g, ms = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_double()
    _check(load().rt_batch_autotune(h, ctypes.byref(c), ctypes.byref(g), ctypes.byref(ms)))
    return c.value, g.value, ms.value


class Batch:
    """Many opacity fields on a few grids, iterated together (see rt_batch_* in rt.h)."""

    def __init__(self, grids, member_grid, stream=None):
        self.grids = list(grids)  # kept alive: the batch uses their geometry
        self.member_grid = list(member_grid)
        self.h = None
        self.h = rt_batch_create([g.h for g in self.grids], member_grid, stream)
        self.nvox = [self.grids[q].nvox for q in self.member_grid]

    def close(self):
        if self.h:
            rt_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_member(self, m, chi, eps, B):
        rt_batch_set_member(self.h, m, chi, eps, B)

    def ali_step(self):
        return rt_batch_ali_step(self.h, len(self.member_grid))

    def solve(self, tol, max_iter):
        return rt_batch_solve(self.h, tol, max_iter, len(self.member_grid))

    def S(self, m):
        return rt_batch_get(self.h, m, 0, self.nvox[m])

    def J(self, m):
        return rt_batch_get(self.h, m, 1, self.nvox[m])

    def Lstar(self, m):
        return rt_batch_get(self.h, m, 2, self.nvox[m])

    def autotune(self):
        return rt_batch_autotune(self.h)


def rt_line_create(grid_handle, phi, wq, use_lstar=RT_LSTAR_DIAG, ng=False, stream=None):
    phi = np.ascontiguousarray(phi, dtype=np.float64)
    wq = np.ascontiguousarray(wq, dtype=np.float64)
    if phi.shape != wq.shape or phi.ndim != 1:
        raise ValueError("phi and wq: one value per frequency each")
    h = ctypes.c_void_p()
    _check(load().rt_line_create(ctypes.byref(h), grid_handle, int(phi.size), ctypes.c_void_p(phi.ctypes.data),
                                 ctypes.c_void_p(wq.ctypes.data), int(use_lstar), int(ng),
                                 stream if stream else None))
    return h


def rt_line_set(h, chi_c, chi_l, eps_l, B):
    ptrs = [_ptr(a) for a in (chi_c, chi_l, eps_l, B)]
    if len({w for _, w, _ in ptrs}) != 1:
        raise TypeError("chi_c, chi_l, eps_l and B must live in the same memory space")
    return _check(load().rt_line_set(h, *[p for p, _, _ in ptrs], ptrs[0][1]))


def rt_line_step(h):
    rel = ctypes.c_double()
    _check(load().rt_line_step(h, ctypes.byref(rel)))
    return rel.value


def rt_line_solve(h, tol, max_iter):
    it = ctypes.c_int32()
    rc = load().rt_line_solve(h, float(tol), int(max_iter), ctypes.byref(it))
    if rc not in (RT_OK, RT_ENOTCONVERGED):
        _check(rc)
    return it.value, rc == RT_OK


def rt_line_get(h, what, n_vox, out=None):
    return _get(lambda hh, p, w: load().rt_line_get(hh, int(what), p, w), h, n_vox, out)


class Line(Batch):
    """Two-level-atom line on one grid, one batch member per frequency (see rt_line_* in rt.h)."""

    def __init__(self, grid, phi, wq, use_lstar=RT_LSTAR_DIAG, ng=False, stream=None):
        self.grids = [grid]
        self.member_grid = [0] * len(phi)
        self.h = None
        self.h = rt_line_create(grid.h, phi, wq, use_lstar, ng, stream)
        self.nvox = [grid.nvox] * len(phi)
        self.n = grid.nvox

    def set(self, chi_c, chi_l, eps_l, B):
        rt_line_set(self.h, chi_c, chi_l, eps_l, B)

    def step(self):
        return rt_line_step(self.h)

    def solve(self, tol, max_iter):
        return rt_line_solve(self.h, tol, max_iter)

    def S_l(self):
        return rt_line_get(self.h, 0, self.n)

    def Jbar(self):
        return rt_line_get(self.h, 1, self.n)

    def Lbar(self):
        return rt_line_get(self.h, 2, self.n)

    def Lbar_nn(self):
        return rt_line_get(self.h, 3, 27 * self.n).reshape(self.n, 27)


class Grid:
    """Owning handle around rt_grid with numpy-friendly accessors."""

    def __init__(self, coord, edges, dirs, weights, **kw):
        self.n = tuple(len(e) - 1 for e in edges)
        self.nvox = int(np.prod(self.n))
        self.n_ang = len(weights)
        self.h = rt_grid_create(coord, edges, dirs, weights, **kw)

    def close(self):
        if self.h:
            rt_grid_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self):
        return rt_get_info(self.h)

    def set_opacity(self, chi, eps, B):
        rt_set_opacity(self.h, chi, eps, B)

    def set_S(self, S):
        rt_set_S(self.h, S)

    def formal_solution(self, precision=None, homog=False):
        if precision is None and not homog:
            rt_formal_solution(self.h)
        else:
            rt_formal_solution_ex(self.h, RT_FP64 if precision is None else precision, homog)

    def ali_step(self):
        return rt_ali_step(self.h)

    def solve(self, tol=1e-8, max_iter=1000):
        return rt_solve(self.h, tol, max_iter)

    def J(self, out=None):
        return rt_get_J(self.h, self.nvox, out)

    def S(self, out=None):
        return rt_get_S(self.h, self.nvox, out)

    def Lstar(self, out=None):
        return rt_get_Lstar(self.h, self.nvox, out)

    def flux(self, out=None):
        return rt_get_flux(self.h, self.nvox, out)

    def Lstar_nn(self, out=None):
        return rt_get_Lstar_nn(self.h, self.nvox, out)

    def history(self):
        return rt_get_history(self.h)

    def crossings(self, omega):
        return rt_get_crossings(self.h, omega)

    def fs_angles(self, omegas, precision=RT_FP64):
        return rt_fs_angles(self.h, omegas, precision, self.nvox)

    def set_precision(self, precision):
        rt_set_precision(self.h, precision)

    def tune(self, knob, value):
        rt_tune(self.h, knob, value)

    def set_timing(self, enable=True):
        rt_set_timing(self.h, enable)

    def timing(self):
        return rt_get_timing(self.h)

    def adjoint(self, dL_dS=None, dL_dJ=None, dL_dF=None, tol=1e-10, max_iter=10000, device=False):
        return rt_adjoint(self.h, self.nvox, dL_dS, dL_dJ, dL_dF, tol, max_iter, device)
