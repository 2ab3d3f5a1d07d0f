"""Formal solution over a solid-angle set processed in chunks (rt_fs_sweep):
the chunked J and flux against one grid holding every angle and against the
oracle (FP64 1e-12, mixed 1e-5), uneven chunk sizes, and the flux vectors of
the outermost voxels of the paper's 65 x 33 x 65 grid becoming radial as the
solid-angle set is refined (Sect. 3.2.2)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_0903_1949_gb300 import build as Bd
from paper_0903_1949_gb300 import inputs as I
from paper_0903_1949_gb300 import rt
from tests.helpers import tiny_problem

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    Bd.build()
    rt.load()


def _sweep(p, S, chunk, precision):
    return rt.rt_fs_sweep(p["coord"], p["edges"], p["dirs"], p["weights"], p["chi"], S, p["B"], chunk,
                          precision=precision, inner_bc=p["inner_bc"])


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


@pytest.mark.parametrize("coord,bc", [(I.SPHERICAL, I.CORE_B), (I.CYLINDRICAL, I.TRANSPARENT)])
def test_sweep_matches_one_grid_and_oracle(coord, bc):
    n3 = (9, 6, 8) if coord == I.SPHERICAL else (8, 7, 6)
    p = tiny_problem(coord, n3, 6, 6, bc, seed=61)
    S = p["B"] * np.random.default_rng(3).uniform(0.5, 2.0, p["nvox"])
    o = O.OracleGrid(p["coord"], p["edges"], p["dirs"], p["weights"], p["inner_bc"])
    J_o, _, F_o, miss = o.formal_solution(S, p["chi"], p["B"])
    assert miss == 0
    g = rt.Grid(p["coord"], p["edges"], p["dirs"], p["weights"], inner_bc=p["inner_bc"], precision=rt.RT_FP64)
    g.set_opacity(p["chi"], p["eps"], p["B"])
    g.set_S(S)
    g.formal_solution(rt.RT_FP64)
    J_g, F_g = g.J(), g.flux()
    g.close()
    for chunk in (36, 7, 5, 1):  # one chunk, uneven chunks, one angle per chunk
        J, F = _sweep(p, S, chunk, rt.RT_FP64)
        assert _rel(J, J_g) < 1e-13 and _rel(F, F_g) < 1e-13, chunk
        assert _rel(J, J_o) < 1e-12 and _rel(F, F_o) < 1e-12, chunk
    J, F = _sweep(p, S, 10, rt.RT_MIXED)
    assert _rel(J, J_o) < 1e-5 and _rel(F, F_o) < 1e-5


def test_sweep_device_buffers():
    """CUDA tensors in and out give the host path's numbers."""
    torch = pytest.importorskip("torch")
    p = tiny_problem(I.SPHERICAL, (9, 6, 8), 6, 6, I.CORE_B, seed=63)
    S = p["B"] * np.random.default_rng(4).uniform(0.5, 2.0, p["nvox"])
    J_h, F_h = _sweep(p, S, 7, rt.RT_FP64)
    dev = [torch.tensor(a, dtype=torch.float64, device="cuda") for a in (p["chi"], S, p["B"])]
    J_d = torch.empty(p["nvox"], dtype=torch.float64, device="cuda")
    F_d = torch.empty((p["nvox"], 3), dtype=torch.float64, device="cuda")
    rt.rt_fs_sweep(p["coord"], p["edges"], p["dirs"], p["weights"], *dev, 7, precision=rt.RT_FP64,
                   inner_bc=p["inner_bc"], J=J_d, F=F_d)
    torch.cuda.synchronize()
    assert np.array_equal(J_d.cpu().numpy(), J_h) and np.array_equal(F_d.cpu().numpy(), F_h)


def test_sweep_argument_checks():
    p = tiny_problem(I.SPHERICAL, (5, 4, 6), 4, 4, I.CORE_B, seed=62)
    for kw in (dict(chunk=0), dict(precision=7)):
        with pytest.raises(rt.RtError) as ei:
            rt.rt_fs_sweep(p["coord"], p["edges"], p["dirs"], p["weights"], p["chi"], p["B"], p["B"],
                           kw.get("chunk", 4), precision=kw.get("precision", rt.RT_FP64), inner_bc=p["inner_bc"])
        assert ei.value.code == rt.RT_EINVAL
    with pytest.raises(rt.RtError) as ei:  # weights must sum to 1
        rt.rt_fs_sweep(p["coord"], p["edges"], p["dirs"], 2 * p["weights"], p["chi"], p["B"], p["B"], 4,
                       inner_bc=p["inner_bc"])
    assert ei.value.code == rt.RT_EINVAL


def test_full_size_outer_flux_vectors_become_radial():
    """A frequency of the eps_l = 1 line (S = B, spherically symmetric) where the
    outermost voxels are optically thin, on the 65 x 33 x 65 grid: F_phi and the
    scatter of F_r over the outermost shell fall from 8^2 to 48^2 solid angles,
    and F_theta does not grow (the polar rows set its floor)."""
    q = I.line_problem("sph65", n_freq=32, ratio=1e6, eps_l=1.0, noise=0.0)
    tau = 1e-2 * (1.0 + 1e6 * q["phi"])
    k = int(np.argmin(np.abs(np.log(tau / 10.0))))
    chi = q["chi_c"] + q["chi_l"] * q["phi"][k]
    res = []
    for na in (8, 48):
        dirs, w = I.angle_set(na, na)
        J, F = rt.rt_fs_sweep(q["coord"], q["edges"], dirs, w, chi, q["B"], q["B"], 1024, inner_bc=q["inner_bc"])
        out = F.reshape(65, 33 * 65, 3)[-1]
        Fr = out[:, 0].mean()
        assert np.all(np.isfinite(F)) and Fr > 0
        res.append((out[:, 0].max() / out[:, 0].min() - 1.0, np.abs(out[:, 1]).max() / Fr,
                    np.abs(out[:, 2]).max() / Fr))
    assert res[1][0] < 0.5 * res[0][0] and res[1][2] < 0.5 * res[0][2], res
    assert res[1][1] <= res[0][1], res
