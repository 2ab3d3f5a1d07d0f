"""Gradients of the converged ALI solution with respect to chi, eps and B
(rt_adjoint and the torch.autograd wrapper) against central finite
differences: of the GPU's own FP64 solve on seeded voxels, and brute force of
the FP64 oracle's solve on a tiny grid.

The loss is L = a_S . S + a_J . J + a_F . F with seeded random weights, so
dL/dS = a_S etc.; S is the fixed point S = (1 - eps) J(S) + eps B (Sect.
3.2.1) and J, F the formal solution at it (Sect. 2)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_0903_1949_gb300 import build as Bd
from paper_0903_1949_gb300 import inputs as I
from paper_0903_1949_gb300 import rt
from tests.helpers import tiny_problem

pytestmark = pytest.mark.gpu

H_REL = 1e-6        # central-difference step, relative to the perturbed value
TOL_FD = 1e-6       # |FD - adjoint| <= TOL_FD * max|adjoint| of that field
N_VOX_FD = 20       # seeded voxels per field (GPU finite differences)


@pytest.fixture(scope="module", autouse=True)
def _built():
    Bd.build()
    rt.load()


def _case(name):
    rng = np.random.default_rng({"sph_core": 11, "cyl_hole": 12, "sph_linear": 13}[name])
    if name == "sph_core":
        p = tiny_problem(I.SPHERICAL, (7, 5, 9), 4, 4, I.CORE_B, eps=0.1, seed=3)
        interp = rt.RT_PARABOLIC
    elif name == "cyl_hole":
        p = tiny_problem(I.CYLINDRICAL, (6, 7, 5), 4, 4, I.TRANSPARENT, eps=0.05, seed=4)
        interp = rt.RT_PARABOLIC
    else:
        p = tiny_problem(I.SPHERICAL, (6, 4, 6), 4, 4, I.CORE_B, eps=0.2, seed=5)
        interp = rt.RT_LINEAR
    n = p["nvox"]
    p["eps"] = p["eps"] * (0.5 + rng.uniform(size=n))
    p["B"] = 1.0 + 0.5 * rng.uniform(size=n)
    w = dict(S=rng.standard_normal(n), J=rng.standard_normal(n), F=rng.standard_normal((n, 3)))
    return p, interp, w


def _grid(p, interp):
    return rt.Grid(p["coord"], p["edges"], p["dirs"], p["weights"], inner_bc=p["inner_bc"], interp=interp,
                   precision=rt.RT_FP64, ng=True)


def _converge(g, max_iter=3000, floor=1e-14):
    """ALI steps until max rel dS reaches the FP64 rounding floor.  The ALI amplifies
    the rounding of J by up to (1 - eps) / (1 - (1 - eps) Lambda) ~ 1 / eps in thick
    media, so at small eps the floor is higher: there the steps go on until max rel dS
    has not reached a new low for 20 steps (it then fluctuates at the floor)."""
    rel, best, best_it = 1.0, np.inf, 0
    for it in range(max_iter):
        rel = g.ali_step()
        if rel < 0.1 * floor:
            break
        if rel < best:
            best, best_it = rel, it
        elif best < floor and it - best_it >= 20:
            break
    assert min(rel, best) < floor, rel


def _loss_gpu(g, w, kinds, chi, eps, B):
    g.set_opacity(chi, eps, B)
    g.set_S(B)
    _converge(g)
    g.formal_solution(rt.RT_FP64)
    L = 0.0
    if "S" in kinds:
        L += w["S"] @ g.S()
    if "J" in kinds:
        L += w["J"] @ g.J()
    if "F" in kinds:
        L += np.sum(w["F"] * g.flux())
    return L


def _adjoint(g, w, kinds, p):
    g.set_opacity(p["chi"], p["eps"], p["B"])
    g.set_S(p["B"])
    _converge(g)
    dchi, deps, dB, it, ok = g.adjoint(w["S"] if "S" in kinds else None, w["J"] if "J" in kinds else None,
                                       w["F"].reshape(-1) if "F" in kinds else None, tol=1e-14, max_iter=5000)
    assert ok and it > 0
    return dict(chi=dchi, eps=deps, B=dB)


def _fd_check(loss, p, grads, fields, voxels, h_rel=None):
    for f in fields:
        gmax = np.max(np.abs(grads[f]))
        for v in voxels:
            args = {k: p[k].copy() for k in ("chi", "eps", "B")}
            h = (h_rel or {}).get(f, H_REL) * args[f][v]
            args[f][v] += h
            Lp = loss(args["chi"], args["eps"], args["B"])
            args[f][v] -= 2.0 * h
            Lm = loss(args["chi"], args["eps"], args["B"])
            fd = (Lp - Lm) / (2.0 * h)
            assert abs(fd - grads[f][v]) <= TOL_FD * gmax, (f, v, fd, grads[f][v], gmax)


@pytest.mark.parametrize("name,kinds", [("sph_core", "S"), ("sph_core", "J"), ("sph_core", "F"),
                                        ("cyl_hole", "SJF"), ("sph_linear", "SJF")])
def test_adjoint_matches_gpu_finite_differences(name, kinds):
    p, interp, w = _case(name)
    g = _grid(p, interp)
    grads = _adjoint(g, w, kinds, p)
    for f in ("chi", "eps", "B"):
        assert np.all(np.isfinite(grads[f])) and np.max(np.abs(grads[f])) > 0, f
    voxels = np.random.default_rng(99).choice(p["nvox"], N_VOX_FD, replace=False)
    _fd_check(lambda c, e, b: _loss_gpu(g, w, kinds, c, e, b), p, grads, ("chi", "eps", "B"), voxels)
    g.close()


@pytest.mark.parametrize("name", ["sph_core", "cyl_hole"])
def test_adjoint_matches_oracle_finite_differences(name):
    p, interp, w = _case(name)
    g = _grid(p, interp)
    grads = _adjoint(g, w, "SJF", p)
    g.close()
    o = O.OracleGrid(p["coord"], p["edges"], p["dirs"], p["weights"], p["inner_bc"])

    def loss(chi, eps, B):
        S, it, _ = o.solve(chi, eps, B, tol=1e-15, max_iter=400, ng=True)
        J, _, F, miss = o.formal_solution(S, chi, B)
        assert miss == 0
        return w["S"] @ S + w["J"] @ J + np.sum(w["F"] * F)

    voxels = np.random.default_rng(98).choice(p["nvox"], N_VOX_FD, replace=False)
    _fd_check(loss, p, grads, ("chi", "eps", "B"), voxels)


def test_autograd_wrapper_matches_rt_adjoint():
    torch = pytest.importorskip("torch")
    from paper_0903_1949_gb300 import autograd as A
    p, interp, w = _case("sph_core")
    g = _grid(p, interp)
    ref = _adjoint(g, w, "SJF", p)
    dev = "cuda"
    chi = torch.tensor(p["chi"], device=dev, requires_grad=True)
    eps = torch.tensor(p["eps"], device=dev, requires_grad=True)
    B = torch.tensor(p["B"], device=dev, requires_grad=True)
    S, J, F = A.solve(g, chi, eps, B, tol=1e-14, max_iter=5000, adj_tol=1e-14, adj_max_iter=5000)
    loss = (torch.tensor(w["S"], device=dev) * S).sum() + (torch.tensor(w["J"], device=dev) * J).sum() + \
        (torch.tensor(w["F"], device=dev) * F).sum()
    loss.backward()
    for name, t in (("chi", chi), ("eps", eps), ("B", B)):
        gref = ref[name]
        assert np.max(np.abs(t.grad.cpu().numpy() - gref)) <= 1e-9 * np.max(np.abs(gref)), name
    g.close()


def test_adjoint_reports_non_convergence_and_bad_arguments():
    p, interp, w = _case("sph_core")
    g = _grid(p, interp)
    g.set_opacity(p["chi"], p["eps"], p["B"])
    g.set_S(p["B"])
    _, _, _, it, ok = g.adjoint(w["S"], None, None, tol=1e-300, max_iter=2)
    assert not ok and it == 2
    with pytest.raises(rt.RtError) as ei:
        g.adjoint(w["S"], tol=0.0)
    assert ei.value.code == rt.RT_EINVAL
    g.close()


def _nn_case(eps_scale, chi_scale, seed):
    rng = np.random.default_rng(seed)
    p = tiny_problem(I.SPHERICAL, (7, 5, 9), 4, 4, I.CORE_B, eps=1.0, seed=seed)
    n = p["nvox"]
    p["chi"] = p["chi"] * chi_scale
    p["eps"] = eps_scale * (0.5 + rng.uniform(size=n))
    p["B"] = 1.0 + 0.5 * rng.uniform(size=n)
    w = dict(S=rng.standard_normal(n), J=rng.standard_normal(n), F=rng.standard_normal((n, 3)))
    return p, w


def _nn_grid(p, lstar):
    return rt.Grid(p["coord"], p["edges"], p["dirs"], p["weights"], inner_bc=p["inner_bc"], precision=rt.RT_FP64,
                   ng=True, use_lstar=lstar)


def test_nn_preconditioned_adjoint_equals_diagonal_one_in_fewer_sweeps():
    """Where the diagonal-Lambda* adjoint iteration converges, the NN-preconditioned one
    reaches the same adjoint (the fixed point does not depend on the preconditioner)."""
    p, w = _nn_case(0.05, 3.0, 31)
    out = {}
    for lstar in (rt.RT_LSTAR_DIAG, rt.RT_LSTAR_NN):
        g = _nn_grid(p, lstar)
        g.set_opacity(p["chi"], p["eps"], p["B"])
        g.set_S(p["B"])
        _converge(g)
        dchi, deps, dB, it, ok = g.adjoint(w["S"], w["J"], w["F"].reshape(-1), tol=1e-14, max_iter=20000)
        assert ok, lstar
        out[lstar] = (dict(chi=dchi, eps=deps, B=dB), it)
        g.close()
    (gd, itd), (gn, itn) = out[rt.RT_LSTAR_DIAG], out[rt.RT_LSTAR_NN]
    print("adjoint sweeps: diagonal %d, nearest-neighbour %d" % (itd, itn))
    assert itn < itd
    for f in ("chi", "eps", "B"):
        assert np.max(np.abs(gn[f] - gd[f])) <= 1e-10 * np.max(np.abs(gd[f])), f


def test_nn_preconditioned_adjoint_matches_finite_differences_at_small_eps():
    """eps ~ 1e-4 in an optically thick tiny grid, where the diagonal-Lambda* iteration is
    impractically slow: the NN-preconditioned adjoint against central differences of
    NN-converged FP64 solves, on seeded voxels of chi, eps and B."""
    p, w = _nn_case(1e-4, 30.0, 32)
    g = _nn_grid(p, rt.RT_LSTAR_NN)
    g.set_opacity(p["chi"], p["eps"], p["B"])
    g.set_S(p["B"])
    _converge(g, max_iter=1000, floor=1e-12)
    # the adjoint iterate carries the same ~1/eps amplification of FP64 rounding as S: 1e-11
    dchi, deps, dB, it, ok = g.adjoint(w["S"], w["J"], w["F"].reshape(-1), tol=1e-11, max_iter=2000)
    assert ok and it < 500, it
    print("NN adjoint sweeps at eps ~ 1e-4: %d" % it)
    grads = dict(chi=dchi, eps=deps, B=dB)
    voxels = np.random.default_rng(33).choice(p["nvox"], 6, replace=False)
    def loss(c, e, b):
        g.set_opacity(c, e, b)
        g.set_S(b)
        _converge(g, max_iter=1000, floor=1e-12)
        g.formal_solution(rt.RT_FP64)
        return w["S"] @ g.S() + w["J"] @ g.J() + np.sum(w["F"] * g.flux())

    # the converged loss carries ~1e-13 of FP64 noise (see _converge), which a central difference
    # divides by 2h: at eps ~ 1e-4 a step of 1e-4 eps leaves that noise at about the 1e-6 bar, so eps
    # is stepped by 1e-3 of itself (the h^2 truncation, ~(h/eps)^2 of the derivative, stays 1e2
    # below) and chi by 1e-5; L is linear in B (S is), so a step of 1e-2 B is exact there
    _fd_check(loss, p, grads, ("chi", "eps", "B"), voxels, h_rel={"chi": 1e-5, "eps": 1e-3, "B": 1e-2})
    g.close()


def test_nn_adjoint_in_the_tau_1e4_eps_1e8_regime():
    """The C5 regime (chi ~ r^-2 with radial tau 1e4, eps 1e-8) on a 33 x 17 x 33 grid
    with 8 x 8 solid angles: the forward NN solve and the NN-preconditioned adjoint both
    converge (their OS steps do not rely on contracting Jacobi sweeps).  S, J and F are
    linear in B, so central differences in B (h = 1e-2 B) carry only the solves' noise and
    resolve the B gradient; in chi and eps the ~1/eps conditioning of the fixed point
    leaves differences of FP64-converged solves too noisy for a 1e-6 check."""
    p = I.make_problem("sph65", n=(33, 17, 33), n_mu=8, n_phi=8, tau=1e4, eps=1e-8, noise=0.0)
    n = p["chi"].size
    rng = np.random.default_rng(5)
    w = dict(S=rng.standard_normal(n), J=rng.standard_normal(n), F=rng.standard_normal((n, 3)))
    g = rt.Grid(p["coord"], p["edges"], p["dirs"], p["weights"], inner_bc=p["inner_bc"], precision=rt.RT_FP64,
                use_lstar=rt.RT_LSTAR_NN)
    try:
        def loss(B):
            g.set_opacity(p["chi"], p["eps"], B)
            g.set_S(B)
            it, ok = g.solve(1e-9, 2000)
            assert ok, g.history()[-3:]
            g.formal_solution(rt.RT_FP64)
            return w["S"] @ g.S() + w["J"] @ g.J() + np.sum(w["F"] * g.flux())

        loss(p["B"])
        _, _, dB, it, ok = g.adjoint(w["S"], w["J"], w["F"].reshape(-1), tol=1e-9, max_iter=3000)
        assert ok, it
        print("NN adjoint sweeps at tau 1e4, eps 1e-8: %d" % it)
        gmax = np.max(np.abs(dB))
        for v in np.random.default_rng(33).choice(n, 6, replace=False):
            B = p["B"].copy()
            h = 1e-2 * B[v]
            B[v] += h
            Lp = loss(B)
            B[v] -= 2.0 * h
            Lm = loss(B)
            fd = (Lp - Lm) / (2.0 * h)
            assert abs(fd - dB[v]) <= 3e-5 * gmax, (v, fd, dB[v], gmax)
    finally:
        g.close()
