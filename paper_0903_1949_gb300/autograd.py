"""torch.autograd interface of the converged ALI solution.

`solve(grid, chi, eps, B)` runs the ALI iteration of the grid (Sect. 3.2.1) to
convergence from per-voxel chi, eps and B given as CUDA float64 tensors and
returns (S, J, F).  Its backward pass is the adjoint of the fixed point
S = (1 - eps) J(S; chi, B) + eps B, computed by rt_adjoint: one adjoint ALI
solve with the ray march run backwards along the characteristics, then one
pass for the chi and B sensitivities.  The parabola-or-linear choice of every
segment counts as fixed (it changes only where dtau_{k+1} = dtau_k / 2).
"""
import torch

from . import rt


class _Solve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, grid, chi, eps, B, tol, max_iter, adj_tol, adj_max_iter):
        for name, x in (("chi", chi), ("eps", eps), ("B", B)):
            if not (x.is_cuda and x.dtype == torch.float64):
                raise TypeError("%s must be a CUDA float64 tensor" % name)
        grid.set_opacity(chi.detach().contiguous(), eps.detach().contiguous(), B.detach().contiguous())
        it, ok = grid.solve(tol, max_iter)
        if not ok:
            raise rt.RtError(rt.RT_ENOTCONVERGED, "ALI did not converge in %d iterations" % max_iter)
        n = grid.nvox
        S = torch.empty(n, dtype=torch.float64, device=chi.device)
        J = torch.empty(n, dtype=torch.float64, device=chi.device)
        F = torch.empty(3 * n, dtype=torch.float64, device=chi.device)
        grid.S(S)
        grid.J(J)
        rt.rt_get_flux(grid.h, n, F)
        ctx.grid = grid
        ctx.adj = (adj_tol, adj_max_iter)
        return S, J, F.view(n, 3)

    @staticmethod
    def backward(ctx, gS, gJ, gF):
        grid = ctx.grid
        args = [None if g is None else g.detach().contiguous().to(torch.float64) for g in (gS, gJ, gF)]
        if args[2] is not None:
            args[2] = args[2].reshape(-1)
        dchi, deps, dB, it, ok = grid.adjoint(args[0], args[1], args[2], tol=ctx.adj[0], max_iter=ctx.adj[1],
                                              device=True)
        if not ok:
            raise rt.RtError(rt.RT_ENOTCONVERGED, "adjoint ALI did not converge in %d sweeps" % ctx.adj[1])
        return None, dchi, deps, dB, None, None, None, None


def solve(grid, chi, eps, B, tol=1e-12, max_iter=20000, adj_tol=1e-12, adj_max_iter=20000):
    """Converged (S, J, F) of `grid` (an rt.Grid) for the given fields, differentiable in chi, eps and B.

    The gradients hold at the forward's converged S (the grid's state when backward runs:
    do not solve another field on the same grid between forward and backward)."""
    return _Solve.apply(grid, chi, eps, B, tol, max_iter, adj_tol, adj_max_iter)
