"""Differentiable load step: J = TCV after one load step of Algorithm 2 as a
torch function of the pressure p, the toughness G_c and the per-cell modulus E_K.

forward  runs the Newton / PDAS load step (pff_newton_pdas_step) and keeps the
         converged state (u, phi, phi_old, active set) as its checkpoint;
backward runs one adjoint solve at that state (pff_tcv_adjoint: transposed
         constrained Jacobian, GMRES with the block V-cycle, then the VJP of the
         residual with respect to the parameters).
"""
import torch

from . import newton_step, tcv_adjoint


class TCVLoadStep(torch.autograd.Function):
    """J = TCV(U(p, G_c, E)) for one load step; see ``tcv_load_step``."""

    @staticmethod
    def forward(ctx, p, Gc, E_cells, problem, mg, u, phi, phi_old, active, newton_kw, adjoint_kw):
        problem.set_params(p=float(p), Gc=float(Gc))
        problem.set_cell_modulus(None if E_cells is None else E_cells.detach().contiguous())
        info = newton_step(problem, mg, u, phi, phi_old, active, **newton_kw)
        J = problem.tcv(u, phi)
        ctx.problem, ctx.mg, ctx.adjoint_kw, ctx.info = problem, mg, adjoint_kw, info
        ctx.has_E = E_cells is not None
        ctx.save_for_backward(u.detach().clone(), phi.detach().clone(), phi_old.detach().clone(),
                              active.detach().clone())
        return torch.tensor(J, dtype=torch.float64, device=u.device)

    @staticmethod
    def backward(ctx, gJ):
        u, phi, phi_old, active = ctx.saved_tensors
        gE = torch.empty(ctx.problem.mesh.info["n_leaf_cells"], dtype=torch.float64, device=u.device) \
            if ctx.has_E else None
        r = tcv_adjoint(ctx.problem, ctx.mg, u, phi, phi_old, active, gE=gE, **ctx.adjoint_kw)
        ctx.adjoint = r
        g_p = gJ * r["p"]
        g_gc = gJ * r["Gc"]
        g_e = gJ * gE if gE is not None else None
        return g_p, g_gc, g_e, None, None, None, None, None, None, None, None


def tcv_load_step(problem, mg, p, Gc, E_cells, u, phi, phi_old, active, newton_kw=None, adjoint_kw=None):
    """Differentiable J = integral of u . grad phi after one load step.

    p, Gc: 0-dim float64 tensors; E_cells: float64 device tensor (n_leaf_cells, leaf
    order) or None; u (2, n_slots), phi, phi_old (n_slots,) float64 and active
    (n_slots,) uint8 device tensors, updated in place to the converged step."""
    return TCVLoadStep.apply(p, Gc, E_cells, problem, mg, u, phi, phi_old, active, newton_kw or {},
                             adjoint_kw or {})
