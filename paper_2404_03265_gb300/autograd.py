"""Differentiable load steps: J = TCV (Sec. 4) after one or several load steps of
Algorithm 2 as a torch function of the pressures p, the toughness G_c and the
per-cell modulus E_K.

One step (TCVLoadStep):
forward  runs the Newton / PDAS load step (pff_newton_pdas_step) and keeps the
         converged state (u, phi, phi_old, active set) as its checkpoint;
backward runs one adjoint solve at that state (pff_tcv_adjoint: transposed
         constrained Jacobian, GMRES with the block V-cycle, then the VJP of the
         residual with respect to the parameters).
Several steps (TCVLoadSteps), step n from phi_old = phi^(n-1) with phi_tilde =
phi^(n-1), or extrapolated (Sec. 2) as clip(2 phi^(n-1) - phi^(n-2), 0, 1) for n >= 2:
forward  runs the N load steps and keeps every step's converged state (u^n,
         phi^n, active set A^n) as the checkpoints;
backward runs the checkpointed adjoint chain (pff_tcv_adjoint_steps): one
         adjoint solve per step, last to first, each passing its phi-sensitivity
         to the steps before through phi_tilde (one step back, or two when
         extrapolated) and the active rows.
"""
import torch

from . import newton_step, tcv_adjoint, tcv_adjoint_steps


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


class TCVLoadSteps(torch.autograd.Function):
    """J = TCV(U^N) after N load steps; see ``tcv_load_steps``."""

    @staticmethod
    def forward(ctx, ps, Gc, E_cells, problem, mg, u0, phi0, newton_kw, adjoint_kw, out, extrapolated):
        problem.set_params(Gc=float(Gc))
        problem.set_cell_modulus(None if E_cells is None else E_cells.detach().contiguous())
        pl = [float(v) for v in ps.detach().cpu().reshape(-1)]
        us = [u0.detach().clone()]
        phis = [phi0.detach().clone()]
        acts = []
        act = torch.zeros(phi0.numel(), dtype=torch.uint8, device=phi0.device)
        infos = []
        phit = torch.empty_like(phi0) if extrapolated and len(pl) >= 2 else None
        for n, p in enumerate(pl, start=1):
            problem.set_pressure(p)
            u = us[-1].clone()
            phi = phis[-1].clone()
            kw = dict(newton_kw)
            if extrapolated and n >= 2:
                problem.extrapolate_phi(phis[-1], phis[-2], phit)
                kw["phi_tilde"] = phit
            infos.append(newton_step(problem, mg, u, phi, phis[-1], act, **kw))
            us.append(u)
            phis.append(phi)
            acts.append(act.clone())
        J = problem.tcv(us[-1], phis[-1])
        ctx.problem, ctx.mg, ctx.adjoint_kw, ctx.extrapolated = problem, mg, adjoint_kw, extrapolated
        ctx.checkpoints = (us, phis, acts, pl)
        ctx.has_E = E_cells is not None
        ctx.dev_p, ctx.dev_gc = ps.device, Gc.device if torch.is_tensor(Gc) else torch.device("cpu")
        if out is not None:
            out.update(u=us, phi=phis, active=acts, info=infos)
        return torch.tensor(J, dtype=torch.float64, device=phi0.device)

    @staticmethod
    def backward(ctx, gJ):
        us, phis, acts, pl = ctx.checkpoints
        dev = phis[0].device
        gE = torch.empty(ctx.problem.mesh.info["n_leaf_cells"], dtype=torch.float64, device=dev) \
            if ctx.has_E else None
        r = tcv_adjoint_steps(ctx.problem, ctx.mg, us, phis, acts, pl, gE=gE, extrapolated=ctx.extrapolated,
                              **ctx.adjoint_kw)
        ctx.adjoint = r
        g_ps = (gJ.cpu() * torch.tensor(r["p"], dtype=torch.float64)).to(ctx.dev_p)
        g_gc = (gJ * r["Gc"]).to(ctx.dev_gc)
        g_e = gJ * gE if gE is not None else None
        return g_ps, g_gc, g_e, None, None, None, None, None, None, None, None


def tcv_load_steps(problem, mg, ps, Gc, E_cells, u0, phi0, newton_kw=None, adjoint_kw=None, out=None,
                   extrapolated=False):
    """Differentiable J = integral of u . grad phi after len(ps) load steps.

    ps: float64 tensor of the N pressures (CPU); Gc: 0-dim float64 tensor; E_cells:
    float64 device tensor (n_leaf_cells, leaf order) or None; u0 (2, n_slots) and
    phi0 (n_slots,): the initial state (phi0 also the first step's obstacle).
    out (dict, optional) receives the step states (u, phi, active lists) and the
    Newton infos.  extrapolated: phi_tilde of steps n >= 2 is clip(2 phi^(n-1) -
    phi^(n-2), 0, 1) (Problem.extrapolate_phi) instead of phi^(n-1).  The backward
    pass leaves the problem's state, active set and multigrid at the first step."""
    return TCVLoadSteps.apply(ps, Gc, E_cells, problem, mg, u0, phi0, newton_kw or {}, adjoint_kw or {}, out,
                              bool(extrapolated))
