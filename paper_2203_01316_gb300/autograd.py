"""Gradients of a heat-transfer objective with respect to the per-node heat
source theta and the wall temperatures, through the hand-written adjoint of
the library (include/lbm.h, "adjoint of the h evolution").

J(theta, T_w) = sum over levels k in [window[0], window[1]] of
weight * F(s^k), F a linear flux of the post-collision h state (the surface
heat flux of a wall, Sec. 4.4, or the x-flux through a plane), over nsteps
steps from a saved state s^0.

Forward: runs the steps, keeping a device checkpoint of the state every
`every` steps.  Backward: for each segment, last first, restores its
checkpoint, recomputes the velocity of every level of the segment, then runs
the adjoint kernel level by level.  For the central-moment kinds the h step
is affine and its adjoint needs only u, so the recomputation advances f only;
the Cumulants-1st collision is nonlinear in h, so there the recomputation
advances h as well and keeps each level's post-collision h for the adjoint.

Two-level checkpointing (every2 < every): the backward first re-runs each
segment from its checkpoint keeping a second-level checkpoint every `every2`
steps, then treats each sub-segment as above.  Memory: nsteps/every + every/
every2 states plus every2 levels of records instead of nsteps/every states
plus every levels of records, for one more forward pass; the recomputed
states and records are the same bits, so the gradients are too.  All
arithmetic runs in the CUDA library; this module only orders the calls and
owns the device buffers (torch tensors).
"""
from __future__ import annotations

import torch

from .lbm import Solver


class ThermalObjective(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta, T_wall, solver: Solver, state0, nsteps: int, window, objective, every: int,
                every2=None):
        if every < 1 or (every2 is not None and every2 < 1):
            raise ValueError("checkpoint intervals must be >= 1")
        dev = state0.device
        # the solver runs on its own stream: order it after torch's work on
        # the inputs, and torch's later work after the solver's
        torch.cuda.synchronize(dev)
        solver.set_source(theta.detach().to(device=dev, dtype=torch.float32))
        torch.cuda.synchronize(dev)
        for w, T in enumerate(T_wall.detach().cpu().tolist()):
            solver.set_bc(w, T)
        solver.load_state(state0)
        J = torch.zeros(1, dtype=torch.float64, device=dev)
        ckpts = {}
        for k in range(nsteps + 1):
            if k % every == 0 and k < nsteps:
                ckpts[k] = solver.save_state(torch.empty_like(state0))
            if window[0] <= k <= window[1]:
                solver.objective_accumulate(objective, J)
            if k < nsteps:
                solver.step(1)
        solver.sync()
        ctx.solver, ctx.ckpts, ctx.nsteps, ctx.window = solver, ckpts, nsteps, window
        ctx.objective, ctx.every, ctx.n_walls = objective, every, T_wall.numel()
        ctx.every2 = every2
        ctx.theta_dtype, ctx.Tw_dtype = theta.dtype, T_wall.dtype
        ctx.theta_device, ctx.Tw_device = theta.device, T_wall.device
        return J[0]

    @staticmethod
    def backward(ctx, gJ):
        s: Solver = ctx.solver
        N, qh = s.N, s.qh
        dev = next(iter(ctx.ckpts.values())).device if ctx.ckpts else torch.device("cuda")
        rdt = torch.float64 if s.params.storage == 1 else torch.float32
        mu_next = torch.zeros(qh * N, dtype=rdt, device=dev)
        mu_out = torch.empty_like(mu_next)
        dtheta = torch.zeros(N, dtype=torch.float64, device=dev)
        torch.cuda.synchronize(dev)  # zeroed buffers before the solver's stream uses them
        s.adjoint_wall_gradient(ctx.n_walls, reset=True)
        lo, hi = ctx.window
        starts = sorted(ctx.ckpts)
        every2 = ctx.every2 if ctx.every2 is not None else ctx.every
        for seg_start in reversed(starts):
            seg_end = min(seg_start + ctx.every, ctx.nsteps)
            s.load_state(ctx.ckpts[seg_start])
            if every2 < seg_end - seg_start:  # second level: states every every2 steps of the segment
                inner = {}
                for k in range(seg_start, seg_end):
                    if (k - seg_start) % every2 == 0:
                        inner[k] = s.save_state(torch.empty_like(ctx.ckpts[seg_start]))
                    s.step(1)
            else:
                inner = {seg_start: None}
            for sub_start in sorted(inner, reverse=True):
                sub_end = min(sub_start + every2, seg_end)
                L = sub_end - sub_start
                if inner[sub_start] is not None:
                    s.load_state(inner[sub_start])
                urec = torch.empty(L * 3 * N, dtype=rdt, device=dev)
                hrec = torch.empty(L * qh * N, dtype=rdt, device=dev) if s.cumulant_h else None
                s.step_record(L, urec, advance_h=False, h_rec=hrec)
                for k in range(sub_end, sub_start, -1):
                    obj = ctx.objective if lo <= k <= hi else None
                    j = k - sub_start - 1
                    u_k = urec[j * 3 * N:(j + 1) * 3 * N]
                    h_k = hrec[j * qh * N:(j + 1) * qh * N] if hrec is not None else None
                    s.adjoint_step(u_k, mu_next, mu_out, obj, dtheta, h_level=h_k)
                    mu_next, mu_out = mu_out, mu_next
        # level 0: the initial state is given; only its objective and wall terms remain
        obj0 = ctx.objective if lo <= 0 <= hi else None
        s.adjoint_step(None, mu_next, mu_out, obj0, None)
        dTw = s.adjoint_wall_gradient(ctx.n_walls, reset=True)  # synchronises the solver's stream
        gJ = gJ.to(torch.float64)
        g_theta = (gJ.to(dtheta.device) * dtheta).to(device=ctx.theta_device, dtype=ctx.theta_dtype)
        g_Tw = (gJ.cpu() * torch.from_numpy(dTw)).to(device=ctx.Tw_device, dtype=ctx.Tw_dtype)
        return g_theta, g_Tw, None, None, None, None, None, None, None


def thermal_objective(theta, T_wall, solver, state0, nsteps, window, objective, every=50, every2=None):
    """J(theta, T_wall) with gradients by the adjoint (see module docstring).
    state0: CUDA uint8 tensor from solver.save_state(out=...); every2 (optional,
    below every) turns on the second checkpoint level."""
    return ThermalObjective.apply(theta, T_wall, solver, state0, nsteps, window, objective, every, every2)


class FlowObjective(torch.autograd.Function):
    """The same objective as ThermalObjective, differentiable also with
    respect to the flow's parameters: the body force F[3] and the inlet
    velocity u_in[3] (equilibrium inlet plane).  The backward runs the
    adjoint of the coupled f + h evolution (include/lbm.h, "adjoint of the
    coupled f + h evolution"): per segment it restores the checkpoint,
    recomputes the segment recording each level's pre-collision arrivals, and
    runs the coupled adjoint level by level.  FP32 or FP64 storage."""

    @staticmethod
    def forward(ctx, theta, T_wall, F, u_in, solver: Solver, state0, nsteps: int, window, objective, every: int,
                every2=None):
        if every < 1 or (every2 is not None and every2 < 1):
            raise ValueError("checkpoint intervals must be >= 1")
        dev = state0.device
        torch.cuda.synchronize(dev)
        solver.set_source(theta.detach().to(device=dev, dtype=torch.float32))
        torch.cuda.synchronize(dev)
        for w, T in enumerate(T_wall.detach().cpu().tolist()):
            solver.set_bc(w, T)
        solver.set_force(F.detach().cpu().tolist())
        T_in = solver.inlet[1] if getattr(solver, "inlet", None) else 0.0
        solver.set_inlet(u_in.detach().cpu().tolist(), T_in)
        solver.load_state(state0)
        J = torch.zeros(1, dtype=torch.float64, device=dev)
        ckpts = {}
        for k in range(nsteps + 1):
            if k % every == 0 and k < nsteps:
                ckpts[k] = solver.save_state(torch.empty_like(state0))
            if window[0] <= k <= window[1]:
                solver.objective_accumulate(objective, J)
            if k < nsteps:
                solver.step(1)
        solver.sync()
        ctx.solver, ctx.ckpts, ctx.nsteps, ctx.window = solver, ckpts, nsteps, window
        ctx.objective, ctx.every, ctx.n_walls = objective, every, T_wall.numel()
        ctx.every2 = every2
        ctx.meta = [(t.dtype, t.device) for t in (theta, T_wall, F, u_in)]
        return J[0]

    @staticmethod
    def backward(ctx, gJ):
        s: Solver = ctx.solver
        N, qh = s.N, s.qh
        dev = next(iter(ctx.ckpts.values())).device if ctx.ckpts else torch.device("cuda")
        rdt = torch.float64 if s.params.storage == 1 else torch.float32
        muf = [torch.zeros(27 * N, dtype=rdt, device=dev), torch.empty(27 * N, dtype=rdt, device=dev)]
        muh = [torch.zeros(qh * N, dtype=rdt, device=dev), torch.empty(qh * N, dtype=rdt, device=dev)]
        dtheta = torch.zeros(N, dtype=torch.float64, device=dev)
        torch.cuda.synchronize(dev)
        s.adjoint_wall_gradient(ctx.n_walls, reset=True)
        s.adjoint_flow_gradient(reset=True)
        lo, hi = ctx.window
        cur = 0
        FR, HR = s.flow_record_size()
        every2 = ctx.every2 if ctx.every2 is not None else ctx.every
        for seg_start in sorted(ctx.ckpts, reverse=True):
            seg_end = min(seg_start + ctx.every, ctx.nsteps)
            s.load_state(ctx.ckpts[seg_start])
            if every2 < seg_end - seg_start:  # second level, as in ThermalObjective
                inner = {}
                for k in range(seg_start, seg_end):
                    if (k - seg_start) % every2 == 0:
                        inner[k] = s.save_state(torch.empty_like(ctx.ckpts[seg_start]))
                    s.step(1)
            else:
                inner = {seg_start: None}
            for sub_start in sorted(inner, reverse=True):
                sub_end = min(sub_start + every2, seg_end)
                L = sub_end - sub_start
                if inner[sub_start] is not None:
                    s.load_state(inner[sub_start])
                frec = torch.empty(L * FR, dtype=rdt, device=dev)
                hrec = torch.empty(L * HR, dtype=rdt, device=dev)
                s.step_record_pre(L, frec, hrec)
                for k in range(sub_end, sub_start, -1):
                    obj = ctx.objective if lo <= k <= hi else None
                    j = k - sub_start - 1
                    s.adjoint_flow_step(frec[j * FR:(j + 1) * FR], hrec[j * HR:(j + 1) * HR],
                                        muf[cur], muh[cur], muf[1 - cur], muh[1 - cur], obj, dtheta)
                    cur = 1 - cur
        obj0 = ctx.objective if lo <= 0 <= hi else None
        s.adjoint_flow_step(None, None, muf[cur], muh[cur], muf[1 - cur], muh[1 - cur], obj0, None)
        dTw = s.adjoint_wall_gradient(ctx.n_walls, reset=True)
        dF, duin = s.adjoint_flow_gradient(reset=True)  # synchronises the solver's stream
        gJ = gJ.detach().to(torch.float64).cpu()
        grads = [dtheta.cpu(), torch.from_numpy(dTw), torch.from_numpy(dF), torch.from_numpy(duin)]
        out = [(gJ * g).to(dtype=dt, device=dv) for g, (dt, dv) in zip(grads, ctx.meta)]
        return out[0], out[1], out[2], out[3], None, None, None, None, None, None, None


def flow_objective(theta, T_wall, F, u_in, solver, state0, nsteps, window, objective, every=50, every2=None):
    """J(theta, T_wall, F, u_in) with gradients by the coupled adjoint."""
    return FlowObjective.apply(theta, T_wall, F, u_in, solver, state0, nsteps, window, objective, every, every2)
