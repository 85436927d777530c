"""Differentiable RK3 steps and trajectories on top of libjf (Section 7.2:
end-to-end optimisation through the solver; Section 4.5: ``feed_forward`` with
a fixed step).

``rk3_step(solver, U, dt)``   one fixed-dt step as a torch.autograd.Function;
                              its backward is jf_rk3_step_vjp.
``rollout(solver, U0, n, dt, ckpt_every=20)``
                              n fixed-dt steps whose backward pass recomputes
                              each segment of ``ckpt_every`` steps from a stored
                              checkpoint (memory: n / ckpt_every + ckpt_every
                              states instead of n; with the default scheme the
                              replay keeps each step's two stage states for
                              jf_rk3_step_vjp_stages, 3 ckpt_every states).
``density_l2(solver, U, target)``
                              sum_cells (rho - target)^2 dV (jf_loss_density_l2)
                              with its gradient.
``feed_forward(batch, U0s, n, dt, theta=None)``
                              Section 4.5: the trajectories of a batch of
                              (uneven) simulations, differentiable w.r.t. the
                              initial states (reverse sweep on the stored
                              trajectory with jf_rk3_step_vjp) and, for the
                              Rusanov-NN flux of Section 7.4, w.r.t. the
                              network parameters theta (jf_rk3_step_vjp_params).
``trajectory_mse(trajs, refs)``
                              Section 7.2: 1/N_T sum_i MSE(U^i, U^i_ref).
``primitive_mse(owner, U, Uref, ncomp=4)``
                              Section 7.4: MSE of the primitive state
                              vectors (jf_loss_primitive_mse) with its
                              gradient.

dt is a float64 CUDA scalar tensor and is not differentiated (the paper's
feed_forward uses a fixed step).  Every computation runs in libjf's kernels.
"""
from __future__ import annotations

import torch


class _RK3Step(torch.autograd.Function):
    @staticmethod
    def forward(ctx, U, solver, dt):
        ctx.solver = solver
        ctx.save_for_backward(U, dt)
        out = U.detach().clone()
        solver.rk3_step(out, dt)
        return out

    @staticmethod
    def backward(ctx, grad):
        U, dt = ctx.saved_tensors
        lam = ctx.solver.rk3_step_vjp(U.detach(), dt, grad.contiguous())
        return lam, None, None


def rk3_step(solver, U, dt):
    return _RK3Step.apply(U, solver, dt)


class _Rollout(torch.autograd.Function):
    @staticmethod
    def forward(ctx, U0, solver, dt, nsteps, ckpt_every):
        U = U0.detach().clone()
        ckpts = [U.clone()]
        for k in range(nsteps):
            solver.rk3_step(U, dt)
            if (k + 1) % ckpt_every == 0 and k + 1 < nsteps:
                ckpts.append(U.clone())
        ctx.solver, ctx.nsteps, ctx.ckpt_every = solver, nsteps, ckpt_every
        ctx.ckpts = ckpts
        ctx.save_for_backward(dt)
        return U

    @staticmethod
    def backward(ctx, grad):
        (dt,) = ctx.saved_tensors
        s, n, c = ctx.solver, ctx.nsteps, ctx.ckpt_every
        lam = grad.contiguous().clone()
        lam_next = torch.empty_like(lam)
        # the default scheme keeps the stage states of the segment's replay, so
        # the step adjoints do not recompute them (memory: 3 states per step)
        keep = s.supports_stage_vjp()
        for seg in reversed(range(len(ctx.ckpts))):
            start = seg * c
            length = min(c, n - start)
            states = [ctx.ckpts[seg]]
            stages = []
            for k in range(length):
                if keep:
                    U1, U2 = s.empty(), s.empty()
                    if k < length - 1:
                        nxt = states[-1].clone()
                        s.rk3_step_keep(nxt, dt, U1, U2)
                        states.append(nxt)
                    else:  # the last step's result is not needed, only its stages
                        s.stage(states[k], None, U1, 0.0, 1.0, dt)
                        s.stage(U1, states[k], U2, 0.75, 0.25, dt)
                    stages.append((U1, U2))
                elif k < length - 1:
                    nxt = states[-1].clone()
                    s.rk3_step(nxt, dt)
                    states.append(nxt)
            for k in reversed(range(length)):
                if keep:
                    U1, U2 = stages[k]
                    s.rk3_step_vjp_stages(states[k], U1, U2, dt, lam, lam_next)
                    stages[k] = None
                else:
                    s.rk3_step_vjp(states[k], dt, lam, lam_next)
                lam, lam_next = lam_next, lam
        ctx.ckpts = None
        return lam, None, None, None, None


def rollout(solver, U0, nsteps, dt, ckpt_every=20):
    return _Rollout.apply(U0, solver, dt, int(nsteps), int(ckpt_every))


class _DensityL2(torch.autograd.Function):
    @staticmethod
    def forward(ctx, U, solver, target):
        loss, seed = solver.loss_density_l2(U.detach(), target)
        ctx.save_for_backward(seed)
        return loss[0]

    @staticmethod
    def backward(ctx, grad):
        (seed,) = ctx.saved_tensors
        return seed * grad, None, None


def density_l2(solver, U, target):
    return _DensityL2.apply(U, solver, target)


class _FeedForward(torch.autograd.Function):
    """Trajectories of a batch (jf_batch_feed_forward) with the reverse sweep
    of each simulation: for U^{t+1} = S(U^t), dL/dU^t = g_t + J_t^T dL/dU^{t+1},
    J_t^T applied by jf_rk3_step_vjp of a single-grid solver of the same grid
    and scheme, on the stored trajectory (no recomputation of states).  With
    the network parameters theta (the Rusanov-NN flux), the same sweep runs
    jf_rk3_step_vjp_params, which also sums dL/dtheta over the steps and
    simulations."""

    @staticmethod
    def forward(ctx, batch, nsteps, dt, theta, *U0s):
        if theta is not None and (batch._nn is None or batch._nn.data_ptr() != theta.data_ptr()):
            raise ValueError("theta must be the tensor the batch holds (Batch.set_nn)")
        trajs = batch.feed_forward([U.detach().contiguous() for U in U0s], nsteps, dt)
        ctx.batch, ctx.nsteps, ctx.with_theta = batch, nsteps, theta is not None
        ctx.dts = [float(dt)] * batch.nsim if not hasattr(dt, "__len__") else [float(x) for x in dt]
        ctx.save_for_backward(*trajs)
        return tuple(trajs)

    @staticmethod
    def backward(ctx, *grads):
        trajs = ctx.saved_tensors
        theta_bar = torch.zeros_like(ctx.batch._nn) if ctx.with_theta else None

        # the C ABI wants 16-byte aligned states, which a trajectory slot of a
        # state whose size is not a multiple of 16 bytes is not: such slots are
        # passed as aligned copies
        def aligned(x):
            return x if x.data_ptr() % 16 == 0 else x.clone()

        if ctx.batch.supports_step_vjp():
            # every simulation of the batch in the same launches, one call per step
            g = [torch.zeros_like(tr) if gi is None else gi.contiguous() for tr, gi in zip(trajs, grads)]
            dt = torch.tensor(ctx.dts, dtype=torch.float64, device=trajs[0].device)
            lam = [gi[ctx.nsteps].clone() for gi in g]
            nxt = [torch.empty_like(x) for x in lam]
            if theta_bar is not None:  # one parameter-gradient launch for the whole sweep
                ctx.batch.param_grad_begin(ctx.nsteps)
            for t in reversed(range(ctx.nsteps)):
                ctx.batch.step_vjp([aligned(tr[t]) for tr in trajs], dt, lam, nxt, [aligned(gi[t]) for gi in g],
                                   theta_bar)
                lam, nxt = nxt, lam
            if theta_bar is not None:
                ctx.batch.param_grad_end(theta_bar)
            return (None, None, None, theta_bar, *lam)
        out = []
        for i, (traj, g) in enumerate(zip(trajs, grads)):
            solver = ctx.batch.solver(i)
            dt = solver.scalar(ctx.dts[i])
            g = torch.zeros_like(traj) if g is None else g.contiguous()
            lam = g[ctx.nsteps].clone()
            for t in reversed(range(ctx.nsteps)):
                if theta_bar is not None:
                    lam, _ = solver.rk3_step_vjp_params(aligned(traj[t]), dt, lam, theta_bar=theta_bar)
                else:
                    lam = solver.rk3_step_vjp(aligned(traj[t]), dt, lam)
                lam += g[t]
            out.append(lam)
        return (None, None, None, theta_bar, *out)


def feed_forward(batch, U0s, nsteps, dt, theta=None):
    """Section 4.5 feed_forward, differentiable: per simulation of ``batch``
    (a jf.Batch; sizes may differ) the trajectory (nsteps + 1, 5, nz, ny, nx)
    of fixed-dt steps from U0s[i]; gradients flow back to every U0s[i] and,
    when given, to the Rusanov-NN parameters theta (the tensor the batch holds
    through Batch.set_nn, updated in place by an optimizer)."""
    return list(_FeedForward.apply(batch, int(nsteps), dt, theta, *U0s))


class _PrimitiveMSE(torch.autograd.Function):
    @staticmethod
    def forward(ctx, U, Uref, owner, ncomp):
        from . import jf
        loss, grad = jf.loss_primitive_mse(owner, U.detach(), Uref.detach(), ncomp, want_grad=U.requires_grad)
        ctx.save_for_backward(grad if grad is not None else loss)
        ctx.has_grad = grad is not None
        return loss[0]

    @staticmethod
    def backward(ctx, g):
        (grad,) = ctx.saved_tensors
        return (grad * g if ctx.has_grad else None), None, None, None


def primitive_mse(owner, U, Uref, ncomp=4):
    """Section 7.4 loss, the mean squared difference of the primitive state
    vectors of U and Uref (jf_loss_primitive_mse; ncomp 4: rho, u, v, p), with
    its gradient w.r.t. U; owner is the jf.Solver or jf.Batch whose gamma
    applies.  Uref is not differentiated."""
    return _PrimitiveMSE.apply(U, Uref, owner, int(ncomp))


def trajectory_mse(trajs, refs):
    """Section 7.2 trajectory loss L = 1/N_T sum_{i=1..N_T} MSE(U^i, U^i_ref)
    (the initial state excluded), averaged over the simulations of a batch.
    trajs / refs: lists of (N_T + 1, 5, ...) tensors."""
    total = 0.0
    for traj, ref in zip(trajs, refs):
        nt = traj.shape[0] - 1
        total = total + sum(torch.mean((traj[i] - ref[i]) ** 2) for i in range(1, nt + 1)) / nt
    return total / len(trajs)
