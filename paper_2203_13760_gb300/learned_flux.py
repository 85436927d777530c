"""Section 7.4: the dissipation of the Rusanov flux learned end to end through
the solver (the Rusanov-NN flux).

Ground truth: the implosion of ``inputs.implosion`` on 128 x 128 cells with
WENO3-JS, HLLC and TVD-RK2 at the fixed step 2.5e-4, sampled every 4 steps
(dt_CG = 1e-3) and coarse-grained to 32 x 32 cells (cell averages of the
conservative state over 4 x 4 blocks).  Model: the same scheme on the coarse
grid with the Rusanov-NN flux and dt = 1e-3.  Training: windows of N_T steps
starting at the samples of the first ``n_train`` time steps, batches of
simulations, the loss L = 1/N_T sum_{i=1..N_T} MSE(W_i^NN, W_i^CG) over the
primitive variables (rho, u, v, p), Adam.  Every solver step and every
gradient through it runs in libjf's kernels (jf_batch_feed_forward,
jf_rk3_step_vjp_params), and so does the loss of the primitive variables
with its gradient (jf_loss_primitive_mse); PyTorch holds the parameters and
takes the Adam step.

``ground_truth(...)``        coarse-grained reference trajectory
``primitives(U)``            (rho, u, v, p) of conservative states
``trajectory_loss(...)``     the loss above for a batch of windows (PyTorch
                             reference of its definition)
``trajectory_loss_jf(...)``  the same loss by libjf, as the trainer uses it
``Trainer``                  batches, forward / backward through the solver, Adam
``rollout_errors(...)``      relative L1 errors of rho and p along a run of the model
"""
from __future__ import annotations

import numpy as np
import torch

from . import autograd, inputs, jf

GAMMA = 1.4
WALLS = (inputs.WALL,) * 4 + (1, 1)


def coarse_grain(U, factor: int):
    """Cell averages of U (5, nz, ny, nx) over factor x factor blocks in (x, y)."""
    c, nz, ny, nx = U.shape
    return U.reshape(c, nz, ny // factor, factor, nx // factor, factor).mean(dim=(3, 5))


def ground_truth(n_fine: int = 128, factor: int = 4, nsamples: int = 1001, dt: float = 2.5e-4, every: int = 4,
                 dtype: str = "f64"):
    """(nsamples, 5, 1, n, n) coarse-grained states, n = n_fine / factor:
    sample k is the fine run after k * every steps of dt."""
    case = inputs.implosion(n_fine)
    s = jf.Solver.from_case(case, dtype=dtype)
    U = torch.tensor(case.U, dtype=s.dtype, device="cuda")
    dtd = s.scalar(dt)
    n = n_fine // factor
    out = torch.empty((nsamples, 5, 1, n, n), dtype=s.dtype, device="cuda")
    out[0] = coarse_grain(U, factor)
    for k in range(1, nsamples):
        s.run(U, every, dtd)
        out[k] = coarse_grain(U, factor)
    s.sync()
    s.close()
    return out


def primitives(U, gamma: float = GAMMA):
    """(..., 5, nz, ny, nx) conservative -> (..., 4, nz, ny, nx): rho, u, v, p."""
    rho = U[..., 0, :, :, :]
    u = U[..., 1, :, :, :] / rho
    v = U[..., 2, :, :, :] / rho
    w = U[..., 3, :, :, :] / rho
    p = (gamma - 1.0) * (U[..., 4, :, :, :] - 0.5 * rho * (u * u + v * v + w * w))
    return torch.stack([rho, u, v, p], dim=-4)


def trajectory_loss(trajs, refs, gamma: float = GAMMA):
    """Mean over the windows of 1/N_T sum_{i=1..N_T} MSE(W_i, W_i^ref): each
    window is an (N_T + 1, 5, ...) trajectory, slot 0 the shared initial state;
    MSE averages over the four primitive variables and the cells."""
    if all(t.shape == trajs[0].shape for t in trajs) and all(r.shape == trajs[0].shape for r in refs):
        # equal windows: one stacked computation (the mean of equal-size means)
        d = primitives(torch.stack(trajs)[:, 1:], gamma) - primitives(torch.stack(refs)[:, 1:], gamma)
        return (d * d).mean()
    total = 0.0
    for traj, ref in zip(trajs, refs):
        d = primitives(traj[1:], gamma) - primitives(ref[1:], gamma)
        total = total + (d * d).mean()
    return total / len(trajs)


def trajectory_loss_jf(owner, trajs, refs):
    """trajectory_loss evaluated by libjf (jf_loss_primitive_mse, with its
    gradient), for CUDA trajectories; owner: the jf.Batch (or jf.Solver)
    whose gas applies."""
    if all(t.shape == trajs[0].shape for t in trajs) and all(r.shape == trajs[0].shape for r in refs):
        return autograd.primitive_mse(owner, torch.stack(trajs)[:, 1:], torch.stack(refs)[:, 1:], 4)
    total = 0.0
    for traj, ref in zip(trajs, refs):
        total = total + autograd.primitive_mse(owner, traj[1:], ref[1:], 4)
    return total / len(trajs)


def model_batch(n: int, nsim: int, dtype: str, theta=None, flux: str = "rusanov-nn"):
    """A jf.Batch of nsim coarse implosion grids with the model's scheme."""
    grids = [jf.make_grid((n, n, 1), bc=WALLS) for _ in range(nsim)]
    return jf.Batch(grids, dtype=dtype, gamma=GAMMA, flux=flux, recon="weno3-js", integrator="rk2", nn=theta)


class Trainer:
    """Adam on the network parameters theta over windows of the reference.

    cg: the coarse reference (nsamples, 5, 1, n, n) on the GPU; theta0: the
    initial parameters (jf.NN_PARAMS values, e.g. ``inputs.nn_params``)."""

    def __init__(self, cg, theta0, batch: int = 20, unroll: int = 15, lr: float = 5e-4, dt: float = 1e-3,
                 n_train: int = 1000, dtype: str = "f32"):
        self.t = torch.float32 if dtype == "f32" else torch.float64
        self.cg = cg.to(self.t).contiguous()
        self.n = int(cg.shape[-1])
        self.unroll, self.dt, self.bsize = int(unroll), float(dt), int(batch)
        self.n_train = min(int(n_train), int(cg.shape[0]))
        self.theta = torch.tensor(np.asarray(theta0), dtype=self.t, device="cuda").requires_grad_(True)
        self.batch = model_batch(self.n, self.bsize, dtype, self.theta)
        self.opt = torch.optim.Adam([self.theta], lr=lr)
        self.starts = np.arange(0, self.n_train - self.unroll)

    def loss_and_grad(self, starts):
        """Loss of the windows starting at `starts` and d loss / d theta."""
        U0s = [self.cg[s] for s in starts]
        trajs = autograd.feed_forward(self.batch, U0s, self.unroll, self.dt, theta=self.theta)
        refs = [self.cg[s:s + self.unroll + 1] for s in starts]
        loss = trajectory_loss_jf(self.batch, trajs, refs)
        if self.theta.grad is not None:
            self.theta.grad = None
        loss.backward()
        return loss.detach(), self.theta.grad.detach().clone()

    def step(self, starts) -> float:
        """One Adam step on the windows starting at `starts` (len == batch)."""
        loss, _ = self.loss_and_grad(starts)
        self.opt.step()
        self.batch.sync()
        value = float(loss.item())
        if not np.isfinite(value):
            raise FloatingPointError("training loss is not finite")
        return value

    def epoch(self, rng) -> float:
        """One pass over the shuffled window starts in batches (the remainder
        that does not fill a batch is left out); the mean loss."""
        order = rng.permutation(self.starts)
        losses = [self.step(order[i:i + self.bsize]) for i in range(0, len(order) - self.bsize + 1, self.bsize)]
        return float(np.mean(losses))


def rollout_errors(cg, nsteps: int, flux: str = "rusanov-nn", theta=None, dt: float = 1e-3, dtype: str = "f32"):
    """Run the coarse model from cg[0] for nsteps steps of dt; returns the
    relative L1 errors sum|q - q_CG| / sum|q_CG| of rho and p after each step
    (arrays of nsteps)."""
    t = torch.float32 if dtype == "f32" else torch.float64
    n = int(cg.shape[-1])
    th = torch.tensor(np.asarray(theta), dtype=t, device="cuda") if theta is not None else None
    b = model_batch(n, 1, dtype, th, flux)
    traj = b.feed_forward([cg[0].to(t).contiguous()], nsteps, dt)[0]
    b.sync()
    W = primitives(traj[1:].double())
    Wr = primitives(cg[1:nsteps + 1].double())
    err = []
    for k in (0, 3):
        num = (W[:, k] - Wr[:, k]).abs().flatten(1).sum(1)
        den = Wr[:, k].abs().flatten(1).sum(1)
        err.append((num / den).cpu().numpy())
    b.close()
    return err[0], err[1]


def train(epochs: int = 200, batch: int = 20, unroll: int = 15, lr: float = 5e-4, n_train: int = 1000,
          nsamples: int = 2501, dtype: str = "f32", seed: int = 0, eval_steps=None, log=None):
    """The Section 7.4 experiment: reference, training, and the rollout errors
    of the trained Rusanov-NN flux and of the Rusanov flux over the whole
    reference.  Returns a dict of the settings, timings, losses and errors."""
    import time
    t0 = time.perf_counter()
    cg = ground_truth(nsamples=nsamples)
    torch.cuda.synchronize()
    t_ref = time.perf_counter() - t0
    tr = Trainer(cg, inputs.nn_params(seed=seed), batch=batch, unroll=unroll, lr=lr, n_train=n_train, dtype=dtype)
    rng = np.random.default_rng(seed)
    losses = []
    steps = 0
    t0 = time.perf_counter()
    for e in range(epochs):
        losses.append(tr.epoch(rng))
        steps += len(tr.starts) // tr.bsize
        if log:
            log(f"epoch {e + 1}/{epochs}: loss {losses[-1]:.6e}")
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    nsteps = int(eval_steps or (nsamples - 1))
    theta = tr.theta.detach().cpu().numpy()
    nn_rho, nn_p = rollout_errors(cg, nsteps, theta=theta, dtype=dtype)
    rs_rho, rs_p = rollout_errors(cg, nsteps, flux="rusanov", dtype=dtype)
    marks = [k for k in (10, 100, 500, 1000, 1500, 2000, 2500) if k <= nsteps]
    return {
        "settings": dict(epochs=epochs, batch=batch, unroll=unroll, lr=lr, n_train=n_train, nsamples=nsamples,
                         dtype=dtype, seed=seed),
        "reference_seconds": t_ref,
        "train_seconds": t_train,
        "optimizer_steps": steps,
        "ms_per_optimizer_step": 1e3 * t_train / max(steps, 1),
        "epoch_losses": losses,
        "rel_l1_after_steps": {str(k): {"rusanov_nn": [float(nn_rho[k - 1]), float(nn_p[k - 1])],
                                        "rusanov": [float(rs_rho[k - 1]), float(rs_p[k - 1])]} for k in marks},
        "mean_rel_l1": {"rusanov_nn": [float(nn_rho.mean()), float(nn_p.mean())],
                        "rusanov": [float(rs_rho.mean()), float(rs_p.mean())]},
        "theta": theta.tolist(),
    }


if __name__ == "__main__":
    import argparse
    import json
    import sys
    ap = argparse.ArgumentParser(description="Section 7.4: train the Rusanov-NN dissipation through the solver")
    ap.add_argument("--epochs", type=int, default=200)
    ap.add_argument("--batch", type=int, default=20)
    ap.add_argument("--unroll", type=int, default=15)
    ap.add_argument("--lr", type=float, default=5e-4)
    ap.add_argument("--n-train", type=int, default=1000)
    ap.add_argument("--samples", type=int, default=2501)
    ap.add_argument("--dtype", default="f32")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--out", default="")
    a = ap.parse_args()
    res = train(a.epochs, a.batch, a.unroll, a.lr, a.n_train, a.samples, a.dtype, a.seed,
                log=lambda m: print(m, file=sys.stderr, flush=True))
    text = json.dumps(res)
    if a.out:
        with open(a.out, "w") as f:
            f.write(text)
    summary = {k: v for k, v in res.items() if k != "theta"}
    print(json.dumps(summary))
