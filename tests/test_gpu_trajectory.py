"""Section 4.5 feed_forward for batches of uneven simulations
(jf_batch_feed_forward) and its gradient (Section 7.2 trajectory loss).

* Slot t of every trajectory equals t fixed-dt steps of the single-grid path,
  bit for bit, with each simulation's own dt.
* The gradient of the trajectory MSE w.r.t. the initial states equals the
  per-step autograd chain of the single-grid solver (FP64, to rounding) and a
  directional central difference.
"""
import pytest

from paper_2203_13760_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2203_13760_gb300 import autograd as jfa  # noqa: E402
from paper_2203_13760_gb300 import jf  # noqa: E402


def make_batch(cases, dtype, **kw):
    grids = [jf.make_grid(c.n, c.lo, c.hi, c.bc) for c in cases]
    p = dict(cases[0].params(), **kw)
    return jf.Batch(grids, dtype=dtype, **{k: p[k] for k in ("gamma", "R", "mu", "Pr", "eps", "cfl", "viscous",
                                                               "heat", "flux", "recon", "speeds", "integrator")})


@pytest.mark.parametrize("integrator", ["rk3", "rk2", "euler"])
@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_feed_forward_equals_single_grid(dtype, integrator):
    cases = inputs.four_quadrant_batch(nsim=3, sides=(32, 48, 40), seed=11)
    b = make_batch(cases, dtype, integrator=integrator)
    t = torch.float32 if dtype == "f32" else torch.float64
    U0s = [torch.tensor(c.U, dtype=t, device="cuda") for c in cases]
    dts = [2e-4, 3e-4, 1.5e-4]
    trajs = b.feed_forward(U0s, 5, dts)
    b.sync()
    for i, c in enumerate(cases):
        assert tuple(trajs[i].shape) == (6, 5, c.n[2], c.n[1], c.n[0])
        assert torch.equal(trajs[i][0], U0s[i])
        s = b.solver(i)
        U = U0s[i].clone()
        dt = s.scalar(dts[i])
        for k in range(1, 6):
            s.rk3_step(U, dt)
            assert torch.equal(trajs[i][k], U), (i, k)
    b.close()


def test_feed_forward_leaves_initial_states():
    cases = inputs.four_quadrant_batch(nsim=2, sides=(32, 40), seed=3)
    b = make_batch(cases, "f32")
    U0s = [torch.tensor(c.U, dtype=torch.float32, device="cuda") for c in cases]
    keep = [U.clone() for U in U0s]
    b.feed_forward(U0s, 3, 1e-4)
    b.sync()
    assert all(torch.equal(a, k) for a, k in zip(U0s, keep))
    trajs = b.feed_forward(U0s, 0, 1e-4)  # nsteps = 0: the initial states only
    b.sync()
    assert all(torch.equal(tr[0], U) for tr, U in zip(trajs, U0s))


def _kh(n, seed):
    return inputs.kelvin_helmholtz(n, seed=seed)


def test_trajectory_loss_gradient_fp64():
    """Uneven batch (two Kelvin-Helmholtz grids, 24^2 and 32^2): dL/dU0 of the
    Section 7.2 trajectory MSE through feed_forward equals the single-grid
    per-step autograd chain and a central difference."""
    cases = [_kh(24, 1), _kh(32, 2)]
    targets = [_kh(24, 5), _kh(32, 6)]
    b = make_batch(cases, "f64")
    nsteps = 6
    dts = []
    for i, c in enumerate(cases):
        s = b.solver(i)
        dts.append(0.4 * s.compute_dt(torch.tensor(c.U, dtype=torch.float64, device="cuda")).item())
    U0s = [torch.tensor(c.U, dtype=torch.float64, device="cuda", requires_grad=True) for c in cases]
    with torch.no_grad():
        refs = b.feed_forward([torch.tensor(c.U, dtype=torch.float64, device="cuda") for c in targets], nsteps, dts)
    loss = jfa.trajectory_mse(jfa.feed_forward(b, U0s, nsteps, dts), refs)
    loss.backward()
    g_ff = [U.grad.clone() for U in U0s]
    # the same loss through per-step single-grid autograd
    V0s = [U.detach().clone().requires_grad_(True) for U in U0s]
    trajs = []
    for i, V in enumerate(V0s):
        s = b.solver(i)
        dt = s.scalar(dts[i])
        states = [V]
        for _ in range(nsteps):
            states.append(jfa.rk3_step(s, states[-1], dt))
        trajs.append(torch.stack(states))
    jfa.trajectory_mse(trajs, refs).backward()
    for a, V in zip(g_ff, V0s):
        assert torch.allclose(a, V.grad, rtol=1e-12, atol=1e-15 * a.abs().max().item())
    # directional central difference along smooth random fields
    vs = [torch.tensor(inputs.random_smooth(c.n, seed=20 + i).U - 1.0, dtype=torch.float64, device="cuda")
          for i, c in enumerate(cases)]

    def L(eps):
        with torch.no_grad():
            tr = b.feed_forward([U.detach() + eps * v for U, v in zip(U0s, vs)], nsteps, dts)
            return jfa.trajectory_mse(tr, refs).item()

    # sanity bound: the WENO weights make the loss's higher derivatives large,
    # so the central difference carries a relative error of ~1e-5 (the exact
    # check is the chain above and the oracle-Jacobian tests of the adjoint)
    eps = 1e-6
    fd = (L(eps) - L(-eps)) / (2 * eps)
    ad = sum(float((g * v).sum()) for g, v in zip(g_ff, vs))
    assert abs(fd - ad) <= 3e-5 * abs(ad)
    b.close()
