"""Section 7.4 end to end on the GPU: the implosion reference, the gradient
of the trajectory loss with respect to the network parameters (through
jf_batch_feed_forward and jf_rk3_step_vjp_params) against central
differences, training that lowers the loss, and the loss kernel
(jf_loss_primitive_mse) against its definition."""
import numpy as np
import pytest

from paper_2203_13760_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2203_13760_gb300 import autograd as jfa  # noqa: E402
from paper_2203_13760_gb300 import jf  # noqa: E402
from paper_2203_13760_gb300 import learned_flux as lf  # noqa: E402


@pytest.fixture(scope="module")
def small_reference():
    # 32^2 fine run (WENO3-JS / HLLC / TVD-RK2, dt 5e-4), every 2 steps, on 16^2
    return lf.ground_truth(n_fine=32, factor=2, nsamples=14, dt=5e-4, every=2, dtype="f64")


def test_reference_is_symmetric_about_the_diagonal(small_reference):
    """Initial state and walls are symmetric under x <-> y (with u <-> v)."""
    cg = small_reference
    rho = cg[:, 0, 0]
    assert torch.allclose(rho, rho.transpose(-1, -2), rtol=1e-12, atol=0)
    assert torch.allclose(cg[:, 1, 0], cg[:, 2, 0].transpose(-1, -2), rtol=1e-10, atol=1e-13)
    assert torch.all(torch.isfinite(cg)).item()


def test_loss_gradient_matches_central_differences(small_reference):
    tr = lf.Trainer(small_reference, inputs.nn_params(seed=7, alpha=2.0), batch=2, unroll=3, n_train=10,
                    dtype="f64")
    starts = [1, 6]
    loss, grad = tr.loss_and_grad(starts)
    rng = np.random.default_rng(3)
    d = torch.tensor(rng.standard_normal(grad.numel()), dtype=torch.float64, device="cuda")
    d /= d.norm()
    eps = 1e-6
    vals = []
    with torch.no_grad():
        base = tr.theta.detach().clone()
        for sgn in (1, -1):
            tr.theta.copy_(base + sgn * eps * d)
            trajs = lf.autograd.feed_forward(tr.batch, [tr.cg[s] for s in starts], tr.unroll, tr.dt)
            vals.append(float(lf.trajectory_loss(trajs, [tr.cg[s:s + 4] for s in starts])))
        tr.theta.copy_(base)
    fd = (vals[0] - vals[1]) / (2 * eps)
    ad = float(grad @ d)
    assert abs(ad) > 0
    assert abs(fd - ad) <= 1e-6 * abs(ad) + 1e-12 * float(loss), (fd, ad)


def test_training_lowers_the_loss(small_reference):
    tr = lf.Trainer(small_reference, inputs.nn_params(seed=7, alpha=2.0), batch=4, unroll=4, lr=2e-3, n_train=10,
                    dtype="f32")
    rng = np.random.default_rng(0)
    first = tr.step(rng.choice(tr.starts, 4, replace=False))
    for _ in range(40):
        last = tr.step(rng.choice(tr.starts, 4, replace=False))
    losses = [tr.step(s) for s in ([0, 2, 4, 6], [1, 3, 5, 6])]
    assert np.isfinite(last) and max(losses) < first


def test_rollout_errors_are_finite(small_reference):
    e_rho, e_p = lf.rollout_errors(small_reference, 10, flux="rusanov", dtype="f64")
    assert e_rho.shape == (10,) and np.all(np.isfinite(e_rho)) and np.all(np.isfinite(e_p))
    e2, _ = lf.rollout_errors(small_reference, 10, theta=inputs.nn_params(seed=7), dtype="f64")
    assert np.all(np.isfinite(e2))


@pytest.mark.parametrize("dtype,ncomp,tol", [("f64", 4, 1e-13), ("f64", 5, 1e-13), ("f32", 4, 1e-6)])
def test_primitive_mse_kernel_matches_definition(dtype, ncomp, tol):
    """jf_loss_primitive_mse against the Section 7.4 loss written out in
    PyTorch (FP64): the loss and its gradient w.r.t. the predicted states
    (autograd of the written-out definition), on a stack of ragged states."""
    t = torch.float32 if dtype == "f32" else torch.float64
    cases = [inputs.random_blocks((13, 11, 1), seed=s) for s in range(6)]
    refs = [inputs.random_smooth((13, 11, 1), seed=10 + s) for s in range(6)]
    U = torch.tensor(np.stack([c.U for c in cases]), dtype=t, device="cuda").reshape(2, 3, 5, 1, 11, 13)
    R = torch.tensor(np.stack([c.U for c in refs]), dtype=t, device="cuda").reshape(2, 3, 5, 1, 11, 13)
    grids = [jf.make_grid((13, 11, 1))]
    b = jf.Batch(grids, dtype=dtype)
    loss, grad = jf.loss_primitive_mse(b, U, R, ncomp)
    b.sync()

    def prim(X):
        rho = X[..., 0, :, :, :]
        u, v, w = (X[..., k, :, :, :] / rho for k in (1, 2, 3))
        p = 0.4 * (X[..., 4, :, :, :] - 0.5 * rho * (u * u + v * v + w * w))
        comps = [rho, u, v, p] if ncomp == 4 else [rho, u, v, w, p]
        return torch.stack(comps, dim=-4)

    Ud = U.double().clone().requires_grad_(True)
    want = ((prim(Ud) - prim(R.double())) ** 2).mean()
    want.backward()
    assert abs(loss.item() - want.item()) <= tol * abs(want.item())
    gscale = Ud.grad.abs().max().item()
    assert torch.allclose(grad.double(), Ud.grad, rtol=0, atol=tol * 10 * gscale)
    # through autograd, with the loss of a window stack
    X = U.clone().requires_grad_(True)
    autograd_loss = jfa.primitive_mse(b, X, R, ncomp)
    autograd_loss.backward()
    assert torch.equal(X.grad, grad)
    b.close()
