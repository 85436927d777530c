"""Host-side pieces of the Section 7.4 training (CPU): the implosion's
initial state, coarse-graining, the primitive variables and the trajectory
loss."""
import numpy as np
import pytest

from paper_2203_13760_gb300 import inputs

torch = pytest.importorskip("torch")

from paper_2203_13760_gb300 import learned_flux as lf  # noqa: E402


def test_implosion_initial_state():
    case = inputs.implosion(32)
    U = case.U
    assert U.shape == (5, 1, 32, 32) and case.bc == (2, 2, 2, 2, 1, 1)
    rho = U[0, 0]
    # the lower-left triangle x + y <= 0.15 holds the low state, the rest the high one
    assert rho[0, 0] == 0.14 and rho[-1, -1] == 1.0 and rho[0, 4] == 1.0 and rho[1, 2] == 0.14
    assert np.array_equal(rho, rho.T)  # symmetric about the diagonal
    assert np.all(U[1:4] == 0)
    p = (1.4 - 1) * U[4, 0]
    assert set(np.unique(p)) == {0.125, 1.0}
    assert case.recon == "weno3-js" and case.integrator == "rk2" and case.dt == 2.5e-4


def test_coarse_grain_keeps_totals_and_averages():
    rng = np.random.default_rng(0)
    U = torch.tensor(rng.uniform(0.5, 2.0, (5, 1, 8, 12)))
    C = lf.coarse_grain(U, 4)
    assert C.shape == (5, 1, 2, 3)
    assert torch.allclose(C.sum(dim=(1, 2, 3)) * 16, U.sum(dim=(1, 2, 3)), rtol=1e-14)
    assert torch.isclose(C[2, 0, 1, 2], U[2, 0, 4:8, 8:12].mean(), rtol=1e-14)


def test_primitives_invert_conservative():
    rng = np.random.default_rng(1)
    rho, u, v, p = rng.uniform(0.5, 2, (4, 1, 3, 4))
    U = inputs.conservative(rho, u, v, 0.0, p, 1.4)
    W = lf.primitives(torch.tensor(U)).numpy()
    for got, want in zip(W, (rho, u, v, p)):
        np.testing.assert_allclose(got, want, rtol=1e-13)


def test_trajectory_loss_definition():
    """1/N_T sum_i mean((W_i - W_i^ref)^2) over (rho, u, v, p) and cells,
    averaged over the windows; slot 0 does not count."""
    rng = np.random.default_rng(2)
    states = []
    for _ in range(4):
        rho, u, v, p = rng.uniform(0.5, 2, (4, 1, 2, 3))
        states.append(inputs.conservative(rho, u, v, 0.0, p, 1.4))
    ref = torch.tensor(np.stack(states))
    pred = ref.clone()
    pred[0] += 5.0  # the initial state is not part of the loss
    assert lf.trajectory_loss([pred], [ref]).item() == 0.0
    pred = ref.clone()
    pred[2, 0] *= 1.1  # density of step 2 up by 10 %
    W, Wr = lf.primitives(pred), lf.primitives(ref)
    want = float(((W[1:] - Wr[1:]) ** 2).mean())
    assert lf.trajectory_loss([pred, ref], [ref, ref]).item() == pytest.approx(want / 2, rel=1e-14)
    assert want > 0
