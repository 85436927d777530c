"""The Section 7.2 trajectory loss of the autograd layer (plain torch; CPU)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2203_13760_gb300 import autograd as jfa  # noqa: E402


def test_trajectory_mse_definition():
    """1/N_T sum_{i=1..N_T} mean((U^i - U^i_ref)^2), slot 0 excluded, averaged
    over the simulations."""
    rng = np.random.default_rng(0)
    a = [torch.tensor(rng.standard_normal((4, 5, 1, 3, 2))), torch.tensor(rng.standard_normal((4, 5, 1, 2, 2)))]
    r = [torch.tensor(rng.standard_normal((4, 5, 1, 3, 2))), torch.tensor(rng.standard_normal((4, 5, 1, 2, 2)))]
    want = np.mean([np.mean([np.mean((x[i] - y[i]).numpy() ** 2) for i in range(1, 4)]) for x, y in zip(a, r)])
    assert jfa.trajectory_mse(a, r).item() == pytest.approx(want, rel=1e-14)
