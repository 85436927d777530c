"""Parity at the full sizes of the benchmark workloads, in the launch
configuration bench.py times (default variant, jf_rk3_run graph), on sampled
cells that the oracle computes one at a time (oracle.sample_cells), plus
properties that hold at any size."""
import numpy as np
import pytest

from paper_2203_13760_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2203_13760_gb300 import jf  # noqa: E402


def _samples(n, count, seed):
    rng = np.random.default_rng(seed)
    cells = np.stack([rng.integers(0, n[d], count) for d in range(3)], axis=1)
    # corners and faces of the domain too
    corners = np.array([[0, 0, 0], [n[0] - 1, n[1] - 1, n[2] - 1], [0, n[1] - 1, 0], [n[0] - 1, 0, n[2] - 1]])
    return np.concatenate([cells, corners])


@pytest.mark.parametrize("n,dtype,tol", [(256, "f32", 1e-5), (128, "f64", 1e-12)])
def test_tgv_one_step_sampled(orc, n, dtype, tol):
    """Compressible TGV (Re 1600, Ma 0.1, viscous + heat) at the benchmark's
    256^3 FP32 size (and 128^3 FP64): one CFL RK3 step through jf_rk3_run,
    compared with the oracle on sampled cells; the oracle computes dt itself
    from the full state."""
    case = inputs.taylor_green(n)
    npdt = np.float32 if dtype == "f32" else np.float64
    U0 = case.U.astype(npdt)
    c = orc.config(**case.params())
    dt_ref = orc.compute_dt(c, U0.astype(np.float64))
    s = jf.Solver.from_case(case, dtype=dtype)
    U = torch.from_numpy(U0).cuda()
    hist = s.scalar()
    s.run(U, 1, None, hist)
    s.sync()
    assert hist.item() == pytest.approx(dt_ref, rel=1e-6 if dtype == "f32" else 1e-13)
    cells = _samples(case.n, 24, 1)
    want = orc.sample_cells(c, U0.astype(np.float64), cells, 1, dt_ref)
    got = U.cpu().numpy()
    got = np.stack([got[:, k, j, i] for i, j, k in cells])
    err = 0.0
    for g in ((0,), (1, 2, 3), (4,)):  # mass, momentum vector, energy
        scale = np.abs(U0[list(g)]).max()
        err = max(err, np.abs(got[:, list(g)] - want[:, list(g)]).max() / scale)
    assert err <= tol


def test_hit384_rhs_sampled_and_invariants(orc):
    """Inviscid solenoidal turbulence at 384^3 FP32 (the sustained-bandwidth
    workload): right-hand side on sampled cells against the oracle, and the
    telescoping property sum_cells L(U) = 0 on the periodic box."""
    case = inputs.solenoidal_turbulence(384, device="cuda")
    U0 = case.U.astype(np.float32)
    c = orc.config(**case.params())
    s = jf.Solver.from_case(case, dtype="f32")
    U = torch.from_numpy(U0).cuda()
    r = s.rhs(U)
    s.sync()
    cells = _samples(case.n, 24, 2)
    want = orc.sample_cells(c, U0.astype(np.float64), cells, 0)
    got = r.cpu().numpy()
    got = np.stack([got[:, k, j, i] for i, j, k in cells])
    # FP32 right-hand side: a difference of fluxes over dx, compared relative
    # to the flux scale max(|L|, |U| a / h) of each conserved quantity
    rate = case.cfl / orc.compute_dt(c, U0.astype(np.float64))
    for g in ((0,), (1, 2, 3), (4,)):
        scale = max(np.abs(want[:, list(g)]).max(), np.abs(U0[list(g)]).max() * rate)
        assert np.abs(got[:, list(g)] - want[:, list(g)]).max() / scale <= 1e-5
    total = r.double().sum(dim=(1, 2, 3)).abs().cpu().numpy()
    mag = r.double().abs().sum(dim=(1, 2, 3)).cpu().numpy()
    assert np.all(total <= 1e-5 * mag)
