"""Section 4.5 feed_forward and the Section 7.2 trajectory loss against the
oracle (not only against the GPU's own single-grid path).

* Slot t of each trajectory of an uneven batch equals t fixed-dt oracle steps
  of that simulation (FP64, relative L-infinity per conserved quantity
  <= 1e-12), for every integrator.
* The gradient of the trajectory MSE w.r.t. the initial states satisfies the
  dot-product identity <dL/dU0, v> = dL(U0 + e v)/de at e = 0, the right side
  formed from the oracle's dual-number JVPs of the trajectory (each step's
  tangent propagated by forward mode) and the oracle's own trajectory; the
  reference trajectories are oracle runs too.  FP64, 1e-10 of the sum of the
  terms' magnitudes.
"""
import numpy as np
import pytest

from paper_2203_13760_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2203_13760_gb300 import autograd as jfa  # noqa: E402
from paper_2203_13760_gb300 import jf  # noqa: E402

GROUPS = ((0,), (1, 2, 3), (4,))


def rel_err(a, b):
    a = np.asarray(a, dtype=np.float64).reshape(5, -1)
    b = np.asarray(b, dtype=np.float64).reshape(5, -1)
    return max(np.abs(a[list(g)] - b[list(g)]).max() / np.abs(b[list(g)]).max() for g in GROUPS)


def make_batch(cases, dtype, **kw):
    grids = [jf.make_grid(c.n, c.lo, c.hi, c.bc) for c in cases]
    p = dict(cases[0].params(), **kw)
    return jf.Batch(grids, dtype=dtype, **{k: p[k] for k in ("gamma", "R", "mu", "Pr", "eps", "cfl", "viscous",
                                                               "heat", "flux", "recon", "speeds", "integrator")})


def dev(U):
    return torch.tensor(np.ascontiguousarray(U), dtype=torch.float64, device="cuda")


@pytest.mark.parametrize("integrator", ["rk3", "rk2", "euler"])
def test_feed_forward_slots_match_oracle(orc, integrator):
    """Uneven four-quadrant batch (ragged sides), each simulation with its own
    fixed step: every slot against the oracle's fixed-dt steps."""
    cases = inputs.four_quadrant_batch(nsim=3, sides=(37, 48, 29), seed=21)
    dts = []
    for c in cases:
        oc = orc.config(**dict(c.params(), integrator=integrator))
        dts.append(0.8 * orc.compute_dt(oc, c.U))
    nsteps = 6
    b = make_batch(cases, "f64", integrator=integrator)
    trajs = b.feed_forward([dev(c.U) for c in cases], nsteps, dts)
    b.sync()
    for i, c in enumerate(cases):
        oc = orc.config(**dict(c.params(), integrator=integrator))
        want = c.U.copy()
        assert rel_err(trajs[i][0].cpu().numpy(), want) == 0.0
        for t in range(1, nsteps + 1):
            want = orc.run(oc, want, 1, dts[i])[0]
            err = rel_err(trajs[i][t].cpu().numpy(), want)
            assert err <= 1e-12, (i, t, err)
    b.close()


def oracle_trajectory_derivative(orc, cases, dts, nsteps, refs, vs):
    """dL/de of the Section 7.2 loss along the tangents vs, by the oracle:
    per simulation the trajectory U^t and its tangent V^t = J_t ... J_1 v
    (dual-number forward mode, one step at a time), then
    dL = 1/S sum_s 1/N_T sum_t 2/M_s sum (U^t - ref^t) V^t."""
    total = 0.0
    for c, dt, ref, v in zip(cases, dts, refs, vs):
        oc = orc.config(**c.params())
        U, V = c.U.copy(), v.copy()
        m = U.size
        acc = 0.0
        for t in range(1, nsteps + 1):
            U, V = orc.jvp_run(oc, U, V, 1, dt)
            acc += 2.0 / m * float(np.sum((U - ref[t]) * V))
        total += acc / nsteps
    return total / len(cases)


def oracle_refs(orc, cases, dts, nsteps):
    out = []
    for c, dt in zip(cases, dts):
        oc = orc.config(**c.params())
        traj = [c.U.copy()]
        for _ in range(nsteps):
            traj.append(orc.run(oc, traj[-1], 1, dt)[0])
        out.append(np.stack(traj))
    return out


@pytest.mark.parametrize("kind", ["viscous_kh", "inviscid_quadrants"])
def test_trajectory_loss_gradient_against_oracle_jvp(orc, kind):
    """Viscous Kelvin-Helmholtz grids take the per-simulation tiled adjoint;
    inviscid four-quadrant grids take the batched per-face adjoint
    (jf_batch_step_vjp).  Both against the oracle's forward mode."""
    if kind == "viscous_kh":
        cases = [inputs.kelvin_helmholtz(21, seed=1), inputs.kelvin_helmholtz(28, seed=2)]
        targets = [inputs.kelvin_helmholtz(21, seed=5), inputs.kelvin_helmholtz(28, seed=6)]
    else:
        cases = inputs.four_quadrant_batch(nsim=2, sides=(24, 33), seed=13)
        targets = inputs.four_quadrant_batch(nsim=2, sides=(24, 33), seed=13)
        targets = [inputs.Case(t.name, t.n, t.lo, t.hi, t.bc, t.U * 1.01) for t in targets]
    nsteps = 5
    dts = [0.5 * orc.compute_dt(orc.config(**c.params()), c.U) for c in cases]
    refs = oracle_refs(orc, targets, dts, nsteps)
    b = make_batch(cases, "f64")
    U0s = [dev(c.U).requires_grad_(True) for c in cases]
    loss = jfa.trajectory_mse(jfa.feed_forward(b, U0s, nsteps, dts), [dev(r) for r in refs])
    loss.backward()
    vs = [inputs.random_smooth(c.n, seed=40 + i).U - 1.0 for i, c in enumerate(cases)]
    lhs_terms = [float((U.grad * dev(v)).sum()) for U, v in zip(U0s, vs)]
    lhs = sum(lhs_terms)
    rhs = oracle_trajectory_derivative(orc, cases, dts, nsteps, refs, vs)
    scale = sum(float((U.grad.abs() * dev(np.abs(v))).sum()) for U, v in zip(U0s, vs))
    assert abs(lhs - rhs) <= 1e-10 * scale, (lhs, rhs, scale)
    b.close()
