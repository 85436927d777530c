"""Adjoint of the RK3 step (jf_rk3_step_vjp) against the oracle.

* The full vector J^T w of the GPU (FP64) equals the one assembled from the
  oracle's dual-number JVPs J e_k (every basis vector), element by element.
* Dot-product identity <VJP(w), v> = <w, JVP(v)> (FP64 and FP32).
* Section 7.3 protocol: gradient of the entropy increase of a Mach-2 shock
  after 5 steps of dt = 1e-2 w.r.t. the shock Mach number, against the
  oracle's forward-mode gradient and central differences (second order).
* Checkpointed trajectory gradient (autograd) against finite differences.
* Kept stage states: jf_rk3_step_keep equals jf_rk3_step and the stage calls
  bit for bit, and jf_rk3_step_vjp_stages equals jf_rk3_step_vjp.
"""
import math

import numpy as np
import pytest

from conftest import golden
from paper_2203_13760_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2203_13760_gb300 import autograd as jfa  # noqa: E402
from paper_2203_13760_gb300 import jf  # noqa: E402

CASES = {
    "1d_blocks_zg": lambda: inputs.random_blocks((14, 1, 1), seed=3),
    "1d_smooth_visc_periodic": lambda: inputs.random_smooth((12, 1, 1), seed=4, viscous=True, mu=0.02),
    "2d_smooth_visc_periodic": lambda: inputs.random_smooth((9, 8, 1), seed=5, viscous=True, mu=0.02),
    "2d_blocks_mixed_bc": lambda: inputs.random_blocks((8, 7, 1), seed=6, bc=(0, 0, 1, 1, 1, 1)),
    "2d_kh_visc": lambda: inputs.kelvin_helmholtz(10, seed=1),
    "2d_smooth_zg_visc": lambda: inputs.random_smooth((7, 9, 1), seed=8, bc=(1,) * 6, viscous=True, mu=0.03),
    "3d_smooth_visc_periodic": lambda: inputs.random_smooth((6, 5, 5), seed=9, viscous=True, mu=0.02),
    "3d_blocks_mixed_bc": lambda: inputs.random_blocks((5, 6, 5), seed=10, bc=(0, 0, 1, 1, 0, 0)),
    "3d_smooth_zg_visc_ragged": lambda: inputs.random_smooth((9, 5, 6), seed=12, bc=(1,) * 6, viscous=True,
                                                             mu=0.03),
}


def oracle_jacobian_T(orc, case, dt, w):
    """J^T w from the oracle's JVPs on every basis vector."""
    c = orc.config(**case.params())
    n = case.U.size
    out = np.zeros(n)
    wf = w.reshape(-1)
    for k in range(n):
        e = np.zeros(n)
        e[k] = 1.0
        _, Je = orc.jvp_run(c, case.U, e.reshape(case.U.shape), 1, dt)
        out[k] = np.dot(wf, Je.reshape(-1))
    return out.reshape(case.U.shape)


@pytest.mark.parametrize("name", sorted(CASES))
def test_vjp_fp64_equals_oracle_jacobian(orc, name):
    case = CASES[name]()
    c = orc.config(**case.params())
    dt = 0.5 * orc.compute_dt(c, case.U)
    rng = np.random.default_rng(11)
    w = rng.standard_normal(case.U.shape)
    want = oracle_jacobian_T(orc, case, dt, w)
    s = jf.Solver.from_case(case, dtype="f64")
    Un = torch.tensor(case.U, dtype=torch.float64, device="cuda")
    got = s.rk3_step_vjp(Un, s.scalar(dt), torch.tensor(w, dtype=torch.float64, device="cuda"))
    s.sync()
    got = got.cpu().numpy()
    scale = np.abs(want).max()
    assert np.abs(got - want).max() <= 1e-11 * scale
    # Un is not modified
    assert np.array_equal(Un.cpu().numpy(), case.U)


def _tgv_off_symmetry(n):
    """Taylor-Green field with a 1e-6 seeded perturbation: the exact field is
    mirror-symmetric, so on its symmetry planes the HLLC contact speed S* is
    exactly 0, where the flux is continuous but not differentiable (the two
    one-sided derivatives differ and any rounding picks one of them)."""
    case = inputs.taylor_green(n)
    rng = np.random.default_rng(4)
    case.U = case.U * (1.0 + 1e-6 * rng.standard_normal(case.U.shape))
    return case


# FP32: the reverse pass chains O(100) dependent FP32 operations per output
# value (approximate reciprocals included, <= 2 ulp each), so the identity
# holds to a few hundred FP32 epsilons (6e-8) of the sum of |terms|: 3e-5.
@pytest.mark.parametrize("dtype,tol,make", [
    ("f64", 1e-12, lambda: inputs.kelvin_helmholtz(32, seed=3)),
    ("f32", 3e-5, lambda: inputs.kelvin_helmholtz(32, seed=3)),
    ("f64", 1e-12, lambda: _tgv_off_symmetry(12)),
    ("f32", 3e-5, lambda: _tgv_off_symmetry(16)),
    # several ragged 2D boxes against zero-gradient and mixed boundaries: the
    # ghost-cell fold of the halo accumulator, edges and corners included
    ("f64", 1e-12, lambda: inputs.random_blocks((37, 21, 1), seed=13, bc=(1,) * 6)),
    ("f32", 3e-5, lambda: inputs.random_blocks((37, 21, 1), seed=13, bc=(1,) * 6)),
    ("f64", 1e-12, lambda: inputs.random_smooth((35, 19, 1), seed=14, bc=(0, 0, 1, 1, 1, 1), viscous=True,
                                                mu=0.02)),
    ("f64", 1e-12, lambda: inputs.random_smooth((18, 34, 1), seed=15, bc=(1, 1, 0, 0, 1, 1), viscous=True,
                                                mu=0.02)),
    # several 3D boxes: periodic 16^3 (every box has all its neighbours), and
    # zero-gradient 24^3 (the middle box away from the boundary, the others
    # folding ghost cotangents)
    ("f64", 1e-12, lambda: _tgv_off_symmetry(16)),
    ("f64", 1e-12, lambda: inputs.random_smooth((24, 24, 24), seed=16, bc=(1,) * 6, viscous=True, mu=0.02)),
    # the z-marching 3D kernel: ragged columns (45 = 32 + 13 along x in FP32,
    # 2 x 16 + 13 in FP64), the upper boundary faces of zero-gradient axes,
    # a periodic axis between them, several z chunks
    ("f64", 1e-12, lambda: inputs.random_smooth((45, 19, 13), seed=17, bc=(1, 1, 0, 0, 1, 1), viscous=True,
                                                mu=0.02)),
    ("f32", 3e-5, lambda: inputs.random_smooth((45, 19, 13), seed=17, bc=(1, 1, 0, 0, 1, 1), viscous=True,
                                               mu=0.02)),
    ("f64", 1e-12, lambda: inputs.random_blocks((45, 19, 13), seed=18, bc=(0, 0, 1, 1, 1, 1))),
])
def test_dot_product_identity(orc, dtype, tol, make):
    case = make()
    c = orc.config(**case.params())
    dt = orc.compute_dt(c, case.U)
    rng = np.random.default_rng(5)
    w = rng.standard_normal(case.U.shape)
    v = rng.standard_normal(case.U.shape)
    t = torch.float32 if dtype == "f32" else torch.float64
    U0 = case.U.astype(np.float32).astype(np.float64) if dtype == "f32" else case.U
    _, Jv = orc.jvp_run(c, U0, v, 1, dt)
    s = jf.Solver.from_case(case, dtype=dtype)
    lam = s.rk3_step_vjp(torch.tensor(U0, dtype=t, device="cuda"), s.scalar(dt),
                         torch.tensor(w, dtype=t, device="cuda"))
    s.sync()
    lam = lam.double().cpu().numpy().reshape(-1)
    lhs = float(np.dot(lam, v.reshape(-1)))
    rhs = float(np.dot(w.reshape(-1), Jv.reshape(-1)))
    # rounding scale of the two dot products: the sums of their absolute terms
    scale = float(np.abs(lam * v.reshape(-1)).sum() + np.abs(w.reshape(-1) * Jv.reshape(-1)).sum())
    assert abs(lhs - rhs) <= tol * scale


def _entropy_and_grad(U, gamma):
    """S = sum rho s dx with s = ln(p / rho^gamma) / (gamma - 1) (dx applied
    by the caller) and dS/dU per cell."""
    rho, m, E = U[0], U[1], U[4]
    u = m / rho
    p = (gamma - 1) * (E - 0.5 * rho * u * u)
    S = rho * (np.log(p) - gamma * np.log(rho)) / (gamma - 1)
    dS_drho = (np.log(p) - gamma * np.log(rho) - gamma) / (gamma - 1)
    dS_dp = rho / (p * (gamma - 1))
    g = np.zeros_like(U)
    g[0] = dS_drho + dS_dp * (gamma - 1) * 0.5 * u * u
    g[1] = -dS_dp * (gamma - 1) * u
    g[4] = dS_dp * (gamma - 1)
    return S.sum(), g


def test_shock_entropy_gradient_section_7_3(orc):
    """d(Delta S^n)/dM_S: GPU adjoint vs oracle forward mode (exact to
    round-off) vs central differences (second-order convergence)."""
    gd = golden("gradient_section_7_3.json")
    Ms, dt, n = gd["shock_mach"], gd["dt"], gd["steps"]
    gamma = gd["gamma"]
    case, dU0 = inputs.moving_shock(Ms, gamma=gamma)
    dx = (case.hi[0] - case.lo[0]) / case.n[0]
    c = orc.config(**case.params())
    s = jf.Solver.from_case(case, dtype="f64")
    dtd = s.scalar(dt)
    # forward on the GPU, storing the step inputs
    states = [torch.tensor(case.U, dtype=torch.float64, device="cuda")]
    for _ in range(n):
        nxt = states[-1].clone()
        s.rk3_step(nxt, dtd)
        states.append(nxt)
    Un = states[-1].cpu().numpy()
    _, gN = _entropy_and_grad(Un, gamma)
    _, g0 = _entropy_and_grad(case.U, gamma)
    lam = torch.tensor(gN * dx, dtype=torch.float64, device="cuda")
    for k in reversed(range(n)):
        lam = s.rk3_step_vjp(states[k], dtd, lam)
    s.sync()
    g_ad = float(np.sum((lam.cpu().numpy() - g0 * dx) * dU0))
    # oracle forward mode
    Uo, dUn = orc.jvp_run(c, case.U, dU0, n, dt)
    assert np.allclose(Uo, Un, rtol=1e-12, atol=1e-12)
    g_fm = float(np.sum(gN * dx * dUn) - np.sum(g0 * dx * dU0))
    assert abs(g_ad - g_fm) <= 1e-10 * abs(g_fm)

    def delta_S(M):
        cs, _ = inputs.moving_shock(M, gamma=gamma)
        U, _, _ = orc.run(c, cs.U, n, dt)
        return (_entropy_and_grad(U, gamma)[0] - _entropy_and_grad(cs.U, gamma)[0]) * dx

    errs = []
    for eps in gd["fd_eps"]:
        g_fd = (delta_S(Ms + eps) - delta_S(Ms - eps)) / (2 * eps)
        errs.append(abs(g_fd - g_ad))
    errs = np.array(errs)
    eps = np.array(gd["fd_eps"])
    # second order: the error falls like eps^2 over the paper's range
    slope = np.polyfit(np.log(eps[:5]), np.log(errs[:5]), 1)[0]
    assert slope > 1.7, (slope, errs)
    assert errs[-1] < 1e-6 * abs(g_ad)


def test_checkpointed_rollout_gradient():
    """d loss / d U0 through 45 steps (checkpoints every 20) equals the
    per-step autograd chain and the directional finite difference."""
    case = inputs.kelvin_helmholtz(32, seed=2)
    target_case = inputs.kelvin_helmholtz(32, seed=7)
    s = jf.Solver.from_case(case, dtype="f64")
    dt = s.scalar(0.4 * s.compute_dt(torch.tensor(case.U, dtype=torch.float64, device="cuda")).item())
    target = torch.tensor(target_case.U[0], dtype=torch.float64, device="cuda").contiguous()
    U0 = torch.tensor(case.U, dtype=torch.float64, device="cuda", requires_grad=True)
    loss = jfa.density_l2(s, jfa.rollout(s, U0, 45, dt, ckpt_every=20), target)
    loss.backward()
    g_ckpt = U0.grad.clone()
    U0.grad = None
    U = U0
    for _ in range(45):
        U = jfa.rk3_step(s, U, dt)
    jfa.density_l2(s, U, target).backward()
    assert torch.allclose(g_ckpt, U0.grad, rtol=1e-12, atol=1e-14)
    # a smooth direction (random Fourier modes): noise would put the WENO
    # weights in their stiff regime and the finite difference would measure that
    v = torch.tensor(inputs.random_smooth((32, 32, 1), seed=3).U - 1.0, dtype=torch.float64, device="cuda")

    def L(x):
        y = x.detach().clone()
        s.run(y, 45, dt)
        return s.loss_density_l2(y, target, want_seed=False)[0].item()

    eps = 1e-6
    fd = (L(U0 + eps * v) - L(U0 - eps * v)) / (2 * eps)
    ad = float((g_ckpt * v).sum())
    assert abs(fd - ad) <= 1e-5 * abs(ad)


@pytest.mark.parametrize("dtype,rtol", [("f64", 1e-13), ("f32", 2e-5)])
@pytest.mark.parametrize("make", [lambda: inputs.kelvin_helmholtz(48, seed=5),
                                  lambda: inputs.random_smooth((12, 10, 9), seed=6, viscous=True, mu=0.02),
                                  lambda: inputs.random_blocks((40, 1, 1), seed=7)])
def test_kept_stage_states(make, dtype, rtol):
    case = make()
    s = jf.Solver.from_case(case, dtype=dtype)
    assert s.supports_stage_vjp()
    t = s.dtype
    Un = torch.tensor(case.U, dtype=t, device="cuda")
    dt = s.scalar(0.5 * s.compute_dt(Un).item())
    Ua, Ub = Un.clone(), Un.clone()
    U1, U2 = s.empty(), s.empty()
    s.rk3_step_keep(Ua, dt, U1, U2)
    s.rk3_step(Ub, dt)
    assert torch.equal(Ua, Ub)
    assert torch.equal(U1, s.stage(Un, None, s.empty(), 0.0, 1.0, dt))
    assert torch.equal(U2, s.stage(U1, Un, s.empty(), 0.75, 0.25, dt))
    g = torch.Generator(device="cpu").manual_seed(11)
    lam = torch.randn(s.shape, generator=g, dtype=torch.float64).to(device="cuda", dtype=t)
    a = s.rk3_step_vjp(Un, dt, lam)
    b = s.rk3_step_vjp_stages(Un, U1, U2, dt, lam)
    s.sync()
    scale = float(a.abs().max())
    assert float((a - b).abs().max()) <= rtol * scale


def test_kept_stage_states_refused_elsewhere():
    case = inputs.kelvin_helmholtz(32, seed=5)
    s = jf.Solver.from_case(case, dtype="f64", flux="hll")
    assert not s.supports_stage_vjp()
    Un = torch.tensor(case.U, dtype=torch.float64, device="cuda")
    dt = s.scalar(1e-3)
    U1, U2 = s.empty(), s.empty()
    with pytest.raises(jf.JFError) as e:
        s.rk3_step_vjp_stages(Un, U1, U2, dt, Un.clone())
    assert e.value.status == jf.JF_ERR_UNSUPPORTED
    r = jf.Solver.from_case(case, dtype="f64", integrator="rk2")
    with pytest.raises(jf.JFError) as e:
        r.rk3_step_keep(Un.clone(), dt, U1, U2)
    assert e.value.status == jf.JF_ERR_UNSUPPORTED
