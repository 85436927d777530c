"""Adjoint of the run-time schemes on the GPU (the per-face adjoint): slip
walls, WENO3-JS, HLLC and the Rusanov-NN flux with its parameter gradient,
TVD-RK3 / TVD-RK2 / Euler, against the oracle's dual-number JVPs through the
dot-product identity <VJP(w), v> = <w, JVP(v)>.

Bars: FP64 1e-11 of the sum of the absolute terms of the two dot products
(the atomic summation order varies); FP32 3e-5 (the bar of the tiled
adjoint's FP32 identity)."""
import numpy as np
import pytest

from paper_2203_13760_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2203_13760_gb300 import jf  # noqa: E402

W = inputs.WALL
THETA = inputs.nn_params(seed=5, alpha=2.0)

CASES = {
    "1d_walls": lambda: inputs.random_smooth((40, 1, 1), seed=2, bc=(W, W, 1, 1, 1, 1)),
    "2d_box": lambda: inputs.random_smooth((21, 17, 1), seed=3, bc=(W, W, W, W, 1, 1)),
    "2d_wall_periodic": lambda: inputs.random_smooth((20, 19, 1), seed=4, bc=(0, 0, 1, W, 1, 1)),
    "3d_mixed": lambda: inputs.random_smooth((11, 10, 9), seed=6, bc=(W, 1, 0, 0, W, W)),
}
SCHEMES = {
    "nn_weno3_rk2": dict(flux="rusanov-nn", recon="weno3-js", integrator="rk2"),
    "nn_weno5_rk3": dict(flux="rusanov-nn"),
    "nn_weno3_euler": dict(flux="rusanov-nn", recon="weno3-js", integrator="euler"),
    "hllc_weno3_rk2": dict(recon="weno3-js", integrator="rk2"),
    "hllc_weno5_rk3": dict(),
}


def with_scheme(case, **kw):
    for k, v in kw.items():
        setattr(case, k, v)
    return case


def dot_check(lhs_vec, v, w, Jv, tol):
    lhs = float(np.dot(lhs_vec.reshape(-1), v.reshape(-1)))
    rhs = float(np.dot(w.reshape(-1), Jv.reshape(-1)))
    scale = float(np.abs(lhs_vec.reshape(-1) * v.reshape(-1)).sum() + np.abs(w.reshape(-1) * Jv.reshape(-1)).sum())
    assert abs(lhs - rhs) <= tol * scale, (lhs, rhs, scale)


def run_case(orc, name, scheme, dtype, tol, nn_grad=False):
    case = with_scheme(CASES[name](), **SCHEMES[scheme])
    nn = case.flux == "rusanov-nn"
    c = orc.config(**case.params(), nn=THETA if nn else None)
    U0 = case.U.astype(np.float32).astype(np.float64) if dtype == "f32" else case.U
    dt = 0.5 * orc.compute_dt(c, U0)
    rng = np.random.default_rng(11)
    w = rng.standard_normal(case.U.shape)
    v = rng.standard_normal(case.U.shape)
    t = torch.float32 if dtype == "f32" else torch.float64
    theta = torch.tensor(THETA, dtype=t, device="cuda") if nn else None
    s = jf.Solver.from_case(case, dtype=dtype, nn=theta)
    Ud = torch.tensor(U0, dtype=t, device="cuda")
    wd = torch.tensor(w, dtype=t, device="cuda")
    if nn_grad:
        lam, tb = s.rk3_step_vjp_params(Ud, s.scalar(dt), wd)
    else:
        lam, tb = s.rk3_step_vjp(Ud, s.scalar(dt), wd), None
    s.sync()
    _, Jv = orc.jvp_run(c, U0, v, 1, dt)
    dot_check(lam.double().cpu().numpy(), v, w, Jv, tol)
    if nn_grad:
        td = rng.standard_normal(jf.NN_PARAMS)
        _, Jt = orc.jvp_params_run(c, U0, 1, dt, td)
        dot_check(tb.double().cpu().numpy(), td, w, Jt, tol)
        assert np.abs(tb.double().cpu().numpy()).max() > 0


@pytest.mark.parametrize("scheme", sorted(SCHEMES))
@pytest.mark.parametrize("name", sorted(CASES))
def test_state_adjoint_fp64(orc, name, scheme):
    run_case(orc, name, scheme, "f64", 1e-11)


@pytest.mark.parametrize("scheme", ["nn_weno3_rk2", "nn_weno5_rk3", "nn_weno3_euler"])
@pytest.mark.parametrize("name", sorted(CASES))
def test_parameter_gradient_fp64(orc, name, scheme):
    run_case(orc, name, scheme, "f64", 1e-11, nn_grad=True)


@pytest.mark.parametrize("scheme", ["nn_weno3_rk2", "hllc_weno3_rk2"])
@pytest.mark.parametrize("name", ["2d_box", "3d_mixed"])
def test_adjoint_fp32(orc, name, scheme):
    run_case(orc, name, scheme, "f32", 3e-5, nn_grad=scheme.startswith("nn"))


def test_parameter_gradient_accumulates_over_calls(orc):
    """theta_bar is added to: two calls give twice one call (to rounding)."""
    case = with_scheme(CASES["2d_box"](), **SCHEMES["nn_weno3_rk2"])
    s = jf.Solver.from_case(case, dtype="f64", nn=torch.tensor(THETA, dtype=torch.float64, device="cuda"))
    U = torch.tensor(case.U, dtype=torch.float64, device="cuda")
    w = torch.ones_like(U)
    dt = s.scalar(1e-3)
    _, once = s.rk3_step_vjp_params(U, dt, w)
    tb = torch.zeros(jf.NN_PARAMS, dtype=torch.float64, device="cuda")
    s.rk3_step_vjp_params(U, dt, w, theta_bar=tb)
    s.rk3_step_vjp_params(U, dt, w, theta_bar=tb)
    s.sync()
    assert torch.allclose(tb, 2 * once, rtol=1e-12, atol=1e-14 * once.abs().max().item())


def test_unsupported_adjoints_are_refused():
    visc = with_scheme(inputs.random_smooth((16, 12, 1), seed=1, bc=(W, W, 1, 1, 1, 1), viscous=True, mu=0.01))
    s = jf.Solver.from_case(visc, dtype="f64")
    U = torch.tensor(visc.U, dtype=torch.float64, device="cuda")
    with pytest.raises(jf.JFError) as e:
        s.rk3_step_vjp(U, s.scalar(1e-3), torch.ones_like(U))
    assert e.value.status == jf.JF_ERR_UNSUPPORTED
    hll = with_scheme(inputs.random_smooth((16, 12, 1), seed=1), flux="hll")
    s = jf.Solver.from_case(hll, dtype="f64")
    with pytest.raises(jf.JFError) as e:
        s.rk3_step_vjp(U, s.scalar(1e-3), torch.ones_like(U))
    assert e.value.status == jf.JF_ERR_UNSUPPORTED
    with pytest.raises(jf.JFError) as e:  # parameter gradient of a flux without parameters
        s.rk3_step_vjp_params(U, s.scalar(1e-3), torch.ones_like(U))
    assert e.value.status == jf.JF_ERR_ARG


@pytest.mark.parametrize("scheme", ["nn_weno3_rk2", "hllc_weno5_rk3", "nn_weno3_euler"])
def test_batch_adjoint_equals_single_grids(scheme):
    """jf_batch_step_vjp over an uneven batch (with walls) equals each grid's
    single-grid adjoint plus the addend, and its theta_bar the sum of the
    single-grid parameter gradients (FP64, to rounding: atomic order)."""
    cases = [with_scheme(c, **SCHEMES[scheme]) for c in inputs.four_quadrant_batch(nsim=3, sides=(32, 48), seed=7)]
    for c in cases:
        c.bc = (W, W, W, 1, 1, 1)
    nn = cases[0].flux == "rusanov-nn"
    theta = torch.tensor(THETA, dtype=torch.float64, device="cuda") if nn else None
    p = cases[0].params()
    b = jf.Batch([jf.make_grid(c.n, c.lo, c.hi, c.bc) for c in cases], dtype="f64", nn=theta,
                 **{k: p[k] for k in ("gamma", "R", "mu", "Pr", "eps", "cfl", "viscous", "heat", "flux", "recon",
                                      "speeds", "integrator")})
    assert b.supports_step_vjp()
    rng = np.random.default_rng(4)
    Us = [torch.tensor(c.U, dtype=torch.float64, device="cuda") for c in cases]
    lams = [torch.tensor(rng.standard_normal(c.U.shape), device="cuda") for c in cases]
    adds = [torch.tensor(rng.standard_normal(c.U.shape), device="cuda") for c in cases]
    dts = [2e-4, 3e-4, 2.5e-4]
    tb = torch.zeros(jf.NN_PARAMS, dtype=torch.float64, device="cuda") if nn else None
    got = b.step_vjp(Us, torch.tensor(dts, dtype=torch.float64, device="cuda"), lams, None, adds, tb)
    b.sync()
    tb_ref = torch.zeros_like(tb) if nn else None
    for i, c in enumerate(cases):
        s = b.solver(i)
        if nn:
            want, _ = s.rk3_step_vjp_params(Us[i], s.scalar(dts[i]), lams[i], theta_bar=tb_ref)
        else:
            want = s.rk3_step_vjp(Us[i], s.scalar(dts[i]), lams[i])
        s.sync()
        want = want + adds[i]
        assert (got[i] - want).abs().max().item() <= 1e-12 * want.abs().max().item(), i
    if nn:
        assert (tb - tb_ref).abs().max().item() <= 1e-12 * tb_ref.abs().max().item()


@pytest.mark.parametrize("scheme", ["nn_weno3_rk2", "nn_weno3_euler"])
def test_deferred_parameter_gradient(scheme):
    """jf_batch_param_grad_begin / end: the parameter gradient of several
    batch adjoint steps summed in one launch equals the sum of the per-call
    gradients (FP64, to rounding), the state cotangents are unchanged, and
    the record store refuses more steps than it was opened for."""
    cases = [with_scheme(c, **SCHEMES[scheme]) for c in inputs.four_quadrant_batch(nsim=3, sides=(32, 48), seed=9)]
    for c in cases:
        c.bc = (W, W, W, 1, 1, 1)
    theta = torch.tensor(THETA, dtype=torch.float64, device="cuda")
    p = cases[0].params()
    b = jf.Batch([jf.make_grid(c.n, c.lo, c.hi, c.bc) for c in cases], dtype="f64", nn=theta,
                 **{k: p[k] for k in ("gamma", "R", "mu", "Pr", "eps", "cfl", "viscous", "heat", "flux", "recon",
                                      "speeds", "integrator")})
    rng = np.random.default_rng(5)
    Us = [torch.tensor(c.U, dtype=torch.float64, device="cuda") for c in cases]
    dt = torch.tensor([2e-4, 3e-4, 2.5e-4], dtype=torch.float64, device="cuda")
    lams = [[torch.tensor(rng.standard_normal(c.U.shape), device="cuda") for c in cases] for _ in range(3)]
    tb_each = torch.zeros(jf.NN_PARAMS, dtype=torch.float64, device="cuda")
    outs_each = [b.step_vjp(Us, dt, lams[k], None, None, tb_each) for k in range(3)]
    tb_once = torch.zeros_like(tb_each)
    b.param_grad_begin(3)
    outs_once = [b.step_vjp(Us, dt, lams[k], None, None, tb_once) for k in range(3)]
    assert float(tb_once.abs().max()) == 0.0  # nothing added before the end call
    b.param_grad_end(tb_once)
    b.sync()
    for a, c in zip(outs_each, outs_once):
        for x, y in zip(a, c):
            assert (x - y).abs().max().item() <= 1e-12 * x.abs().max().item()
    assert (tb_once - tb_each).abs().max().item() <= 1e-12 * tb_each.abs().max().item()
    # the store holds max_steps steps; the end call needs a begin
    b.param_grad_begin(1)
    b.step_vjp(Us, dt, lams[0], None, None, tb_once)
    with pytest.raises(jf.JFError) as e:
        b.step_vjp(Us, dt, lams[1], None, None, tb_once)
    assert e.value.status == jf.JF_ERR_ARG
    b.param_grad_end(tb_once)
    with pytest.raises(jf.JFError) as e:
        b.param_grad_end(tb_once)
    assert e.value.status == jf.JF_ERR_ARG
