"""Scheme variants of Table 2 on the GPU (HLL, Rusanov, Davis and Toro
signal speeds, WENO5-Z, TVD-RK2, Euler) and the flux-splitting ROE setup
against the oracle, through the C ABI.

Same norms and bars as test_gpu_parity.py: FP64 <= 1e-12 (right-hand side
relative to the flux scale, states per conserved group), FP32 <= 1e-5 after
ten steps.  The batch form of each integrator is bitwise the single-grid
path."""
import numpy as np
import pytest

from paper_2203_13760_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2203_13760_gb300 import jf  # noqa: E402
from test_gpu_parity import rate_err, rel_err, to_dev  # noqa: E402

SCHEMES = {
    "hll_einfeldt": dict(flux="hll"),
    "hll_davis_z": dict(flux="hll", speeds="davis", recon="weno5-z"),
    "hll_toro": dict(flux="hll", speeds="toro"),
    "rusanov": dict(flux="rusanov"),
    "rusanov_z": dict(flux="rusanov", recon="weno5-z"),
    "hllc_davis": dict(speeds="davis"),
    "hllc_toro_z": dict(speeds="toro", recon="weno5-z"),
    "hllc_z_rk2": dict(recon="weno5-z", integrator="rk2"),
    "hll_euler": dict(flux="hll", integrator="euler"),
    "roe": dict(flux="roe"),
    "roe_z_rk2": dict(flux="roe", recon="weno5-z", integrator="rk2"),
}

CASES = {
    "1d_blocks_zg": lambda: inputs.random_blocks((37, 1, 1), seed=1),
    "2d_blocks_mixed_ragged": lambda: inputs.random_blocks((40, 33, 1), seed=4, bc=(0, 0, 1, 1, 1, 1)),
    "3d_smooth_visc_ragged": lambda: inputs.random_smooth((19, 13, 11), seed=6, viscous=True, mu=0.01),
}


def with_scheme(case, **kw):
    for k, v in kw.items():
        setattr(case, k, v)
    return case


@pytest.mark.parametrize("scheme", sorted(SCHEMES))
@pytest.mark.parametrize("name", sorted(CASES))
def test_variant_rhs_and_steps_fp64(orc, scheme, name):
    case = with_scheme(CASES[name](), **SCHEMES[scheme])
    c = orc.config(**case.params())
    s = jf.Solver.from_case(case, dtype="f64")
    U = to_dev(case.U, "f64")
    rate = case.cfl / orc.compute_dt(c, case.U)
    got = s.rhs(U).cpu().numpy()
    assert rate_err(got, orc.rhs(c, case.U), case.U, rate) <= 1e-12
    want = case.U.copy()
    used = s.scalar()
    for _ in range(4):
        dt = orc.compute_dt(c, want)
        want = orc.rk3_step(c, want, dt)   # one step of the configured integrator
        s.rk3_step(U, None, used)
        assert used.item() == pytest.approx(dt, rel=1e-13)
    s.sync()
    assert rel_err(U.cpu().numpy(), want) <= 1e-12


@pytest.mark.parametrize("scheme", ["hll_davis_z", "rusanov", "hllc_toro_z", "hllc_z_rk2", "hll_euler", "roe"])
def test_variant_ten_steps_fp32(orc, scheme):
    case = with_scheme(inputs.random_smooth((19, 13, 11), seed=6, viscous=True, mu=0.01), **SCHEMES[scheme])
    c = orc.config(**case.params())
    U32 = case.U.astype(np.float32)
    dt = 0.5 * orc.compute_dt(c, U32.astype(np.float64))
    want, _, _ = orc.run(c, U32.astype(np.float64), 10, dt)
    s = jf.Solver.from_case(case, dtype="f32")
    U = to_dev(U32, "f32")
    dtd = s.scalar(dt)
    for _ in range(10):
        s.rk3_step(U, dtd)
    s.sync()
    assert rel_err(U.cpu().numpy(), want) <= 1e-5


@pytest.mark.parametrize("problem", ["sod", "lax"])
@pytest.mark.parametrize("scheme", ["hll_einfeldt", "hll_toro", "rusanov", "hllc_davis", "hllc_toro_z", "roe"])
def test_shock_tubes_gpu(orc, problem, scheme):
    """Section 5.1.2 at the paper's N = 100: the FP64 GPU run to the end time
    equals the oracle's run, and both follow the exact Riemann solution."""
    if problem == "sod":
        WL, WR, T = inputs.SOD_LEFT, inputs.SOD_RIGHT, 0.2
    else:
        WL, WR, T = inputs.LAX_LEFT, inputs.LAX_RIGHT, inputs.LAX_END_TIME
    case = with_scheme(inputs.riemann_1d(100, WL, WR), **SCHEMES[scheme])
    c = orc.config(**case.params())
    want, t, nsteps = orc.run(c, case.U, 100000, 0.0, T)
    # replay the oracle's step sequence on the GPU: CFL steps, the last one cut to reach T
    s = jf.Solver.from_case(case, dtype="f64")
    U = to_dev(case.U, "f64")
    ref = case.U.copy()
    t_gpu = 0.0
    for k in range(nsteps):
        dt = orc.compute_dt(c, ref)
        if t_gpu + dt > T:
            dt = T - t_gpu
        ref = orc.rk3_step(c, ref, dt)
        s.rk3_step(U, s.scalar(dt))
        t_gpu += dt
    s.sync()
    got = U.cpu().numpy()
    assert t_gpu == pytest.approx(t, rel=1e-14)
    assert rel_err(got, want) <= 1e-12
    ex = orc.exact_sample(WL, WR, inputs.centres(100, 0.0, 1.0), T)
    assert np.mean(np.abs(got[0, 0, 0] - ex[:, 0])) < (6.5e-3 if problem == "sod" else 2.2e-2)


@pytest.mark.parametrize("scheme", ["hll_euler", "hllc_z_rk2", "hll_toro", "roe"])
@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_batch_variant_equals_single_grid(scheme, dtype):
    """The batch form of each integrator and solver (stage codes and the
    Euler copy) is bitwise the single-grid path, with its own dt."""
    cases = [with_scheme(c, **SCHEMES[scheme]) for c in inputs.four_quadrant_batch(nsim=4, sides=(32, 48), seed=7)]
    grids = [jf.make_grid(c.n, c.lo, c.hi, c.bc) for c in cases]
    p = cases[0].params()
    b = jf.Batch(grids, dtype=dtype, **{k: p[k] for k in ("gamma", "R", "mu", "Pr", "eps", "cfl", "viscous", "heat",
                                                           "flux", "recon", "speeds", "integrator")})
    t = torch.float32 if dtype == "f32" else torch.float64
    Us = [torch.tensor(c.U, dtype=t, device="cuda") for c in cases]
    dts = b.step(Us, 5)
    b.sync()
    for i, c in enumerate(cases):
        s = jf.Solver.from_case(c, dtype=dtype)
        U = torch.tensor(c.U, dtype=t, device="cuda")
        used = s.scalar()
        for _ in range(5):
            s.rk3_step(U, None, used)
        s.sync()
        assert torch.equal(U, Us[i]), f"simulation {i} differs"
        assert dts[i].item() == used.item()


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_roe_launch_variants_agree(dtype):
    """Every compiled tile shape of the ROE kernels computes the same bits."""
    case = with_scheme(inputs.random_smooth((19, 13, 11), seed=6, viscous=True, mu=0.01), flux="roe")
    s = jf.Solver.from_case(case, dtype=dtype)
    U0 = to_dev(case.U, dtype)
    ref = None
    for v in range(len(s.variants())):
        s.set_variant(v)
        out = s.rhs(U0)
        s.sync()
        if ref is None:
            ref = out
        else:
            assert torch.equal(out, ref), s.variants()[v]


def test_adjoint_rejects_variant_schemes():
    case = with_scheme(inputs.random_smooth((12, 10, 1), seed=1), flux="hll")
    s = jf.Solver.from_case(case, dtype="f64")
    U = to_dev(case.U, "f64")
    with pytest.raises(jf.JFError) as e:
        s.rk3_step_vjp(U, s.scalar(1e-3), torch.ones_like(U))
    assert e.value.status == jf.JF_ERR_UNSUPPORTED
