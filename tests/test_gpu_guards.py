"""Out-of-bounds write detection without a sanitizer: every buffer an entry
point writes sits inside a larger allocation whose margins hold a NaN canary
bit pattern; after the call the margins must be bit-for-bit unchanged and the
written region finite.  Grids are small and ragged for every tile shape."""
import numpy as np
import pytest

from paper_2203_13760_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2203_13760_gb300 import jf  # noqa: E402

GUARD = 4096  # elements on each side (a multiple of 4: the view stays 16-byte aligned)
CANARY = {torch.float32: 0x7FC0DEAD, torch.float64: 0x7FF8DEADBEEFDEAD}


class Guarded:
    """A tensor of `shape` inside a canary-filled allocation."""

    def __init__(self, shape, dtype, init=None):
        n = int(np.prod(shape))
        itype = torch.int32 if dtype == torch.float32 else torch.int64
        self.raw = torch.full((n + 2 * GUARD,), CANARY[dtype], dtype=itype, device="cuda").view(dtype)
        self.t = self.raw[GUARD:GUARD + n].view(shape)
        if init is not None:
            self.t.copy_(init)
        self.itype = itype

    def check(self):
        torch.cuda.synchronize()
        bits = self.raw.view(self.itype)
        c = CANARY[self.raw.dtype]
        assert torch.all(bits[:GUARD] == c).item(), "write below the buffer"
        assert torch.all(bits[-GUARD:] == c).item(), "write above the buffer"
        assert torch.isfinite(self.t).all().item(), "part of the buffer not written / not finite"


CASES = {
    "1d": lambda: inputs.random_blocks((37, 1, 1), seed=1),
    "2d_visc": lambda: inputs.random_smooth((37, 19, 1), seed=3, viscous=True, mu=0.01),
    "3d_visc": lambda: inputs.random_smooth((19, 13, 11), seed=6, viscous=True, mu=0.01),
    "3d_blocks": lambda: inputs.random_blocks((21, 17, 9), seed=7, bc=(0, 0, 1, 1, 0, 0)),
}


@pytest.mark.parametrize("flux", ["hllc", "hll", "roe"])
@pytest.mark.parametrize("dtype", ["f32", "f64"])
@pytest.mark.parametrize("name", sorted(CASES))
def test_single_grid_entry_points_stay_in_bounds(name, dtype, flux):
    case = CASES[name]()
    case.flux = flux
    s = jf.Solver.from_case(case, dtype=dtype)
    t = s.dtype
    U0 = torch.tensor(case.U, dtype=t, device="cuda")
    shape = tuple(U0.shape)
    # right-hand side
    out = Guarded(shape, t)
    s.rhs(U0, out.t)
    out.check()
    # RK3 steps in place (fixed small dt: this test is about bounds, not
    # stability), graph run
    U = Guarded(shape, t, U0)
    dt_small = s.scalar(1e-5)
    s.rk3_step(U.t, dt_small)
    s.run(U.t, 3, dt_small)
    U.check()
    # one stage into a separate output
    U1 = Guarded(shape, t)
    s.stage(U0, None, U1.t, 0.0, 1.0, s.scalar(1e-4))
    U1.check()
    # CFL step into a guarded scalar
    dt = Guarded((1,), torch.float64)
    s.compute_dt(U0, dt.t)
    dt.check()
    s.sync()


@pytest.mark.parametrize("dtype", ["f32", "f64"])
@pytest.mark.parametrize("name", ["1d", "2d_visc", "3d_visc"])
def test_adjoint_stays_in_bounds(name, dtype):
    case = CASES[name]()
    s = jf.Solver.from_case(case, dtype=dtype)
    t = s.dtype
    U0 = torch.tensor(case.U, dtype=t, device="cuda")
    lam_out = torch.ones_like(U0)
    lam_in = Guarded(tuple(U0.shape), t)
    dt = 0.5 * s.compute_dt(U0).item()
    s.rk3_step_vjp(U0, s.scalar(dt), lam_out, lam_in.t)
    lam_in.check()
    s.sync()


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_batch_and_trajectories_stay_in_bounds(dtype):
    cases = inputs.four_quadrant_batch(nsim=3, sides=(32, 48, 40), seed=11)
    grids = [jf.make_grid(c.n, c.lo, c.hi, c.bc) for c in cases]
    b = jf.Batch(grids, dtype=dtype)
    t = torch.float32 if dtype == "f32" else torch.float64
    Us = [Guarded(c.U.shape, t, torch.tensor(c.U, dtype=t, device="cuda")) for c in cases]
    dts = Guarded((len(cases),), torch.float64)
    b.step([g.t for g in Us], 4, dts.t)
    for g in Us:
        g.check()
    dts.check()
    trajs = [Guarded((4,) + c.U.shape, t) for c in cases]
    dt_dev = torch.tensor([1e-4] * len(cases), dtype=torch.float64, device="cuda")
    u0 = (jf.ctypes.c_void_p * len(cases))(*[g.t.data_ptr() for g in Us])
    tp = (jf.ctypes.c_void_p * len(cases))(*[g.t.data_ptr() for g in trajs])
    assert jf.lib().jf_batch_feed_forward(b.h, u0, tp, 3, jf._ptr(dt_dev), jf._stream()) == jf.JF_OK
    for g in trajs:
        g.check()
    b.sync()


def test_density_loss_stays_in_bounds():
    case = inputs.kelvin_helmholtz(24, seed=1)
    s = jf.Solver.from_case(case, dtype="f64")
    U = torch.tensor(case.U, dtype=torch.float64, device="cuda")
    target = torch.tensor(case.U[0], dtype=torch.float64, device="cuda").contiguous() * 1.01
    seed = Guarded(tuple(U.shape), torch.float64)
    loss = Guarded((1,), torch.float64)
    s.loss_density_l2(U, target, loss.t, seed.t)
    seed.check()
    loss.check()
    s.sync()


def test_roe_blow_up_is_reported_like_the_oracle(orc):
    """The ROE setup (no entropy fix or positivity limiter: the paper names
    none) loses positivity on the random-block field at CFL 0.5 in the oracle;
    the GPU run of the same step reports it through the device flag."""
    case = CASES["3d_blocks"]()
    case.flux = "roe"
    c = orc.config(**case.params())
    want = orc.rk3_step(c, case.U, orc.compute_dt(c, case.U))
    assert not np.isfinite(want).all()
    s = jf.Solver.from_case(case, dtype="f64")
    U = torch.tensor(case.U, dtype=torch.float64, device="cuda")
    s.rk3_step(U)
    with pytest.raises(jf.JFError) as e:
        s.sync()
    assert e.value.status == jf.JF_ERR_NONPHYSICAL


@pytest.mark.parametrize("dtype", ["f32", "f64"])
@pytest.mark.parametrize("n", [(37, 1, 1), (37, 19, 1), (13, 11, 9)])
def test_per_face_adjoint_stays_in_bounds(dtype, n):
    """The per-face adjoint (walls, WENO3-JS, Rusanov-NN, TVD-RK2) with its
    parameter gradient: lam_in and theta_bar inside canary margins."""
    W = inputs.WALL
    case = inputs.random_smooth(n, seed=3, bc=(W, W, W, 1, W, W))
    case.flux, case.recon, case.integrator = "rusanov-nn", "weno3-js", "rk2"
    t = torch.float32 if dtype == "f32" else torch.float64
    theta = torch.tensor(inputs.nn_params(seed=5), dtype=t, device="cuda")
    s = jf.Solver.from_case(case, dtype=dtype, nn=theta)
    U0 = torch.tensor(case.U, dtype=t, device="cuda")
    lam_in = Guarded(tuple(U0.shape), t)
    tb = Guarded((jf.NN_PARAMS,), t, torch.zeros(jf.NN_PARAMS, dtype=t, device="cuda"))
    s.rk3_step_vjp_params(U0, s.scalar(1e-4), torch.ones_like(U0), lam_in.t, tb.t)
    lam_in.check()
    tb.check()
    s.sync()


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_batch_adjoint_stays_in_bounds(dtype):
    """jf_batch_step_vjp over an uneven walled batch with the Rusanov-NN flux:
    every lam_in and theta_bar inside canary margins."""
    W = inputs.WALL
    cases = inputs.four_quadrant_batch(nsim=3, sides=(32, 48, 40), seed=11)
    for c in cases:
        c.bc = (W, W, W, 1, 1, 1)
    t = torch.float32 if dtype == "f32" else torch.float64
    theta = torch.tensor(inputs.nn_params(seed=5), dtype=t, device="cuda")
    b = jf.Batch([jf.make_grid(c.n, c.lo, c.hi, c.bc) for c in cases], dtype=dtype, flux="rusanov-nn",
                 recon="weno3-js", integrator="rk2", nn=theta)
    Us = [torch.tensor(c.U, dtype=t, device="cuda") for c in cases]
    lams = [torch.ones_like(U) for U in Us]
    outs = [Guarded(tuple(U.shape), t) for U in Us]
    tb = Guarded((jf.NN_PARAMS,), t, torch.zeros(jf.NN_PARAMS, dtype=t, device="cuda"))
    dt = torch.full((3,), 1e-4, dtype=torch.float64, device="cuda")
    b.step_vjp(Us, dt, lams, [g.t for g in outs], lams, tb.t)
    for g in outs:
        g.check()
    tb.check()
    b.sync()
