"""FP32 parity on shocked data and at a benchmark size, and the safe
reconstruction fallback, against the oracle.

* The four-quadrant batch (64 Riemann problems, sides {64, 128, 256, 512})
  through the persistent FP32 batch kernel, 10 CFL steps: each simulation
  against the FP64 oracle started from the same FP32-rounded state and fed the
  GPU's per-simulation dt (the GPU's dt itself is checked against the
  oracle's CFL step).  Relative L-infinity per conserved quantity <= 1e-5 over
  the whole field: no cell needs an allowance at the discontinuities.
* FP32 Sod (200 cells, t = 0.2, the oracle's dt sequence) and Lax (100 cells,
  t = 0.14) shock tubes against the oracle (<= 1e-5) and Sod against the exact
  Riemann solution.
* Taylor-Green 128^3 FP32 Navier-Stokes, 10 fixed-dt steps, the whole field
  against the oracle (<= 1e-5).
* is_safe_reconstruction (Appendix A; a face side whose reconstructed density
  or pressure is not positive takes its cell value) in FP64 against the
  oracle (<= 1e-12), with near-vacuum gaps along x, y and z.
"""
import numpy as np
import pytest

from paper_2203_13760_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2203_13760_gb300 import jf  # noqa: E402

GROUPS = ((0,), (1, 2, 3), (4,))
FP32_BAR = 1e-5


def cell_err(a, b):
    """Per-cell relative error: max over the conserved quantities of
    |a - b| / ||b_q||_inf (mass, momentum vector, energy)."""
    a = np.asarray(a, dtype=np.float64).reshape(5, -1)
    b = np.asarray(b, dtype=np.float64).reshape(5, -1)
    e = np.zeros(a.shape[1])
    for g in GROUPS:
        g = list(g)
        e = np.maximum(e, np.abs(a[g] - b[g]).max(axis=0) / np.abs(b[g]).max())
    return e


def rate_err(got, want, U, rate):
    got = np.asarray(got, dtype=np.float64).reshape(5, -1)
    want = np.asarray(want, dtype=np.float64).reshape(5, -1)
    U = np.asarray(U, dtype=np.float64).reshape(5, -1)
    worst = 0.0
    for g in GROUPS:
        g = list(g)
        scale = max(np.abs(want[g]).max(), np.abs(U[g]).max() * rate, 1e-300)
        worst = max(worst, np.abs(got[g] - want[g]).max() / scale)
    return worst


def f32_dev(U):
    return torch.tensor(np.ascontiguousarray(U, dtype=np.float32), device="cuda")


def test_four_quadrant_batch_fp32_persistent_vs_oracle(orc):
    cases = inputs.four_quadrant_batch()
    assert len(cases) == 64 and {c.n[0] for c in cases} <= {64, 128, 256, 512}
    grids = [jf.make_grid(c.n, c.lo, c.hi, c.bc) for c in cases]
    b = jf.Batch(grids, dtype="f32")
    assert "persistent" in b.variants()[0]
    Us = [f32_dev(c.U) for c in cases]
    nsteps = 10
    dts = []
    for _ in range(nsteps):
        dts.append(b.step(Us, 1).cpu().numpy().copy())
    b.sync()
    for i, c in enumerate(cases):
        oc = orc.config(**c.params())
        W = c.U.astype(np.float32).astype(np.float64)
        for k in range(nsteps):
            # FP32 rates, FP64 reduction: the CFL step to FP32 rounding
            assert dts[k][i] == pytest.approx(orc.compute_dt(oc, W), rel=1e-6)
            W = orc.rk3_step(oc, W, float(dts[k][i]))
        e = cell_err(Us[i].cpu().numpy(), W)
        assert e.max() <= FP32_BAR, (i, c.n, e.max(), int((e > FP32_BAR).sum()))
    b.close()


def _tube_dts(orc, case, t_end):
    """The oracle's CFL step sequence to t_end (last step clipped) and its
    final state, from the FP32-rounded initial state."""
    oc = orc.config(**case.params())
    W = case.U.astype(np.float32).astype(np.float64)
    t, seq, states = 0.0, [], [W]
    while t < t_end - 1e-15:
        dt = min(orc.compute_dt(oc, W), t_end - t)
        W = orc.rk3_step(oc, W, dt)
        seq.append(dt)
        states.append(W)
        t += dt
    return seq, states


@pytest.mark.parametrize("tube", ["sod", "lax"])
def test_shock_tubes_fp32_vs_oracle(orc, tube):
    case = inputs.sod(200) if tube == "sod" else inputs.lax(100)
    t_end = 0.2 if tube == "sod" else inputs.LAX_END_TIME
    seq, states = _tube_dts(orc, case, t_end)
    s = jf.Solver.from_case(case, dtype="f32")
    U = f32_dev(case.U)
    for k, dt in enumerate(seq):
        s.rk3_step(U, s.scalar(dt))
        if k + 1 == 10:
            assert cell_err(U.cpu().numpy(), states[10]).max() <= FP32_BAR
    s.sync()
    e = cell_err(U.cpu().numpy(), states[-1])
    assert e.max() <= FP32_BAR, (len(seq), e.max())
    if tube == "sod":
        x = inputs.centres(200, 0, 1)
        ex = orc.exact_sample([1, 0, 1], [0.125, 0, 0.1], x, 0.2)
        assert np.mean(np.abs(U[0, 0, 0].cpu().numpy() - ex[:, 0])) < 3e-3


def test_taylor_green_128_fp32_ten_steps_whole_field(orc):
    """The benchmark flow at 128^3 (Navier-Stokes, Ma = 0.1, Re = 1600):
    every cell after 10 steps."""
    case = inputs.taylor_green(128)
    oc = orc.config(**case.params())
    U32 = case.U.astype(np.float32)
    dt = orc.compute_dt(oc, U32.astype(np.float64))
    want, _, _ = orc.run(oc, U32.astype(np.float64), 10, dt)
    s = jf.Solver.from_case(case, dtype="f32")
    U = torch.from_numpy(U32).cuda()
    d = s.scalar(dt)
    for _ in range(10):
        s.rk3_step(U, d)
    s.sync()
    assert cell_err(U.cpu().numpy(), want).max() <= FP32_BAR


# --- safe reconstruction, FP64 -------------------------------------------------

# the 26-cell gap row of tests/test_oracle_pins.py: a pressure gap (cells 3..7)
# and a density gap (cells 15..19) where WENO5-JS reconstructs non-positive
# states, with colliding velocities at the gaps
P_GAP = [1.0, 1.0, 1.0, 1e-2, 1e-5, 1e-8, 3e-8, 1e-8] + [1.0] * 18
RHO_GAP = ([1.0, 1.0, 0.9, 0.8, 0.7, 0.6, 0.65, 0.7, 1.2, 1.2, 1.1, 1.0, 1.0, 1.0, 1.0]
           + [1e-2, 1e-5, 1e-8, 3e-8, 1e-8] + [1.0] * 6)
U_GAP = [0.05] * 26
U_GAP[5], U_GAP[6], U_GAP[17], U_GAP[18] = 0.2, -0.2, 0.2, -0.2


def gap_case(axis, dims, n_other):
    """The gap row along `axis` (0, 1, 2) of a `dims`-dimensional grid,
    repeated over the other active axes (n_other cells each) with a mild
    velocity across the row that varies along those axes; zero-gradient along
    the row, periodic across."""
    n = [1, 1, 1]
    n[axis] = 26
    for a in range(dims):
        if a != axis:
            n[a] = n_other
    shape = (n[2], n[1], n[0])
    row = [1, 1, 1]
    row[2 - axis] = 26

    def along(v):
        return np.broadcast_to(np.asarray(v, dtype=np.float64).reshape(row), shape)

    rho, p, un = along(RHO_GAP), along(P_GAP), along(U_GAP)
    vel = [np.zeros(shape), np.zeros(shape), np.zeros(shape)]
    vel[axis] = un
    Z, Y, X = np.meshgrid(*(np.arange(k, dtype=np.float64) for k in shape), indexing="ij")
    coord = [X, Y, Z]
    for a in range(dims):
        if a != axis:  # periodic variation across the row
            vel[a] = 0.1 * np.sin(2 * np.pi * (coord[a] + 0.5) / n[a])
    U = inputs.conservative(rho, vel[0], vel[1], vel[2], p, 1.4)
    bc = [0, 0, 0, 0, 0, 0]
    bc[2 * axis] = bc[2 * axis + 1] = 1
    hi = tuple(float(k) for k in n)
    return inputs.Case(f"gap{axis}", tuple(n), (0.0, 0.0, 0.0), hi, tuple(bc), U.reshape(5, *shape))


@pytest.mark.parametrize("axis,dims,n_other", [(0, 1, 1), (0, 2, 13), (1, 2, 19), (2, 3, 11), (0, 3, 9)])
def test_safe_reconstruction_fp64_vs_oracle(orc, axis, dims, n_other):
    case = gap_case(axis, dims, n_other)
    c = orc.config(**case.params(), safe=True)
    s = jf.Solver.from_case(case, dtype="f64", safe=True)
    U = torch.tensor(case.U, dtype=torch.float64, device="cuda")
    want = orc.rhs(c, case.U)
    assert np.all(np.isfinite(want))
    got = s.rhs(U).cpu().numpy()
    # the right-hand side is a difference of face fluxes whose rounding floor
    # scales with the fastest wave (c ~ 1e4 in the density gap): compare it
    # relative to max(|L_q|, |U_q| a / h), a / h = CFL / dt, as the other
    # right-hand-side parity tests do
    rate = case.cfl / orc.compute_dt(c, case.U)
    assert rate_err(got, want, case.U, rate) <= 1e-12
    # three CFL steps
    W = case.U.copy()
    used = s.scalar()
    for _ in range(3):
        dt = orc.compute_dt(c, W)
        W = orc.rk3_step(c, W, dt)
        s.rk3_step(U, None, used)
        assert used.item() == pytest.approx(dt, rel=1e-13)
    s.sync()
    assert cell_err(U.cpu().numpy(), W).max() <= 1e-12
