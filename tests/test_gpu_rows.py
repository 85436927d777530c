"""Row tiles of 2D grids (the DIM_Y2 kernels: one row of BX cells per CTA,
marching along y over a chunk of rows with the six-slot ring of the 3D
kernel; selected with set_variant, described "ymarch").  Against the oracle
at the FP64 bar (one right-hand side, ten CFL steps) on ragged grids with
periodic, zero-gradient and mixed boundaries and several chunk lengths, at
the FP32 bar after ten steps, and through the batch (persistent FP32 kernel,
per-simulation FP64 launches)."""
import numpy as np
import pytest

from paper_2203_13760_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2203_13760_gb300 import jf  # noqa: E402

GROUPS = ((0,), (1, 2, 3), (4,))


def rel_err(a, b):
    a = np.asarray(a, dtype=np.float64).reshape(5, -1)
    b = np.asarray(b, dtype=np.float64).reshape(5, -1)
    return max(np.abs(a[list(g)] - b[list(g)]).max() / max(np.abs(b[list(g)]).max(), 1e-300) for g in GROUPS)


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


def dev(U, dtype):
    return torch.tensor(np.ascontiguousarray(U), dtype=torch.float32 if dtype == "f32" else torch.float64,
                        device="cuda")


def row_variants(obj, chunk=None):
    """Indices of the row-tile variants of a Solver or Batch (chunk: the
    z chunk text of a Solver variant, e.g. "auto" or "8")."""
    out = []
    for v, d in enumerate(obj.variants()):
        if "ymarch" not in d:
            continue
        if chunk is not None and f"zchunk={chunk}" not in d and not (chunk == "auto" and "zchunk=auto" in d):
            continue
        out.append(v)
    return out


CASES = {
    "smooth_visc_ragged": lambda: inputs.random_smooth((37, 19, 1), seed=3, viscous=True, mu=0.01),
    "blocks_zg_ragged": lambda: inputs.random_blocks((40, 33, 1), seed=4),
    "mixed_bc_x_periodic": lambda: inputs.random_smooth((33, 24, 1), seed=5, bc=(0, 0, 1, 1, 1, 1), viscous=True,
                                                         mu=0.01),
    "mixed_bc_y_periodic_wide": lambda: inputs.random_smooth((150, 41, 1), seed=8, bc=(1, 1, 0, 0, 1, 1),
                                                              viscous=True, mu=0.01),
    "blocks_periodic_wide": lambda: inputs.random_blocks((260, 23, 1), seed=9, bc=(0, 0, 0, 0, 1, 1)),
}


@pytest.mark.parametrize("chunk", ["auto", "8"])
@pytest.mark.parametrize("name", sorted(CASES))
def test_rows_fp64_vs_oracle(orc, name, chunk):
    case = CASES[name]()
    c = orc.config(**case.params())
    want_rhs = orc.rhs(c, case.U)
    rate = case.cfl / orc.compute_dt(c, case.U)
    s = jf.Solver.from_case(case, dtype="f64")
    vs = row_variants(s, chunk)
    assert vs, s.variants()
    s.set_variant(vs[0])
    got = s.rhs(dev(case.U, "f64")).cpu().numpy()
    assert rate_err(got, want_rhs, case.U, rate) <= 1e-12
    U = dev(case.U, "f64")
    dt_used = s.scalar()
    want = case.U.copy()
    for _ in range(10):
        dt_ref = orc.compute_dt(c, want)
        want = orc.rk3_step(c, want, dt_ref)
        s.rk3_step(U, None, dt_used)
        assert dt_used.item() == pytest.approx(dt_ref, rel=1e-13)
    s.sync()
    assert rel_err(U.cpu().numpy(), want) <= 1e-12


@pytest.mark.parametrize("scheme", [dict(flux="hll", recon="weno5-z"), dict(speeds="davis"),
                                    dict(flux="rusanov", speeds="toro")])
@pytest.mark.parametrize("name", ["blocks_zg_ragged", "mixed_bc_y_periodic_wide"])
def test_rows_run_time_schemes_fp64_vs_oracle(orc, name, scheme):
    """The row tiles of the run-time Godunov schemes (Table 2 variants):
    right-hand side and four CFL steps against the oracle at 1e-12."""
    case = CASES[name]()
    for k, v in scheme.items():
        setattr(case, k, v)
    c = orc.config(**case.params())
    s = jf.Solver.from_case(case, dtype="f64")
    vs = row_variants(s, "8")
    assert vs, s.variants()
    s.set_variant(vs[0])
    rate = case.cfl / orc.compute_dt(c, case.U)
    got = s.rhs(dev(case.U, "f64")).cpu().numpy()
    assert rate_err(got, orc.rhs(c, case.U), case.U, rate) <= 1e-12
    U = dev(case.U, "f64")
    dt_used = s.scalar()
    want = case.U.copy()
    for _ in range(4):
        want = orc.rk3_step(c, want, orc.compute_dt(c, want))
        s.rk3_step(U, None, dt_used)
    s.sync()
    assert rel_err(U.cpu().numpy(), want) <= 1e-12


@pytest.mark.parametrize("name", ["smooth_visc_ragged", "mixed_bc_y_periodic_wide", "kh64"])
def test_rows_fp32_ten_steps_vs_oracle(orc, name):
    """Every FP32 row width (auto chunk and 8 rows) within 1e-5 of the oracle
    after ten CFL steps, each side with its own dt, on smooth flows."""
    case = inputs.kelvin_helmholtz(64) if name == "kh64" else CASES[name]()
    c = orc.config(**case.params())
    W = case.U.astype(np.float32).astype(np.float64)
    want = W.copy()
    for _ in range(10):
        want = orc.rk3_step(c, want, orc.compute_dt(c, want))
    s = jf.Solver.from_case(case, dtype="f32")
    vs = row_variants(s, "auto") + row_variants(s, "8")
    assert len(vs) >= 6, s.variants()
    for v in vs:
        s.set_variant(v)
        U = dev(case.U, "f32")
        s.run(U, 10)
        s.sync()
        assert rel_err(U.double().cpu().numpy(), want) <= 1e-5, s.variants()[v]


def test_rows_repeat_is_bitwise():
    case = inputs.kelvin_helmholtz(64)
    s = jf.Solver.from_case(case, dtype="f32")
    s.set_variant(row_variants(s, "8")[0])
    U0 = dev(case.U, "f32")
    a = s.rhs(U0).clone()
    b = s.rhs(U0).clone()
    s.sync()
    assert torch.equal(a, b)


def _batch(cases, dtype):
    grids = [jf.make_grid(c.n, c.lo, c.hi, c.bc) for c in cases]
    return jf.Batch(grids, dtype=dtype)


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_rows_batch_vs_oracle(orc, dtype):
    """Four-quadrant problems of uneven and ragged sizes (several column
    tiles and row chunks each) through the row-tile batch variant: ten CFL
    steps against the oracle per simulation (FP64: 1e-12; FP32: the batch's
    shocked-data bar, 1e-5 per cell relative to the quantity's maximum)."""
    cases = inputs.four_quadrant_batch(nsim=5, sides=(48, 64, 100, 130, 200), seed=11)
    b = _batch(cases, dtype)
    vs = row_variants(b)
    assert vs and "persistent" in b.variants()[vs[0]], b.variants()
    b.set_variant(vs[0])
    Us = [dev(c.U, dtype) for c in cases]
    dts = [b.step(Us, 1).cpu().numpy().copy() for _ in range(10)]
    b.sync()
    for i, c in enumerate(cases):
        oc = orc.config(**c.params())
        W = c.U if dtype == "f64" else c.U.astype(np.float32).astype(np.float64)
        for k in range(10):
            W = orc.rk3_step(oc, W, float(dts[k][i]))
        tol = 1e-12 if dtype == "f64" else 1e-5
        assert rel_err(Us[i].double().cpu().numpy(), W) <= tol, (i, c.n)
    b.close()


def test_rows_batch_close_to_tiles():
    """The row-tile and 32 x 7 batch variants agree to FP32 rounding after
    three steps (separate instantiations: not bitwise)."""
    cases = inputs.four_quadrant_batch(nsim=3, sides=(64,), seed=4)
    b = _batch(cases, "f32")
    ref = [dev(c.U, "f32") for c in cases]
    b.step(ref, 3)
    b.set_variant(row_variants(b)[0])
    U = [dev(c.U, "f32") for c in cases]
    b.step(U, 3)
    b.sync()
    for x, y in zip(ref, U):
        assert rel_err(y.double().cpu().numpy(), x.double().cpu().numpy()) <= 1e-5
    b.close()


@pytest.mark.parametrize("n,rows,dtype", [((2048, 350, 1), True, "f32"), ((1024, 1024, 1), True, "f32"),
                                          ((2048, 300, 1), False, "f32"), ((512, 512, 1), False, "f32"),
                                          ((64, 64, 1), False, "f32"), ((1024, 1024, 1), True, "f64"),
                                          ((512, 512, 1), False, "f64")])
def test_2d_default_tiles(n, rows, dtype):
    """FP32 2D handles default to the row tiles (automatic chunk) when the
    rows padded to whole tiles cover at most 8 % more cells than 32 x 7
    tiles do and there are at least 12 rows of row tiles per resident CTA
    (152 SMs x 3 CTAs: 2048 x 350 has 16 x 350 = 5600 >= 5472, 1024^2 8192),
    else to the 32 x 7 tiles (2048 x 300: 4800 row tiles; 512^2: 2048;
    64 x 64: 8192 padded cells against 4480).  FP64 (row tiles at 2 CTAs
    per SM, 32 x 8 tiles): 1024^2 has 26.9 rows per resident CTA, 512^2 6.7.
    The default launch is bitwise the launch of that variant."""
    case = inputs.random_smooth(n, seed=21, viscous=True, mu=0.01)
    s = jf.Solver.from_case(case, dtype=dtype)
    U0 = dev(case.U, dtype)
    dflt = s.rhs(U0).clone()
    want = row_variants(s, "auto")[0] if rows else 0
    s.set_variant(want)
    tile = "tile=32x7" if dtype == "f32" else "tile=32x8"
    assert "ymarch" in s.variants()[want] if rows else tile in s.variants()[want]
    got = s.rhs(U0)
    s.sync()
    assert torch.equal(dflt, got)


def test_batch_default_is_rows_for_the_four_quadrant_batch():
    """The 64 four-quadrant problems (about 106 rows of row tiles per
    resident CTA) default to the row tiles with 32 rows per work item."""
    cases = inputs.four_quadrant_batch(nsim=64)
    b = _batch(cases, "f32")
    Us = [dev(c.U, "f32") for c in cases]
    b.step(Us, 2)
    v = row_variants(b)[0]
    assert "tile=128x1 ymarch rows=32 persistent" == b.variants()[v]
    b.set_variant(v)
    Vs = [dev(c.U, "f32") for c in cases]
    b.step(Vs, 2)
    b.sync()
    for x, y in zip(Us, Vs):
        assert torch.equal(x, y)
    b.close()
