"""Batched simulations (jf_batch_create / jf_batch_step): every simulation of
the batch equals the same simulation advanced alone through the single-grid
path (same tile code, same arithmetic: bitwise in FP32 and FP64), and the FP64
batch matches the oracle per simulation."""
import numpy as np
import pytest

from paper_2203_13760_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2203_13760_gb300 import jf  # noqa: E402


def rel_err(a, b):
    a = np.asarray(a, dtype=np.float64).reshape(5, -1)
    b = np.asarray(b, dtype=np.float64).reshape(5, -1)
    return max(np.abs(a[g] - b[g]).max() / np.abs(b[g]).max() for g in ([0], [1, 2, 3], [4]))


def batch_of(cases, dtype, **kw):
    grids = [jf.make_grid(c.n, c.lo, c.hi, c.bc) for c in cases]
    p = cases[0].params()
    return jf.Batch(grids, gamma=p["gamma"], R=p["R"], mu=p["mu"], Pr=p["Pr"], dtype=dtype, eps=p["eps"],
                    cfl=p["cfl"], viscous=p["viscous"], heat=p["heat"], **kw)


def fields(cases, dtype):
    t = torch.float32 if dtype == "f32" else torch.float64
    return [torch.tensor(c.U, dtype=t, device="cuda") for c in cases]


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_batch_equals_single_grid_path(dtype):
    """Four-quadrant problems of uneven (and ragged) sizes: after 12 CFL steps
    each simulation is bitwise the single-grid result, with its own dt."""
    cases = inputs.four_quadrant_batch(nsim=7, sides=(32, 48, 64, 80), seed=5)
    b = batch_of(cases, dtype)
    Us = fields(cases, dtype)
    dt = b.step(Us, 12)
    b.sync()
    for i, c in enumerate(cases):
        s = jf.Solver.from_case(c, dtype=dtype)
        U = fields([c], dtype)[0]
        used = s.scalar()
        for _ in range(12):
            s.rk3_step(U, None, used)
        s.sync()
        assert torch.equal(U, Us[i]), f"simulation {i} ({c.n}) differs"
        assert dt[i].item() == used.item()


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_batch_ragged_cell_counts(dtype):
    """Cell counts that are and are not multiples of the 16-byte vector
    (37 x 19 = 703, 40 x 33 = 1320, 129 x 130, 31 x 64): the batch CFL reads
    the first with scalar loads and the others in vectors within one launch;
    dt and the states stay bitwise those of the single-grid path."""
    cases = [inputs.random_blocks((37, 19, 1), seed=1), inputs.random_blocks((40, 33, 1), seed=2),
             inputs.random_blocks((129, 130, 1), seed=3), inputs.random_blocks((31, 64, 1), seed=4)]
    b = batch_of(cases, dtype)
    Us = fields(cases, dtype)
    dt = b.step(Us, 5)
    b.sync()
    for i, c in enumerate(cases):
        s = jf.Solver.from_case(c, dtype=dtype)
        U = fields([c], dtype)[0]
        used = s.scalar()
        for _ in range(5):
            s.rk3_step(U, None, used)
        s.sync()
        assert dt[i].item() == used.item(), i
        assert torch.equal(U, Us[i]), i


def test_batch_fp64_matches_oracle(orc):
    cases = inputs.four_quadrant_batch(nsim=4, sides=(24, 40), seed=9)
    b = batch_of(cases, "f64")
    Us = fields(cases, "f64")
    b.step(Us, 3)
    b.sync()
    for c, U in zip(cases, Us):
        oc = orc.config(**c.params())
        want = c.U.copy()
        for _ in range(3):
            want = orc.rk3_step(oc, want, orc.compute_dt(oc, want))
        assert rel_err(U.cpu().numpy(), want) <= 1e-12


def test_batch_graph_replay_and_rebinding():
    """The captured graph is replayed; new field tensors are rebound."""
    cases = inputs.four_quadrant_batch(nsim=5, sides=(32, 64), seed=2)
    b = batch_of(cases, "f32")
    A = fields(cases, "f32")
    B = fields(cases, "f32")
    b.step(A, 4)
    b.step(A, 4)      # replay: A advanced 8 steps
    b.step(B, 8)      # rebinding to B, new graph for 8 steps
    b.sync()
    for a, bb in zip(A, B):
        assert torch.equal(a, bb)


def test_batch_1d_and_viscous():
    cases = [inputs.random_blocks((n, 1, 1), seed=n) for n in (40, 64, 129)]
    b = batch_of(cases, "f32")
    Us = fields(cases, "f32")
    b.step(Us, 6)
    b.sync()
    for c, U in zip(cases, Us):
        s = jf.Solver.from_case(c, dtype="f32")
        V = fields([c], "f32")[0]
        s.run(V, 6)
        s.sync()
        assert torch.equal(U, V)
    visc = [inputs.kelvin_helmholtz(n, seed=n) for n in (32, 48)]
    b = batch_of(visc, "f64")
    Us = fields(visc, "f64")
    b.step(Us, 3)
    b.sync()
    for c, U in zip(visc, Us):
        s = jf.Solver.from_case(c, dtype="f64")
        V = fields([c], "f64")[0]
        s.run(V, 3)
        s.sync()
        assert torch.equal(U, V)


def test_batch_variants_agree():
    """The 2D tile shapes compute the same bits (one expression per face,
    compiled per tile shape); the row tiles (ymarch, their own kernel
    instantiations) agree to FP32 rounding (test_gpu_rows.py)."""
    cases = inputs.four_quadrant_batch(nsim=3, sides=(64,), seed=4)
    b = batch_of(cases, "f32")
    ref = fields(cases, "f32")
    b.step(ref, 3)
    names = b.variants()
    for v in range(len(names)):
        b.set_variant(v)
        U = fields(cases, "f32")
        b.step(U, 3)
        b.sync()
        for x, y in zip(ref, U):
            if "ymarch" in names[v]:
                assert rel_err(y.cpu().numpy(), x.cpu().numpy()) <= 1e-5, names[v]
            else:
                assert torch.equal(x, y), names[v]


def test_batch_rejects_mixed_dimensions():
    grids = [jf.make_grid((32, 32, 1)), jf.make_grid((32, 1, 1))]
    with pytest.raises(jf.JFError):
        jf.Batch(grids)


def test_autotuner_picks_and_caches(tmp_path):
    """The autotuner times every variant, selects the fastest, caches it,
    and a new handle of the same configuration picks it from the cache."""
    from paper_2203_13760_gb300 import autotune
    cases = inputs.four_quadrant_batch(nsim=4, sides=(64, 128), seed=3)
    b = batch_of(cases, "f32")
    Us = fields(cases, "f32")
    path = str(tmp_path / "tune.json")
    rec = autotune.tune(b, Us, steps=2, reps=2, path=path)
    assert set(rec["ms"]) == set(b.variants())
    b2 = batch_of(cases, "f32")
    assert autotune.apply(b2, path=path) == rec["variant"]
    # the tuned batch still computes the same bits as the single-grid path
    # with the same tiles (row tiles: the same row width and chunk)
    import re
    tuned = b2.variants()[rec["variant"]]
    m = re.match(r"tile=(\d+)x1 ymarch rows=(\d+) persistent", tuned)
    V = fields(cases, "f32")
    b2.step(V, 2)
    b2.sync()
    for c, U in zip(cases, V):
        s = jf.Solver.from_case(c, dtype="f32")
        names = s.variants()
        if m:
            s.set_variant(names.index(next(d for d in names if d.startswith(f"tile={m[1]}x1 ymarch zchunk={m[2]} "))))
        else:
            s.set_variant(names.index(next(d for d in names if d.startswith(tuned.split()[0] + " "))))
        W = fields([c], "f32")[0]
        s.run(W, 2)
        s.sync()
        assert torch.equal(U, W), (tuned, s.variants())
    case = inputs.taylor_green(48)
    s = jf.Solver.from_case(case, dtype="f32")
    U = torch.tensor(case.U, dtype=torch.float32, device="cuda")
    rec = autotune.tune(s, U, steps=2, reps=2, path=path)
    assert rec["description"] == s.variants()[rec["variant"]]
