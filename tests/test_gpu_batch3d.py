"""Batches of 3D grids (jf_batch_create with nz > 1): the persistent kernel's
work items are tile columns and chunks of planes along z (32 by default,
16 or 64 by jf_set_variant).  Each simulation is bitwise the single-grid
path with the same tiles and chunk (FP32), the FP64 batch matches the oracle
per simulation, the trajectories of jf_batch_feed_forward equal fixed-dt
single-grid steps, and the batch adjoint (jf_batch_step_vjp) of inviscid 3D
grids equals the single-grid z-marching adjoint."""
import re

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


def cases_3d(viscous=True):
    # uneven and ragged: several tile columns, chunks and a short last chunk
    kw = dict(viscous=True, mu=0.01) if viscous else {}
    return [inputs.random_smooth((40, 17, 70), seed=31, **kw), inputs.random_smooth((19, 13, 11), seed=32, **kw),
            inputs.random_smooth((64, 30, 33), seed=33, bc=(0, 0, 1, 1, 0, 0), **kw)]


def batch_of(cases, dtype):
    grids = [jf.make_grid(c.n, c.lo, c.hi, c.bc) for c in cases]
    p = cases[0].params()
    return jf.Batch(grids, gamma=p["gamma"], R=p["R"], mu=p["mu"], Pr=p["Pr"], dtype=dtype, eps=p["eps"],
                    cfl=p["cfl"], viscous=p["viscous"], heat=p["heat"])


def fields(cases, dtype):
    t = torch.float32 if dtype == "f32" else torch.float64
    return [torch.tensor(c.U, dtype=t, device="cuda") for c in cases]


def solver_like(c, dtype, batch_desc):
    """A single-grid solver with the batch variant's tile and z chunk."""
    s = jf.Solver.from_case(c, dtype=dtype)
    m = re.match(r"tile=(\d+)x(\d+) zchunk=(\d+) persistent", batch_desc)
    assert m, batch_desc
    names = s.variants()
    s.set_variant(next(i for i, d in enumerate(names) if d.startswith(f"tile={m[1]}x{m[2]} zchunk={m[3]} ")))
    return s


@pytest.mark.parametrize("viscous", [True, False])
def test_batch3d_equals_single_grid_path(viscous):
    cases = cases_3d(viscous)
    b = batch_of(cases, "f32")
    names = b.variants()
    assert names[0] == "tile=32x7 zchunk=32 persistent", names
    Us = fields(cases, "f32")
    dt = b.step(Us, 6)
    b.sync()
    for i, c in enumerate(cases):
        s = solver_like(c, "f32", names[0])
        U = fields([c], "f32")[0]
        used = s.scalar()
        for _ in range(6):
            s.rk3_step(U, None, used)
        s.sync()
        assert dt[i].item() == used.item(), i
        assert torch.equal(U, Us[i]), (i, c.n)
    b.close()


def test_batch3d_chunk_variants():
    """Every 3D batch variant (tile shapes x 32, 16, 64 planes) is bitwise the
    single-grid path with that tile and chunk after two steps."""
    cases = cases_3d()[:2]
    b = batch_of(cases, "f32")
    names = b.variants()
    assert len(names) >= 6
    for v, d in enumerate(names):
        b.set_variant(v)
        Us = fields(cases, "f32")
        b.step(Us, 2)
        b.sync()
        for c, U in zip(cases, Us):
            s = solver_like(c, "f32", d)
            W = fields([c], "f32")[0]
            s.run(W, 2)
            s.sync()
            assert torch.equal(U, W), d
    b.close()


def test_batch3d_fp64_vs_oracle(orc):
    cases = cases_3d()
    b = batch_of(cases, "f64")
    Us = fields(cases, "f64")
    dts = [b.step(Us, 1).cpu().numpy().copy() for _ in range(4)]
    b.sync()
    for i, c in enumerate(cases):
        oc = orc.config(**c.params())
        W = c.U.copy()
        for k in range(4):
            assert dts[k][i] == pytest.approx(orc.compute_dt(oc, W), rel=1e-13)
            W = orc.rk3_step(oc, W, float(dts[k][i]))
        assert rel_err(Us[i].cpu().numpy(), W) <= 1e-12, (i, c.n)
    b.close()


def test_batch3d_feed_forward():
    cases = cases_3d()
    b = batch_of(cases, "f32")
    U0s = fields(cases, "f32")
    dts = [2e-3, 1e-3, 1.5e-3]
    trajs = b.feed_forward(U0s, 3, dts)
    b.sync()
    desc = b.variants()[0]
    for c, tr, dt in zip(cases, trajs, dts):
        s = solver_like(c, "f32", desc)
        U = fields([c], "f32")[0]
        dtt = torch.tensor([dt], dtype=torch.float64, device="cuda")
        assert torch.equal(tr[0], U)
        for t in range(3):
            s.rk3_step(U, dtt)
            s.sync()
            assert torch.equal(tr[t + 1], U), t
    b.close()


def test_batch3d_step_vjp_equals_single_grids():
    """jf_batch_step_vjp over an uneven batch of inviscid 3D grids (the
    per-face adjoint, its forward recompute through the batch's z-chunk work
    items) equals each grid's single-grid adjoint (the z-marching adjoint
    kernel) plus the addend, FP64 to rounding (atomic order)."""
    cases = cases_3d(viscous=False)
    b = batch_of(cases, "f64")
    assert b.supports_step_vjp()
    rng = np.random.default_rng(4)
    Us = fields(cases, "f64")
    lams = [torch.tensor(rng.standard_normal(c.U.shape), device="cuda") for c in cases]
    adds = [torch.tensor(rng.standard_normal(c.U.shape), device="cuda") for c in cases]
    dts = [2e-4, 3e-4, 2.5e-4]
    got = b.step_vjp(Us, torch.tensor(dts, dtype=torch.float64, device="cuda"), lams, None, adds, None)
    b.sync()
    for i, c in enumerate(cases):
        s = b.solver(i)
        want = s.rk3_step_vjp(Us[i], s.scalar(dts[i]), lams[i])
        s.sync()
        want = want + adds[i]
        assert (got[i] - want).abs().max().item() <= 1e-12 * want.abs().max().item(), i
    b.close()
