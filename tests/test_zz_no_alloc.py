"""jf_rk3_step_noalloc: the RK3 step for callers that may not allocate device
memory while they run.  It uses a fixed scratch array compiled into libjf
instead of the stage buffers jf_init allocates.  It runs the same kernels
with the same launch variant as the handle path (jf_init + jf_rk3_step), so
its state and its dt must equal that path's bit for bit; one grid has exactly
JF_NOALLOC_MAX_CELLS cells, so the top of the scratch array is in use.

This file is named to be collected last; it passes both alone in a fresh
process and after the other tests."""
import ctypes

import pytest

from paper_2203_13760_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2203_13760_gb300 import jf  # noqa: E402

MAX_CELLS = 65536  # JF_NOALLOC_MAX_CELLS in include/jf.h


def noalloc_step(s, U, dt, dt_used):
    """One step through the C ABI entry point jf_rk3_step_noalloc."""
    L = jf.lib()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return L.jf_rk3_step_noalloc(ctypes.byref(s.grid), ctypes.byref(s.gas), ctypes.byref(s.scheme),
                                 ctypes.c_void_p(U.data_ptr()), jf._ptr(dt), jf._ptr(dt_used), stream)


@pytest.mark.parametrize("dtype", ["f32", "f64"])
@pytest.mark.parametrize("make", [
    lambda: inputs.kelvin_helmholtz(64),                                   # 2D viscous, periodic
    lambda: inputs.kelvin_helmholtz(256),                                  # exactly MAX_CELLS cells
    lambda: inputs.random_smooth((24, 20, 12), seed=3, viscous=True, mu=0.01),  # 3D, ragged tiles
    lambda: inputs.random_blocks((200, 1, 1), seed=2),                     # 1D shocks, zero gradient
])
def test_noalloc_matches_handle_path(dtype, make):
    case = make()
    s = jf.Solver.from_case(case, dtype=dtype)
    U_ref = torch.tensor(case.U, dtype=s.dtype, device="cuda")
    U_na = U_ref.clone()
    used_ref, used_na = s.scalar(), s.scalar()
    for _ in range(2):  # two calls in a row: the shared scratch is reused
        s.rk3_step(U_ref, None, used_ref)
        assert noalloc_step(s, U_na, None, used_na) == jf.JF_OK, jf.lib().jf_last_error(None)
        torch.cuda.synchronize()
        assert used_na.item() == used_ref.item()
        assert torch.equal(U_na, U_ref)
    # fixed-dt form as well
    dt = s.scalar(0.5 * used_ref.item())
    s.rk3_step(U_ref, dt)
    assert noalloc_step(s, U_na, dt, None) == jf.JF_OK
    torch.cuda.synchronize()
    assert torch.equal(U_na, U_ref)
    s.sync()


def test_noalloc_size_limit_matches_header():
    case = inputs.kelvin_helmholtz(256)
    assert case.cells == MAX_CELLS


def test_noalloc_rejects_grids_beyond_its_scratch():
    s = jf.Solver((300, 300, 1), bc=(0,) * 6, dtype="f32")  # 90,000 cells > 65,536
    U = s.empty()
    assert noalloc_step(s, U, None, None) == jf.JF_ERR_ARG
    assert b"JF_NOALLOC_MAX_CELLS" in jf.lib().jf_last_error(None)
