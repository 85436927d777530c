"""The C-ABI library loads and exports every entry point include/*.h
declares, and rejects bad arguments before touching the GPU.  CPU only."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?\w[\w\s\*]*?\b(jf_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def libjf():
    from paper_2203_13760_gb300 import _build
    _build.build()
    from paper_2203_13760_gb300 import jf
    return jf


def test_header_declares_the_boundary():
    names = declared_functions()
    for want in ["jf_init", "jf_destroy", "jf_rhs", "jf_compute_dt", "jf_rk3_step", "jf_rk3_step_vjp",
                 "jf_batch_create", "jf_batch_step", "jf_status_sync", "jf_last_error", "jf_stage", "jf_rk3_run"]:
        assert want in names


def test_every_declared_symbol_is_exported(libjf):
    L = ctypes.CDLL(libjf.LIB_PATH)
    for name in declared_functions():
        assert hasattr(L, name), name
    # the binding knows every declared entry point
    assert set(declared_functions()) <= set(libjf.SIGNATURES)


def test_bad_arguments_rejected_on_host(libjf):
    L = libjf.lib()
    h = ctypes.c_void_p()
    gas = libjf.GasParams(1.4, 1.0, 0.0, 0.72)
    sch = libjf.make_scheme("f32")
    for grid in [libjf.make_grid((3, 1, 1)), libjf.make_grid((16, 1, 8)), libjf.make_grid((16, 16, 1), bc=(0, 1, 1, 1, 1, 1)),
                 libjf.make_grid((16, 1, 1), lo=(1, 0, 0), hi=(0, 1, 1))]:
        st = L.jf_init(ctypes.byref(grid), ctypes.byref(gas), ctypes.byref(sch), ctypes.byref(h))
        assert st in (libjf.JF_ERR_ARG, libjf.JF_ERR_UNSUPPORTED)
        assert L.jf_last_error(None)
    grid = libjf.make_grid((16, 1, 1))
    bad_gas = libjf.GasParams(1.0, 1.0, 0.0, 0.72)
    assert L.jf_init(ctypes.byref(grid), ctypes.byref(bad_gas), ctypes.byref(sch), ctypes.byref(h)) == libjf.JF_ERR_ARG
    visc = libjf.make_scheme("f32", viscous=True)  # viscous with mu = 0
    assert L.jf_init(ctypes.byref(grid), ctypes.byref(gas), ctypes.byref(visc), ctypes.byref(h)) == libjf.JF_ERR_ARG
    assert L.jf_init(None, None, None, None) == libjf.JF_ERR_ARG
    # boundary codes 0..2 (periodic, zero gradient, slip wall)
    for code in (3, -1):
        g = libjf.make_grid((16, 1, 1), bc=(code, 1, 1, 1, 1, 1))
        assert L.jf_init(ctypes.byref(g), ctypes.byref(gas), ctypes.byref(sch), ctypes.byref(h)) == libjf.JF_ERR_ARG
    # scheme options out of range (flux 0..4, recon 0..2, speeds and integrators 0..2)
    for field, value in (("flux", 5), ("recon", 3), ("signal_speed", 3), ("integrator", -1)):
        bad = libjf.make_scheme("f32")
        setattr(bad, field, value)
        assert L.jf_init(ctypes.byref(grid), ctypes.byref(gas), ctypes.byref(bad), ctypes.byref(h)) == libjf.JF_ERR_ARG
        assert field.split("_")[0].encode() in L.jf_last_error(None)
        assert L.jf_batch_create(ctypes.byref(grid), 1, ctypes.byref(gas), ctypes.byref(bad),
                                 ctypes.byref(h)) == libjf.JF_ERR_ARG
    assert L.jf_rhs(None, None, None, None) == libjf.JF_ERR_ARG
    assert L.jf_destroy(None) == libjf.JF_OK
    assert L.jf_version().startswith(b"jf")
    assert L.jf_set_nn(None, None, 0) == libjf.JF_ERR_ARG
    assert L.jf_rk3_step_keep(None, None, None, None, None, None) == libjf.JF_ERR_ARG
    out = ctypes.c_double(0.0)
    assert L.jf_fma_peak(7, 10, ctypes.byref(out), None) == libjf.JF_ERR_ARG
    assert L.jf_fma_peak(libjf.JF_F32, 0, ctypes.byref(out), None) == libjf.JF_ERR_ARG
    assert L.jf_fma_peak(libjf.JF_F32, 10, None, None) == libjf.JF_ERR_ARG
    assert L.jf_batch_param_grad_begin(None, 1) == libjf.JF_ERR_ARG
    assert L.jf_batch_param_grad_end(None, None, None) == libjf.JF_ERR_ARG
    assert L.jf_rk3_step_vjp_stages(None, None, None, None, None, None, None, None) == libjf.JF_ERR_ARG
    # the Rusanov-NN flux runs only through a handle that holds parameters
    nn = libjf.make_scheme("f32", flux="rusanov-nn")
    U = ctypes.c_void_p(16)
    assert L.jf_rk3_step_noalloc(ctypes.byref(grid), ctypes.byref(gas), ctypes.byref(nn), U, None, None,
                                 None) == libjf.JF_ERR_UNSUPPORTED
    assert b"jf_set_nn" in L.jf_last_error(None)


def test_network_size_matches_the_header(libjf):
    import oracle
    text = open(os.path.join(ROOT, "include", "jf.h")).read()
    assert "#define JF_NN_HIDDEN 32" in text
    assert libjf.NN_PARAMS == oracle.NN_PARAMS == 2305
