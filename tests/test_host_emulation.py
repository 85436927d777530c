"""The stage kernel's own source, compiled for the CPU (tests/host_emu: one
std::thread per CUDA thread, a std::barrier per CTA, exact-size heap buffers
for the shared memory and the fields) and run under AddressSanitizer and
UBSan where the toolchain has them: every shared-memory and global access of
the tiles stays inside its buffer, and the results match the oracle -- FP64
to 1e-12 (right-hand side, rate norm; one stage), FP32 to 1e-5 -- for the 2D
tiles, the row tiles of 2D grids (several row widths and chunk lengths), the
3D z-march, and the run-time-scheme kernels (HLL, Rusanov, Davis and Toro
speeds, WENO5-Z) on ragged grids with periodic, zero-gradient and mixed
boundaries.  The persistent batch form (descriptors and work items, with
chunks of planes for the z-march kernels) is checked the same way: every
simulation of an emulated batch stage equals the emulated single-grid stage
with the same chunk, bit for bit.  This checks the kernels' index arithmetic
on the CPU, without a GPU; the GPU parity tests check the compiled kernels
themselves."""
import ctypes
import json
import os
import shutil
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if __name__ == "__main__":
    sys.path.insert(0, ROOT)

from paper_2203_13760_gb300 import inputs  # noqa: E402

CSRC = os.path.join(ROOT, "paper_2203_13760_gb300", "csrc")
HERE = os.path.join(ROOT, "tests", "host_emu")
GROUPS = ((0,), (1, 2, 3), (4,))
SMEM_DECL = "extern __shared__ __align__(16) unsigned char smem_raw[];"

CASES = {
    "2d_smooth_visc_mixed": lambda: inputs.random_smooth((37, 19, 1), seed=3, bc=(0, 0, 1, 1, 1, 1), viscous=True,
                                                         mu=0.01),
    "2d_blocks_zg": lambda: inputs.random_blocks((40, 33, 1), seed=4),
    "2d_wide_y_periodic": lambda: inputs.random_smooth((150, 41, 1), seed=8, bc=(1, 1, 0, 0, 1, 1), viscous=True,
                                                       mu=0.01),
    "3d_smooth_visc_ragged": lambda: inputs.random_smooth((19, 13, 11), seed=6, viscous=True, mu=0.01),
}


def _scheme(make, **kw):
    def f():
        c = make()
        for k, v in kw.items():
            setattr(c, k, v)
        return c
    return f


# run-time-scheme kernels (Table 2 Godunov variants, per-cell reconstruction)
CASES.update({
    "2d_blocks_hll_z": _scheme(CASES["2d_blocks_zg"], flux="hll", recon="weno5-z"),
    "2d_visc_davis": _scheme(CASES["2d_smooth_visc_mixed"], speeds="davis"),
    "3d_visc_rusanov_z": _scheme(CASES["3d_smooth_visc_ragged"], flux="rusanov", recon="weno5-z"),
    "3d_visc_toro": _scheme(CASES["3d_smooth_visc_ragged"], speeds="toro"),
})

# (case, precision, kernel, z chunk): kernels as in emu.cpp (0: 2D tiles,
# 1/2/3: row tiles 128/96/224 wide, 4: 3D tiles, 5/6/7: run-time-scheme 2D
# tiles, 3D tiles and 2D row tiles)
RUNS = [
    ("2d_smooth_visc_mixed", "f64", 0, 1), ("2d_smooth_visc_mixed", "f64", 1, 5),
    ("2d_smooth_visc_mixed", "f64", 1, 1000), ("2d_blocks_zg", "f64", 1, 7), ("2d_wide_y_periodic", "f64", 1, 16),
    ("2d_wide_y_periodic", "f32", 2, 3), ("2d_wide_y_periodic", "f32", 3, 41), ("2d_blocks_zg", "f32", 1, 1),
    ("3d_smooth_visc_ragged", "f64", 4, 4), ("3d_smooth_visc_ragged", "f32", 4, 11),
    ("2d_blocks_hll_z", "f64", 5, 1), ("2d_visc_davis", "f64", 5, 1), ("2d_blocks_hll_z", "f32", 5, 1),
    ("3d_visc_rusanov_z", "f64", 6, 4), ("3d_visc_toro", "f64", 6, 5), ("3d_visc_rusanov_z", "f32", 6, 11),
    ("2d_blocks_hll_z", "f64", 7, 6), ("2d_visc_davis", "f64", 7, 4), ("2d_visc_davis", "f32", 7, 1000),
]


def _sanitizer_libs():
    libs = []
    for name in ("libasan.so", "libubsan.so"):
        p = subprocess.run(["gcc", "-print-file-name=" + name], capture_output=True, text=True).stdout.strip()
        if not os.path.isabs(p) or not os.path.exists(p):
            return []
        libs.append(p)
    return libs


@pytest.fixture(scope="module")
def emu_lib(tmp_path_factory):
    if shutil.which("g++") is None:
        pytest.skip("g++ not available")
    d = tmp_path_factory.mktemp("host_emu")
    src = d / "src"
    src.mkdir()
    for f in ("stage.cuh", "jf_math.cuh"):
        shutil.copy(os.path.join(CSRC, f), src / f)
    text = (src / "stage.cuh").read_text()
    assert text.count(SMEM_DECL) == 1
    text = text.replace(SMEM_DECL, "unsigned char* smem_raw = emu_smem();")
    text = text.replace("namespace jf {\n", "unsigned char* emu_smem();\nnamespace jf {\n", 1)
    (src / "stage.cuh").write_text(text)
    san = _sanitizer_libs()
    lib = d / "libemu.so"
    cmd = ["g++", "-std=c++20", "-O1", "-g1", "-fno-omit-frame-pointer", "-shared", "-fPIC",
           "-I", os.path.join(HERE, "cuda_stub"), "-I", str(src), os.path.join(HERE, "emu.cpp"), "-o", str(lib),
           "-lpthread"]
    if san:
        cmd[1:1] = ["-fsanitize=address,undefined", "-fno-sanitize-recover=undefined"]
    out = subprocess.run(cmd, capture_output=True, text=True)
    if out.returncode != 0 and "barrier" in out.stderr:
        pytest.skip("the C++ library has no std::barrier")
    assert out.returncode == 0, out.stderr[-3000:]
    return str(lib), san


def _params(case):
    p = case.params()
    n = [int(x) for x in p["n"]]
    periodic = [1 if p["bc"][2 * a] == 0 else 0 for a in range(3)]
    inv_h = [n[a] / (p["hi"][a] - p["lo"][a]) for a in range(3)]
    mu = p["mu"] if p["viscous"] else 0.0
    lam = p["mu"] * p["gamma"] * p["R"] / ((p["gamma"] - 1.0) * p["Pr"]) if p["heat"] else 0.0
    codes = {"flux": {"hllc": 0, "hll": 1, "rusanov": 2}, "recon": {"weno5-js": 0, "weno5-z": 1},
             "speeds": {"einfeldt": 0, "davis": 1, "toro": 2}}
    scheme = [float(codes[k][p[k]]) for k in ("flux", "recon", "speeds")]
    return n, periodic, inv_h, [p["gamma"], p["R"], mu, lam, p["eps"]] + scheme


def emulate(lib_path, case, dtype, kernel, zchunk, rhs_only=True, a=0.0, b=1.0, dt=0.0, Un=None):
    L = ctypes.CDLL(lib_path)
    n, periodic, inv_h, gas = _params(case)
    t = np.float64 if dtype == "f64" else np.float32
    U = np.ascontiguousarray(case.U, dtype=t)
    N = np.ascontiguousarray(Un, dtype=t) if Un is not None else None
    out = np.zeros_like(U)
    ip = lambda v: (ctypes.c_int * 3)(*v)  # noqa: E731
    dp = lambda v: (ctypes.c_double * len(v))(*v)  # noqa: E731
    fn = L.emu_stage_f64 if dtype == "f64" else L.emu_stage_f32
    fn.restype = ctypes.c_int
    flag = fn(kernel, ip(n), ip(periodic), dp(inv_h), dp(gas), int(zchunk), int(rhs_only), ctypes.c_double(a),
              ctypes.c_double(b), ctypes.c_double(dt), U.ctypes.data_as(ctypes.c_void_p),
              N.ctypes.data_as(ctypes.c_void_p) if N is not None else None, out.ctypes.data_as(ctypes.c_void_p))
    assert flag == 0, flag
    return out.astype(np.float64)


def emulate_batch_stage1(lib_path, cases, kernel, rows, ctas, dts):
    """Stage 1 (U1 = U + dt L(U)) of every simulation through the persistent
    batch form (FP64)."""
    L = ctypes.CDLL(lib_path)
    ps = [_params(c) for c in cases]
    n = [x for p in ps for x in p[0]]
    per = [x for p in ps for x in p[1]]
    ih = [x for p in ps for x in p[2]]
    Us = [np.ascontiguousarray(c.U, dtype=np.float64) for c in cases]
    outs = [np.zeros_like(U) for U in Us]
    vp = ctypes.c_void_p
    L.emu_batch_stage1_f64.restype = ctypes.c_int
    flag = L.emu_batch_stage1_f64(kernel, len(cases), (ctypes.c_int * len(n))(*n), (ctypes.c_int * len(per))(*per),
                                  (ctypes.c_double * len(ih))(*ih), (ctypes.c_double * 8)(*ps[0][3]), int(rows),
                                  int(ctas), (ctypes.c_double * len(dts))(*dts),
                                  (vp * len(Us))(*[U.ctypes.data for U in Us]),
                                  (vp * len(outs))(*[o.ctypes.data for o in outs]))
    assert flag == 0, flag
    return outs


def _run_children(lib_path, san, jobs):
    """Runs this file as a script in child processes (the sanitizer runtime
    must be loaded first, with LD_PRELOAD), a few at a time, one per job (a
    list of arguments); returns {job: (returncode, JSON result or output)}."""
    env = dict(os.environ)
    if san:
        env["LD_PRELOAD"] = " ".join(san)
        env["ASAN_OPTIONS"] = "detect_leaks=0:abort_on_error=1"
    env["PYTHONPATH"] = ROOT + os.pathsep + env.get("PYTHONPATH", "")
    width = max(1, min(4, (os.cpu_count() or 1) // 2))
    out, running, queue = {}, [], list(jobs)
    while queue or running:
        while queue and len(running) < width:
            job = queue.pop(0)
            p = subprocess.Popen([sys.executable, os.path.abspath(__file__), lib_path, *map(str, job)],
                                 stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True, env=env)
            running.append((job, p))
        job, p = running.pop(0)
        so, se = p.communicate(timeout=900)
        out[tuple(job)] = (0, json.loads(so.strip().splitlines()[-1])) if p.returncode == 0 else \
            (p.returncode, so[-2000:] + se[-4000:])
    return out


@pytest.fixture(scope="module")
def results(emu_lib):
    lib_path, san = emu_lib
    jobs = [["single", *r] for r in RUNS] + [["batch", *b] for b in BATCH_RUNS]
    return _run_children(lib_path, san, jobs)


def _result(results, job):
    rc, res = results[tuple(job)]
    assert rc == 0, res
    return res


def _child(lib_path, name, dtype, kernel, zchunk):
    import oracle as orc
    case = CASES[name]()
    c = orc.config(**case.params())
    U = case.U if dtype == "f64" else case.U.astype(np.float32).astype(np.float64)
    want = orc.rhs(c, U)
    rate = case.cfl / orc.compute_dt(c, U)
    got = emulate(lib_path, case, dtype, kernel, zchunk)
    err = 0.0
    for g in GROUPS:
        g = list(g)
        w, x, u = want.reshape(5, -1)[g], got.reshape(5, -1)[g], U.reshape(5, -1)[g]
        err = max(err, np.abs(x - w).max() / max(np.abs(w).max(), np.abs(u).max() * rate, 1e-300))
    res = {"rhs": err}
    if dtype == "f64":
        # one stage of the Shu-Osher form: out = 3/4 Un + 1/4 (Us + dt L(Us))
        Un = inputs.random_smooth(tuple(case.n), seed=77).U
        dt = 0.3 * orc.compute_dt(c, U)
        want_s = 0.75 * Un + 0.25 * (U + dt * want)
        got_s = emulate(lib_path, case, dtype, kernel, zchunk, rhs_only=False, a=0.75, b=0.25, dt=dt, Un=Un)
        res["stage"] = float(np.abs(got_s - want_s).max() / np.abs(want_s).max())
    return res


BATCHES = {
    "3d": (4, lambda: [inputs.random_smooth((19, 13, 11), seed=6, viscous=True, mu=0.01),
                       inputs.random_smooth((40, 9, 7), seed=7, viscous=True, mu=0.01),
                       inputs.random_smooth((8, 16, 20), seed=8, viscous=True, mu=0.01)]),
    "2d_rows": (1, lambda: [inputs.random_blocks((150, 41, 1), seed=9), inputs.random_blocks((37, 19, 1), seed=10),
                            inputs.random_blocks((40, 33, 1), seed=11)]),
    "2d_tiles": (0, lambda: [inputs.random_blocks((37, 19, 1), seed=10), inputs.random_blocks((40, 33, 1), seed=11)]),
}


def _child_batch(lib_path, name, rows, ctas):
    kernel, make = BATCHES[name]
    cases = make()
    dts = [1e-3 * (k + 1) for k in range(len(cases))]
    outs = emulate_batch_stage1(lib_path, cases, kernel, rows, ctas, dts)
    same = []
    for c, o, dt in zip(cases, outs, dts):
        want = emulate(lib_path, c, "f64", kernel, rows, rhs_only=False, a=0.0, b=1.0, dt=dt)
        same.append(bool(np.array_equal(o, want)))
    return {"same": same}


BATCH_RUNS = [("3d", 4, 5), ("3d", 16, 64), ("2d_rows", 8, 7), ("2d_tiles", 1, 3)]


@pytest.mark.parametrize("name,rows,ctas", BATCH_RUNS)
def test_emulated_batch_equals_single_grid(results, name, rows, ctas):
    res = _result(results, ["batch", name, rows, ctas])
    assert all(res["same"]), res


@pytest.mark.parametrize("run", RUNS, ids=[f"{r[0]}-{r[1]}-k{r[2]}-z{r[3]}" for r in RUNS])
def test_emulated_kernel_vs_oracle(results, run):
    res = _result(results, ["single", *run])
    tol = 1e-12 if run[1] == "f64" else 1e-5
    assert res["rhs"] <= tol, res
    if "stage" in res:
        assert res["stage"] <= 1e-13, res


if __name__ == "__main__":
    if sys.argv[2] == "batch":
        lib, _, name, rows, ctas = sys.argv[1:6]
        print(json.dumps(_child_batch(lib, name, int(rows), int(ctas))))
    else:
        lib, _, name, dtype, kernel, zchunk = sys.argv[1:7]
        print(json.dumps(_child(lib, name, dtype, int(kernel), int(zchunk))))
