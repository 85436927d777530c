"""The oracle: a plain, slow FP64 CPU implementation of the JAX-FLUIDS
finite-volume RK3 stage (arXiv 2203.13760, Sections 2-3), written in C++
(``jf_oracle.hpp``) and loaded here with ctypes.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s ``cpu_baseline`` / ``--impl reference`` legs may import this
package.  The product path (``paper_2203_13760_gb300``) never imports it, and the
two share no code; the seeded input generators in
``paper_2203_13760_gb300/inputs.py`` are the only module both sides use.

Parity status of each function (what pins it is in ``tests/test_oracle_*.py``):
  rhs / rk3_step / run   pinned (free stream, conservation, Sod vs exact
                         Riemann solution, 5th-order convergence, mirror
                         symmetry, manufactured viscous fields)
  weno5                  pinned (polynomial exactness, linear weights on
                         smooth data, non-oscillation at a jump)
  hllc                   pinned (consistency with the physical flux,
                         Rankine-Hugoniot for an isolated shock and contact)
  exact_star/sample      pinned (Rankine-Hugoniot, isentropic and Riemann
                         invariant relations, contact continuity)
  jvp_run                pinned (against central finite differences of run)
  compute_dt             pinned (closed form on uniform states)
  weno5_z                pinned (fifth order at critical points where WENO5-JS
                         drops, non-oscillation at a jump, linear exactness)
  hll / rusanov flux     pinned (consistency, Rankine-Hugoniot across the HLL
                         fan, Rusanov = HLL with symmetric speeds, upwinding,
                         contact diffusion ordering)
  signal_speeds          pinned (equal states give u -+ c; Einfeldt's speed
                         equals the exact shock speed of an isolated
                         Rankine-Hugoniot shock, which only sqrt(rho)-weighted
                         Roe averages give; Toro's factor with the exact p*
                         gives the exact shock speed; PVRS error of second
                         order in the jump)
  safe reconstruction    pinned (the right-hand side with the flag equals the
                         one assembled face by face with each non-positive
                         WENO5 side replaced by its cell value; inert where
                         every face state is positive)
  time_step (rk2/euler)  pinned (temporal orders 1, 2, 3; RK2 = mean of U and
                         two Euler steps)
  shock tubes            Sod and Lax against the exact solution for every
                         solver / speed / reconstruction
  roe_eigensystem /      pinned (L = R^-1; R diag(lambda) L equals the flux
  fs_flux (ROE setup)    Jacobian by finite differences; Roe's property
                         A~ (U_R - U_L) = F_R - F_L; consistency; fifth order
                         on smooth advection; Sod and Lax convergence)
  wall boundary          pinned (equals the mirror-doubled periodic domain to
                         rounding; closed box conserves mass and energy)
  weno3                  pinned (linear exactness, non-oscillation at a jump,
                         third-order convergence)
  flux_nn / nn_alpha /   pinned (constant alpha gives Lax-Friedrichs = HLL
  jvp_params_run         with -+alpha; a network built to compute
                         exp(a . x + b) matches the closed form with the
                         paper's inputs; parameter JVP = central differences)
  count_flops            descriptive only (an operation count, not a result)
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_SOURCES = ["oracle_capi.cpp", "jf_oracle.hpp", "dual.hpp", "exact_riemann.hpp"]
_lock = threading.Lock()
_lib = None

BC_PERIODIC = 0
BC_ZERO_GRADIENT = 1


def build(force: bool = False) -> str:
    """Compile liboracle.so with g++ (FP64, no FMA contraction, OpenMP)."""
    newest = max(os.path.getmtime(os.path.join(_HERE, s)) for s in _SOURCES)
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= newest:
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
           "-fPIC", "-shared", os.path.join(_HERE, "oracle_capi.cpp"), "-o", tmp]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Config(ctypes.Structure):
    """Mirror of ``orc::Config`` in jf_oracle.hpp."""
    _fields_ = [
        ("n", ctypes.c_int * 3),
        ("lo", ctypes.c_double * 3),
        ("hi", ctypes.c_double * 3),
        ("bc", ctypes.c_int * 6),
        ("gamma", ctypes.c_double),
        ("R", ctypes.c_double),
        ("mu", ctypes.c_double),
        ("Pr", ctypes.c_double),
        ("eps", ctypes.c_double),
        ("cfl", ctypes.c_double),
        ("convective", ctypes.c_int),
        ("viscous", ctypes.c_int),
        ("heat", ctypes.c_int),
        ("safe", ctypes.c_int),
        ("flux", ctypes.c_int),
        ("recon", ctypes.c_int),
        ("speeds", ctypes.c_int),
        ("integrator", ctypes.c_int),
        ("nn", ctypes.POINTER(ctypes.c_double)),
        ("nn_dot", ctypes.POINTER(ctypes.c_double)),
    ]


# scheme options (Table 2); 0 is the Appendix A configuration
FLUX = {"hllc": 0, "hll": 1, "rusanov": 2, "roe": 3, "rusanov-nn": 4}
RECON = {"weno5-js": 0, "weno5-z": 1, "weno3-js": 2}
NN_PARAMS = 32 * 4 + 32 + 2 * (32 * 32 + 32) + 32 + 1
SPEEDS = {"einfeldt": 0, "davis": 1, "toro": 2}
INTEGRATOR = {"rk3": 0, "rk2": 1, "euler": 2}


def config(n, lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0), bc=(1, 1, 1, 1, 1, 1), gamma=1.4, R=1.0,
           mu=0.0, Pr=0.72, eps=1e-6, cfl=0.5, convective=True, viscous=False, heat=False,
           safe=False, flux="hllc", recon="weno5-js", speeds="einfeldt", integrator="rk3", nn=None) -> Config:
    n = tuple(int(x) for x in n) + (1,) * (3 - len(n))
    c = Config()
    c.n[:] = n
    c.lo[:] = [float(x) for x in lo]
    c.hi[:] = [float(x) for x in hi]
    c.bc[:] = [int(x) for x in bc]
    c.gamma, c.R, c.mu, c.Pr, c.eps, c.cfl = gamma, R, mu, Pr, eps, cfl
    c.convective, c.viscous, c.heat, c.safe = int(convective), int(viscous), int(heat), int(safe)
    c.flux, c.recon = FLUX[flux], RECON[recon]
    c.speeds, c.integrator = SPEEDS[speeds], INTEGRATOR[integrator]
    if nn is not None:
        arr = np.ascontiguousarray(nn, dtype=np.float64)
        if arr.size != NN_PARAMS:
            raise ValueError(f"the Rusanov-NN network has {NN_PARAMS} parameters")
        c._nn_keep = arr  # the structure holds a raw pointer into it
        c.nn = arr.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    return c


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB_PATH)
            P = ctypes.POINTER
            d = ctypes.c_double
            dp = P(d)
            cp = P(Config)
            L.orc_set_threads.argtypes = [ctypes.c_int]
            L.orc_set_threads.restype = ctypes.c_int
            L.orc_rhs.argtypes = [cp, dp, dp]
            L.orc_rhs.restype = ctypes.c_int
            L.orc_compute_dt.argtypes = [cp, dp]
            L.orc_compute_dt.restype = d
            L.orc_run.argtypes = [cp, dp, ctypes.c_int, d, d, dp]
            L.orc_run.restype = ctypes.c_int
            L.orc_jvp_run.argtypes = [cp, dp, dp, ctypes.c_int, d]
            L.orc_jvp_run.restype = ctypes.c_int
            L.orc_weno5.argtypes = [dp, d]
            L.orc_weno5.restype = d
            L.orc_hllc.argtypes = [dp, dp, ctypes.c_int, d, dp]
            L.orc_hllc.restype = None
            L.orc_weno5_z.argtypes = [dp, d]
            L.orc_weno5_z.restype = d
            L.orc_signal_speeds.argtypes = [dp, dp, ctypes.c_int, d, ctypes.c_int, dp]
            L.orc_signal_speeds.restype = None
            L.orc_toro_q.argtypes = [d, d, d]
            L.orc_toro_q.restype = d
            L.orc_flux.argtypes = [dp, dp, ctypes.c_int, d, ctypes.c_int, ctypes.c_int, dp]
            L.orc_flux.restype = None
            L.orc_hll_speeds.argtypes = [dp, dp, ctypes.c_int, d, d, d, dp]
            L.orc_hll_speeds.restype = None
            L.orc_jvp_params_run.argtypes = [cp, dp, dp, ctypes.c_int, d, dp]
            L.orc_jvp_params_run.restype = ctypes.c_int
            L.orc_flux_nn.argtypes = [dp, dp, ctypes.c_int, d, dp, dp]
            L.orc_flux_nn.restype = None
            L.orc_nn_alpha.argtypes = [dp, dp]
            L.orc_nn_alpha.restype = d
            L.orc_weno3.argtypes = [dp, d]
            L.orc_weno3.restype = d
            L.orc_roe_eigensystem.argtypes = [dp, dp, ctypes.c_int, d, dp, dp, dp]
            L.orc_roe_eigensystem.restype = None
            L.orc_fs_flux.argtypes = [dp, ctypes.c_int, d, d, ctypes.c_int, dp]
            L.orc_fs_flux.restype = None
            L.orc_exact_star.argtypes = [dp, dp, d, dp]
            L.orc_exact_star.restype = ctypes.c_int
            L.orc_exact_sample.argtypes = [dp, dp, d, d, d, ctypes.c_int, dp, dp]
            L.orc_exact_sample.restype = ctypes.c_int
            L.orc_sample_cells.argtypes = [cp, dp, ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.c_int, d, dp]
            L.orc_sample_cells.restype = ctypes.c_int
            L.orc_count_flops.argtypes = [cp, dp]
            L.orc_count_flops.restype = ctypes.c_int
            _lib = L
    return _lib


def _ptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _state(c: Config, U) -> np.ndarray:
    U = np.ascontiguousarray(U, dtype=np.float64)
    want = (5, c.n[2], c.n[1], c.n[0])
    if U.size != np.prod(want):
        raise ValueError(f"state has {U.size} values, config wants {want}")
    return U.reshape(want).copy()


def set_threads(n: int) -> int:
    return lib().orc_set_threads(int(n))


def rhs(c: Config, U) -> np.ndarray:
    """dU/dt of Eq. (FVD) for the interior state U[5][nz][ny][nx]."""
    U = _state(c, U)
    out = np.empty_like(U)
    if lib().orc_rhs(ctypes.byref(c), _ptr(U), _ptr(out)) != 0:
        raise ValueError("oracle rejected the configuration")
    return out


def compute_dt(c: Config, U) -> float:
    U = _state(c, U)
    return float(lib().orc_compute_dt(ctypes.byref(c), _ptr(U)))


def run(c: Config, U, nsteps: int, dt: float = 0.0, t_end: float = 0.0):
    """nsteps TVD-RK3 steps (fixed dt if dt > 0, else CFL steps up to t_end).
    Returns (U, t, steps_taken)."""
    U = _state(c, U)
    t = ctypes.c_double(0.0)
    s = lib().orc_run(ctypes.byref(c), _ptr(U), int(nsteps), float(dt), float(t_end), ctypes.byref(t))
    if s < 0:
        raise ValueError("oracle rejected the configuration")
    return U, t.value, s


def rk3_step(c: Config, U, dt: float) -> np.ndarray:
    """One fixed-dt step of the configured integrator (TVD-RK3 by default)."""
    return run(c, U, 1, dt)[0]


def jvp_run(c: Config, U, V, nsteps: int, dt: float):
    """(U_n, J V) for nsteps fixed-dt RK3 steps, by forward-mode dual numbers."""
    U = _state(c, U)
    V = _state(c, V)
    if lib().orc_jvp_run(ctypes.byref(c), _ptr(U), _ptr(V), int(nsteps), float(dt)) != 0:
        raise ValueError("oracle rejected the configuration")
    return U, V


def sample_cells(c: Config, U, cells, nsteps: int, dt: float = 0.0) -> np.ndarray:
    """Values at the given cells [(i, j, k), ...] after nsteps fixed-dt RK3
    steps of the full state U (nsteps == 0: the right-hand side there),
    computed one cell at a time on a local patch.  Returns [len(cells), 5]."""
    U = np.ascontiguousarray(U, dtype=np.float64)
    if U.size != 5 * c.n[0] * c.n[1] * c.n[2]:
        raise ValueError("state does not match the configuration")
    idx = np.ascontiguousarray(np.asarray(cells, dtype=np.int32).reshape(-1, 3))
    out = np.empty((idx.shape[0], 5))
    r = lib().orc_sample_cells(ctypes.byref(c), _ptr(U), idx.shape[0],
                               idx.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), int(nsteps), float(dt), _ptr(out))
    if r != 0:
        raise ValueError("oracle rejected the configuration")
    return out


def weno5(v, eps: float = 1e-6) -> float:
    v = np.ascontiguousarray(v, dtype=np.float64)
    return float(lib().orc_weno5(_ptr(v), float(eps)))


def hllc(WL, WR, d: int = 0, gamma: float = 1.4) -> np.ndarray:
    WL = np.ascontiguousarray(WL, dtype=np.float64)
    WR = np.ascontiguousarray(WR, dtype=np.float64)
    F = np.empty(5)
    lib().orc_hllc(_ptr(WL), _ptr(WR), int(d), float(gamma), _ptr(F))
    return F


def weno5_z(v, eps: float = 1e-6) -> float:
    v = np.ascontiguousarray(v, dtype=np.float64)
    return float(lib().orc_weno5_z(_ptr(v), float(eps)))


def signal_speeds(WL, WR, d: int = 0, gamma: float = 1.4, kind: str = "einfeldt"):
    """(S_L, S_R) of the named estimate."""
    WL = np.ascontiguousarray(WL, dtype=np.float64)
    WR = np.ascontiguousarray(WR, dtype=np.float64)
    out = np.empty(2)
    lib().orc_signal_speeds(_ptr(WL), _ptr(WR), int(d), float(gamma), SPEEDS[kind], _ptr(out))
    return float(out[0]), float(out[1])


def toro_q(p_star: float, pK: float, gamma: float = 1.4) -> float:
    return float(lib().orc_toro_q(float(p_star), float(pK), float(gamma)))


def flux(WL, WR, d: int = 0, gamma: float = 1.4, kind: str = "hllc", speeds: str = "einfeldt") -> np.ndarray:
    WL = np.ascontiguousarray(WL, dtype=np.float64)
    WR = np.ascontiguousarray(WR, dtype=np.float64)
    F = np.empty(5)
    lib().orc_flux(_ptr(WL), _ptr(WR), int(d), float(gamma), FLUX[kind], SPEEDS[speeds], _ptr(F))
    return F


def hll_with_speeds(WL, WR, SL: float, SR: float, d: int = 0, gamma: float = 1.4) -> np.ndarray:
    WL = np.ascontiguousarray(WL, dtype=np.float64)
    WR = np.ascontiguousarray(WR, dtype=np.float64)
    F = np.empty(5)
    lib().orc_hll_speeds(_ptr(WL), _ptr(WR), int(d), float(gamma), float(SL), float(SR), _ptr(F))
    return F


def jvp_params_run(c: Config, U, nsteps: int, dt: float, theta_dot):
    """(U_n, dU_n/dtheta . theta_dot) for nsteps fixed-dt steps of the
    Rusanov-NN configuration, by dual-number parameters."""
    U = _state(c, U)
    V = np.zeros_like(U)
    td = np.ascontiguousarray(theta_dot, dtype=np.float64)
    if lib().orc_jvp_params_run(ctypes.byref(c), _ptr(U), _ptr(V), int(nsteps), float(dt), _ptr(td)) != 0:
        raise ValueError("orc_jvp_params_run failed")
    return U, V


def flux_nn(WL, WR, theta, d: int = 0, gamma: float = 1.4) -> np.ndarray:
    WL = np.ascontiguousarray(WL, dtype=np.float64)
    WR = np.ascontiguousarray(WR, dtype=np.float64)
    th = np.ascontiguousarray(theta, dtype=np.float64)
    F = np.empty(5)
    lib().orc_flux_nn(_ptr(WL), _ptr(WR), int(d), float(gamma), _ptr(th), _ptr(F))
    return F


def nn_alpha(theta, x) -> float:
    th = np.ascontiguousarray(theta, dtype=np.float64)
    xv = np.ascontiguousarray(x, dtype=np.float64)
    return float(lib().orc_nn_alpha(_ptr(th), _ptr(xv)))


def weno3(v, eps: float = 1e-6) -> float:
    v = np.ascontiguousarray(v, dtype=np.float64)
    return float(lib().orc_weno3(_ptr(v), float(eps)))


def roe_eigensystem(WL, WR, d: int = 0, gamma: float = 1.4):
    """(lambda[5], R[5x5], L[5x5]) of the Roe-averaged flux Jacobian along d."""
    WL = np.ascontiguousarray(WL, dtype=np.float64)
    WR = np.ascontiguousarray(WR, dtype=np.float64)
    lam, R, L = np.empty(5), np.empty((5, 5)), np.empty((5, 5))
    lib().orc_roe_eigensystem(_ptr(WL), _ptr(WR), int(d), float(gamma), _ptr(lam), _ptr(R), _ptr(L))
    return lam, R, L


def fs_flux(W6, d: int = 0, gamma: float = 1.4, eps: float = 1e-6, recon: str = "weno5-js") -> np.ndarray:
    """Flux-splitting (ROE setup) face flux from six primitive states
    (cells i-2 .. i+3 of the face x_{i+1/2}) along d."""
    W6 = np.ascontiguousarray(W6, dtype=np.float64).reshape(6, 5)
    F = np.empty(5)
    lib().orc_fs_flux(_ptr(W6), int(d), float(gamma), float(eps), RECON[recon], _ptr(F))
    return F


def exact_star(WL, WR, gamma: float = 1.4):
    """(p*, u*, rho*_L, rho*_R) of the exact Riemann solution; W = (rho, u, p)."""
    WL = np.ascontiguousarray(WL, dtype=np.float64)
    WR = np.ascontiguousarray(WR, dtype=np.float64)
    out = np.empty(4)
    if lib().orc_exact_star(_ptr(WL), _ptr(WR), float(gamma), _ptr(out)) != 0:
        raise ValueError("no exact solution (vacuum)")
    return out


def exact_sample(WL, WR, x, t: float, x0: float = 0.5, gamma: float = 1.4) -> np.ndarray:
    """Exact (rho, u, p) at points x and time t: array of shape (len(x), 3)."""
    WL = np.ascontiguousarray(WL, dtype=np.float64)
    WR = np.ascontiguousarray(WR, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float64)
    W = np.empty((x.size, 3))
    if lib().orc_exact_sample(_ptr(WL), _ptr(WR), float(gamma), float(x0), float(t), x.size, _ptr(x), _ptr(W)) != 0:
        raise ValueError("no exact solution")
    return W


def count_flops(c: Config) -> dict:
    """Floating-point operations of the scheme as defined (see oracle_capi.cpp)."""
    out = np.empty(6)
    if lib().orc_count_flops(ctypes.byref(c), _ptr(out)) != 0:
        raise ValueError("oracle rejected the configuration")
    keys = ["primitives", "convective_faces", "dissipative_faces", "divergence", "rhs_per_cell", "rk_combine"]
    return dict(zip(keys, out.tolist()))
