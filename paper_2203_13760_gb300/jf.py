"""ctypes binding of libjf.so (include/jf.h): argument marshalling only.

Every step of the path runs in the library's CUDA kernels; PyTorch supplies
device memory and streams.  There is no CPU fallback: if libjf.so cannot be
loaded, :func:`lib` raises.

Arrays are torch CUDA tensors, contiguous, shaped [5, nz, ny, nx] (x fastest),
float32 for ``dtype="f32"`` and float64 for ``dtype="f64"``.  Every call is
enqueued on ``torch.cuda.current_stream()``.
"""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libjf.so")

JF_OK, JF_ERR_ARG, JF_ERR_CUDA, JF_ERR_OOM, JF_ERR_NONPHYSICAL, JF_ERR_TIMEOUT, JF_ERR_UNSUPPORTED = 0, -1, -2, -3, -4, -5, -6
JF_F32, JF_F64 = 0, 1
PERIODIC, ZERO_GRADIENT, WALL = 0, 1, 2
_STATUS = {0: "JF_OK", -1: "JF_ERR_ARG", -2: "JF_ERR_CUDA", -3: "JF_ERR_OOM", -4: "JF_ERR_NONPHYSICAL",
           -5: "JF_ERR_TIMEOUT", -6: "JF_ERR_UNSUPPORTED"}


class JFError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


class Grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("lo", ctypes.c_double * 3), ("hi", ctypes.c_double * 3), ("bc", ctypes.c_int * 6)]


class GasParams(ctypes.Structure):
    _fields_ = [("gamma", ctypes.c_double), ("R", ctypes.c_double), ("mu", ctypes.c_double), ("Pr", ctypes.c_double)]


class Scheme(ctypes.Structure):
    _fields_ = [("dtype", ctypes.c_int), ("weno_eps", ctypes.c_double), ("cfl", ctypes.c_double),
                ("viscous", ctypes.c_int), ("heat", ctypes.c_int), ("signal_speed", ctypes.c_int),
                ("safe_recon", ctypes.c_int), ("flux", ctypes.c_int), ("recon", ctypes.c_int),
                ("integrator", ctypes.c_int)]


# scheme options of include/jf.h (0: the default configuration)
FLUX = {"hllc": 0, "hll": 1, "rusanov": 2, "roe": 3, "rusanov-nn": 4}
RECON = {"weno5-js": 0, "weno5-z": 1, "weno3-js": 2}
# parameters of the Rusanov-NN network (JF_NN_PARAMS): W1 [32][4], b1, W2 [32][32], b2, W3 [32][32], b3, W4 [32], b4
NN_HIDDEN = 32
NN_PARAMS = NN_HIDDEN * 4 + NN_HIDDEN + 2 * (NN_HIDDEN * NN_HIDDEN + NN_HIDDEN) + NN_HIDDEN + 1
SPEEDS = {"einfeldt": 0, "davis": 1, "toro": 2}
INTEGRATOR = {"rk3": 0, "rk2": 1, "euler": 2}


# name -> (restype, argtypes) of every entry point in include/jf.h
_VP, _I, _D = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
SIGNATURES = {
    "jf_init": (_I, [ctypes.POINTER(Grid), ctypes.POINTER(GasParams), ctypes.POINTER(Scheme), ctypes.POINTER(_VP)]),
    "jf_destroy": (_I, [_VP]),
    "jf_rhs": (_I, [_VP, _VP, _VP, _VP]),
    "jf_compute_dt": (_I, [_VP, _VP, _VP, _VP]),
    "jf_rk3_step": (_I, [_VP, _VP, _VP, _VP, _VP]),
    "jf_stage": (_I, [_VP, _VP, _VP, _VP, _D, _D, _VP, _VP]),
    "jf_rk3_run": (_I, [_VP, _VP, _I, _VP, _VP, _VP]),
    "jf_rk3_step_host": (_I, [_VP, ctypes.POINTER(_VP), ctypes.POINTER(_VP), _I, _VP, _VP]),
    "jf_rk3_step_vjp": (_I, [_VP, _VP, _VP, _VP, _VP, _VP]),
    "jf_rk3_step_keep": (_I, [_VP, _VP, _VP, _VP, _VP, _VP]),
    "jf_rk3_step_vjp_stages": (_I, [_VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP]),
    "jf_rk3_step_vjp_params": (_I, [_VP, _VP, _VP, _VP, _VP, _VP, _VP]),
    "jf_batch_step_vjp": (_I, [_VP, ctypes.POINTER(_VP), _VP, ctypes.POINTER(_VP), ctypes.POINTER(_VP),
                               ctypes.POINTER(_VP), _VP, _VP]),
    "jf_batch_param_grad_begin": (_I, [_VP, _I]),
    "jf_batch_param_grad_end": (_I, [_VP, _VP, _VP]),
    "jf_loss_density_l2": (_I, [_VP, _VP, _VP, _VP, _VP, _VP]),
    "jf_loss_primitive_mse": (_I, [_VP, _VP, _VP, ctypes.c_longlong, ctypes.c_longlong, _I, _VP, _VP, _VP]),
    "jf_batch_create": (_I, [ctypes.POINTER(Grid), _I, ctypes.POINTER(GasParams), ctypes.POINTER(Scheme),
                             ctypes.POINTER(_VP)]),
    "jf_batch_step": (_I, [_VP, ctypes.POINTER(_VP), _I, _VP, _VP]),
    "jf_batch_feed_forward": (_I, [_VP, ctypes.POINTER(_VP), ctypes.POINTER(_VP), _I, _VP, _VP]),
    "jf_set_variant": (_I, [_VP, _I]),
    "jf_set_nn": (_I, [_VP, _VP, _I]),
    "jf_variant_info": (_I, [_VP, _I, ctypes.c_char_p, _I]),
    "jf_auto_zchunk": (_I, [_I, _I, _I, _I, _I, _I, _I]),
    "jf_status_sync": (_I, [_VP]),
    "jf_last_error": (ctypes.c_char_p, [_VP]),
    "jf_version": (ctypes.c_char_p, []),
    "jf_fma_peak": (_I, [_I, _I, ctypes.POINTER(ctypes.c_double), _VP]),
    "jf_rk3_step_noalloc": (_I, [ctypes.POINTER(Grid), ctypes.POINTER(GasParams), ctypes.POINTER(Scheme), _VP, _VP,
                                 _VP, _VP]),
}

_lib = None
_lock = threading.Lock()


def lib():
    """Load libjf.so (raises if it is missing: there is no fallback path)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise ImportError(f"{LIB_PATH} is missing; build it with "
                                  "`python -c 'import __graft_entry__ as g; g.build()'`")
            L = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in SIGNATURES.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def _check(status: int, handle=None):
    if status != JF_OK:
        msg = lib().jf_last_error(handle)
        raise JFError(status, msg.decode() if msg else "")


def _stream():
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def auto_zchunk(n, tile=(32, 7), ctas_per_sm=2, sms=152):
    """Default planes per CTA of a 3D grid n = (nx, ny, nz) (jf_auto_zchunk;
    host logic, no GPU needed)."""
    return int(lib().jf_auto_zchunk(int(n[0]), int(n[1]), int(n[2]), int(tile[0]), int(tile[1]),
                                    int(ctas_per_sm), int(sms)))


def fma_peak(dtype="f32", iters=None):
    """Measured fused-multiply-add rate of the current device in FLOP/s
    (jf_fma_peak): the ALU roofline of the stage kernels.  iters defaults to
    a launch of roughly 30 ms (30000 loop trips in FP32, 500 in FP64)."""
    code = JF_F32 if dtype in ("f32", "float32") else JF_F64
    if iters is None:
        iters = 30000 if code == JF_F32 else 500
    out = ctypes.c_double(0.0)
    _check(lib().jf_fma_peak(code, int(iters), ctypes.byref(out), _stream()))
    return out.value


def _set_nn(obj, theta):
    """jf_set_nn for a Solver or Batch; keeps theta referenced while the
    handle may read it."""
    import torch
    if (not isinstance(theta, torch.Tensor) or not theta.is_cuda or theta.dtype != obj.dtype
            or not theta.is_contiguous() or theta.numel() != NN_PARAMS):
        raise ValueError(f"theta must be a contiguous CUDA {obj.dtype} tensor of {NN_PARAMS} values")
    _check(lib().jf_set_nn(obj.h, _ptr(theta), NN_PARAMS), obj.h)
    obj._nn = theta


def make_grid(n, lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0), bc=(1, 1, 1, 1, 1, 1)) -> Grid:
    n = tuple(int(x) for x in n) + (1,) * (3 - len(n))
    g = Grid()
    g.nx, g.ny, g.nz = n
    g.lo[:] = [float(x) for x in lo]
    g.hi[:] = [float(x) for x in hi]
    g.bc[:] = [int(x) for x in bc]
    return g


def make_scheme(dtype="f32", eps=1e-6, cfl=0.5, viscous=False, heat=False, safe=False, flux="hllc",
                recon="weno5-js", speeds="einfeldt", integrator="rk3") -> Scheme:
    s = Scheme()
    s.dtype = JF_F32 if dtype in ("f32", "float32") else JF_F64
    s.weno_eps, s.cfl = float(eps), float(cfl)
    s.viscous, s.heat, s.safe_recon = int(bool(viscous)), int(bool(heat)), int(bool(safe))
    s.signal_speed, s.flux, s.recon = SPEEDS[speeds], FLUX[flux], RECON[recon]
    s.integrator = INTEGRATOR[integrator]
    return s


class Solver:
    """One grid (jf_init).  Parameters mirror jf_grid / jf_gas / jf_scheme."""

    def __init__(self, n, lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0), bc=(1, 1, 1, 1, 1, 1), gamma=1.4, R=1.0,
                 mu=0.0, Pr=0.72, dtype="f32", eps=1e-6, cfl=0.5, viscous=False, heat=False, safe=False,
                 flux="hllc", recon="weno5-js", speeds="einfeldt", integrator="rk3", nn=None):
        import torch
        self.grid = make_grid(n, lo, hi, bc)
        self.gas = GasParams(float(gamma), float(R), float(mu), float(Pr))
        self.scheme = make_scheme(dtype, eps, cfl, viscous, heat, safe, flux, recon, speeds, integrator)
        self.dtype = torch.float32 if self.scheme.dtype == JF_F32 else torch.float64
        self.shape = (5, self.grid.nz, self.grid.ny, self.grid.nx)
        h = ctypes.c_void_p()
        _check(lib().jf_init(ctypes.byref(self.grid), ctypes.byref(self.gas), ctypes.byref(self.scheme),
                             ctypes.byref(h)))
        self.h = h
        self._nn = None
        if nn is not None:
            self.set_nn(nn)

    def set_nn(self, theta):
        """Rusanov-NN parameters (jf_set_nn): a CUDA tensor of NN_PARAMS values
        of the solver's dtype, read at every launch (update it in place)."""
        _set_nn(self, theta)

    @classmethod
    def from_case(cls, case, dtype="f32", **over):
        kw = case.params()
        kw.update(over)
        return cls(dtype=dtype, **kw)

    # -- helpers -------------------------------------------------------------
    def _field(self, t, name):
        import torch
        if not isinstance(t, torch.Tensor) or not t.is_cuda:
            raise TypeError(f"{name} must be a CUDA tensor")
        if t.dtype != self.dtype or tuple(t.shape) != self.shape or not t.is_contiguous():
            raise ValueError(f"{name} must be a contiguous {self.dtype} tensor of shape {self.shape}")
        return _ptr(t)

    def empty(self):
        import torch
        return torch.empty(self.shape, dtype=self.dtype, device="cuda")

    def scalar(self, value=0.0):
        import torch
        return torch.full((1,), float(value), dtype=torch.float64, device="cuda")

    # -- entry points ----------------------------------------------------------
    def rhs(self, U, out=None):
        out = self.empty() if out is None else out
        _check(lib().jf_rhs(self.h, self._field(U, "U"), self._field(out, "out"), _stream()), self.h)
        return out

    def compute_dt(self, U, out=None):
        out = self.scalar() if out is None else out
        _check(lib().jf_compute_dt(self.h, self._field(U, "U"), _ptr(out), _stream()), self.h)
        return out

    def rk3_step(self, U, dt=None, dt_used=None):
        """One RK3 step in place; dt: None (CFL) or a float64 CUDA tensor."""
        _check(lib().jf_rk3_step(self.h, self._field(U, "U"), _ptr(dt), _ptr(dt_used), _stream()), self.h)
        return U

    def step_host(self, U_in, U_out, dt=None):
        """Independent RK3 steps of host states (jf_rk3_step_host): U_in /
        U_out are lists of CPU tensors shaped like a state (pinned for
        overlap); U_out[k] receives one step of U_in[k]."""
        if len(U_in) != len(U_out):
            raise ValueError("one output per input state")
        for t_ in list(U_in) + list(U_out):
            if (t_.is_cuda or t_.dtype != self.dtype or tuple(t_.shape) != self.shape or not t_.is_contiguous()):
                raise ValueError(f"host states must be contiguous CPU {self.dtype} tensors of shape {self.shape}")
        n = len(U_in)
        ins = (ctypes.c_void_p * max(n, 1))(*[t_.data_ptr() for t_ in U_in])
        outs = (ctypes.c_void_p * max(n, 1))(*[t_.data_ptr() for t_ in U_out])
        _check(lib().jf_rk3_step_host(self.h, ins, outs, n, _ptr(dt), _stream()), self.h)
        return U_out

    def stage(self, Us, Un, out, a, b, dt):
        """out = a Un + b (Us + dt L(Us)); dt a float64 CUDA scalar tensor."""
        _check(lib().jf_stage(self.h, self._field(Us, "Us"), self._field(Un, "Un") if Un is not None else None,
                              self._field(out, "out"), float(a), float(b), _ptr(dt), _stream()), self.h)
        return out

    def run(self, U, nsteps, dt=None, dt_hist=None):
        """nsteps RK3 steps in place as one CUDA graph."""
        _check(lib().jf_rk3_run(self.h, self._field(U, "U"), int(nsteps), _ptr(dt), _ptr(dt_hist), _stream()),
               self.h)
        return U

    def rk3_step_vjp(self, Un, dt, lam_out, lam_in=None):
        lam_in = self.empty() if lam_in is None else lam_in
        _check(lib().jf_rk3_step_vjp(self.h, self._field(Un, "Un"), _ptr(dt), self._field(lam_out, "lam_out"),
                                     self._field(lam_in, "lam_in"), _stream()), self.h)
        return lam_in

    def supports_stage_vjp(self):
        """True when rk3_step_vjp_stages serves this solver: the default
        scheme (HLLC, Einfeldt speeds, WENO5-JS, TVD-RK3) without walls."""
        s = self.scheme
        return (s.flux == FLUX["hllc"] and s.recon == RECON["weno5-js"] and s.signal_speed == SPEEDS["einfeldt"]
                and s.integrator == INTEGRATOR["rk3"] and WALL not in list(self.grid.bc))

    def rk3_step_keep(self, U, dt, U1, U2):
        """One fixed-dt RK3 step of U in place (as rk3_step), writing the stage
        states U1 and U2 into the given tensors (jf_rk3_step_keep)."""
        _check(lib().jf_rk3_step_keep(self.h, self._field(U, "U"), _ptr(dt), self._field(U1, "U1"),
                                      self._field(U2, "U2"), _stream()), self.h)
        return U

    def rk3_step_vjp_stages(self, Un, U1, U2, dt, lam_out, lam_in=None):
        """rk3_step_vjp from the kept stage states of the step
        (jf_rk3_step_vjp_stages: no recomputation)."""
        lam_in = self.empty() if lam_in is None else lam_in
        _check(lib().jf_rk3_step_vjp_stages(self.h, self._field(Un, "Un"), self._field(U1, "U1"),
                                            self._field(U2, "U2"), _ptr(dt), self._field(lam_out, "lam_out"),
                                            self._field(lam_in, "lam_in"), _stream()), self.h)
        return lam_in

    def rk3_step_vjp_params(self, Un, dt, lam_out, lam_in=None, theta_bar=None):
        """Adjoint of one step of the Rusanov-NN scheme: returns (lam_in,
        theta_bar) with theta_bar += (dU^{n+1}/dtheta)^T lam_out (a zero
        tensor of NN_PARAMS values is made when theta_bar is None)."""
        import torch
        lam_in = self.empty() if lam_in is None else lam_in
        if theta_bar is None:
            theta_bar = torch.zeros(NN_PARAMS, dtype=self.dtype, device="cuda")
        if (theta_bar.dtype != self.dtype or not theta_bar.is_cuda or not theta_bar.is_contiguous()
                or theta_bar.numel() != NN_PARAMS):
            raise ValueError(f"theta_bar must be a contiguous CUDA {self.dtype} tensor of {NN_PARAMS} values")
        _check(lib().jf_rk3_step_vjp_params(self.h, self._field(Un, "Un"), _ptr(dt), self._field(lam_out, "lam_out"),
                                            self._field(lam_in, "lam_in"), _ptr(theta_bar), _stream()), self.h)
        return lam_in, theta_bar

    def loss_density_l2(self, U, target, loss=None, seed=None, want_seed=True):
        import torch
        loss = self.scalar() if loss is None else loss
        if want_seed and seed is None:
            seed = self.empty()
        if target.dtype != self.dtype or target.numel() != self.grid.nx * self.grid.ny * self.grid.nz:
            raise ValueError("target must hold nx*ny*nz densities of the solver's dtype")
        _check(lib().jf_loss_density_l2(self.h, self._field(U, "U"), _ptr(target.contiguous()), _ptr(loss),
                                        _ptr(seed) if want_seed else None, _stream()), self.h)
        return loss, seed

    def set_variant(self, v):
        _check(lib().jf_set_variant(self.h, int(v)), self.h)

    def variants(self):
        buf = ctypes.create_string_buffer(128)
        n = lib().jf_variant_info(self.h, 0, buf, 128)
        out = []
        for v in range(max(n, 0)):
            lib().jf_variant_info(self.h, v, buf, 128)
            out.append(buf.value.decode())
        return out

    def sync(self):
        """Wait for the device and raise if a kernel flagged a non-physical state."""
        _check(lib().jf_status_sync(self.h), self.h)

    def close(self):
        if getattr(self, "h", None):
            lib().jf_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def loss_primitive_mse(owner, U, Uref, ncomp=4, loss=None, grad=None, want_grad=True):
    """Section 7.4 training loss (jf_loss_primitive_mse): the mean squared
    difference of the primitive variables of U and Uref, contiguous CUDA
    tensors of states (..., 5, nz, ny, nx) in the dtype of `owner` (a Solver
    or a Batch, which supplies gamma and the reduction scratch).  ncomp = 4:
    (rho, u, v, p); 5: (rho, u, v, w, p).  Returns (loss, dloss/dU or None)."""
    import torch
    if (not U.is_cuda or U.dtype != owner.dtype or U.shape != Uref.shape or U.dtype != Uref.dtype
            or U.shape[-4] != 5):
        raise ValueError("U and Uref must be CUDA tensors of states (..., 5, nz, ny, nx) in the owner's dtype")
    U = U.contiguous()
    Uref = Uref.contiguous()
    ncells = int(U.shape[-1] * U.shape[-2] * U.shape[-3])
    nstates = int(U.numel() // (5 * ncells))
    loss = torch.empty(1, dtype=torch.float64, device="cuda") if loss is None else loss
    if want_grad and grad is None:
        grad = torch.empty_like(U)
    _check(lib().jf_loss_primitive_mse(owner.h, _ptr(U), _ptr(Uref), nstates, ncells, int(ncomp), _ptr(loss),
                                       _ptr(grad) if want_grad else None, _stream()), owner.h)
    return loss, (grad if want_grad else None)


class Batch:
    """Many independent simulations of uneven sizes (jf_batch_create)."""

    def __init__(self, grids, gamma=1.4, R=1.0, mu=0.0, Pr=0.72, dtype="f32", eps=1e-6, cfl=0.5,
                 viscous=False, heat=False, safe=False, flux="hllc", recon="weno5-js", speeds="einfeldt",
                 integrator="rk3", nn=None):
        import torch
        self.grids = (Grid * len(grids))(*[make_grid(**g) if isinstance(g, dict) else g for g in grids])
        self.nsim = len(grids)
        self.gas = GasParams(float(gamma), float(R), float(mu), float(Pr))
        self.scheme = make_scheme(dtype, eps, cfl, viscous, heat, safe, flux, recon, speeds, integrator)
        self.dtype = torch.float32 if self.scheme.dtype == JF_F32 else torch.float64
        h = ctypes.c_void_p()
        _check(lib().jf_batch_create(self.grids, self.nsim, ctypes.byref(self.gas), ctypes.byref(self.scheme),
                                     ctypes.byref(h)))
        self.h = h
        self._nn = None
        if nn is not None:
            self.set_nn(nn)

    def supports_step_vjp(self):
        """Whether jf_batch_step_vjp covers this batch's scheme (inviscid,
        WENO5-JS / WENO3-JS, HLLC with Einfeldt speeds or Rusanov-NN)."""
        s = self.scheme
        visc = bool(s.viscous or s.heat) and self.gas.mu > 0
        flux_ok = s.flux == FLUX["rusanov-nn"] or (s.flux == FLUX["hllc"] and s.signal_speed == SPEEDS["einfeldt"])
        return (not visc) and s.recon in (RECON["weno5-js"], RECON["weno3-js"]) and flux_ok

    def set_nn(self, theta):
        """Rusanov-NN parameters of every simulation (jf_set_nn; also given to
        the cached single-grid solvers)."""
        _set_nn(self, theta)
        for s in self.__dict__.get("_solvers", {}).values():
            s.set_nn(theta)

    def solver(self, i):
        """A single-grid Solver with simulation i's grid and this batch's gas and
        scheme (cached; used by the batch's adjoint)."""
        cache = self.__dict__.setdefault("_solvers", {})
        if i not in cache:
            g, s, gas = self.grids[i], self.scheme, self.gas
            names = {v: k for k, v in FLUX.items()}, {v: k for k, v in RECON.items()}, \
                {v: k for k, v in SPEEDS.items()}, {v: k for k, v in INTEGRATOR.items()}
            cache[i] = Solver((g.nx, g.ny, g.nz), tuple(g.lo), tuple(g.hi), tuple(g.bc), gas.gamma, gas.R, gas.mu,
                              gas.Pr, "f32" if s.dtype == JF_F32 else "f64", s.weno_eps, s.cfl, bool(s.viscous),
                              bool(s.heat), bool(s.safe_recon), names[0][s.flux], names[1][s.recon],
                              names[2][s.signal_speed], names[3][s.integrator], nn=self._nn)
        return cache[i]

    def _check_fields(self, Us):
        if len(Us) != self.nsim:
            raise ValueError("one field per simulation")
        for i, (U, g) in enumerate(zip(Us, self.grids)):
            if (not U.is_cuda or U.dtype != self.dtype or not U.is_contiguous()
                    or tuple(U.shape) != (5, g.nz, g.ny, g.nx)):
                raise ValueError(f"field {i} has the wrong shape / dtype / device")

    def feed_forward(self, U0s, nsteps, dt):
        """Section 4.5 feed_forward: per simulation the trajectory tensor
        (nsteps + 1, 5, nz, ny, nx), slot 0 = U0, slot t = t steps of the fixed
        step dt (a float, or one value per simulation)."""
        import torch
        self._check_fields(U0s)
        dts = [float(dt)] * self.nsim if not hasattr(dt, "__len__") else [float(x) for x in dt]
        if len(dts) != self.nsim:
            raise ValueError("one dt per simulation")
        dt_dev = torch.tensor(dts, dtype=torch.float64, device="cuda")
        trajs = [torch.empty((int(nsteps) + 1,) + tuple(U.shape), dtype=self.dtype, device="cuda") for U in U0s]
        u0 = (ctypes.c_void_p * self.nsim)(*[U.data_ptr() for U in U0s])
        tp = (ctypes.c_void_p * self.nsim)(*[T.data_ptr() for T in trajs])
        _check(lib().jf_batch_feed_forward(self.h, u0, tp, int(nsteps), _ptr(dt_dev), _stream()), self.h)
        return trajs

    def step_vjp(self, Uns, dt, lams, lam_ins=None, adds=None, theta_bar=None):
        """Adjoint of one fixed-dt step of every simulation (jf_batch_step_vjp):
        lam_ins[i] = J_i^T lams[i] + adds[i]; theta_bar (Rusanov-NN) is added to.
        dt: a float64 CUDA tensor of one step per simulation."""
        import torch
        self._check_fields(Uns)
        self._check_fields(lams)
        lam_ins = [torch.empty_like(L) for L in lams] if lam_ins is None else lam_ins
        self._check_fields(lam_ins)
        if adds is not None:
            self._check_fields(adds)
        arr = lambda ts: (ctypes.c_void_p * self.nsim)(*[x.data_ptr() for x in ts])  # noqa: E731
        if (dt.dtype != torch.float64 or not dt.is_cuda or dt.numel() != self.nsim):
            raise ValueError("dt must be a float64 CUDA tensor of one step per simulation")
        _check(lib().jf_batch_step_vjp(self.h, arr(Uns), _ptr(dt), arr(lams), arr(lam_ins),
                                       arr(adds) if adds is not None else None,
                                       _ptr(theta_bar) if theta_bar is not None else None, _stream()), self.h)
        return lam_ins

    def param_grad_begin(self, max_steps):
        """Keep the face records of the next (at most max_steps) step_vjp calls
        with theta_bar instead of adding to theta_bar
        (jf_batch_param_grad_begin)."""
        _check(lib().jf_batch_param_grad_begin(self.h, int(max_steps)), self.h)

    def param_grad_end(self, theta_bar):
        """Add the parameter gradient of every kept record to theta_bar in one
        launch (jf_batch_param_grad_end)."""
        if (theta_bar.dtype != self.dtype or not theta_bar.is_cuda or not theta_bar.is_contiguous()
                or theta_bar.numel() != NN_PARAMS):
            raise ValueError(f"theta_bar must be a contiguous CUDA {self.dtype} tensor of {NN_PARAMS} values")
        _check(lib().jf_batch_param_grad_end(self.h, _ptr(theta_bar), _stream()), self.h)
        return theta_bar

    def step(self, Us, nsteps, dt_out=None):
        import torch
        self._check_fields(Us)
        ptrs = (ctypes.c_void_p * self.nsim)(*[U.data_ptr() for U in Us])
        dt_out = torch.zeros(self.nsim, dtype=torch.float64, device="cuda") if dt_out is None else dt_out
        _check(lib().jf_batch_step(self.h, ptrs, int(nsteps), _ptr(dt_out), _stream()), self.h)
        return dt_out

    def set_variant(self, v):
        _check(lib().jf_set_variant(self.h, int(v)), self.h)

    def variants(self):
        buf = ctypes.create_string_buffer(128)
        n = lib().jf_variant_info(self.h, 0, buf, 128)
        out = []
        for v in range(max(n, 0)):
            lib().jf_variant_info(self.h, v, buf, 128)
            out.append(buf.value.decode())
        return out

    def sync(self):
        _check(lib().jf_status_sync(self.h), self.h)

    def close(self):
        for s in self.__dict__.pop("_solvers", {}).values():
            s.close()
        if getattr(self, "h", None):
            lib().jf_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
