"""Seeded synthetic initial states shaped like the paper's test cases.

This is the one module that both the GPU path's tests / benchmark and the
oracle consume.  It builds initial data only: primitive fields
W = [rho, u, v, w, p] on cell centres (or cell averages where the paper uses
them), turned into the conservative state U = [rho, rho u, rho v, rho w, E]
with E = p / (gamma - 1) + rho |u|^2 / 2 (Section 2 of the paper).  It holds
none of the right-hand side arithmetic (reconstruction, fluxes, time
integration).

Every state is returned as a float64 array U[5][nz][ny][nx] (x fastest)
inside a :class:`Case` that also carries the grid, gas and scheme parameters.
Random draws come from ``numpy.random.default_rng(seed)`` in the order each
docstring states.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

DEFAULT_SEED = 2203
PERIODIC = 0
ZERO_GRADIENT = 1
WALL = 2
NN_HIDDEN = 32


@dataclasses.dataclass
class Case:
    name: str
    n: tuple            # (nx, ny, nz); an axis with 1 cell is inactive
    lo: tuple
    hi: tuple
    bc: tuple           # (x-lo, x-hi, y-lo, y-hi, z-lo, z-hi)
    U: np.ndarray       # float64 [5][nz][ny][nx]
    gamma: float = 1.4
    R: float = 1.0
    mu: float = 0.0
    Pr: float = 0.72
    viscous: bool = False
    heat: bool = False
    cfl: float = 0.5
    eps: float = 1e-6
    flux: str = "hllc"          # Riemann solver: hllc | hll | rusanov
    recon: str = "weno5-js"     # reconstruction: weno5-js | weno5-z
    speeds: str = "einfeldt"    # signal speeds: einfeldt | davis | toro
    integrator: str = "rk3"     # time integration: rk3 | rk2 | euler
    dt: float = 0.0     # fixed time step if > 0

    @property
    def cells(self) -> int:
        return int(self.n[0] * self.n[1] * self.n[2])

    def params(self) -> dict:
        """Grid / gas / scheme parameters as keyword arguments."""
        return dict(n=self.n, lo=self.lo, hi=self.hi, bc=self.bc, gamma=self.gamma, R=self.R,
                    mu=self.mu, Pr=self.Pr, eps=self.eps, cfl=self.cfl, viscous=self.viscous,
                    heat=self.heat, flux=self.flux, recon=self.recon, speeds=self.speeds,
                    integrator=self.integrator)


def conservative(rho, u, v, w, p, gamma: float) -> np.ndarray:
    """U = [rho, rho u, rho v, rho w, p/(gamma-1) + rho |u|^2 / 2] (Section 2)."""
    rho, u, v, w, p = np.broadcast_arrays(*(np.asarray(a, dtype=np.float64) for a in (rho, u, v, w, p)))
    E = p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v + w * w)
    return np.stack([rho, rho * u, rho * v, rho * w, E]).astype(np.float64)


def centres(n: int, lo: float, hi: float) -> np.ndarray:
    h = (hi - lo) / n
    return lo + (np.arange(n) + 0.5) * h


def _mesh(n, lo, hi):
    """Cell-centre coordinate arrays of shape [nz][ny][nx]."""
    x = centres(n[0], lo[0], hi[0])
    y = centres(n[1], lo[1], hi[1])
    z = centres(n[2], lo[2], hi[2])
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    return X, Y, Z


# ---------------------------------------------------------------------------
def sod(n: int = 200, gamma: float = 1.4) -> Case:
    """Sod shock tube on [0, 1] (Appendix A case file): left (1, 0, 1), right
    (0.125, 0, 0.1), diaphragm at x = 0.5 (cell centres, so no centre lies on
    it for even n), zero-gradient ("transmissive") ends."""
    x = centres(n, 0.0, 1.0)
    left = x <= 0.5
    rho = np.where(left, 1.0, 0.125)
    p = np.where(left, 1.0, 0.1)
    U = conservative(rho, 0.0, 0.0, 0.0, p, gamma).reshape(5, 1, 1, n)
    return Case("sod", (n, 1, 1), (0.0, 0.0, 0.0), (1.0, 1.0, 1.0), (1, 1, 1, 1, 1, 1), U, gamma=gamma)


def riemann_1d(n: int, WL, WR, x0: float = 0.5, length: float = 1.0, gamma: float = 1.4) -> Case:
    """General 1D Riemann problem, W = (rho, u, p) left / right of x0."""
    x = centres(n, 0.0, length)
    left = x <= x0
    rho = np.where(left, WL[0], WR[0])
    u = np.where(left, WL[1], WR[1])
    p = np.where(left, WL[2], WR[2])
    U = conservative(rho, u, 0.0, 0.0, p, gamma).reshape(5, 1, 1, n)
    return Case("riemann1d", (n, 1, 1), (0.0, 0.0, 0.0), (length, 1.0, 1.0), (1, 1, 1, 1, 1, 1), U, gamma=gamma)


# Sod's shock tube (Sod 1978; the Appendix A case): (rho, u, p) left / right.
SOD_LEFT = (1.0, 0.0, 1.0)
SOD_RIGHT = (0.125, 0.0, 0.1)

# Lax's shock tube (Lax 1954), with the states tabulated by Shu & Osher (1989,
# "Efficient implementation of essentially non-oscillatory shock-capturing
# schemes II", Example 2): (rho, u, p) = (0.445, 0.698, 3.528) left and
# (0.5, 0, 0.571) right of x = 0.5 on [0, 1]; run to t = 0.14.
LAX_LEFT = (0.445, 0.698, 3.528)
LAX_RIGHT = (0.5, 0.0, 0.571)
LAX_END_TIME = 0.14


def lax(n: int = 100, gamma: float = 1.4) -> Case:
    """Lax shock tube of Section 5.1.2 (domain [0, 1], N = 100, t = 0.14,
    zero-gradient ends).  The paper only cites Lax (1954) for the states, so
    the classic ones above are used."""
    case = riemann_1d(n, LAX_LEFT, LAX_RIGHT, gamma=gamma)
    case.name = "lax"
    return case


def sine_advection(n: int, gamma: float = 1.4) -> Case:
    """Section 5.1.1 convergence case: rho = 1.5 + sin(2 pi x) as exact cell
    averages, u = 1, p = 1, periodic on [0, 1]."""
    h = 1.0 / n
    xf = np.arange(n + 1) * h
    rho = 1.5 - (np.cos(2 * np.pi * xf[1:]) - np.cos(2 * np.pi * xf[:-1])) / (2 * np.pi * h)
    U = conservative(rho, 1.0, 0.0, 0.0, 1.0, gamma).reshape(5, 1, 1, n)
    return Case("sine", (n, 1, 1), (0.0, 0.0, 0.0), (1.0, 1.0, 1.0), (0,) * 6, U, gamma=gamma)


def sine_exact_average(n: int, t: float) -> np.ndarray:
    """Exact cell averages of rho(x, t) = 1.5 + sin(2 pi (x - t))."""
    h = 1.0 / n
    xf = np.arange(n + 1) * h - t
    return 1.5 - (np.cos(2 * np.pi * xf[1:]) - np.cos(2 * np.pi * xf[:-1])) / (2 * np.pi * h)


def taylor_green(n: int, Ma: float = 0.1, Re: float = 1600.0, gamma: float = 1.4, Pr: float = 0.72,
                 viscous: bool = True) -> Case:
    """Compressible Taylor-Green vortex on [0, 2 pi]^3, periodic (Section 6
    benchmark; textbook initial field, point values at cell centres):
      u = sin x cos y cos z, v = -cos x sin y cos z, w = 0,
      p = p0 + (cos 2x + cos 2y)(cos 2z + 2) / 16, p0 = 1 / (gamma Ma^2),
      rho = p / (R T0), T0 = p0 (rho0 = U0 = R = 1), mu = 1 / Re."""
    L = 2 * np.pi
    X, Y, Z = _mesh((n, n, n), (0, 0, 0), (L, L, L))
    p0 = 1.0 / (gamma * Ma * Ma)
    u = np.sin(X) * np.cos(Y) * np.cos(Z)
    v = -np.cos(X) * np.sin(Y) * np.cos(Z)
    p = p0 + (np.cos(2 * X) + np.cos(2 * Y)) * (np.cos(2 * Z) + 2.0) / 16.0
    rho = p / p0
    U = conservative(rho, u, v, 0.0, p, gamma)
    return Case(f"tgv{n}", (n, n, n), (0.0, 0.0, 0.0), (L, L, L), (0,) * 6, U, gamma=gamma,
                mu=(1.0 / Re) if viscous else 0.0, Pr=Pr, viscous=viscous, heat=viscous)


def solenoidal_turbulence(n: int, Mt: float = 0.3, k0: float = 4.0, seed: int = DEFAULT_SEED,
                          gamma: float = 1.4, device=None) -> Case:
    """Inviscid periodic box [0, 2 pi]^3 with rho = 1, p = 1/gamma (c = 1) and a
    random-phase solenoidal velocity with energy spectrum
    E(k) ~ k^4 exp(-2 (k/k0)^2) (the shape of the paper's decaying-turbulence
    initial spectrum, Section 5.1.4), scaled so that sqrt(<|u|^2>) / c = Mt.

    Draws: three standard-normal complex arrays (real parts, then imaginary
    parts, for u, v, w in that order) of shape (n, n, n) from
    default_rng(seed); each Fourier coefficient vector is projected onto the
    plane normal to k and scaled by k exp(-(k/k0)^2) (so that the shell energy
    goes as E(k)); the velocity is the real part of the inverse FFT.

    ``device`` (a torch device) builds the field with torch.fft there, for
    large n; the draws are the same."""
    rng = np.random.default_rng(seed)
    if device is None:
        kk = np.fft.fftfreq(n, d=1.0 / n)
        KZ, KY, KX = np.meshgrid(kk, kk, kk, indexing="ij")
        K2 = KX * KX + KY * KY + KZ * KZ
        Kmag = np.sqrt(K2)
        amp = Kmag * np.exp(-(Kmag / k0) ** 2)
        K2s = np.where(K2 == 0, 1.0, K2)
        c = [rng.standard_normal((n, n, n)) + 0j for _ in range(3)]
        for a in range(3):
            c[a] = c[a] + 1j * rng.standard_normal((n, n, n))
        kdotc = KX * c[0] + KY * c[1] + KZ * c[2]
        vel = []
        for a, Ka in enumerate((KX, KY, KZ)):
            ca = (c[a] - Ka * kdotc / K2s) * amp
            vel.append(np.real(np.fft.ifftn(ca)))
        u, v, w = vel
    else:
        import torch
        kk = torch.fft.fftfreq(n, d=1.0 / n, device=device, dtype=torch.float64)
        KZ, KY, KX = torch.meshgrid(kk, kk, kk, indexing="ij")
        K2 = KX * KX + KY * KY + KZ * KZ
        Kmag = torch.sqrt(K2)
        amp = Kmag * torch.exp(-(Kmag / k0) ** 2)
        K2s = torch.where(K2 == 0, torch.ones_like(K2), K2)
        re = [torch.from_numpy(rng.standard_normal((n, n, n))).to(device) for _ in range(3)]
        im = [torch.from_numpy(rng.standard_normal((n, n, n))).to(device) for _ in range(3)]
        c = [torch.complex(re[a], im[a]) for a in range(3)]
        kdotc = KX * c[0] + KY * c[1] + KZ * c[2]
        vel = []
        for a, Ka in enumerate((KX, KY, KZ)):
            ca = (c[a] - Ka * kdotc / K2s) * amp
            vel.append(torch.fft.ifftn(ca).real.cpu().numpy())
        u, v, w = vel
    rms = math.sqrt(float(np.mean(u * u + v * v + w * w)))
    s = Mt / rms  # c = 1
    u, v, w = u * s, v * s, w * s
    L = 2 * np.pi
    U = conservative(1.0, u, v, w, 1.0 / gamma, gamma)
    return Case(f"hit{n}", (n, n, n), (0.0, 0.0, 0.0), (L, L, L), (0,) * 6, U, gamma=gamma)


def four_quadrant_batch(nsim: int = 64, sides=(64, 128, 256, 512), seed: int = DEFAULT_SEED,
                        gamma: float = 1.4) -> list:
    """Batched 2D four-quadrant Riemann problems on [0, 1]^2 with zero-gradient
    boundaries, split at (0.5, 0.5).

    Draws from default_rng(seed), per simulation in order: the side (uniform
    over ``sides``), then for the quadrants NE, NW, SW, SE in that order:
    rho ~ U[0.1, 1.5], u ~ U[-1, 1], v ~ U[-1, 1], p ~ U[0.1, 1.5]."""
    rng = np.random.default_rng(seed)
    cases = []
    for s in range(nsim):
        side = int(sides[int(rng.integers(0, len(sides)))])
        states = []
        for _ in range(4):
            rho = rng.uniform(0.1, 1.5)
            u = rng.uniform(-1.0, 1.0)
            v = rng.uniform(-1.0, 1.0)
            p = rng.uniform(0.1, 1.5)
            states.append((rho, u, v, p))
        X, Y, _ = _mesh((side, side, 1), (0, 0, 0), (1, 1, 1))
        east, north = X > 0.5, Y > 0.5
        quad = np.where(north, np.where(east, 0, 1), np.where(east, 3, 2))  # NE, NW, SW, SE
        W = np.zeros((4,) + X.shape)
        for q, st in enumerate(states):
            for m in range(4):
                W[m] = np.where(quad == q, st[m], W[m])
        U = conservative(W[0], W[1], W[2], 0.0, W[3], gamma)
        cases.append(Case(f"quad{s}_{side}", (side, side, 1), (0.0, 0.0, 0.0), (1.0, 1.0, 1.0),
                          (1, 1, 1, 1, 1, 1), U, gamma=gamma))
    return cases


def kelvin_helmholtz(n: int = 256, seed: int = DEFAULT_SEED, Re: float = 1e4, gamma: float = 1.4,
                     Pr: float = 0.72, amplitude: float = 1e-2, delta: float = 0.05) -> Case:
    """Periodic double shear layer on [0, 1]^2: rho = 1, p = 2.5,
      u = 0.5 [tanh((y - 1/4)/delta) - tanh((y - 3/4)/delta) - 1],
      v = amplitude * P(x) * [exp(-(y - 1/4)^2/delta^2) + exp(-(y - 3/4)^2/delta^2)],
      P(x) = sum_{k=1..4} a_k sin(2 pi k x + phi_k) / sum_k a_k,
    with draws from default_rng(seed): a_1..a_4 ~ U[0, 1], then
    phi_1..phi_4 ~ U[0, 2 pi).  mu = 1/Re; heat flux with Prandtl number Pr."""
    rng = np.random.default_rng(seed)
    a = rng.uniform(0.0, 1.0, 4)
    phi = rng.uniform(0.0, 2 * np.pi, 4)
    X, Y, _ = _mesh((n, n, 1), (0, 0, 0), (1, 1, 1))
    u = 0.5 * (np.tanh((Y - 0.25) / delta) - np.tanh((Y - 0.75) / delta) - 1.0)
    P = sum(a[k] * np.sin(2 * np.pi * (k + 1) * X + phi[k]) for k in range(4)) / a.sum()
    v = amplitude * P * (np.exp(-((Y - 0.25) / delta) ** 2) + np.exp(-((Y - 0.75) / delta) ** 2))
    U = conservative(1.0, u, v, 0.0, 2.5, gamma)
    return Case(f"kh{n}", (n, n, 1), (0.0, 0.0, 0.0), (1.0, 1.0, 1.0), (0,) * 6, U, gamma=gamma,
                mu=1.0 / Re, Pr=Pr, viscous=True, heat=True)


def moving_shock(Ms: float = 2.0, n: int = 64, length: float = 4.0, x_shock: float = 1.0,
                 gamma: float = 1.4):
    """Single right-running shock of Mach number Ms into (rho, u, p) = (1, 0, 1)
    (Section 7.3 gradient test), zero-gradient ends.  The post-shock state is
    given by the Rankine-Hugoniot relations,
      p2 = 1 + 2 gamma/(gamma+1) (Ms^2 - 1),
      rho2 = (gamma+1) Ms^2 / ((gamma-1) Ms^2 + 2),
      u2 = c1 2/(gamma+1) (Ms - 1/Ms),  c1 = sqrt(gamma).
    Returns (case, dU/dMs), the second array being the exact derivative of the
    initial state with respect to Ms."""
    c1 = math.sqrt(gamma)
    M2 = Ms * Ms
    p2 = 1.0 + 2.0 * gamma / (gamma + 1.0) * (M2 - 1.0)
    dp2 = 4.0 * gamma / (gamma + 1.0) * Ms
    den = (gamma - 1.0) * M2 + 2.0
    rho2 = (gamma + 1.0) * M2 / den
    drho2 = (gamma + 1.0) * (2.0 * Ms * den - M2 * 2.0 * (gamma - 1.0) * Ms) / (den * den)
    u2 = c1 * 2.0 / (gamma + 1.0) * (Ms - 1.0 / Ms)
    du2 = c1 * 2.0 / (gamma + 1.0) * (1.0 + 1.0 / M2)
    x = centres(n, 0.0, length)
    behind = x <= x_shock
    rho = np.where(behind, rho2, 1.0)
    u = np.where(behind, u2, 0.0)
    p = np.where(behind, p2, 1.0)
    U = conservative(rho, u, 0.0, 0.0, p, gamma).reshape(5, 1, 1, n)
    # derivative of U = [rho, rho u, 0, 0, p/(g-1) + rho u^2 / 2] behind the shock
    dU = np.zeros_like(U)
    b = behind.reshape(1, 1, n)
    dU[0] = np.where(b, drho2, 0.0)
    dU[1] = np.where(b, drho2 * u2 + rho2 * du2, 0.0)
    dU[4] = np.where(b, dp2 / (gamma - 1.0) + 0.5 * drho2 * u2 * u2 + rho2 * u2 * du2, 0.0)
    case = Case("shock", (n, 1, 1), (0.0, 0.0, 0.0), (length, 1.0, 1.0), (1, 1, 1, 1, 1, 1), U, gamma=gamma)
    return case, dU


def random_smooth(n, seed: int = DEFAULT_SEED, bc=None, modes: int = 3, mach: float = 0.5,
                  gamma: float = 1.4, lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0), viscous: bool = False,
                  mu: float = 0.0) -> Case:
    """Smooth random state for parity tests: each primitive is a constant plus
    ``modes`` random Fourier modes per axis (periodic in the unit cell).

    Draws from default_rng(seed), for rho, u, v, w, p in order and for each
    active axis and mode: amplitude ~ U[0, 1], phase ~ U[0, 2 pi).  rho and p
    lie in [0.5, 1.5]; velocities in [-mach, mach] (sound speed ~ 1.2)."""
    n = tuple(int(x) for x in n) + (1,) * (3 - len(n))
    rng = np.random.default_rng(seed)
    X, Y, Z = _mesh(n, lo, hi)
    coords = (X, Y, Z)
    fields = []
    for comp in range(5):
        f = np.zeros_like(X)
        norm = 0.0
        for d in range(3):
            if n[d] == 1:
                continue
            for m in range(1, modes + 1):
                amp = rng.uniform(0.0, 1.0)
                ph = rng.uniform(0.0, 2 * np.pi)
                L = hi[d] - lo[d]
                f = f + amp * np.sin(2 * np.pi * m * (coords[d] - lo[d]) / L + ph)
                norm += amp
        f = f / max(norm, 1e-30)  # in [-1, 1]
        fields.append(f)
    rho = 1.0 + 0.5 * fields[0]
    u, v, w = (mach * fields[1], mach * fields[2], mach * fields[3])
    p = 1.0 + 0.5 * fields[4]
    if bc is None:
        bc = (0,) * 6
    U = conservative(rho, u, v, w, p, gamma)
    return Case("smooth", n, tuple(lo), tuple(hi), tuple(bc), U, gamma=gamma, viscous=viscous,
                heat=viscous, mu=mu)


def random_blocks(n, seed: int = DEFAULT_SEED, bc=None, blocks: int = 3, gamma: float = 1.4,
                  speed: float = 2.0) -> Case:
    """Piecewise-constant random state (discontinuities in every field,
    supersonic regions) for parity tests of every HLLC branch: the domain is
    cut into ``blocks`` slabs per active axis, each block gets
    rho ~ U[0.2, 2], u, v, w ~ U[-speed, speed], p ~ U[0.2, 2] drawn from
    default_rng(seed) block by block (x fastest), components in that order."""
    n = tuple(int(x) for x in n) + (1,) * (3 - len(n))
    rng = np.random.default_rng(seed)
    nb = [blocks if n[d] > 1 else 1 for d in range(3)]
    idx = [np.minimum(np.arange(n[d]) * nb[d] // n[d], nb[d] - 1) for d in range(3)]
    table = np.zeros((nb[2], nb[1], nb[0], 5))
    for bz in range(nb[2]):
        for by in range(nb[1]):
            for bx in range(nb[0]):
                table[bz, by, bx] = [rng.uniform(0.2, 2.0), rng.uniform(-speed, speed),
                                     rng.uniform(-speed, speed), rng.uniform(-speed, speed),
                                     rng.uniform(0.2, 2.0)]
    W = table[np.ix_(idx[2], idx[1], idx[0])]  # [nz][ny][nx][5]
    W = np.moveaxis(W, -1, 0)
    if bc is None:
        bc = (1,) * 6
    U = conservative(W[0], W[1], W[2], W[3], W[4], gamma)
    return Case("blocks", n, (0.0, 0.0, 0.0), (1.0, 1.0, 1.0), tuple(bc), U, gamma=gamma)


def implosion(n: int = 128, gamma: float = 1.4) -> Case:
    """Section 7.4's implosion on [0, 1]^2: (rho, u, v, p) = (0.14, 0, 0,
    0.125) where x + y <= 0.15 and (1, 0, 0, 1) elsewhere, evaluated at cell
    centres; slip walls on all four sides (the shock reflects off the walls
    of the lower-left corner); the ground-truth scheme of the section:
    WENO3-JS, HLLC, TVD-RK2 with the fixed step 2.5e-4."""
    x = centres(n, 0.0, 1.0)
    X, Y = np.meshgrid(x, x, indexing="xy")
    inner = X + Y <= 0.15
    rho = np.where(inner, 0.14, 1.0)
    p = np.where(inner, 0.125, 1.0)
    U = conservative(rho, 0.0, 0.0, 0.0, p, gamma).reshape(5, 1, n, n)
    return Case("implosion", (n, n, 1), (0.0, 0.0, 0.0), (1.0, 1.0, 1.0), (WALL, WALL, WALL, WALL, 1, 1), U,
                gamma=gamma, recon="weno3-js", integrator="rk2", dt=2.5e-4)


def nn_params(seed: int = DEFAULT_SEED, alpha: float = 2.0, spread: float = 0.1) -> np.ndarray:
    """Seeded parameters of the Rusanov-NN network (Section 7.4) in the flat
    layout W1 [32][4], b1, W2 [32][32], b2, W3 [32][32], b3, W4 [32], b4
    (row-major, outputs by inputs): Gaussian weights of variance 2 / fan-in
    (He initialisation) and biases of standard deviation 0.1 for the hidden
    layers, output weights of standard deviation spread / sqrt(32), and output
    bias ln(alpha), so that the dissipation starts near alpha.  Draw order:
    W1, b1, W2, b2, W3, b3, W4."""
    rng = np.random.default_rng(seed)
    H = NN_HIDDEN
    parts = [rng.normal(0.0, math.sqrt(2.0 / 4), (H, 4)), rng.normal(0.0, 0.1, H),
             rng.normal(0.0, math.sqrt(2.0 / H), (H, H)), rng.normal(0.0, 0.1, H),
             rng.normal(0.0, math.sqrt(2.0 / H), (H, H)), rng.normal(0.0, 0.1, H),
             rng.normal(0.0, spread / math.sqrt(H), H), np.array([math.log(alpha)])]
    return np.concatenate([a.ravel() for a in parts]).astype(np.float64)
