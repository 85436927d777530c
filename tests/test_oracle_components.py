"""Pins of the oracle's building blocks against mathematics the paper relies
on (WENO5-JS reconstruction, HLLC flux, exact Riemann solution).  CPU only."""
import math

import numpy as np
import pytest

GAMMA = 1.4


def cell_averages_poly(coef, centres, h):
    """Exact cell averages of the polynomial sum_k coef[k] x^k."""
    out = np.zeros_like(centres)
    for k, a in enumerate(coef):
        # (1/h) int_{x-h/2}^{x+h/2} t^k dt
        out += a * ((centres + h / 2) ** (k + 1) - (centres - h / 2) ** (k + 1)) / ((k + 1) * h)
    return out


def poly(coef, x):
    return sum(a * x ** k for k, a in enumerate(coef))


# --- WENO5-JS ---------------------------------------------------------------

@pytest.mark.parametrize("seed", range(5))
def test_weno5_exact_for_quadratics(orc, seed):
    """For cell averages of a quadratic all three smoothness indicators are
    equal, so the weights are the linear ones and the reconstruction is the
    exact point value at the face (fifth-order linear combination)."""
    rng = np.random.default_rng(seed)
    coef = rng.uniform(-2, 2, 3)
    h = 0.1
    xc = np.arange(-2, 3) * h
    v = cell_averages_poly(coef, xc, h)
    got = orc.weno5(v, 1e-6)
    assert got == pytest.approx(poly(coef, h / 2), abs=1e-13)


def test_weno5_fifth_order_on_smooth_data(orc):
    """Away from critical points the weights tend to d = (1/10, 6/10, 3/10) and
    the face value converges at fifth order (a wrong linear weight or
    candidate stencil drops it to third order)."""
    errs = []
    for h in (0.04, 0.02, 0.01):
        x0 = 0.3  # f' != 0 here
        xc = x0 + np.arange(-2, 3) * h
        v = (np.cos(xc + h / 2) - np.cos(xc - h / 2)) * (-1.0 / h)  # averages of sin
        got = orc.weno5(v, 1e-6)
        errs.append(abs(got - math.sin(x0 + h / 2)))
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(orders > 4.6), orders


def test_weno5_nonoscillatory_at_jump(orc):
    """A jump at the face: the only smooth sub-stencil (all zeros) takes
    essentially all the weight."""
    assert abs(orc.weno5([0.0, 0.0, 0.0, 1.0, 1.0], 1e-6)) < 1e-10
    # jump one cell earlier: the value stays within the data range
    got = orc.weno5([0.0, 0.0, 1.0, 1.0, 1.0], 1e-6)
    assert 0.0 <= got <= 1.0 + 1e-12 and abs(got - 1.0) < 1e-10


def test_weno5_constant(orc):
    assert orc.weno5([2.5] * 5, 1e-6) == pytest.approx(2.5, rel=1e-15)


# --- HLLC ------------------------------------------------------------------

def physical_flux(W, d, gamma=GAMMA):
    """Convective flux F, G, H of Section 2 for W = (rho, u, v, w, p)."""
    rho, p = W[0], W[4]
    vel = np.array(W[1:4])
    E = p / (gamma - 1) + 0.5 * rho * vel @ vel
    un = vel[d]
    F = np.array([rho * un, rho * un * vel[0], rho * un * vel[1], rho * un * vel[2], un * (E + p)])
    F[1 + d] += p
    return F


@pytest.mark.parametrize("d", [0, 1, 2])
def test_hllc_consistency(orc, d):
    """F(U, U) equals the physical flux (consistency of the Riemann solver)."""
    rng = np.random.default_rng(d)
    for _ in range(20):
        W = np.array([rng.uniform(0.2, 2), *rng.uniform(-2, 2, 3), rng.uniform(0.2, 2)])
        np.testing.assert_allclose(orc.hllc(W, W, d), physical_flux(W, d), rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("d", [0, 1, 2])
@pytest.mark.parametrize("un", [0.0, 0.4, -0.7])
def test_hllc_resolves_contact_exactly(orc, d, un):
    """An isolated contact (equal normal velocity and pressure, different
    density and tangential velocity) is resolved exactly by HLLC: the flux is
    the upwind side's physical flux.  A wrong S* or star state breaks this."""
    WL = np.array([1.3, 0.2, -0.1, 0.3, 0.8])
    WR = np.array([0.4, -0.5, 0.6, 0.1, 0.8])
    WL[1 + d] = WR[1 + d] = un
    want = physical_flux(WL if un >= 0 else WR, d)
    np.testing.assert_allclose(orc.hllc(WL, WR, d), want, rtol=1e-13, atol=1e-13)


def test_hllc_supersonic_upwinding(orc):
    """Both states supersonic to the right (left): the flux is F_L (F_R)."""
    WL = np.array([1.0, 3.0, 0.1, 0.0, 1.0])
    WR = np.array([0.5, 2.8, -0.2, 0.3, 0.6])
    np.testing.assert_allclose(orc.hllc(WL, WR, 0), physical_flux(WL, 0), rtol=1e-14)
    WL2 = WL.copy(); WR2 = WR.copy()
    WL2[1] = -2.9; WR2[1] = -3.0
    np.testing.assert_allclose(orc.hllc(WL2, WR2, 0), physical_flux(WR2, 0), rtol=1e-14)


def test_hllc_mirror_symmetry(orc):
    """Mirroring x -> -x swaps the states and flips normal velocities: the
    mirrored flux has mass/tangential/energy components negated."""
    rng = np.random.default_rng(7)
    for _ in range(50):
        WL = np.array([rng.uniform(0.2, 2), *rng.uniform(-2, 2, 3), rng.uniform(0.2, 2)])
        WR = np.array([rng.uniform(0.2, 2), *rng.uniform(-2, 2, 3), rng.uniform(0.2, 2)])
        F = orc.hllc(WL, WR, 0)
        mL, mR = WR.copy(), WL.copy()
        mL[1] *= -1
        mR[1] *= -1
        Fm = orc.hllc(mL, mR, 0)
        np.testing.assert_allclose(Fm, [-F[0], F[1], -F[2], -F[3], -F[4]], rtol=1e-12, atol=1e-12)


def test_hllc_axis_permutation(orc):
    """Flux along y of a state equals the flux along x of the state with u and
    v exchanged (components exchanged back)."""
    rng = np.random.default_rng(3)
    for _ in range(20):
        WL = np.array([rng.uniform(0.2, 2), *rng.uniform(-2, 2, 3), rng.uniform(0.2, 2)])
        WR = np.array([rng.uniform(0.2, 2), *rng.uniform(-2, 2, 3), rng.uniform(0.2, 2)])
        Fy = orc.hllc(WL, WR, 1)
        sw = lambda W: W[[0, 2, 1, 3, 4]]
        Fx = orc.hllc(sw(WL), sw(WR), 0)
        np.testing.assert_allclose(Fy, sw(Fx), rtol=1e-14, atol=1e-14)


# --- exact Riemann solver ----------------------------------------------------

def sound(rho, p, g=GAMMA):
    return math.sqrt(g * p / rho)


def check_wave(side, W, pstar, ustar, rstar, g=GAMMA):
    """Rankine-Hugoniot across a shock, isentropic relation and Riemann
    invariant across a rarefaction."""
    rho, u, p = W
    if pstar > p:  # shock: mass flux across it gives its speed
        S = (rstar * ustar - rho * u) / (rstar - rho)
        m1, m2 = rho * (u - S), rstar * (ustar - S)
        assert m1 == pytest.approx(m2, rel=1e-10)
        assert rho * u * (u - S) + p == pytest.approx(rstar * ustar * (ustar - S) + pstar, rel=1e-10)
        E1 = p / (g - 1) + 0.5 * rho * u * u
        E2 = pstar / (g - 1) + 0.5 * rstar * ustar * ustar
        assert E1 * (u - S) + p * u == pytest.approx(E2 * (ustar - S) + pstar * ustar, rel=1e-9, abs=1e-12)
    else:
        assert p / rho ** g == pytest.approx(pstar / rstar ** g, rel=1e-12)
        sgn = 1.0 if side == "L" else -1.0
        assert u + sgn * 2 * sound(rho, p) / (g - 1) == pytest.approx(
            ustar + sgn * 2 * sound(rstar, pstar) / (g - 1), rel=1e-12, abs=1e-12)


@pytest.mark.parametrize("WL,WR", [
    ([1.0, 0.0, 1.0], [0.125, 0.0, 0.1]),        # Sod: rarefaction + shock
    ([1.0, 2.0, 0.4], [1.0, -2.0, 0.4]),         # two shocks
    ([1.0, -1.0, 0.4], [1.0, 1.0, 0.4]),         # two rarefactions
    ([5.99924, 19.5975, 460.894], [5.99242, -6.19633, 46.095]),  # strong shocks
])
def test_exact_riemann_wave_relations(orc, WL, WR):
    pstar, ustar, rL, rR = orc.exact_star(WL, WR)
    check_wave("L", WL, pstar, ustar, rL)
    check_wave("R", WR, pstar, ustar, rR)


def test_exact_riemann_sample_fan(orc):
    """Inside the Sod rarefaction the solution is isentropic with constant
    left Riemann invariant, and u - c = x/t."""
    WL, WR = [1.0, 0.0, 1.0], [0.125, 0.0, 0.1]
    t = 0.2
    x = np.linspace(0.3, 0.48, 12)
    W = orc.exact_sample(WL, WR, x, t)
    head = -sound(1.0, 1.0)
    inside = (x - 0.5) / t > head
    for (rho, u, p), xi in zip(W[inside], (x[inside] - 0.5) / t):
        if abs(rho - 1.0) < 1e-12:
            continue
        assert p / rho ** GAMMA == pytest.approx(1.0, rel=1e-12)
        assert u + 2 * sound(rho, p) / (GAMMA - 1) == pytest.approx(2 * sound(1.0, 1.0) / (GAMMA - 1), rel=1e-12)
        if u < 0.92:  # still inside the fan
            assert u - sound(rho, p) == pytest.approx(xi, rel=1e-10, abs=1e-12)
