"""Pins of the oracle's full right-hand side and RK3 step against what the
paper and the mathematics fix.  CPU only."""
import math

import numpy as np
import pytest

from conftest import golden
from paper_2203_13760_gb300 import inputs


def test_sod_matches_exact_riemann_solution(orc):
    """Section 5.1.2: the HLLC setup follows the exact solution of the Sod
    problem (Appendix A case).  The L1 density error shrinks under refinement
    and at 200 cells (CFL 0.5) stays below 3e-3."""
    g = golden("sod_appendix_a.json")
    WL = [g["left"]["rho"], g["left"]["u"], g["left"]["p"]]
    WR = [g["right"]["rho"], g["right"]["u"], g["right"]["p"]]
    errs = {}
    for n in (100, 200, 400):
        case = inputs.riemann_1d(n, WL, WR, x0=g["diaphragm"])
        c = orc.config(**case.params())
        U, t, _ = orc.run(c, case.U, 100000, 0.0, g["end_time"])
        assert t == pytest.approx(g["end_time"], rel=1e-14)
        x = inputs.centres(n, 0.0, 1.0)
        ex = orc.exact_sample(WL, WR, x, t, x0=g["diaphragm"])
        errs[n] = float(np.mean(np.abs(U[0, 0, 0] - ex[:, 0])))
    assert errs[200] < 3e-3
    assert errs[100] > errs[200] > errs[400]


def test_fifth_order_convergence(orc):
    """Section 5.1.1 (Eq. SinusDensity): WENO5-JS + TVD-RK3 with dt = 1e-4 to
    t = 1 converges at fifth order in the l1 norm."""
    g = golden("convergence_section_5_1_1.json")
    steps = int(round(g["end_time"] / g["dt"]))
    errs = []
    for n in (20, 40, 80):
        case = inputs.sine_advection(n)
        c = orc.config(**case.params())
        U, t, s = orc.run(c, case.U, steps, g["dt"])
        assert s == steps
        errs.append(np.mean(np.abs(U[0, 0, 0] - inputs.sine_exact_average(n, t))))
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(orders > 0.94 * g["expected_order"]["WENO5-JS"]), orders


@pytest.mark.parametrize("n,bc", [((12, 1, 1), (1,) * 6), ((8, 8, 1), (0,) * 6), ((6, 7, 5), (0, 0, 1, 1, 0, 0))])
def test_free_stream_preserved_exactly(orc, n, bc):
    """A uniform state has a right-hand side of exactly zero (all faces carry
    identical bits), with viscous and heat fluxes on."""
    U = np.empty((5, n[2], n[1], n[0]))
    U[:] = np.array([1.2, 0.3, -0.2, 0.1, 2.7])[:, None, None, None]
    c = orc.config(n, bc=bc, viscous=True, heat=True, mu=0.01)
    assert np.all(orc.rhs(c, U) == 0.0)


@pytest.mark.parametrize("n", [(16, 12, 1), (8, 6, 7)])
def test_conservation_periodic(orc, n):
    """On a periodic grid the face fluxes telescope: sum_cells U dV is
    conserved to round-off (mass, momentum, energy)."""
    case = inputs.random_smooth(n, seed=11, viscous=True, mu=0.02)
    c = orc.config(**case.params())
    U0 = case.U
    U, _, _ = orc.run(c, U0, 5, 0.002)
    s0 = U0.reshape(5, -1).sum(1)
    s1 = U.reshape(5, -1).sum(1)
    scale = np.abs(U0).reshape(5, -1).sum(1)
    assert np.all(np.abs(s1 - s0) <= 1e-13 * scale), (s1 - s0) / scale
    assert np.abs(U - U0).max() > 1e-6  # the state did evolve


def test_sod_mirror_symmetry(orc):
    """x -> 1 - x with the states exchanged and u negated gives the mirrored
    solution."""
    n = 64
    case = inputs.riemann_1d(n, [1.0, 0.3, 1.0], [0.125, -0.2, 0.1])
    mirror = inputs.riemann_1d(n, [0.125, 0.2, 0.1], [1.0, -0.3, 1.0])
    c = orc.config(**case.params())
    U, _, _ = orc.run(c, case.U, 20, 0.002)
    M, _, _ = orc.run(c, mirror.U, 20, 0.002)
    M = M[:, :, :, ::-1].copy()
    M[1] *= -1
    np.testing.assert_allclose(U, M, rtol=1e-12, atol=1e-12)


def _poly_state(n, h, vel_fn, p_fn):
    x = (np.arange(n[0]) + 0.5) * h
    y = (np.arange(n[1]) + 0.5) * h
    z = (np.arange(n[2]) + 0.5) * h
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    u, v, w = vel_fn(X, Y, Z)
    p = p_fn(X, Y, Z)
    return inputs.conservative(1.0, u, v, w, p, 1.4), (X, Y, Z)


def test_viscous_stress_manufactured_2d(orc):
    """u = 0, v = x^2 y, rho = p = 1: the C4 stencils of Section 3.4 are exact
    for these polynomials, so the momentum right-hand side is the Stokes
    operator mu (lap u + grad(div u) / 3) = mu (2x/3, 2y) in interior cells.
    This exercises the face-normal, the cross (tangential) derivative and the
    -2/3 mu div u term."""
    n, h, mu = (14, 14, 1), 0.1, 0.05
    U, (X, Y, _) = _poly_state(n, h, lambda X, Y, Z: (0 * X, X * X * Y, 0 * X), lambda X, Y, Z: 1 + 0 * X)
    c = orc.config(n, hi=(1.4, 1.4, 1.0), bc=(1,) * 6, convective=False, viscous=True, mu=mu)
    r = orc.rhs(c, U)
    s = (slice(None), slice(4, -4), slice(4, -4))
    np.testing.assert_allclose(r[1][s], (mu * 2 * X / 3)[s], rtol=1e-10, atol=1e-12)
    np.testing.assert_allclose(r[2][s], (mu * 2 * Y)[s], rtol=1e-10, atol=1e-12)
    assert np.all(r[0] == 0.0)


def test_viscous_stress_manufactured_3d(orc):
    """Divergence-free u = (y z^2, x^2 z, x y^2): the momentum right-hand side
    is mu lap u = mu (2y, 2z, 2x), exact for the C4 stencils."""
    n, h, mu = (12, 12, 12), 0.1, 0.03
    U, (X, Y, Z) = _poly_state(n, h, lambda X, Y, Z: (Y * Z * Z, X * X * Z, X * Y * Y), lambda X, Y, Z: 1 + 0 * X)
    c = orc.config(n, hi=(1.2, 1.2, 1.2), bc=(1,) * 6, convective=False, viscous=True, mu=mu)
    r = orc.rhs(c, U)
    s = (slice(4, -4),) * 3
    np.testing.assert_allclose(r[1][s], (mu * 2 * Y)[s], rtol=1e-10, atol=1e-12)
    np.testing.assert_allclose(r[2][s], (mu * 2 * Z)[s], rtol=1e-10, atol=1e-12)
    np.testing.assert_allclose(r[3][s], (mu * 2 * X)[s], rtol=1e-10, atol=1e-12)


def test_heat_flux_manufactured(orc):
    """Fluid at rest with rho = 1 and T = p = 1 + a x^2 (R = 1): the energy
    right-hand side is div(lambda grad T) = 2 a lambda with
    lambda = mu gamma R / ((gamma - 1) Pr)."""
    n, h, mu, Pr, a = (16, 1, 1), 0.1, 0.04, 0.72, 0.3
    U, (X, _, _) = _poly_state(n, h, lambda X, Y, Z: (0 * X, 0 * X, 0 * X), lambda X, Y, Z: 1 + a * X * X)
    c = orc.config(n, hi=(1.6, 1.0, 1.0), bc=(1,) * 6, convective=False, viscous=True, heat=True, mu=mu, Pr=Pr)
    r = orc.rhs(c, U)
    lam = mu * 1.4 / (0.4 * Pr)
    np.testing.assert_allclose(r[4][0, 0, 4:-4], 2 * a * lam, rtol=1e-10)
    assert np.all(np.abs(r[1:4]) < 1e-14)


def test_linear_shear_stress(orc):
    """u = s y (simple shear): tau_xy = mu s is constant, so the momentum
    right-hand side vanishes in the interior, and the energy right-hand side
    is d(u tau_xy)/dy = mu s^2 (u tau_yx flux through y faces)."""
    n, h, mu, s = (8, 16, 1), 0.1, 0.07, 0.9
    U, (X, Y, _) = _poly_state(n, h, lambda X, Y, Z: (s * Y, 0 * X, 0 * X), lambda X, Y, Z: 1 + 0 * X)
    c = orc.config(n, hi=(0.8, 1.6, 1.0), bc=(0, 0, 1, 1, 1, 1), convective=False, viscous=True, mu=mu)
    r = orc.rhs(c, U)
    np.testing.assert_allclose(r[1][:, 4:-4, :], 0.0, atol=1e-12)
    np.testing.assert_allclose(r[4][:, 4:-4, :], mu * s * s, rtol=1e-10)


def test_compute_dt_closed_form(orc):
    """Uniform state: dt = CFL dx / (|u| + c) (convective limit) and the
    viscous limit 3/14 dx^2 / max(mu/rho, lambda/(rho c_v))."""
    n = (10, 10, 1)
    rho, u, v, p = 0.8, 0.5, -0.9, 1.1
    U = np.empty((5, 1, 10, 10))
    U[:] = inputs.conservative(rho, u, v, 0.0, p, 1.4).reshape(5, 1, 1, 1)
    c = orc.config(n, hi=(1.0, 2.0, 1.0), bc=(0,) * 6, cfl=0.5)
    cs = math.sqrt(1.4 * p / rho)
    want = 0.5 * 0.1 / max(abs(u) + cs, abs(v) + cs)
    assert orc.compute_dt(c, U) == pytest.approx(want, rel=1e-14)
    mu = 0.5
    c = orc.config(n, hi=(1.0, 2.0, 1.0), bc=(0,) * 6, cfl=0.5, viscous=True, heat=True, mu=mu)
    lam = mu * 1.4 / (0.4 * 0.72)
    cv = 1.0 / 0.4
    want_v = 0.5 * (3.0 / 14.0) * 0.01 / max(mu / rho, lam / (rho * cv))
    assert orc.compute_dt(c, U) == pytest.approx(min(want, want_v), rel=1e-14)


def test_jvp_matches_central_differences(orc):
    """Forward-mode dual numbers give J v; central differences of the FP64
    step converge to it at second order."""
    case = inputs.random_smooth((10, 8, 1), seed=5, viscous=True, mu=0.01)
    c = orc.config(**case.params())
    rng = np.random.default_rng(1)
    V = rng.standard_normal(case.U.shape)
    dt = 0.002
    _, JV = orc.jvp_run(c, case.U, V, 2, dt)
    errs = []
    for eps in (1e-4, 1e-5):
        up, _, _ = orc.run(c, case.U + eps * V, 2, dt)
        um, _, _ = orc.run(c, case.U - eps * V, 2, dt)
        errs.append(np.abs((up - um) / (2 * eps) - JV).max())
    assert errs[1] < 1e-6 * np.abs(JV).max()
    assert errs[0] / errs[1] > 50.0  # second order: 100x per decade of eps
