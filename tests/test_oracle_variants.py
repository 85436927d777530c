"""Pins of the oracle's scheme variants (Table 2 of the paper): HLL and
Rusanov fluxes, Davis and Toro signal speeds, WENO5-Z, TVD-RK2 and Euler.
Each pin is a property the mathematics fixes, independent of the formula as
coded: conservation across the wave fan, exact shock speeds, orders of
accuracy, non-oscillation, exact solutions of Riemann problems.  CPU only."""
import numpy as np
import pytest

from paper_2203_13760_gb300 import inputs

GAMMA = 1.4
FLUXES = [("hllc", "einfeldt"), ("hllc", "davis"), ("hllc", "toro"), ("hll", "einfeldt"), ("hll", "davis"),
          ("hll", "toro"), ("rusanov", "einfeldt")]


def euler_flux(W, d=0, gamma=GAMMA):
    """Physical flux of the Euler equations along axis d (Section 2)."""
    rho, vel, p = W[0], np.array(W[1:4]), W[4]
    E = p / (gamma - 1) + 0.5 * rho * vel @ vel
    F = np.array([rho * vel[d], rho * vel[0] * vel[d], rho * vel[1] * vel[d], rho * vel[2] * vel[d],
                  vel[d] * (E + p)])
    F[1 + d] += p
    return F


def conserved(W, gamma=GAMMA):
    rho, vel, p = W[0], np.array(W[1:4]), W[4]
    return np.array([rho, *(rho * vel), p / (gamma - 1) + 0.5 * rho * vel @ vel])


def random_states(rng, n, mach=0.8):
    out = []
    for _ in range(n):
        rho = rng.uniform(0.2, 3.0)
        p = rng.uniform(0.2, 3.0)
        c = np.sqrt(GAMMA * p / rho)
        out.append(np.array([rho, *(rng.uniform(-mach, mach, 3) * c), p]))
    return out


@pytest.mark.parametrize("flux,speeds", FLUXES)
def test_flux_consistent_with_physical_flux(orc, flux, speeds):
    """F(W, W) is the physical flux f(W) for every solver and speed estimate."""
    rng = np.random.default_rng(1)
    for W in random_states(rng, 20):
        for d in range(3):
            F = orc.flux(W, W, d, GAMMA, flux, speeds)
            np.testing.assert_allclose(F, euler_flux(W, d), rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("speeds", ["einfeldt", "davis", "toro"])
def test_hll_conserves_across_the_wave_fan(orc, speeds):
    """HLL (Harten, Lax, van Leer 1983) takes the single intermediate state
    U_hll = (S_R U_R - S_L U_L - (F_R - F_L)) / (S_R - S_L) that conserves
    the integral over the fan; its flux satisfies the Rankine-Hugoniot
    relations across both bounding waves: F = F_L + S_L (U_hll - U_L) =
    F_R + S_R (U_hll - U_R)."""
    rng = np.random.default_rng(2)
    L, R = random_states(rng, 30), random_states(rng, 30)
    for WL, WR in zip(L, R):
        SL, SR = orc.signal_speeds(WL, WR, 0, GAMMA, speeds)
        if not (SL < 0 < SR):
            continue
        UL, UR, FL, FR = conserved(WL), conserved(WR), euler_flux(WL), euler_flux(WR)
        Uh = (SR * UR - SL * UL - (FR - FL)) / (SR - SL)
        F = orc.flux(WL, WR, 0, GAMMA, "hll", speeds)
        scale = np.abs(FL).max() + np.abs(FR).max()
        assert np.abs(F - (FL + SL * (Uh - UL))).max() <= 1e-13 * scale
        assert np.abs(F - (FR + SR * (Uh - UR))).max() <= 1e-13 * scale


def test_rusanov_is_hll_with_symmetric_speeds(orc):
    """Local Lax-Friedrichs is the HLL flux with S_L = -a, S_R = a,
    a = max(|u_L| + c_L, |u_R| + c_R)."""
    rng = np.random.default_rng(3)
    for WL, WR in zip(random_states(rng, 20), random_states(rng, 20)):
        for d in range(3):
            a = max(abs(W[1 + d]) + np.sqrt(GAMMA * W[4] / W[0]) for W in (WL, WR))
            np.testing.assert_allclose(orc.flux(WL, WR, d, GAMMA, "rusanov"),
                                       orc.hll_with_speeds(WL, WR, -a, a, d, GAMMA), rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("speeds", ["einfeldt", "davis", "toro"])
def test_upwind_for_supersonic_faces(orc, speeds):
    """All waves right-moving (u > c on both sides): HLL and HLLC give the
    left physical flux; all left-moving: the right one."""
    WL = np.array([1.0, 3.0, 0.2, -0.1, 1.0])
    WR = np.array([0.8, 2.6, 0.0, 0.3, 0.7])
    for flux in ("hll", "hllc"):
        np.testing.assert_array_equal(orc.flux(WL, WR, 0, GAMMA, flux, speeds), euler_flux(WL))
        neg = lambda W: np.array([W[0], -W[1], W[2], W[3], W[4]])  # noqa: E731
        np.testing.assert_array_equal(orc.flux(neg(WR), neg(WL), 0, GAMMA, flux, speeds), euler_flux(neg(WL)))


def test_stationary_contact(orc):
    """A resting contact (u = 0, equal p, density jump): HLLC keeps it exactly
    (zero mass flux, momentum flux p); HLL and Rusanov diffuse mass from the
    dense side.  With Davis's speeds the fan is symmetric (-max c, max c) and
    HLL coincides with Rusanov; Einfeldt's fan is narrower (the Roe-averaged
    sound speed lies between c_L and c_R), so its HLL diffuses less."""
    WL = np.array([1.0, 0.0, 0.0, 0.0, 1.0])
    WR = np.array([0.25, 0.0, 0.0, 0.0, 1.0])
    for speeds in ("einfeldt", "davis", "toro"):
        F = orc.flux(WL, WR, 0, GAMMA, "hllc", speeds)
        assert F[0] == 0.0 and F[1] == 1.0 and F[4] == 0.0
    rus = orc.flux(WL, WR, 0, GAMMA, "rusanov")
    np.testing.assert_allclose(orc.flux(WL, WR, 0, GAMMA, "hll", "davis"), rus, rtol=1e-14)
    hll = orc.flux(WL, WR, 0, GAMMA, "hll", "einfeldt")[0]
    assert 0.0 < hll < rus[0]


@pytest.mark.parametrize("WL,WR", [([1.0, 0.0, 1.0], [0.125, 0.0, 0.1]),        # Sod: right shock
                                   ([0.445, 0.698, 3.528], [0.5, 0.0, 0.571]),  # Lax: right shock
                                   ([1.0, 0.0, 0.1], [1.0, -1.0, 1.0])])         # two shocks
def test_toro_factor_gives_exact_shock_speeds(orc, WL, WR):
    """Toro's speed S_R = u_R + c_R q_R with the exact star pressure p*
    equals the exact shock speed, which mass conservation across the shock
    fixes: S = (rho*_R u* - rho_R u_R) / (rho*_R - rho_R)."""
    p_star, u_star, rho_sL, rho_sR = orc.exact_star(WL, WR, GAMMA)
    if p_star > WR[2]:
        S_exact = (rho_sR * u_star - WR[0] * WR[1]) / (rho_sR - WR[0])
        cR = np.sqrt(GAMMA * WR[2] / WR[0])
        assert WR[1] + cR * orc.toro_q(p_star, WR[2], GAMMA) == pytest.approx(S_exact, rel=1e-12)
    if p_star > WL[2]:
        S_exact = (rho_sL * u_star - WL[0] * WL[1]) / (rho_sL - WL[0])
        cL = np.sqrt(GAMMA * WL[2] / WL[0])
        assert WL[1] - cL * orc.toro_q(p_star, WL[2], GAMMA) == pytest.approx(S_exact, rel=1e-12)


def test_toro_speeds_converge_to_exact_for_weak_shocks(orc):
    """The PVRS pressure is exact to second order in the jump, so Toro's S_R
    approaches the exact shock speed quadratically as the jump shrinks."""
    errs = []
    for delta in (0.05, 0.025, 0.0125):
        WL = [1.0 + delta, delta, 1.0 + 1.4 * delta]
        WR = [1.0, 0.0, 1.0]
        p_star, u_star, _, rho_sR = orc.exact_star(WL, WR, GAMMA)
        S_exact = (rho_sR * u_star) / (rho_sR - 1.0)
        _, SR = orc.signal_speeds([WL[0], WL[1], 0, 0, WL[2]], [1.0, 0.0, 0, 0, 1.0], 0, GAMMA, "toro")
        errs.append(abs(SR - S_exact))
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(orders > 1.8), orders


def test_signal_speeds_equal_states(orc):
    """For equal states every estimate is the characteristic pair u -+ c."""
    rng = np.random.default_rng(4)
    for W in random_states(rng, 10):
        c = np.sqrt(GAMMA * W[4] / W[0])
        for kind in ("einfeldt", "davis", "toro"):
            SL, SR = orc.signal_speeds(W, W, 0, GAMMA, kind)
            assert SL == pytest.approx(W[1] - c, rel=1e-13, abs=1e-13)
            assert SR == pytest.approx(W[1] + c, rel=1e-13, abs=1e-13)


def _henrick_averages(n):
    """Exact cell averages (10-point Gauss-Legendre) of
    f(x) = sin(pi x - sin(pi x) / pi) on [-1, 1] with 3 ghost cells per side;
    f has critical points where f' = 0 and f'' != 0."""
    f = lambda x: np.sin(np.pi * x - np.sin(np.pi * x) / np.pi)  # noqa: E731
    xg, wg = np.polynomial.legendre.leggauss(10)
    h = 2.0 / n
    left = -1.0 + h * (np.arange(n + 6) - 3)
    avg = np.array([0.5 * np.sum(wg * f(a + 0.5 * h * (xg + 1))) for a in left])
    return f, left, h, avg


def test_weno5_z_keeps_fifth_order_at_critical_points(orc):
    """Borges et al. (2008): at critical points WENO5-JS loses order while
    WENO5-Z keeps fifth order (eps = 1e-40 as in their tests), with a smaller
    error at every resolution."""
    errs = {"js": [], "z": []}
    for n in (20, 40, 80, 160):
        f, left, h, avg = _henrick_averages(n)
        e = {"js": 0.0, "z": 0.0}
        for i in range(2, n + 3):
            exact = f(left[i] + h)
            e["js"] = max(e["js"], abs(orc.weno5(avg[i - 2:i + 3], 1e-40) - exact))
            e["z"] = max(e["z"], abs(orc.weno5_z(avg[i - 2:i + 3], 1e-40) - exact))
        errs["js"].append(e["js"])
        errs["z"].append(e["z"])
    oz = np.log2(np.array(errs["z"][:-1]) / np.array(errs["z"][1:]))
    oj = np.log2(np.array(errs["js"][:-1]) / np.array(errs["js"][1:]))
    assert np.all(oz > 4.8), oz
    assert oj[-1] < 4.6, oj
    assert np.all(np.array(errs["z"]) < np.array(errs["js"]))


def test_weno5_z_non_oscillatory_at_a_step(orc):
    """At a jump the reconstruction stays within the values of the two cells
    beside the face (the linear fifth-order scheme overshoots); on linear
    data it is exact."""
    for k in range(5):
        v = np.where(np.arange(5) >= k, 1.0, 0.0)
        r = orc.weno5_z(v)
        assert min(v[2], v[3]) - 1e-6 <= r <= max(v[2], v[3]) + 1e-6
        linear = (2 * v[0] - 13 * v[1] + 47 * v[2] + 27 * v[3] - 3 * v[4]) / 60
        if not (min(v[2], v[3]) <= linear <= max(v[2], v[3])):
            assert abs(r - linear) > 1e-3  # the pin is not vacuous
    v = 0.3 + 0.7 * np.arange(5)
    assert orc.weno5_z(v) == pytest.approx(0.3 + 0.7 * 2.5, rel=1e-14)


@pytest.mark.parametrize("flux,speeds", FLUXES)
@pytest.mark.parametrize("recon", ["weno5-js", "weno5-z"])
def test_shock_tubes_every_scheme(orc, flux, speeds, recon):
    """Section 5.1.2: Sod (t = 0.2) and Lax (t = 0.14) against the exact
    Riemann solution; every solver, speed estimate and reconstruction
    converges under refinement."""
    for WL, WR, T, bound in ((inputs.SOD_LEFT, inputs.SOD_RIGHT, 0.2, 3.2e-3),
                             (inputs.LAX_LEFT, inputs.LAX_RIGHT, inputs.LAX_END_TIME, 1.25e-2)):
        errs = []
        for n in (100, 200, 400):
            case = inputs.riemann_1d(n, WL, WR)
            c = orc.config(**dict(case.params(), flux=flux, recon=recon, speeds=speeds))
            U, t, _ = orc.run(c, case.U, 100000, 0.0, T)
            ex = orc.exact_sample(WL, WR, inputs.centres(n, 0.0, 1.0), t)
            errs.append(np.mean(np.abs(U[0, 0, 0] - ex[:, 0])))
        assert errs[0] > errs[1] > errs[2], errs
        assert errs[1] < bound, errs


def test_shock_tube_dissipation_ordering(orc):
    """On Sod and Lax, the more dissipative the solver the larger the error:
    HLLC < HLL < Rusanov; and WENO5-Z < WENO5-JS for the same solver."""
    for WL, WR, T in ((inputs.SOD_LEFT, inputs.SOD_RIGHT, 0.2),
                      (inputs.LAX_LEFT, inputs.LAX_RIGHT, inputs.LAX_END_TIME)):
        case = inputs.riemann_1d(200, WL, WR)
        ex = orc.exact_sample(WL, WR, inputs.centres(200, 0.0, 1.0), T)
        err = {}
        for flux in ("hllc", "hll", "rusanov"):
            for recon in ("weno5-js", "weno5-z"):
                c = orc.config(**dict(case.params(), flux=flux, recon=recon))
                U, _, _ = orc.run(c, case.U, 100000, 0.0, T)
                err[flux, recon] = np.mean(np.abs(U[0, 0, 0] - ex[:, 0]))
        for recon in ("weno5-js", "weno5-z"):
            assert err["hllc", recon] < err["hll", recon] < err["rusanov", recon]
        for flux in ("hllc", "hll", "rusanov"):
            assert err[flux, "weno5-z"] < err[flux, "weno5-js"]


@pytest.mark.parametrize("integrator,order", [("euler", 1), ("rk2", 2), ("rk3", 3)])
def test_time_integrator_order(orc, integrator, order):
    """Table 2 integrators: on a smooth periodic flow with the space
    discretisation fixed, the error against a converged solution falls at
    the integrator's order as dt halves."""
    case = inputs.sine_advection(32)
    T = 0.05
    ref, _, _ = orc.run(orc.config(**case.params()), case.U, 1600, T / 1600)
    c = orc.config(**dict(case.params(), integrator=integrator))
    errs = []
    for n in (20, 40, 80):
        U, _, _ = orc.run(c, case.U, n, T / n)
        errs.append(np.abs(U - ref).max())
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(np.abs(orders - order) < 0.1), orders


def test_rk2_is_the_average_of_two_euler_steps(orc):
    """Shu-Osher TVD-RK2: U^{n+1} = (U^n + E(E(U^n))) / 2, E the Euler step."""
    case = inputs.random_smooth((16, 12, 1), seed=5, viscous=True, mu=0.02)
    dt = 1e-3
    U2, _, _ = orc.run(orc.config(**dict(case.params(), integrator="rk2")), case.U, 1, dt)
    UE, _, _ = orc.run(orc.config(**dict(case.params(), integrator="euler")), case.U, 2, dt)
    np.testing.assert_allclose(U2, 0.5 * (case.U + UE), rtol=0, atol=1e-14 * np.abs(case.U).max())


# ---------------------------------------------------------------------------
# The ROE setup (Section 3.3 flux-splitting formulation, Section 5): Roe
# average, eigen-decomposition, WENO5 on the split characteristic fluxes.

def _conserved_from_roe_state(rho, u, H, gamma=GAMMA):
    """A state with velocity u and total enthalpy H (p from H = c^2/(gamma-1) + |u|^2/2)."""
    p = (gamma - 1) / gamma * rho * (H - 0.5 * u @ u)
    return np.array([rho, *u, p])


def _jacobian_fd(W, d, gamma=GAMMA, h=1e-6):
    """Flux Jacobian dF/dU of the Euler equations along d by central differences."""
    U0 = conserved(W, gamma)

    def prim(U):
        rho = U[0]
        vel = U[1:4] / rho
        p = (gamma - 1) * (U[4] - 0.5 * rho * vel @ vel)
        return np.array([rho, *vel, p])

    A = np.zeros((5, 5))
    for k in range(5):
        e = np.zeros(5)
        e[k] = h * max(1.0, abs(U0[k]))
        A[:, k] = (euler_flux(prim(U0 + e), d, gamma) - euler_flux(prim(U0 - e), d, gamma)) / (2 * e[k])
    return A


@pytest.mark.parametrize("d", [0, 1, 2])
def test_roe_eigensystem(orc, d):
    """L = R^-1; R diag(lambda) L is the flux Jacobian at the Roe state
    (finite differences of the Euler flux); and the defining property of the
    Roe average: A~ (U_R - U_L) = F(U_R) - F(U_L) exactly."""
    rng = np.random.default_rng(7 + d)
    for WL, WR in zip(random_states(rng, 10), random_states(rng, 10)):
        lam, R, L = orc.roe_eigensystem(WL, WR, d, GAMMA)
        np.testing.assert_allclose(L @ R, np.eye(5), atol=1e-13)
        A = R @ np.diag(lam) @ L
        sL, sR = np.sqrt(WL[0]), np.sqrt(WR[0])
        u = (sL * np.array(WL[1:4]) + sR * np.array(WR[1:4])) / (sL + sR)
        H = lambda W: (conserved(W)[4] + W[4]) / W[0]  # noqa: E731
        Ht = (sL * H(WL) + sR * H(WR)) / (sL + sR)
        Wt = _conserved_from_roe_state(sL * sR, u, Ht)
        np.testing.assert_allclose(A, _jacobian_fd(Wt, d), rtol=1e-7, atol=1e-7 * np.abs(A).max())
        dF = euler_flux(WR, d) - euler_flux(WL, d)
        np.testing.assert_allclose(A @ (conserved(WR) - conserved(WL)), dF, rtol=1e-12,
                                   atol=1e-12 * np.abs(dF).max())


@pytest.mark.parametrize("d", [0, 1, 2])
def test_flux_splitting_consistent(orc, d):
    """A uniform stencil gives the physical flux: WENO of a constant is the
    constant, G+ + G- = G and R L F = F."""
    rng = np.random.default_rng(9)
    for W in random_states(rng, 10):
        np.testing.assert_allclose(orc.fs_flux(np.tile(W, (6, 1)), d), euler_flux(W, d), rtol=1e-13, atol=1e-13)


def test_roe_setup_fifth_order(orc):
    """Section 5.1.1 convergence case with the ROE setup: WENO5 on the
    characteristic fluxes converges at fifth order (dt = 1e-4 to t = 0.2)."""
    errs = []
    steps = 2000
    for n in (20, 40, 80):
        case = inputs.sine_advection(n)
        c = orc.config(**dict(case.params(), flux="roe"))
        U, t, _ = orc.run(c, case.U, steps, 1e-4)
        errs.append(np.mean(np.abs(U[0, 0, 0] - inputs.sine_exact_average(n, t))))
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(orders > 4.6), orders


@pytest.mark.parametrize("recon", ["weno5-js", "weno5-z"])
def test_roe_setup_shock_tubes(orc, recon):
    """Section 5.1.2 with the ROE setup: Sod and Lax converge to the exact
    Riemann solution."""
    for WL, WR, T, bound in ((inputs.SOD_LEFT, inputs.SOD_RIGHT, 0.2, 3.2e-3),
                             (inputs.LAX_LEFT, inputs.LAX_RIGHT, inputs.LAX_END_TIME, 1.25e-2)):
        errs = []
        for n in (100, 200, 400):
            case = inputs.riemann_1d(n, WL, WR)
            c = orc.config(**dict(case.params(), flux="roe", recon=recon))
            U, t, _ = orc.run(c, case.U, 100000, 0.0, T)
            ex = orc.exact_sample(WL, WR, inputs.centres(n, 0.0, 1.0), t)
            errs.append(np.mean(np.abs(U[0, 0, 0] - ex[:, 0])))
        assert errs[0] > errs[1] > errs[2], errs
        assert errs[1] < bound, errs
