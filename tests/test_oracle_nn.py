"""Pins of the oracle's Section 7.4 pieces: the slip-wall boundary, WENO3-JS
(the ground-truth scheme of the Rusanov-NN experiment) and the Rusanov-NN flux
with its parameter derivatives.  CPU only."""
import numpy as np
import pytest

from paper_2203_13760_gb300 import inputs

GAMMA = 1.4


@pytest.mark.parametrize("axis", [0, 1])
def test_wall_equals_mirrored_periodic_domain(orc, axis):
    """Walls on both ends of an axis are symmetry planes: the walled solution
    equals the left half of a periodic domain twice as long holding the
    field and its mirror image (normal momentum negated), to rounding."""
    case = inputs.random_smooth((12, 10, 1), seed=3, viscous=True, mu=0.02)
    p = case.params()
    n = list(p["n"])
    bc = [0, 0, 0, 0, 1, 1]
    bc[2 * axis] = bc[2 * axis + 1] = 2
    cw = orc.config(**dict(p, bc=tuple(bc)))
    U = case.U
    ax = 3 - axis  # array axis of the grid axis in [5][nz][ny][nx]
    mirror = np.flip(U, axis=ax).copy()
    mirror[1 + axis] *= -1
    Ud = np.concatenate([U, mirror], axis=ax)
    nd, hi = list(n), list(p["hi"])
    nd[axis] *= 2
    hi[axis] *= 2
    cp = orc.config(**dict(p, n=tuple(nd), hi=tuple(hi), bc=(0, 0, 0, 0, 1, 1)))
    dt = 0.3 * orc.compute_dt(cw, U)
    Uw, _, _ = orc.run(cw, U, 3, dt)
    Up, _, _ = orc.run(cp, Ud, 3, dt)
    half = Up[:, :, :, :n[0]] if axis == 0 else Up[:, :, :n[1], :]
    assert np.abs(Uw - half).max() <= 1e-13 * np.abs(Uw).max()


def test_wall_keeps_mass_and_stops_normal_flux(orc):
    """A closed box (walls everywhere): mass and energy are conserved, and
    the momentum normal to a wall changes only by the pressure force."""
    case = inputs.random_smooth((14, 12, 1), seed=5)
    c = orc.config(**dict(case.params(), bc=(2, 2, 2, 2, 1, 1)))
    U, _, _ = orc.run(c, case.U, 5, 0.3 * orc.compute_dt(c, case.U))
    for m in (0, 4):
        assert abs(U[m].sum() - case.U[m].sum()) <= 1e-13 * np.abs(case.U[m]).sum()


def test_weno3_js_definition_properties(orc):
    """Linear data are reproduced exactly; at a jump the value stays within
    the two cells beside the face; on smooth advection the scheme converges
    at third order once eps dominates the smoothness indicators."""
    assert orc.weno3([0.3, 1.0, 1.7]) == pytest.approx(1.35, rel=1e-14)
    for v in ([0.0, 0.0, 1.0], [0.0, 1.0, 1.0], [1.0, 0.0, 0.0]):
        r = orc.weno3(v)
        assert min(v[1], v[2]) - 1e-6 <= r <= max(v[1], v[2]) + 1e-6
    errs = []
    for n in (40, 80, 160, 320):
        case = inputs.sine_advection(n)
        c = orc.config(**dict(case.params(), recon="weno3-js"))
        U, t, _ = orc.run(c, case.U, 400, 2.5e-4)
        errs.append(np.mean(np.abs(U[0, 0, 0] - inputs.sine_exact_average(n, t))))
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(np.diff(errs) < 0) and orders[-1] > 2.8, orders


def _theta_const(alpha):
    th = np.zeros(orc_nn_params())
    th[-1] = np.log(alpha)
    return th


def orc_nn_params():
    import oracle
    return oracle.NN_PARAMS


def _theta_linear(a, b):
    """A network computing alpha = exp(a . x + b) for x with x0, x2, x3 >= 0:
    layer 1 passes x0, x2, x3 and the two signed parts of x1 through ReLU,
    layers 2 and 3 copy them, the output weights recombine them."""
    H = 32
    W1 = np.zeros((H, 4))
    W1[0, 0] = W1[1, 2] = W1[2, 3] = 1.0
    W1[3, 1], W1[4, 1] = 1.0, -1.0
    W2 = np.zeros((H, H))
    W3 = np.zeros((H, H))
    for i in range(5):
        W2[i, i] = W3[i, i] = 1.0
    W4 = np.zeros(H)
    W4[:5] = [a[0], a[2], a[3], a[1], -a[1]]
    return np.concatenate([W1.ravel(), np.zeros(H), W2.ravel(), np.zeros(H), W3.ravel(), np.zeros(H), W4, [b]])


def _states(rng, k):
    out = []
    for _ in range(k):
        rho, p = rng.uniform(0.3, 2.0, 2)
        c = np.sqrt(GAMMA * p / rho)
        out.append(np.array([rho, *(rng.uniform(-0.8, 0.8, 3) * c), p]))
    return out


def test_rusanov_nn_with_constant_alpha_is_lax_friedrichs(orc):
    """Zero weights: alpha = exp(b4), and the flux is HLL with speeds -+alpha."""
    rng = np.random.default_rng(1)
    th = _theta_const(1.7)
    for WL, WR in zip(_states(rng, 10), _states(rng, 10)):
        for d in range(3):
            np.testing.assert_allclose(orc.flux_nn(WL, WR, th, d), orc.hll_with_speeds(WL, WR, -1.7, 1.7, d),
                                       rtol=1e-13, atol=1e-13)


def test_rusanov_nn_inputs_and_network(orc):
    """A network built to compute alpha = exp(a . x + b): the flux equals
    (F_L + F_R)/2 - alpha (U_R - U_L)/2 with x = (|du_n|, mean u_n, mean c,
    |ds|), s = ln(p / rho^gamma) / (gamma - 1), evaluated in the test."""
    rng = np.random.default_rng(2)
    a, b = np.array([0.3, -0.4, 0.5, 0.2]), -0.1
    th = _theta_linear(a, b)
    for WL, WR in zip(_states(rng, 10), _states(rng, 10)):
        for d in range(3):
            cL, cR = np.sqrt(GAMMA * WL[4] / WL[0]), np.sqrt(GAMMA * WR[4] / WR[0])
            s = lambda W: np.log(W[4] / W[0] ** GAMMA) / (GAMMA - 1)  # noqa: E731
            x = np.array([abs(WR[1 + d] - WL[1 + d]), 0.5 * (WL[1 + d] + WR[1 + d]), 0.5 * (cL + cR),
                          abs(s(WR) - s(WL))])
            alpha = np.exp(a @ x + b)
            assert orc.nn_alpha(th, x) == pytest.approx(alpha, rel=1e-13)
            hll = orc.hll_with_speeds(WL, WR, -alpha, alpha, d)
            np.testing.assert_allclose(orc.flux_nn(WL, WR, th, d), hll, rtol=1e-12, atol=1e-13)


def test_rusanov_nn_parameter_jvp_matches_finite_differences(orc):
    """d U_n / d theta along a random direction by dual numbers equals the
    central difference of the runs (walls, two steps)."""
    rng = np.random.default_rng(3)
    th = 0.2 * rng.standard_normal(orc_nn_params())
    th[-1] = 0.3
    td = rng.standard_normal(orc_nn_params())
    case = inputs.random_smooth((10, 9, 1), seed=4)
    p = dict(case.params(), bc=(2, 2, 2, 2, 1, 1), flux="rusanov-nn")
    dt = 0.2 * orc.compute_dt(orc.config(**p, nn=th), case.U)
    U, J = orc.jvp_params_run(orc.config(**p, nn=th), case.U, 2, dt, td)
    eps = 1e-7  # small enough that no ReLU kink lies within +-eps along td
    Up, _, _ = orc.run(orc.config(**p, nn=th + eps * td), case.U, 2, dt)
    Um, _, _ = orc.run(orc.config(**p, nn=th - eps * td), case.U, 2, dt)
    fd = (Up - Um) / (2 * eps)
    assert np.abs(J).max() > 1e-8
    assert np.abs(J - fd).max() <= 1e-6 * np.abs(J).max()
