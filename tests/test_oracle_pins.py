"""Pins of two oracle functions that the smooth-data and shock-tube tests do not
reach: Einfeldt's Roe-averaged signal speeds (Section 3.3, Table 2; the speed
estimate Appendix A selects) and the "is_safe_reconstruction" fallback
(Appendix A; read as: a face side whose reconstructed density or pressure is
not positive takes its cell value).  CPU only."""
import math

import numpy as np
import pytest

from paper_2203_13760_gb300 import inputs

GAMMA = 1.4


def shock_states(Ms, d, u0=0.0, vt=(0.0, 0.0), gamma=GAMMA):
    """A single shock of Mach number Ms running in +d into (rho, p) = (1, 1)
    at rest in a frame moving with u0 along d, tangential velocity vt on both
    sides.  Rankine-Hugoniot gives the state behind it; the shock speed comes
    from mass conservation across the shock, S = (rho2 u2 - rho1 u1) /
    (rho2 - rho1).  Returns (W_behind, W_ahead, S) with W = (rho, u, v, w, p)."""
    M2 = Ms * Ms
    rho2 = (gamma + 1.0) * M2 / ((gamma - 1.0) * M2 + 2.0)
    p2 = 1.0 + 2.0 * gamma / (gamma + 1.0) * (M2 - 1.0)
    u2 = math.sqrt(gamma) * 2.0 / (gamma + 1.0) * (Ms - 1.0 / Ms)
    S = (rho2 * (u2 + u0) - 1.0 * u0) / (rho2 - 1.0)
    t = [m for m in range(3) if m != d]
    Wb = np.zeros(5)
    Wa = np.zeros(5)
    Wb[0], Wb[4], Wb[1 + d] = rho2, p2, u2 + u0
    Wa[0], Wa[4], Wa[1 + d] = 1.0, 1.0, u0
    for k, m in enumerate(t):
        Wb[1 + m] = Wa[1 + m] = vt[k]
    return Wb, Wa, S


def mirror(W, d):
    out = np.array(W, dtype=np.float64)
    out[1 + d] = -out[1 + d]
    return out


@pytest.mark.parametrize("d", [0, 1, 2])
@pytest.mark.parametrize("Ms", [1.5, 2.0, 3.0])
@pytest.mark.parametrize("u0,vt", [(0.0, (0.0, 0.0)), (0.3, (0.7, -0.4))])
def test_einfeldt_speed_is_exact_shock_speed(orc, d, Ms, u0, vt):
    """Roe's linearisation resolves an isolated shock exactly: the jump of the
    two states is an eigenvector of the Roe matrix, with the shock speed as
    eigenvalue (u~ + c~ for a shock running to the right).  Einfeldt's S_R =
    max(u_R + c_R, u~ + c~) therefore equals the exact shock speed, and for the
    mirrored (left-running) shock S_L does.  Only the sqrt(rho) weights of the
    Roe averages (and H~ formed from the total enthalpy, |u~|^2 over all three
    components) have this property."""
    Wb, Wa, S = shock_states(Ms, d, u0, vt)
    SL, SR = orc.signal_speeds(Wb, Wa, d, GAMMA, "einfeldt")
    assert SR == pytest.approx(S, rel=1e-12, abs=1e-12)
    # the left wave of the same pair is bounded by the state behind the shock
    cb = math.sqrt(GAMMA * Wb[4] / Wb[0])
    assert SL <= Wb[1 + d] - cb + 1e-12
    # mirrored problem: the shock runs to the left into the state on the right
    SL_m, _ = orc.signal_speeds(mirror(Wa, d), mirror(Wb, d), d, GAMMA, "einfeldt")
    assert SL_m == pytest.approx(-S, rel=1e-12, abs=1e-12)


def test_einfeldt_pin_discriminates_the_weights(orc):
    """The pin above is sharp: the same speed formed with arithmetic means of
    the velocity and enthalpy misses the shock speed by far more than the
    tolerance (written out here only to show the test would catch it)."""
    for Ms in (1.5, 2.0, 3.0):
        Wb, Wa, S = shock_states(Ms, 0)
        H = [(W[4] / (GAMMA - 1.0) + 0.5 * W[0] * W[1] ** 2 + W[4]) / W[0] for W in (Wb, Wa)]
        u_a = 0.5 * (Wb[1] + Wa[1])
        H_a = 0.5 * (H[0] + H[1])
        wrong = u_a + math.sqrt((GAMMA - 1.0) * (H_a - 0.5 * u_a * u_a))
        assert abs(wrong - S) > 0.05
        assert orc.signal_speeds(Wb, Wa, 0, GAMMA, "einfeldt")[1] == pytest.approx(S, rel=1e-12)


# --- is_safe_reconstruction --------------------------------------------------

# A row of 26 cells with two near-vacuum gaps before jumps.  Pressure gap at
# cells 3..7: WENO5-JS reconstructs a negative pressure on both sides of the
# face between cells 5 and 6 and on the left side of the face between cells
# 7 and 8.  Density gap at cells 15..19 (pressure 1): negative density on both
# sides of the face between cells 17 and 18 and on the left of the face
# between 19 and 20.  The cells on either side of each such face differ in
# every primitive variable and collide (u = +-0.2), so both face states enter
# the flux and taking the wrong cell's value would show.
P_GAP = [1.0, 1.0, 1.0, 1e-2, 1e-5, 1e-8, 3e-8, 1e-8] + [1.0] * 18
RHO_GAP = ([1.0, 1.0, 0.9, 0.8, 0.7, 0.6, 0.65, 0.7, 1.2, 1.2, 1.1, 1.0, 1.0, 1.0, 1.0]
           + [1e-2, 1e-5, 1e-8, 3e-8, 1e-8] + [1.0] * 6)
U_GAP = [0.05] * 26
U_GAP[5], U_GAP[6], U_GAP[17], U_GAP[18] = 0.2, -0.2, 0.2, -0.2
GAP_FACES = {(5, "both"), (7, "left"), (17, "both"), (19, "left")}   # (cell left of the face, sides)
GAP_CELLS = (5, 6, 7, 8, 17, 18, 19, 20)


def gap_case():
    p, rho, u = np.array(P_GAP), np.array(RHO_GAP), np.array(U_GAP)
    n = p.size
    U = inputs.conservative(rho, u, 0.0, 0.0, p, GAMMA).reshape(5, 1, 1, n)
    return inputs.Case("gap", (n, 1, 1), (0.0, 0.0, 0.0), (float(n), 1.0, 1.0), (1, 1, 1, 1, 1, 1), U)


def primitives(U, gamma=GAMMA):
    rho = U[0]
    vel = U[1:4] / rho
    p = (gamma - 1.0) * (U[4] - 0.5 * rho * (vel ** 2).sum(0))
    return np.concatenate([rho[None], vel, p[None]])


def test_weno5_reconstructs_non_positive_states_in_the_gaps(orc):
    """The field is built so that the fallback has something to do: exactly
    the face sides listed in GAP_FACES reconstruct a non-positive density or
    pressure."""
    p, rho = np.array(P_GAP), np.array(RHO_GAP)
    found = set()
    for i in range(2, p.size - 3):
        for v, name in ((p, "p"), (rho, "rho")):
            left = orc.weno5(v[i - 2:i + 3]) <= 0.0
            right = orc.weno5(v[[i + 3, i + 2, i + 1, i, i - 1]]) <= 0.0
            if left or right:
                found.add((i, "both" if left and right else ("left" if left else "right")))
    assert found == GAP_FACES


def test_safe_reconstruction_takes_cell_values(orc):
    """With the flag on, each face side whose WENO5-JS density or pressure is
    not positive is replaced by the primitive state of the cell on that side
    before the HLLC flux; the right-hand side then follows Eq. (FVD).  The
    expected right-hand side is assembled here face by face from the pinned
    WENO5-JS and HLLC functions on a zero-gradient (clamped) padded row."""
    case = gap_case()
    n = case.n[0]
    h = 1.0
    W = primitives(case.U.reshape(5, n))
    Wp = np.concatenate([np.repeat(W[:, :1], 3, 1), W, np.repeat(W[:, -1:], 3, 1)], axis=1)
    flux = []
    fallbacks = 0
    for f in range(n + 1):           # face f sits between cells f-1 and f
        c = f - 1 + 3                # padded index of the cell left of the face
        left = np.array([orc.weno5(Wp[m, c - 2:c + 3]) for m in range(5)])
        right = np.array([orc.weno5(Wp[m, [c + 3, c + 2, c + 1, c, c - 1]]) for m in range(5)])
        if not (left[0] > 0 and left[4] > 0):
            left = Wp[:, c].copy()
            fallbacks += 1
        if not (right[0] > 0 and right[4] > 0):
            right = Wp[:, c + 1].copy()
            fallbacks += 1
        flux.append(orc.hllc(left, right, 0, GAMMA))
    flux = np.array(flux)
    want = -(flux[1:] - flux[:-1]).T / h
    assert fallbacks == 6
    c = orc.config(**case.params(), safe=True)
    got = orc.rhs(c, case.U).reshape(5, n)
    scale = np.abs(want).max(axis=1, keepdims=True)
    assert np.all(np.abs(got - want) <= 1e-13 * scale + 1e-300)
    # without the flag the cells beside those faces change (the negative face
    # pressures enter the flux); cells whose faces kept positive states are
    # bit for bit the same
    off = orc.rhs(orc.config(**case.params(), safe=False), case.U).reshape(5, n)
    for i in GAP_CELLS:
        assert not np.allclose(off[:, i], got[:, i], rtol=1e-9, atol=0.0)  # NaN counts as different
    keep = [i for i in range(n) if i not in GAP_CELLS]
    np.testing.assert_array_equal(off[:, keep], got[:, keep])


def test_safe_reconstruction_is_inert_on_positive_faces(orc):
    """Where every reconstructed density and pressure is positive the flag
    changes nothing, bit for bit."""
    case = inputs.random_blocks((21, 17, 1), seed=3)
    on = orc.rhs(orc.config(**case.params(), safe=True), case.U)
    off = orc.rhs(orc.config(**case.params(), safe=False), case.U)
    np.testing.assert_array_equal(on, off)
