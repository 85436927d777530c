// Exact solution of the 1D Riemann problem for an ideal gas.
//
// TEST INFRASTRUCTURE ONLY (see oracle/jf_oracle.hpp).
//
// The paper validates its shock-tube results against "an exact Riemann
// solver" (Section 5.1.2, citing Toro's textbook).  This is that textbook
// construction written from its definition: the star pressure p* solves
//   f_L(p) + f_R(p) + (u_R - u_L) = 0,
// where f_K is the shock branch (Rankine-Hugoniot) for p > p_K and the
// rarefaction branch (isentropic, Riemann invariant) for p <= p_K:
//   shock:       f_K = (p - p_K) sqrt(A_K / (p + B_K)),
//                A_K = 2 / ((gamma + 1) rho_K),  B_K = (gamma - 1)/(gamma + 1) p_K
//   rarefaction: f_K = 2 c_K / (gamma - 1) ((p / p_K)^((gamma - 1)/(2 gamma)) - 1)
// solved by Newton iteration; u* = (u_L + u_R)/2 + (f_R(p*) - f_L(p*))/2.
// The self-similar solution W(x/t) is then sampled wave by wave.
#pragma once
#include <algorithm>
#include <cmath>

namespace orc {

struct Prim1 { double rho, u, p; };

struct ExactRiemann {
  Prim1 L, R;
  double g;
  double pstar = 0.0, ustar = 0.0;

  double sound(const Prim1& s) const { return std::sqrt(g * s.p / s.rho); }

  // f_K(p) and its derivative for side K
  void fk(double p, const Prim1& s, double& f, double& df) const {
    const double c = sound(s);
    if (p > s.p) {
      const double A = 2.0 / ((g + 1.0) * s.rho);
      const double B = (g - 1.0) / (g + 1.0) * s.p;
      const double q = std::sqrt(A / (p + B));
      f = (p - s.p) * q;
      df = q * (1.0 - 0.5 * (p - s.p) / (B + p));
    } else {
      const double r = p / s.p;
      f = 2.0 * c / (g - 1.0) * (std::pow(r, (g - 1.0) / (2.0 * g)) - 1.0);
      df = 1.0 / (s.rho * c) * std::pow(r, -(g + 1.0) / (2.0 * g));
    }
  }

  // Newton iteration on f(p) = 0 from the two-rarefaction guess; returns
  // false if the data generate vacuum or the iteration does not converge.
  bool solve() {
    const double cL = sound(L), cR = sound(R);
    if (2.0 * (cL + cR) / (g - 1.0) <= R.u - L.u) return false;  // vacuum
    const double z = (g - 1.0) / (2.0 * g);
    double p = std::pow((cL + cR - 0.5 * (g - 1.0) * (R.u - L.u)) /
                            (cL / std::pow(L.p, z) + cR / std::pow(R.p, z)),
                        1.0 / z);
    p = std::max(p, 1e-14);
    for (int it = 0; it < 100; ++it) {
      double fL, dfL, fR, dfR;
      fk(p, L, fL, dfL);
      fk(p, R, fR, dfR);
      const double f = fL + fR + (R.u - L.u);
      double pn = p - f / (dfL + dfR);
      if (pn < 0.0) pn = 0.5 * p;
      const double change = 2.0 * std::fabs(pn - p) / (pn + p);
      p = pn;
      if (change < 1e-15) break;
    }
    double fL, dfL, fR, dfR;
    fk(p, L, fL, dfL);
    fk(p, R, fR, dfR);
    pstar = p;
    ustar = 0.5 * (L.u + R.u) + 0.5 * (fR - fL);
    return std::isfinite(pstar) && std::isfinite(ustar);
  }

  // density on the star side of wave K
  double star_density(const Prim1& s) const {
    const double r = pstar / s.p;
    if (pstar > s.p) {
      const double k = (g - 1.0) / (g + 1.0);
      return s.rho * (r + k) / (k * r + 1.0);
    }
    return s.rho * std::pow(r, 1.0 / g);
  }

  // sample the solution at xi = x / t
  Prim1 sample(double xi) const {
    if (xi <= ustar) {
      const double c = sound(L);
      if (pstar > L.p) {  // left shock
        const double S = L.u - c * std::sqrt((g + 1.0) / (2.0 * g) * pstar / L.p + (g - 1.0) / (2.0 * g));
        if (xi <= S) return L;
        return Prim1{star_density(L), ustar, pstar};
      }
      const double head = L.u - c;  // left rarefaction
      const double cstar = c * std::pow(pstar / L.p, (g - 1.0) / (2.0 * g));
      const double tail = ustar - cstar;
      if (xi <= head) return L;
      if (xi >= tail) return Prim1{star_density(L), ustar, pstar};
      const double base = 2.0 / (g + 1.0) + (g - 1.0) / ((g + 1.0) * c) * (L.u - xi);
      return Prim1{L.rho * std::pow(base, 2.0 / (g - 1.0)),
                   2.0 / (g + 1.0) * (c + 0.5 * (g - 1.0) * L.u + xi),
                   L.p * std::pow(base, 2.0 * g / (g - 1.0))};
    }
    const double c = sound(R);
    if (pstar > R.p) {  // right shock
      const double S = R.u + c * std::sqrt((g + 1.0) / (2.0 * g) * pstar / R.p + (g - 1.0) / (2.0 * g));
      if (xi >= S) return R;
      return Prim1{star_density(R), ustar, pstar};
    }
    const double head = R.u + c;  // right rarefaction
    const double cstar = c * std::pow(pstar / R.p, (g - 1.0) / (2.0 * g));
    const double tail = ustar + cstar;
    if (xi >= head) return R;
    if (xi <= tail) return Prim1{star_density(R), ustar, pstar};
    const double base = 2.0 / (g + 1.0) - (g - 1.0) / ((g + 1.0) * c) * (R.u - xi);
    return Prim1{R.rho * std::pow(base, 2.0 / (g - 1.0)),
                 2.0 / (g + 1.0) * (-c + 0.5 * (g - 1.0) * R.u + xi),
                 R.p * std::pow(base, 2.0 * g / (g - 1.0))};
  }
};

}  // namespace orc
