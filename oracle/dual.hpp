// Forward-mode dual numbers for the oracle.
//
// TEST INFRASTRUCTURE ONLY (see oracle/jf_oracle.hpp).
//
// A Dual carries a value and one directional derivative.  Running the oracle's
// RK3 step on Dual inputs (value = U, derivative = V) returns J(U)·V exactly
// up to rounding, where J is the Jacobian of the step.  This is the
// differentiated form of the forward pass that the paper obtains with JAX
// automatic differentiation (Section 6.2, "Validation of Automatic
// Differentiation Gradients"); here it serves as an independent check of the
// hand-written adjoint (VJP) kernels through <VJP(w), v> = <w, JVP(v)>.
//
// Comparisons, min/max and branch selections act on the value only, so the
// derivative follows the branch the value takes.
#pragma once
#include <cmath>

namespace orc {

struct Dual {
  double v;  // value
  double d;  // directional derivative
  Dual() : v(0.0), d(0.0) {}
  Dual(double x) : v(x), d(0.0) {}  // NOLINT: constants promote implicitly
  Dual(double x, double dx) : v(x), d(dx) {}
};

inline Dual operator+(const Dual& a, const Dual& b) { return Dual(a.v + b.v, a.d + b.d); }
inline Dual operator-(const Dual& a, const Dual& b) { return Dual(a.v - b.v, a.d - b.d); }
inline Dual operator-(const Dual& a) { return Dual(-a.v, -a.d); }
inline Dual operator*(const Dual& a, const Dual& b) { return Dual(a.v * b.v, a.d * b.v + a.v * b.d); }
inline Dual operator/(const Dual& a, const Dual& b) {
  // d(a/b) = (da*b - a*db)/b^2
  return Dual(a.v / b.v, (a.d * b.v - a.v * b.d) / (b.v * b.v));
}
inline Dual operator+(const Dual& a, double b) { return Dual(a.v + b, a.d); }
inline Dual operator+(double a, const Dual& b) { return Dual(a + b.v, b.d); }
inline Dual operator-(const Dual& a, double b) { return Dual(a.v - b, a.d); }
inline Dual operator-(double a, const Dual& b) { return Dual(a - b.v, -b.d); }
inline Dual operator*(const Dual& a, double b) { return Dual(a.v * b, a.d * b); }
inline Dual operator*(double a, const Dual& b) { return Dual(a * b.v, a * b.d); }
inline Dual operator/(const Dual& a, double b) { return Dual(a.v / b, a.d / b); }
inline Dual operator/(double a, const Dual& b) { return Dual(a / b.v, -a * b.d / (b.v * b.v)); }
inline Dual& operator+=(Dual& a, const Dual& b) { a = a + b; return a; }
inline Dual& operator-=(Dual& a, const Dual& b) { a = a - b; return a; }

inline bool operator<(const Dual& a, const Dual& b) { return a.v < b.v; }
inline bool operator>(const Dual& a, const Dual& b) { return a.v > b.v; }
inline bool operator<=(const Dual& a, const Dual& b) { return a.v <= b.v; }
inline bool operator>=(const Dual& a, const Dual& b) { return a.v >= b.v; }
inline bool operator<(const Dual& a, double b) { return a.v < b; }
inline bool operator>(const Dual& a, double b) { return a.v > b; }
inline bool operator<=(const Dual& a, double b) { return a.v <= b; }
inline bool operator>=(const Dual& a, double b) { return a.v >= b; }

inline Dual sqrt(const Dual& a) {
  const double s = std::sqrt(a.v);
  return Dual(s, a.d / (2.0 * s));
}
inline Dual log(const Dual& a) { return Dual(std::log(a.v), a.d / a.v); }
inline Dual exp(const Dual& a) {
  const double e = std::exp(a.v);
  return Dual(e, e * a.d);
}
inline Dual fabs(const Dual& a) { return a.v < 0.0 ? -a : a; }

// double overloads, so that unqualified calls inside namespace orc resolve to
// the exact double function rather than converting to Dual
inline double sqrt(double x) { return std::sqrt(x); }
inline double log(double x) { return std::log(x); }
inline double exp(double x) { return std::exp(x); }
inline double fabs(double x) { return std::fabs(x); }

inline double value_of(double x) { return x; }
inline double value_of(const Dual& x) { return x.v; }

}  // namespace orc
