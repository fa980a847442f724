/*
 * Forward-mode dual numbers for the oracle (TEST INFRASTRUCTURE ONLY).
 *
 * A dual number a + b e with e^2 = 0 carries a value and its derivative along one
 * input direction; every arithmetic operation applies the chain rule, so running
 * the oracle's own step with real = dual gives the exact directional derivative
 * (Jacobian-vector product) of the discrete forward map, to rounding.  The tests use
 * it as the reference gradient of the outlet-temperature loss with respect to the
 * viscosity, the heat-source field and the wall heat flux (the quantities that the
 * paper's thermal LBE of Sec. 2.2 takes as inputs).
 *
 * Compiled only into the C++ build of lbm_oracle.c (-DORACLE_DUAL).  Comparisons
 * and the branch in the Gauss-Jordan pivot look at values only: the derivative of a
 * piecewise definition is that of the piece the value selects.
 */
#pragma once
#include <cmath>

struct dual {
  double v, d;
  dual() = default;
  dual(double a) : v(a), d(0.0) {}  // NOLINT: constants enter as dual numbers
  dual(double a, double b) : v(a), d(b) {}
  explicit operator double() const { return v; }
  dual &operator+=(const dual &o) { d += o.d; v += o.v; return *this; }
  dual &operator-=(const dual &o) { d -= o.d; v -= o.v; return *this; }
  dual &operator*=(const dual &o) { d = d * o.v + v * o.d; v *= o.v; return *this; }
  dual &operator/=(const dual &o) { d = (d * o.v - v * o.d) / (o.v * o.v); v /= o.v; return *this; }
};

inline dual operator+(dual a, const dual &b) { return a += b; }
inline dual operator-(dual a, const dual &b) { return a -= b; }
inline dual operator*(dual a, const dual &b) { return a *= b; }
inline dual operator/(dual a, const dual &b) { return a /= b; }
inline dual operator-(const dual &a) { return dual(-a.v, -a.d); }
inline dual operator+(const dual &a) { return a; }
inline bool operator==(const dual &a, const dual &b) { return a.v == b.v; }
inline bool operator!=(const dual &a, const dual &b) { return a.v != b.v; }
inline bool operator<(const dual &a, const dual &b) { return a.v < b.v; }
inline bool operator>(const dual &a, const dual &b) { return a.v > b.v; }
inline bool operator<=(const dual &a, const dual &b) { return a.v <= b.v; }
inline bool operator>=(const dual &a, const dual &b) { return a.v >= b.v; }

/* d sqrt(a) = da / (2 sqrt(a)); d |a| = sign(a) da; d a^n = n a^(n-1) da */
inline dual sqrt(const dual &a) {
  const double s = std::sqrt(a.v);
  return dual(s, s > 0.0 ? a.d / (2.0 * s) : 0.0);
}
inline dual fabs(const dual &a) { return a.v < 0.0 ? -a : a; }
inline dual pow(const dual &a, int n) {
  if (n == 0) return dual(1.0);
  return dual(std::pow(a.v, n), n * std::pow(a.v, n - 1) * a.d);
}
