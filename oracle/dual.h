// Dual numbers x = v + d*eps (eps^2 = 0) for the forward-mode tangent build of
// the oracle (TEST INFRASTRUCTURE ONLY).  Each operation computes its value
// with exactly the double operation of the plain build (both builds use
// -ffp-contract=off), so the tangent build reproduces the plain oracle's
// values bit for bit; the tangent part follows the chain rule.  Where a
// function is not differentiable (|x| at 0, max/min at a tie) the derivative
// of the branch the value takes is used.
#pragma once

#include <cmath>

struct Dual {
  double v, d;
  Dual() : v(0.0), d(0.0) {}
  Dual(double x) : v(x), d(0.0) {}  // NOLINT: constants promote implicitly
  Dual(double x, double dx) : v(x), d(dx) {}
  Dual& operator+=(const Dual& b) {
    v += b.v;
    d += b.d;
    return *this;
  }
  Dual& operator-=(const Dual& b) {
    v -= b.v;
    d -= b.d;
    return *this;
  }
  Dual& operator*=(const Dual& b) {
    d = d * b.v + v * b.d;
    v *= b.v;
    return *this;
  }
  Dual& operator/=(const Dual& b) {
    const double q = v / b.v;
    d = (d - q * b.d) / b.v;
    v = q;
    return *this;
  }
};

inline Dual operator+(const Dual& a, const Dual& b) { return Dual(a.v + b.v, a.d + b.d); }
inline Dual operator-(const Dual& a, const Dual& b) { return Dual(a.v - b.v, a.d - b.d); }
inline Dual operator-(const Dual& a) { return Dual(-a.v, -a.d); }
inline Dual operator+(const Dual& a) { return a; }
inline Dual operator*(const Dual& a, const Dual& b) { return Dual(a.v * b.v, a.d * b.v + a.v * b.d); }
inline Dual operator/(const Dual& a, const Dual& b) {
  const double q = a.v / b.v;
  return Dual(q, (a.d - q * b.d) / b.v);
}
inline bool operator<(const Dual& a, const Dual& b) { return a.v < b.v; }
inline bool operator>(const Dual& a, const Dual& b) { return a.v > b.v; }
inline bool operator<=(const Dual& a, const Dual& b) { return a.v <= b.v; }
inline bool operator>=(const Dual& a, const Dual& b) { return a.v >= b.v; }
inline bool operator==(const Dual& a, const Dual& b) { return a.v == b.v; }
inline bool operator!=(const Dual& a, const Dual& b) { return a.v != b.v; }

inline Dual sqrt(const Dual& a) {
  const double s = std::sqrt(a.v);
  return Dual(s, a.d / (2.0 * s));
}
inline Dual log(const Dual& a) { return Dual(std::log(a.v), a.d / a.v); }
inline Dual exp(const Dual& a) {
  const double e = std::exp(a.v);
  return Dual(e, e * a.d);
}
inline Dual fabs(const Dual& a) { return Dual(std::fabs(a.v), a.v >= 0.0 ? a.d : -a.d); }
inline Dual pow(const Dual& a, const Dual& b) {
  // a^b = exp(b log a); the value is the library pow of the plain build
  const double p = std::pow(a.v, b.v);
  double dp = b.v * std::pow(a.v, b.v - 1.0) * a.d;
  if (b.d != 0.0) dp += p * std::log(a.v) * b.d;
  return Dual(p, dp);
}
inline bool isfinite(const Dual& a) { return std::isfinite(a.v); }

// Holds a coefficient at its value: the tangent through it is dropped (the
// "frozen coefficient" linearisation of the stabilisation maps).
inline void freeze(Dual& a) { a.d = 0.0; }

inline double val(const Dual& a) { return a.v; }
inline double tan_of(const Dual& a) { return a.d; }
