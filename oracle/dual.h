// Forward-mode dual numbers for the oracle's tangent-linear mode (test infrastructure only).
//
// Dual<K> carries a value and K directional derivatives. Every operation computes its value with
// exactly the double operation the primal oracle performs (so the value part of a dual run is
// bit-identical to a plain double run) and its derivatives by the chain rule. Comparisons,
// branches and max/min act on values: branch decisions are frozen, as in any discrete derivative.
#ifndef IMEXDS_ORACLE_DUAL_H
#define IMEXDS_ORACLE_DUAL_H
#include <cmath>

namespace orcdual {

template <int K>
struct Dual {
  double v;
  double d[K];
  Dual() : v(0.0) {
    for (int k = 0; k < K; ++k) d[k] = 0.0;
  }
  Dual(double x) : v(x) {  // NOLINT: implicit promotion of constants
    for (int k = 0; k < K; ++k) d[k] = 0.0;
  }
  Dual& operator+=(const Dual& b) { return *this = *this + b; }
  Dual& operator-=(const Dual& b) { return *this = *this - b; }
  Dual& operator*=(const Dual& b) { return *this = *this * b; }
  friend Dual operator+(const Dual& a, const Dual& b) {
    Dual r;
    r.v = a.v + b.v;
    for (int k = 0; k < K; ++k) r.d[k] = a.d[k] + b.d[k];
    return r;
  }
  friend Dual operator-(const Dual& a, const Dual& b) {
    Dual r;
    r.v = a.v - b.v;
    for (int k = 0; k < K; ++k) r.d[k] = a.d[k] - b.d[k];
    return r;
  }
  friend Dual operator-(const Dual& a) {
    Dual r;
    r.v = -a.v;
    for (int k = 0; k < K; ++k) r.d[k] = -a.d[k];
    return r;
  }
  friend Dual operator*(const Dual& a, const Dual& b) {
    Dual r;
    r.v = a.v * b.v;
    for (int k = 0; k < K; ++k) r.d[k] = a.d[k] * b.v + a.v * b.d[k];
    return r;
  }
  friend Dual operator/(const Dual& a, const Dual& b) {
    Dual r;
    r.v = a.v / b.v;
    for (int k = 0; k < K; ++k) r.d[k] = (a.d[k] - r.v * b.d[k]) / b.v;
    return r;
  }
  friend bool operator<(const Dual& a, const Dual& b) { return a.v < b.v; }
  friend bool operator>(const Dual& a, const Dual& b) { return a.v > b.v; }
  friend bool operator<=(const Dual& a, const Dual& b) { return a.v <= b.v; }
  friend bool operator>=(const Dual& a, const Dual& b) { return a.v >= b.v; }
};

template <int K>
Dual<K> sqrt(const Dual<K>& a) {
  Dual<K> r;
  r.v = std::sqrt(a.v);
  for (int k = 0; k < K; ++k) r.d[k] = 0.5 * a.d[k] / r.v;
  return r;
}
template <int K>
Dual<K> log(const Dual<K>& a) {
  Dual<K> r;
  r.v = std::log(a.v);
  for (int k = 0; k < K; ++k) r.d[k] = a.d[k] / a.v;
  return r;
}
template <int K>
Dual<K> exp(const Dual<K>& a) {
  Dual<K> r;
  r.v = std::exp(a.v);
  for (int k = 0; k < K; ++k) r.d[k] = a.d[k] * r.v;
  return r;
}
template <int K>
Dual<K> fabs(const Dual<K>& a) {
  return (a.v < 0.0) ? -a : a;
}

// true for the dual-number types (derivative-carrying), false for double and the counting type
template <class T>
struct is_dual {
  static constexpr bool value = false;
};
template <int K>
struct is_dual<Dual<K>> {
  static constexpr bool value = true;
};

inline double val(double x) { return x; }

// The value v with the derivatives of `same`, an expression equal to the one that gave v. Used where the
// defining formula's derivative has a removable 0 * inf (a square root at zero) that an equal form avoids.
inline double with_value(double v, double /*same*/) { return v; }
template <int K>
Dual<K> with_value(double v, const Dual<K>& same) {
  Dual<K> r = same;
  r.v = v;
  return r;
}
template <int K>
double val(const Dual<K>& x) {
  return x.v;
}

// std::max / std::min semantics on values: max returns a unless a < b, min returns a unless b < a.
template <class T>
T tmax(const T& a, const T& b) {
  return (val(a) < val(b)) ? b : a;
}
template <class T>
T tmin(const T& a, const T& b) {
  return (val(b) < val(a)) ? b : a;
}

}  // namespace orcdual
#endif
