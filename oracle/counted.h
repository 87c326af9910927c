// Operation-counting scalar for the oracle (test infrastructure only).
//
// Counted carries a double and tallies, per thread, the floating-point operations performed on it: adds
// and subtracts, multiplies, divides, square roots, logarithms and exponentials. Its value part is the
// exact double operation, so a counted run reproduces the plain oracle bit for bit; comparisons act on
// values and are not counted (they are decisions, not arithmetic). Run through the oracle's templated
// scheme it gives the scheme's operation mix per cell-step, the algorithmic work of a roofline.
#ifndef IMEXDS_ORACLE_COUNTED_H
#define IMEXDS_ORACLE_COUNTED_H
#include <cmath>

namespace orcdual {

struct OpCount {
  long long add = 0, mul = 0, div = 0, sqrt = 0, log = 0, exp = 0;
};
inline thread_local OpCount op_count;

struct Counted {
  double v;
  Counted() : v(0.0) {}
  Counted(double x) : v(x) {}  // NOLINT: implicit promotion of constants
  Counted& operator+=(const Counted& b) { return *this = *this + b; }
  Counted& operator-=(const Counted& b) { return *this = *this - b; }
  Counted& operator*=(const Counted& b) { return *this = *this * b; }
  friend Counted operator+(const Counted& a, const Counted& b) {
    ++op_count.add;
    return Counted(a.v + b.v);
  }
  friend Counted operator-(const Counted& a, const Counted& b) {
    ++op_count.add;
    return Counted(a.v - b.v);
  }
  friend Counted operator-(const Counted& a) { return Counted(-a.v); }  // a sign flip
  friend Counted operator*(const Counted& a, const Counted& b) {
    ++op_count.mul;
    return Counted(a.v * b.v);
  }
  friend Counted operator/(const Counted& a, const Counted& b) {
    ++op_count.div;
    return Counted(a.v / b.v);
  }
  friend bool operator<(const Counted& a, const Counted& b) { return a.v < b.v; }
  friend bool operator>(const Counted& a, const Counted& b) { return a.v > b.v; }
  friend bool operator<=(const Counted& a, const Counted& b) { return a.v <= b.v; }
  friend bool operator>=(const Counted& a, const Counted& b) { return a.v >= b.v; }
};

inline Counted sqrt(const Counted& a) {
  ++op_count.sqrt;
  return Counted(std::sqrt(a.v));
}
inline Counted log(const Counted& a) {
  ++op_count.log;
  return Counted(std::log(a.v));
}
inline Counted exp(const Counted& a) {
  ++op_count.exp;
  return Counted(std::exp(a.v));
}
inline Counted fabs(const Counted& a) { return Counted(std::fabs(a.v)); }  // a sign operation
inline double val(const Counted& x) { return x.v; }
inline Counted with_value(double v, const Counted& /*same*/) { return Counted(v); }

}  // namespace orcdual
#endif
