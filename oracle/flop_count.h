// TEST INFRASTRUCTURE ONLY -- instrumented FP64 scalar for the oracle's
// operation count (the algorithmic FLOPs of a cell-update).  Compiled into
// the oracle only with -DORACLE_COUNT_FLOPS (a separate, single-threaded
// build); the ordinary oracle uses plain double.
//
// Counting rule: each add, subtract, multiply, divide and square root whose
// result depends on the data counts 1 (the oracle has no fused multiply-add;
// an FMA would count 2).  Not counted: negation, absolute value, min/max and
// comparisons (no arithmetic), and the identity operations of the oracle's
// dense 7x7 matrix formulation -- adding or subtracting an exact zero,
// multiplying by an exact 0 or +-1, dividing by +-1 -- which an
// implementation that uses the structure of the matrices never performs.
// Operations on the parameters alone (gamma, eps_k, dt/dx) are plain double
// arithmetic and are not counted: they are loop invariants.
// The value of every operation is the IEEE double result, so a counting run
// gives the same bits as the ordinary oracle.
#pragma once

#include <cmath>

namespace flopcount {

enum Section {
  SEC_NONE = 0,
  SEC_CELL,     // sweep: zone primitives and zone flux, per zone of a pencil
  SEC_FACE,     // sweep: Roe state, eigen-system, alpha_k, nu_k, g-tilde, mean flux, per face
  SEC_HLL,      // sweep: HLL flux of a protected face
  SEC_LIMIT,    // sweep: g_k (SWEBY limiter), per zone of a pencil
  SEC_EMIT,     // sweep: gamma_k, beta_k and u-bar, per output face
  SEC_EREF,     // Step 2: reference EMF, per zone
  SEC_EDGE,     // Steps 3, 9: corner EMF, per edge
  SEC_CT,       // Steps 4, 11: constrained transport, per face
  SEC_TRANS,    // Steps 5, 7: transverse state incl. div B source, per zone and direction
  SEC_EREFH,    // Step 8: half-step reference EMF, per zone
  SEC_UPDATE,   // Step 10: conservative update, per zone
  SEC_FINAL,    // Step 11 epilogue: zone field, floors, per zone
  SEC_DT,       // CFL rate, per zone
  SEC_COUNT
};

extern long long flops[SEC_COUNT];
extern long long units[SEC_COUNT];
extern int section;

inline void tick() { ++flops[section]; }
inline void unit(int s) { ++units[s]; }
inline void enter(int s) { section = s; }

struct real {
  double v;
  real() : v(0.0) {}
  real(double x) : v(x) {}  // NOLINT: literals and loaded values enter freely
  explicit operator double() const { return v; }
  real& operator+=(const real& o) { *this = *this + o; return *this; }
  real& operator-=(const real& o) { *this = *this - o; return *this; }
  real& operator*=(const real& o) { *this = *this * o; return *this; }
  real& operator/=(const real& o) { *this = *this / o; return *this; }
  friend real operator+(const real& a, const real& b) {
    if (a.v != 0.0 && b.v != 0.0) tick();
    return real(a.v + b.v);
  }
  friend real operator-(const real& a, const real& b) {
    if (a.v != 0.0 && b.v != 0.0) tick();
    return real(a.v - b.v);
  }
  friend real operator*(const real& a, const real& b) {
    if (a.v != 0.0 && b.v != 0.0 && a.v != 1.0 && a.v != -1.0 && b.v != 1.0 && b.v != -1.0)
      tick();
    return real(a.v * b.v);
  }
  friend real operator/(const real& a, const real& b) {
    if (a.v != 0.0 && b.v != 1.0 && b.v != -1.0) tick();
    return real(a.v / b.v);
  }
  friend real operator-(const real& a) { return real(-a.v); }
  friend bool operator<(const real& a, const real& b) { return a.v < b.v; }
  friend bool operator>(const real& a, const real& b) { return a.v > b.v; }
  friend bool operator<=(const real& a, const real& b) { return a.v <= b.v; }
  friend bool operator>=(const real& a, const real& b) { return a.v >= b.v; }
  friend bool operator==(const real& a, const real& b) { return a.v == b.v; }
  friend bool operator!=(const real& a, const real& b) { return a.v != b.v; }
};

inline real r_sqrt(const real& x) {
  if (x.v != 0.0 && x.v != 1.0) tick();
  return real(std::sqrt(x.v));
}
inline real r_fabs(const real& x) { return real(std::fabs(x.v)); }
inline real r_fmin(const real& a, const real& b) { return real(std::fmin(a.v, b.v)); }
inline real r_fmax(const real& a, const real& b) { return real(std::fmax(a.v, b.v)); }
inline bool r_isfinite(const real& x) { return std::isfinite(x.v); }
inline double to_d(const real& x) { return x.v; }

}  // namespace flopcount
