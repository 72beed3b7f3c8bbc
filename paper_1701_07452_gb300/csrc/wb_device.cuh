// Device-side definitions shared by the CUDA translation units of the
// GB300-native WOMBAT step (Mendygral et al. 2017, arXiv:1701.07452).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#define WB_NG 5  // boundary zones per patch (Sec. "MHD in Two Dimensions")

// zone-centred state fields
enum { F_RHO = 0, F_MX = 1, F_MY = 2, F_MZ = 3, F_EN = 4, F_BX = 5, F_BY = 6, F_BZ = 7 };

struct WbPhys {
  double gamma, gm1, gm2, g_over_gm1, inv_gm1, gm2_over_gm1, cfl;
  float gamma_f;  // gamma for the FP32 screen of the signal rate
  double hgm2;  // (gamma - 2) / 2
  double eps[7], two_eps[7], four_eps[7], inv16eps[7];
  double inv4eps_m1[7];  // 1/(4 eps_k) - 1: Q_k(nu) - nu^2 = nu^2 (1/(4 eps) - 1) + eps
  int eps_zero;  // bit k set when eps_k == 0
  double sweby;
  int minmod;  // sweby == 1
  double rho_floor, p_floor;
  double prot_rho, prot_p;  // protection floors (App. A)
  int prot;                 // a protection floor is > 0
};

// Geometry of one patch and its padded storage (x fastest).
struct WbGeo {
  int n[3];         // interior zones
  int pd[3];        // padded dims n + 2 NG
  long long sy, sz; // strides of j and k
  long long V;      // padded volume (doubles per field per patch)
  double dx[3], idx[3];
};

// Zone (i, j, k) lies in the padded storage of a patch (a z index is free in
// the one-plane storage of a 2D box, whose z stride is 0).
__host__ __device__ __forceinline__ bool wb_zone_ok(const WbGeo& g, int i, int j, int k) {
  return i >= -WB_NG && i < g.pd[0] - WB_NG && j >= -WB_NG && j < g.pd[1] - WB_NG &&
         (g.sz == 0 || (k >= -WB_NG && k < g.pd[2] - WB_NG));
}

// The checked build (-DWB_CHECKED; a substitute for a memory checker, which
// this GPU pool does not offer): every zone index a kernel forms is tested
// against the padded storage; a bad one sets a bit in the translation unit's
// check word (read through wb_check_flags) and wb_at redirects it to zone
// (0, 0, 0), so the access stays inside the array.
#ifdef WB_CHECKED
static __device__ unsigned wb_check_word;
#define WB_CHECK_ZONE(g, i, j, k)                                        \
  do {                                                                   \
    if (!wb_zone_ok((g), (i), (j), (k))) atomicOr(&wb_check_word, 1u);  \
  } while (0)
#else
#define WB_CHECK_ZONE(g, i, j, k) \
  do {                            \
  } while (0)
#endif

// Host accessor of a translation unit's check word: returns it and clears it
// (0 in an unchecked build).  Each .cu file defines one with WB_CHECK_ACCESSOR.
#ifdef WB_CHECKED
#define WB_CHECK_ACCESSOR(name)                                     \
  unsigned name() {                                                 \
    unsigned v = 0, z = 0;                                          \
    cudaMemcpyFromSymbol(&v, wb_check_word, sizeof(v));             \
    cudaMemcpyToSymbol(wb_check_word, &z, sizeof(z));               \
    return v;                                                       \
  }
#else
#define WB_CHECK_ACCESSOR(name) \
  unsigned name() { return 0u; }
#endif

__host__ __device__ __forceinline__ long long wb_at(const WbGeo& g, int i, int j, int k) {
#if defined(WB_CHECKED) && defined(__CUDA_ARCH__)
  if (!wb_zone_ok(g, i, j, k)) {
    atomicOr(&wb_check_word, 1u);
    i = j = k = 0;
  }
#endif
  return (long long)(k + WB_NG) * g.sz + (long long)(j + WB_NG) * g.sy + (i + WB_NG);
}

template <int D>
__host__ __device__ __forceinline__ long long wb_stride(const WbGeo& g) {
  return D == 0 ? 1LL : (D == 1 ? g.sy : g.sz);
}

// Inclusive index box relative to the patch interior.
struct WbBox {
  int lo[3], hi[3];
};

// Device scalars of a grid (time step control and error counters).
struct WbScalars {
  double dt;              // dt of the current step (0 = skip)
  double t;               // time since load
  unsigned long long wmax_lag;   // lagged dt: signal rate of the previous step's start state (0: none)
  unsigned long long wmax_next;  // accumulated by the final update for the next step
  unsigned int rate_screen;      // running max of the FP32 screen of the signal rate (float bits)
  unsigned int pad_;
  long long steps;
  long long floor_hits;
  long long unphysical;
  long long timeouts;
  long long hll_faces;
};


// magnitude comparison on the IEEE bit pattern (integer pipe): |a| < |b|
// The sign bit is dropped by a left shift, not by a mask: the compiler turns
// a masked sign bit into an FP64 absolute value, which costs an FP64-pipe
// instruction on this GPU (measured), while the shift stays on the integer
// pipe.
__device__ __forceinline__ bool wb_abs_less(double a, double b) {
  const unsigned long long ua = (unsigned long long)__double_as_longlong(a) << 1;
  const unsigned long long ub = (unsigned long long)__double_as_longlong(b) << 1;
  return ua < ub;
}

// |x| on the integer pipe: the sign bit of the high word is cleared in PTX
// (fabs, or a 64-bit mask, becomes an FP64-pipe instruction on this GPU).
__device__ __forceinline__ double wb_fabs(double x) {
  int hi = __double2hiint(x), h2;
  asm("and.b32 %0, %1, 0x7fffffff;" : "=r"(h2) : "r"(hi));
  return __hiloint2double(h2, __double2loint(x));
}

// -x on the integer pipe: the sign bit of the high word flipped in PTX.  A
// negated double that feeds a select or an integer-pipe test, rather than an
// FMA operand (where the negation is free), otherwise costs an FP64 DADD.
__device__ __forceinline__ double wb_flip(double x) {
  int hi = __double2hiint(x), h2;
  asm("xor.b32 %0, %1, 0x80000000;" : "=r"(h2) : "r"(hi));
  return __hiloint2double(h2, __double2loint(x));
}

// minmod(a, b) on the integer pipe: the argument of smaller magnitude when the
// signs agree, else 0 (the SWEBY limiter with beta = 1, App. A).
__device__ __forceinline__ double wb_minmod(double a, double b) {
  long long ia = __double_as_longlong(a), ib = __double_as_longlong(b);
  double r = wb_abs_less(a, b) ? a : b;
  return ((ia ^ ib) >= 0) ? r : 0.0;
}

// Reciprocal and reciprocal square root for FP64 without the library
// division/sqrt sequences: the PTX approximations rcp.approx.ftz.f64 and
// rsqrt.approx.ftz.f64 (relative error ~1e-6, measured) refined by one
// third-order correction from the series of (1-e)^-1 and (1-e)^-1/2:
//   1/x:       e = 1 - x y,    y <- y (1 + e + e^2)
//   1/sqrt(x): e = 1 - x y^2,  y <- y (1 + e/2 + 3 e^2 / 8)
// The truncation error is O(e^3) ~ 1e-18, below one ulp.  Inputs must be
// positive, finite and normal: the approximations flush subnormal inputs to
// zero (callers test with wb_normal_pos or know the range).
__device__ __forceinline__ double wb_rcp(double x) {
  double y;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
  double e = __fma_rn(-x, y, 1.0);
  double p = __fma_rn(e, e, e);
  return __fma_rn(y, p, y);
}

__device__ __forceinline__ double wb_rsqrt(double x) {
  double y;
  asm("rsqrt.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
  double h = __dmul_rn(x, y);
  double e = __fma_rn(-h, y, 1.0);
  double p = __fma_rn(0.375, e, 0.5);
  return __fma_rn(__dmul_rn(y, e), p, y);
}

// Comparisons on the IEEE bit patterns (integer pipe; the FP64 pipe is the
// scarce unit on this GPU).
// x > 0, finite (false for +inf and NaN)
__device__ __forceinline__ bool wb_pos(double x) {
  const long long b = __double_as_longlong(x);
  return b > 0 && b < 0x7ff0000000000000LL;
}
// x < 0 (false for -0.0 and NaN)
__device__ __forceinline__ bool wb_neg(double x) {
  const long long b = __double_as_longlong(x);
  const unsigned long long m = (unsigned long long)b << 1;  // |x| bits, shifted (see wb_abs_less)
  return b < 0 && m != 0 && m <= 0xffe0000000000000ULL;
}
// x is finite (exponent field not all ones; tested on the high word)
__device__ __forceinline__ bool wb_finite(double x) {
  return ((__double2hiint(x) >> 20) & 0x7ff) != 0x7ff;
}
// x < f for a floor f that is finite and >= +0: exact for every x, false
// for NaN (the bit patterns of non-negative doubles order as their values;
// an FP64 compare costs an FP64-pipe instruction on this GPU)
__device__ __forceinline__ bool wb_below_floor(double x, double f) {
  const long long bx = __double_as_longlong(x), bf = __double_as_longlong(f);
  if (bx < 0) {
    const unsigned long long m = (unsigned long long)bx << 1;
    if (m > 0xffe0000000000000ULL) return false;  // NaN
    return m != 0 || bf != 0;                      // x < 0 < ... ; -0 < f unless f = +0
  }
  return bx < bf;                                  // NaN (bx > inf >= bf) gives false
}
// x is a positive normal finite double (>= 2^-1022; false for subnormals,
// zero, negatives, inf and NaN)
__device__ __forceinline__ bool wb_normal_pos(double x) {
  const long long b = __double_as_longlong(x);
  return b >= 0x0010000000000000LL && b < 0x7ff0000000000000LL;
}
// x == 0 (either sign), on the integer pipe.  The sign bit is shifted out of
// the high word in PTX: written as a C expression on the bit pattern the test
// is exactly x == 0.0, which the compiler emits as an FP64 compare (an
// FP64-pipe instruction, counted by a probe kernel's counters).
__device__ __forceinline__ bool wb_zero(double x) {
  int h;
  asm("shl.b32 %0, %1, 1;" : "=r"(h) : "r"(__double2hiint(x)));
  return (h | __double2loint(x)) == 0;
}
// a <= b for a, b >= 0 (non-negative, non-NaN operands)
__device__ __forceinline__ bool wb_le_nonneg(double a, double b) {
  return __double_as_longlong(a) <= __double_as_longlong(b);
}
// 2 x, exact: the exponent field raised by one on the integer pipe for a
// normal x whose double is normal; zero, subnormals, the top binade, inf and
// NaN take an FP64 add (rare).
__device__ __forceinline__ double wb_twice(double x) {
  const int hi = __double2hiint(x);
  const int ex = (hi >> 20) & 0x7ff;
  if (ex != 0 && ex < 0x7fe) return __hiloint2double(hi + (1 << 20), __double2loint(x));
  return __dadd_rn(x, x);
}
// a < b in the order of the bit patterns read as sign and magnitude (the
// order of the values, with -0 before +0; not for NaN), on the integer pipe
__device__ __forceinline__ bool wb_order_less(double a, double b) {
  long long ka = __double_as_longlong(a), kb = __double_as_longlong(b);
  ka ^= (ka >> 63) & 0x7fffffffffffffffLL;
  kb ^= (kb >> 63) & 0x7fffffffffffffffLL;
  return ka < kb;
}
// min(max(x, 0), 1)
__device__ __forceinline__ double wb_clamp01(double x) {
  const long long b = __double_as_longlong(x);
  if (b <= 0) return 0.0;                                 // negative or zero
  return b > 0x3ff0000000000000LL ? 1.0 : x;              // above 1 (or NaN -> 1)
}

// x / 2^s for s = 1, 2 on the integer pipe: the exponent field is lowered by
// s, which is exact for every normal x whose quotient is normal.  Inputs
// below 2^(s-1022) in magnitude (zero, subnormals, the lowest binades) give a
// zero of the same sign instead of a subnormal; inf and NaN pass unchanged.
template <int S>
__device__ __forceinline__ double wb_pow2_div(double x) {
  const int hi = __double2hiint(x);
  const int lo = __double2loint(x);
  const int ex = (hi >> 20) & 0x7ff;
  int h = hi & (int)0x80000000;
  int l = 0;
  if (ex > S) {
    h = hi - (S << 20);
    l = lo;
  }
  if (ex == 0x7ff) {
    h = hi;
    l = lo;
  }
  return __hiloint2double(h, l);
}
__device__ __forceinline__ double wb_half(double x) { return wb_pow2_div<1>(x); }
__device__ __forceinline__ double wb_quarter(double x) { return wb_pow2_div<2>(x); }

// +1 for x >= 0 (including -0.0), -1 for x < 0
__device__ __forceinline__ double wb_sgn(double x) { return wb_neg(x) ? -1.0 : 1.0; }

// SWEBY limiter g = SIGN(a) max(0, min(beta|a|, s b), min(|a|, beta s b)), s = SIGN(a)
__device__ __forceinline__ double wb_sweby(double a, double b, double beta, int minmod) {
  if (minmod) return wb_minmod(a, b);
  double s = wb_sgn(a);
  double aa = fabs(a);
  double m1 = fmin(beta * aa, s * b);
  double m2 = fmin(aa, beta * s * b);
  return s * fmax(0.0, fmax(m1, m2));
}

// x * s for s = +1 or -1: the sign bit of s flips x (integer pipe)
__device__ __forceinline__ double wb_xsgn(double x, double s) {
  const long long sg = __double_as_longlong(s) & (long long)0x8000000000000000ULL;
  return __longlong_as_double(__double_as_longlong(x) ^ sg);
}

// |x| with the sign of s (integer pipe)
__device__ __forceinline__ double wb_copysign_abs(double mag, double s) {
  long long m = __double_as_longlong(mag) & 0x7fffffffffffffffLL;
  long long sg = __double_as_longlong(s) & (long long)0x8000000000000000ULL;
  return __longlong_as_double(m | sg);
}

// Key of a signal rate w for an unsigned atomicMax: the bits of w > 0, 0 for
// w <= 0, the canonical NaN for any NaN (so that a NaN rate poisons the max),
// from the bit pattern alone: the FP64 compares (w >= 0, w != w) would each
// take an FP64-pipe instruction.
__device__ __forceinline__ unsigned long long wb_rate_bits(double w) {
  const long long b = __double_as_longlong(w);
  int mh;
  asm("and.b32 %0, %1, 0x7fffffff;" : "=r"(mh) : "r"(__double2hiint(w)));
  const bool nan = mh > 0x7ff00000 || (mh == 0x7ff00000 && __double2loint(w) != 0);
  return nan ? 0x7ff8000000000000ULL : (b > 0 ? (unsigned long long)b : 0ULL);
}

// atomic max of a non-negative double through its bit pattern (exact, order independent)
__device__ __forceinline__ void wb_atomic_max_pos(unsigned long long* addr, double v) {
  if (v >= 0.0) atomicMax(addr, (unsigned long long)__double_as_longlong(v));
  else if (!(v >= 0.0) && v != v) atomicMax(addr, 0x7ff8000000000000ULL);  // NaN poisons
}
