// Device "units" of the CTU+CT MHDTVD step (Sec. "MHD in Three Dimensions",
// Steps 1-11 with the App. A flux): one function per stage, each working on
// one index (zone, face, edge or pencil segment) of one box.  The per-stage
// kernels of a grid (wb_stages.cu, wb_sweep.cu) and the persistent batch
// kernel (wb_batch.cu) call the same functions.
#pragma once
#include "wb_device.cuh"

// Field pointers of one box (or one patch slot).  F[d][F_BX + d] is unused.
struct WbView {
  WbGeo geo;
  double* q[8];
  double* b[3];
  double* Fp[3][8];
  double* Fc[3][8];
  double* Eref[3];
  double* Eedge[3];
  double* bh[3];
  double* qh[3][8];
  double* Erefh[3];
  double* Eedgeh[3];
  WbScalars* scal;
};

namespace wbu {

// ---------------------------------------------------------------- sweep ----
constexpr int kBlock = 64;

// waves 2, 4, 6 (Alfven, entropy, Alfven) have eps = 0 (the default eps_k):
// the mask of the sweep specialisation that drops their Q-branch arithmetic
constexpr int kEpsZeroLD = (1 << 1) | (1 << 3) | (1 << 5);

struct Cell {
  double rho, ir, sr, isr;        // rho, 1/rho, sqrt(rho), 1/sqrt(rho)
  double vn, vt1, vt2;
  double bt1, bt2;
  double eref;                    // E - bn^2/2 (energy referred to the face field)
  double hr;                      // (gamma/(gamma-1) P + rho v^2/2 + |Bt|^2) / rho
  double F[7];                    // half the Sec. 3 flux (rho, Mn, Mt1, Mt2, Bt1, Bt2, E)
  double mn, mt1, mt2;
};

// Loads of fields a launch only reads may use the non-coherent read-only path
// (NC = true); the persistent batch kernel writes the same arrays in other
// stages of one launch and uses coherent loads (NC = false).
template <bool NC>
__device__ __forceinline__ double ld(const double* p) {
  if (NC) return __ldg(p);
  return *p;
}

// Zone state of a sweep.  The arithmetic is written with explicit rounding
// (no contraction left to the compiler): a zone is loaded both before and
// inside the march over a segment, and the two inlined copies must round
// identically, or a face's flux would depend on where a segment starts.
template <int D, bool NC>
__device__ __forceinline__ void load_cell(const double* const* q, long long off, const WbPhys& P,
                                          Cell& c) {
  constexpr int T1 = (D + 1) % 3, T2 = (D + 2) % 3;
  c.rho = ld<NC>(q[F_RHO] + off);
  c.mn = ld<NC>(q[F_MX + D] + off);
  c.mt1 = ld<NC>(q[F_MX + T1] + off);
  c.mt2 = ld<NC>(q[F_MX + T2] + off);
  const double e = ld<NC>(q[F_EN] + off);
  const double bn = ld<NC>(q[F_BX + D] + off);
  c.bt1 = ld<NC>(q[F_BX + T1] + off);
  c.bt2 = ld<NC>(q[F_BX + T2] + off);
  c.isr = wb_rsqrt(c.rho);
  c.ir = __dmul_rn(c.isr, c.isr);
  c.sr = __dmul_rn(c.rho, c.isr);
  c.vn = __dmul_rn(c.mn, c.ir);
  c.vt1 = __dmul_rn(c.mt1, c.ir);
  c.vt2 = __dmul_rn(c.mt2, c.ir);
  const double ke = wb_half(__fma_rn(c.mt2, c.vt2, __fma_rn(c.mt1, c.vt1, __dmul_rn(c.mn, c.vn))));
  const double bt2 = __fma_rn(c.bt2, c.bt2, __dmul_rn(c.bt1, c.bt1));
  const double bn2 = __dmul_rn(bn, bn);
  const double me = wb_half(__dadd_rn(bn2, bt2));
  const double p = __dmul_rn(P.gm1, __dsub_rn(__dsub_rn(e, ke), me));
  const double pstar = __dadd_rn(p, me);
  const double ep = __dadd_rn(e, pstar);
  c.eref = __dsub_rn(e, wb_half(bn2));
  // rho h = gamma/(gamma-1) P + rho v^2/2 + |B_t|^2 = (E + P*) - B_n^2
  c.hr = __dmul_rn(__dsub_rn(ep, bn2), c.ir);
  // half fluxes: the face needs (F_L + F_R) / 2
  const double hmn = wb_half(c.mn), hvn = wb_half(c.vn), hbn = wb_half(bn);
  c.F[0] = hmn;
  c.F[1] = __fma_rn(hmn, c.vn, wb_half(__dsub_rn(pstar, bn2)));
  c.F[2] = __fma_rn(hmn, c.vt1, __dmul_rn(-hbn, c.bt1));
  c.F[3] = __fma_rn(hmn, c.vt2, __dmul_rn(-hbn, c.bt2));
  c.F[4] = __fma_rn(c.bt1, hvn, __dmul_rn(-hbn, c.vt1));
  c.F[5] = __fma_rn(c.bt2, hvn, __dmul_rn(-hbn, c.vt2));
  const double bv = __fma_rn(c.bt2, c.vt2, __fma_rn(c.bt1, c.vt1, __dmul_rn(bn, c.vn)));
  c.F[6] = __fma_rn(ep, hvn, __dmul_rn(-hbn, bv));
}

// Per-face record (shared memory, structure of arrays over the block).
// R_PG = rho a^2 / (gamma-1); R_KX = (gamma-2)/(gamma-1) X - v^2/2 (= K - v^2 for the
// K = v^2/2 + (gamma-2)/(gamma-1) X of the energy row);
// R_AFCF = alpha_f c_f, R_ASCS = alpha_s c_s.
enum {
  R_AL = 0, R_NU = 7, R_RHO = 14, R_SRHO, R_A, R_PG, R_CF, R_ASCS, R_AFCF, R_AF, R_AS, R_B1, R_B2, R_S,
  R_VN, R_VT1, R_VT2, R_BTM, R_KX, R_FAVG, R_WORDS = R_FAVG + 7
};

// One thread's face record in shared memory, word w at p[w * BS] (the block's
// records interleaved, BS = threads per block).
template <int BS>
struct RecT {
  double* p;
  __device__ __forceinline__ double& operator[](int w) const { return p[w * BS]; }
};
using Rec = RecT<kBlock>;

// The flux arithmetic below is written with explicit rounding: every product
// that feeds a sum is one fused multiply-add (__fma_rn), every other operation
// is rounded on its own (__dmul_rn, __dadd_rn, __dsub_rn), and nothing is left
// to the compiler's contraction.  An interface then gives the same bits in
// every kernel this code is inlined into (the grid sweeps, both forms of the
// batch path), whatever else the kernel holds.  Shorthands:
#define WB_FMA __fma_rn
#define WB_MUL __dmul_rn
#define WB_ADD __dadd_rn
#define WB_SUB __dsub_rn

// Q_k(nu) - nu^2 for the g-tilde of App. A.  Waves in the compile-time mask
// EZ have eps_k = 0, where Q is |nu|; the branch test runs on the integer pipe.
template <int EZ>
__device__ __forceinline__ double Qk_m_nu2(double nu, int k, const WbPhys& P) {
  if (EZ & (1 << k)) return WB_FMA(-nu, nu, wb_fabs(nu));
  // |nu| - nu^2, or for |nu| < 2 eps nu^2 / (4 eps) + eps - nu^2 = nu^2 (1/(4 eps) - 1) + eps:
  // one FMA of operands chosen on the integer pipe, FMA(x, nu, y) with (x, y) = (-nu, |nu|)
  // or (nu (1/(4 eps) - 1), eps), so that no warp issues both forms
  const bool band = wb_abs_less(nu, P.two_eps[k]);
  const double x = band ? WB_MUL(nu, P.inv4eps_m1[k]) : wb_flip(nu);
  return WB_FMA(x, nu, band ? P.eps[k] : wb_fabs(nu));
}

// Gas pressure of a zone from its sweep-frame fields (Sec. 3, Eq. totenergy)
__device__ __forceinline__ double zone_pressure(const Cell& c, const WbPhys& P) {
  const double mv = WB_FMA(c.mt2, c.vt2, WB_FMA(c.mt1, c.vt1, WB_MUL(c.mn, c.vn)));
  const double bb = WB_FMA(c.bt2, c.bt2, WB_MUL(c.bt1, c.bt1));
  return WB_MUL(P.gm1, WB_SUB(WB_SUB(c.eref, wb_half(mv)), wb_half(bb)));
}

// Protection floor of App. A: true when a zone state, or an intermediate
// state w_L + sum_{j<=k} alpha_j r_j of the linearised Riemann problem, has a
// density or pressure below the floors.  The density / pressure rows of r_k
// (k = 1..6) are rho_ af / rho_ a^2 af, 0 / 0, rho_ as / rho_ a^2 as, 1 / 0,
// rho_ as / rho_ a^2 as, 0 / 0.
__device__ __forceinline__ bool protection_hit(const Cell& L, const Cell& R, double rho, double ra2,
                                               double af, double as, const double al[7],
                                               const WbPhys& P) {
  const double pL = zone_pressure(L, P), pR = zone_pressure(R, P);
  if (L.rho < P.prot_rho || pL < P.prot_p || R.rho < P.prot_rho || pR < P.prot_p) return true;
  const double r1 = WB_FMA(al[0], WB_MUL(rho, af), L.rho), p1 = WB_FMA(al[0], WB_MUL(ra2, af), pL);
  if (r1 < P.prot_rho || p1 < P.prot_p) return true;
  const double r3 = WB_FMA(al[2], WB_MUL(rho, as), r1), p3 = WB_FMA(al[2], WB_MUL(ra2, as), p1);
  if (r3 < P.prot_rho || p3 < P.prot_p) return true;
  const double r4 = WB_ADD(r3, al[3]);
  if (r4 < P.prot_rho) return true;
  const double r5 = WB_FMA(al[4], WB_MUL(rho, as), r4), p5 = WB_FMA(al[4], WB_MUL(ra2, as), p3);
  return r5 < P.prot_rho || p5 < P.prot_p;
}

// Fast speed of one zone along the sweep axis with its own zone field (Sec. 3)
__device__ __forceinline__ double zone_fast_speed(const Cell& c, double bn, const WbPhys& P) {
  const double a2 = WB_MUL(P.gamma, zone_pressure(c, P)) / c.rho;
  const double bn2 = WB_MUL(bn, bn);
  const double b2 = WB_FMA(c.bt2, c.bt2, WB_FMA(c.bt1, c.bt1, bn2)) / c.rho;
  const double s = WB_ADD(a2, b2);
  double disc = WB_FMA(s, s, -(WB_MUL(WB_MUL(4.0, a2), bn2) / c.rho));
  if (disc < 0.0) disc = 0.0;
  return sqrt(wb_half(WB_ADD(s, sqrt(disc))));
}

// Marker of a face record that holds a finished HLL flux (a Roe density is > 0)
constexpr double kHllFace = -1.0;

// HLL flux of App. A into the record of one face:
//   b+ = max(a_max, vR + cfR, 0), b- = min(a_min, vL - cfL, 0),
//   u = (b+ F_L - b- F_R + b+ b- (q_R - q_L)) / (b+ - b-),
// with a_max, a_min = vn_ +- cf_ of the Roe state when it exists (roe), the
// Einfeldt sign of the F_R term (the printed +b- F_R is not consistent), and
// bounds +-max(|v| + c_f) if both speeds vanish.  Rare path.
template <class Rc>
__device__ __forceinline__ void hll_face(const Cell& L, const Cell& R, double bnL, double bnR, bool roe,
                                      const WbPhys& P, const Rc& f) {
  const double cfL = zone_fast_speed(L, bnL, P), cfR = zone_fast_speed(R, bnR, P);
  double bp = fmax(WB_ADD(R.vn, cfR), 0.0);
  double bm = fmin(WB_SUB(L.vn, cfL), 0.0);
  if (roe) {
    bp = fmax(bp, WB_ADD(f[R_VN], f[R_CF]));
    bm = fmin(bm, WB_SUB(f[R_VN], f[R_CF]));
  }
  if (!(WB_SUB(bp, bm) > 0.0)) {
    const double sp = fmax(WB_ADD(fabs(L.vn), cfL), WB_ADD(fabs(R.vn), cfR));
    bp = sp;
    bm = -sp;
  }
  const double dq[7] = {WB_SUB(R.rho, L.rho), WB_SUB(R.mn, L.mn), WB_SUB(R.mt1, L.mt1), WB_SUB(R.mt2, L.mt2),
                        WB_SUB(R.bt1, L.bt1), WB_SUB(R.bt2, L.bt2), WB_SUB(R.eref, L.eref)};
  const double inv = 1.0 / WB_SUB(bp, bm);
  const double bpm = WB_MUL(bp, bm);
#pragma unroll
  for (int m = 0; m < 7; ++m) {
    // the zone fluxes hold F/2
    const double FL = WB_MUL(2.0, L.F[m]), FR = WB_MUL(2.0, R.F[m]);
    f[R_FAVG + m] = WB_MUL(WB_FMA(bpm, dq[m], WB_FMA(bp, FL, -WB_MUL(bm, FR))), inv);
  }
  f[R_RHO] = kHllFace;
}

// Roe state, eigen-system, alpha_k, nu_k and g-tilde_k (doubled) of one interface.
// Returns 0 for an MHDTVD face, 1 when the protection floor asks for the HLL
// flux (the record holds the Roe state), 2 when the Roe state has no real
// sound speed (HLL without Roe speeds).  The protection test is compiled in
// only when PROT is set.
template <int EZ, bool PROT, class Rc>
__device__ __forceinline__ int face_system(const Cell& L, const Cell& R, double b, double dtdx,
                                           const WbPhys& P, const Rc& f, double gt[7]) {
  const double iD = wb_rcp(WB_ADD(L.sr, R.sr));
  const double wL = WB_MUL(L.sr, iD), wR = WB_MUL(R.sr, iD);
  const double rho = WB_MUL(L.sr, R.sr);
  const double irho = WB_MUL(L.isr, R.isr);
  const double vn = WB_FMA(wL, L.vn, WB_MUL(wR, R.vn));
  const double vt1 = WB_FMA(wL, L.vt1, WB_MUL(wR, R.vt1));
  const double vt2 = WB_FMA(wL, L.vt2, WB_MUL(wR, R.vt2));
  const double bt1 = WB_FMA(wR, L.bt1, WB_MUL(wL, R.bt1));
  const double bt2 = WB_FMA(wR, L.bt2, WB_MUL(wL, R.bt2));
  const double b2 = WB_MUL(b, b);
  // H = wL (h_L + b^2)/rho_L + wR (h_R + b^2)/rho_R, with wL/rho_L + wR/rho_R = 1/rho_
  const double H = WB_FMA(b2, irho, WB_FMA(wL, L.hr, WB_MUL(wR, R.hr)));
  const double dbt1 = WB_SUB(R.bt1, L.bt1), dbt2 = WB_SUB(R.bt2, L.bt2);
  const double gX = WB_MUL(P.hgm2, WB_MUL(WB_FMA(dbt1, dbt1, WB_MUL(dbt2, dbt2)), WB_MUL(iD, iD)));  // (gamma-2) X
  const double hv2 = wb_half(WB_FMA(vn, vn, WB_FMA(vt1, vt1, WB_MUL(vt2, vt2))));
  const double bt2s = WB_FMA(bt1, bt1, WB_MUL(bt2, bt2));
  const double a2 = WB_FMA(P.gm1, WB_FMA(-WB_ADD(b2, bt2s), irho, WB_SUB(H, hv2)), -gX);
  if (!wb_normal_pos(a2)) return 2;
  const double isrho = wb_rsqrt(rho);
  const double srho = WB_MUL(rho, isrho);
  const double ca2 = WB_MUL(b2, irho), ct2 = WB_MUL(bt2s, irho);
  const double dac = WB_SUB(a2, ca2);
  const double disc = WB_FMA(dac, dac, WB_MUL(ct2, WB_FMA(2.0, WB_ADD(a2, ca2), ct2)));
  const double sum = WB_ADD(WB_ADD(a2, ca2), ct2);
  double rsd = 0.0, sd = 0.0;
  if (wb_normal_pos(disc)) {  // a subnormal discriminant is degenerate (sd ~ 0)
    rsd = wb_rsqrt(disc);
    sd = WB_MUL(disc, rsd);
  }
  const double cf2 = wb_half(WB_ADD(sum, sd));
  const double icf = wb_rsqrt(cf2);
  const double ia = wb_rsqrt(a2);
  const double a = WB_MUL(a2, ia);
  const double ca = WB_MUL(wb_fabs(b), isrho);
  const double cf = WB_MUL(cf2, icf);
  const double cs = WB_MUL(WB_MUL(a, ca), icf);  // c_f c_s = a c_a
  // 1/|B_t| and c_t = |B_t| / sqrt(rho_); a transverse field whose square is
  // not a normal double (underflowing noise ahead of a front) counts as 0
  double ib = 0.0, ct = 0.0, btm = 0.0;  // btm = |B_t|
  if (wb_normal_pos(bt2s)) {
    ib = wb_rsqrt(bt2s);
    btm = WB_MUL(bt2s, ib);
    ct = WB_MUL(btm, isrho);
  }
  double af, as;
  if (wb_le_nonneg(sd, WB_MUL(1e-12, sum))) {
    const bool fast = wb_le_nonneg(ca2, a2);
    af = fast ? 1.0 : 0.0;
    as = fast ? 0.0 : 1.0;
  } else {
    // With t1 = ca^2 + ct^2 - a^2: alpha_f^2 = (sd - t1) / (2 sd) and
    // alpha_s^2 = (sd + t1) / (2 sd) (cf^2 + cs^2 = a^2 + ca^2 + ct^2,
    // cf^2 - cs^2 = sd), and (sd - t1)(sd + t1) = disc - t1^2 = 4 a^2 ct^2,
    // so alpha_f alpha_s = a ct / sd.  The larger of the two is sqrt(m / (2 sd))
    // with m = sd + |t1| (no cancellation), = m r for r = 1/sqrt(2 sd m), and
    // the smaller a ct / (sd m r) = 2 a ct r: one reciprocal square root.
    // t1 takes the difference ca^2 - a^2 first: it is exact where the two
    // nearly cancel (the degenerate neighbourhood, where sd is small).
    const double t1 = WB_ADD(WB_SUB(ca2, a2), ct2);
    const bool slow_major = !wb_neg(t1);
    const double m = WB_ADD(sd, slow_major ? t1 : wb_flip(t1));
    const double r = wb_rsqrt(wb_twice(WB_MUL(sd, m)));
    const double major = WB_MUL(m, r);
    const double minor = WB_MUL(WB_MUL(a, ct), wb_twice(r));
    af = slow_major ? minor : major;
    as = slow_major ? major : minor;
  }
  const double ra2 = WB_MUL(rho, a2);
  double b1n, b2n;
  if (wb_le_nonneg(bt2s, WB_MUL(1e-24, WB_ADD(WB_ADD(ra2, b2), bt2s)))) {
    b1n = b2n = 0.70710678118654752440;
  } else {
    b1n = WB_MUL(bt1, ib);
    b2n = WB_MUL(bt2, ib);
  }
  const double S = wb_sgn(b);
  // primitive differences of the 7-variable system; the velocity differences
  // are kept times rho_ (dv' = rho_ dv), the 1/rho_ goes into the coefficients
  const double drho = WB_SUB(R.rho, L.rho);
  const double dmn = WB_SUB(R.mn, L.mn), dmt1 = WB_SUB(R.mt1, L.mt1), dmt2 = WB_SUB(R.mt2, L.mt2);
  const double de = WB_SUB(R.eref, L.eref);
  const double dvn = WB_FMA(-vn, drho, dmn);
  const double dvt1 = WB_FMA(-vt1, drho, dmt1);
  const double dvt2 = WB_FMA(-vt2, drho, dmt2);
  const double vdm = WB_FMA(vn, dmn, WB_FMA(vt1, dmt1, WB_MUL(vt2, dmt2)));
  const double bdb = WB_FMA(bt1, dbt1, WB_MUL(bt2, dbt2));
  const double dp = WB_FMA(-gX, drho, WB_MUL(P.gm1, WB_SUB(WB_FMA(hv2, drho, WB_SUB(de, vdm)), bdb)));
  // projections on the transverse field direction beta and its normal; S = sign(b)
  const double dvbS = wb_xsgn(WB_FMA(b1n, dvt1, WB_MUL(b2n, dvt2)), S);
  const double dvp = WB_FMA(-b2n, dvt1, WB_MUL(b1n, dvt2));
  const double dbb = WB_FMA(b1n, dbt1, WB_MUL(b2n, dbt2));
  const double dbpS = wb_xsgn(WB_FMA(-b2n, dbt1, WB_MUL(b1n, dbt2)), S);
  const double ia2 = WB_MUL(ia, ia);
  const double hir = wb_half(irho), hisr = wb_half(isrho);
  const double i2ra = WB_MUL(hisr, ia);   // 1 / (2 sqrt(rho) a)
  const double ri2a2 = WB_MUL(hir, ia2);  // 1 / (2 rho a^2)
  const double dpr = WB_MUL(dp, ri2a2);
  const double afcf = WB_MUL(af, cf), ascs = WB_MUL(as, cs);
  const double dbbi = WB_MUL(dbb, i2ra);
  // alpha_{1,7} = Cf -+ Xf / (2 rho a^2), alpha_{3,5} = Cs -+ Xs / (2 rho a^2): the factor
  // goes into the FMAs that form them
  const double Xf = WB_FMA(afcf, dvn, -WB_MUL(ascs, dvbS));
  const double Cf = WB_FMA(as, dbbi, WB_MUL(af, dpr));
  const double Xs = WB_FMA(ascs, dvn, WB_MUL(afcf, dvbS));
  const double Cs = WB_FMA(-af, dbbi, WB_MUL(as, dpr));
  const double hAa = WB_MUL(hisr, dbpS);
  double al[7];
  al[0] = WB_FMA(-ri2a2, Xf, Cf);
  al[6] = WB_FMA(ri2a2, Xf, Cf);
  al[2] = WB_FMA(-ri2a2, Xs, Cs);
  al[4] = WB_FMA(ri2a2, Xs, Cs);
  al[1] = WB_FMA(hir, dvp, hAa);
  al[5] = WB_FMA(hir, dvp, -hAa);
  al[3] = WB_FMA(-dp, ia2, drho);
  // nu_k = (dt/dx) a_k for the eigenvalues a_1..a_7 (Sec. 3)
  const double tvn = WB_MUL(dtdx, vn);
  const double nuk[7] = {WB_FMA(-dtdx, cf, tvn), WB_FMA(-dtdx, ca, tvn), WB_FMA(-dtdx, cs, tvn), tvn,
                         WB_FMA(dtdx, cs, tvn),  WB_FMA(dtdx, ca, tvn),  WB_FMA(dtdx, cf, tvn)};
#pragma unroll
  for (int k = 0; k < 7; ++k) {
    const double nu = nuk[k];
    f[R_AL + k] = al[k];
    f[R_NU + k] = nu;
    gt[k] = WB_MUL(Qk_m_nu2<EZ>(nu, k, P), al[k]);  // 2 g-tilde
  }
  f[R_RHO] = rho; f[R_SRHO] = srho; f[R_A] = a; f[R_PG] = WB_MUL(ra2, P.inv_gm1); f[R_CF] = cf;
  f[R_ASCS] = ascs; f[R_AFCF] = afcf; f[R_AF] = af; f[R_AS] = as; f[R_B1] = b1n; f[R_B2] = b2n; f[R_S] = S;
  f[R_VN] = vn; f[R_VT1] = vt1; f[R_VT2] = vt2; f[R_BTM] = btm;
  f[R_KX] = WB_FMA(gX, P.inv_gm1, -hv2);  // K - v^2 (the energy row of face_flux)
#pragma unroll
  for (int m = 0; m < 7; ++m) f[R_FAVG + m] = WB_ADD(L.F[m], R.F[m]);
  if (PROT && P.prot && protection_hit(L, R, rho, ra2, af, as, al, P)) return 1;
  return 0;
}

// beta_k of App. A from the limited slopes carried doubled, G = 2 g (the
// limiter commutes with the factor 2), without forming gamma_k.  With
// w = nu alpha + g_{i+1} - g_i, Q(nu + gamma) alpha = Q(w / alpha) alpha.  Where
// Q(x) = |x| (eps_k = 0, or |w| >= 2 eps |alpha|) that is |w| sign(alpha), and
// beta = |w| sign(alpha) - (g_i + g_{i+1}) is nu alpha - G_i when w has the sign
// of alpha, else -nu alpha - G_{i+1}: the larger of the two for alpha > 0, the
// smaller for alpha < 0, one FMA after an integer-pipe choice of operands.
// Inside the band, Q(x) alpha = w^2 / (4 eps alpha) + eps alpha, with
// 2 w = 2 nu alpha + G_{i+1} - G_i.  alpha = 0 needs no case of its own: this
// face's g-tilde is then 0, the limiter makes G_i = G_{i+1} = 0 and either form
// gives 0.
template <int EZ>
__device__ __forceinline__ double beta_k(double al, double nu, double Gi, double Gi1, int k,
                                         const WbPhys& P) {
  if (EZ & (1 << k)) {
    const double b1 = WB_FMA(nu, al, -Gi), b2 = WB_FMA(-nu, al, -Gi1);
    return (wb_order_less(b1, b2) != wb_neg(al)) ? b2 : b1;
  }
  const double d = WB_FMA(wb_twice(nu), al, WB_SUB(Gi1, Gi));  // 2 w
  if (!wb_abs_less(d, WB_MUL(P.four_eps[k], al))) {
    const bool same = (__double_as_longlong(d) ^ __double_as_longlong(al)) >= 0;
    return WB_FMA(same ? nu : wb_flip(nu), al, -(same ? Gi : Gi1));
  }
  // |nu + gamma| < 2 eps: beta = (2 w)^2 / (16 eps alpha) + eps alpha - (g_i + g_{i+1})
  const double t = WB_FMA(P.eps[k], al, -wb_half(WB_ADD(Gi, Gi1)));
  if (wb_abs_less(al, 1e-290)) return t;  // (2 w)^2 / (16 eps alpha) < eps |alpha|
  return WB_FMA(WB_MUL(WB_MUL(d, d), P.inv16eps[k]), wb_rcp(al), t);
}

// u-bar = (F_L + F_R)/2 - (dx/(2 dt)) sum_k beta_k R_k  (App. A)
template <int EZ, class Rc>
__device__ __forceinline__ void face_flux(const Rc& f, const double gi[7], const double gi1[7],
                                          double dx_2dt, const WbPhys& P, double out[7]) {
  double be[7];
#pragma unroll
  for (int k = 0; k < 7; ++k) be[k] = beta_k<EZ>(f[R_AL + k], f[R_NU + k], gi[k], gi1[k], k, P);
  const double rho = f[R_RHO], af = f[R_AF], as = f[R_AS];
  const double S = f[R_S], b1 = f[R_B1], b2 = f[R_B2];
  // sum_k beta_k r_k in w = (rho, vn, vt, Bt, p)
  const double sf = WB_ADD(be[0], be[6]), df = WB_SUB(be[6], be[0]);
  const double ss = WB_ADD(be[2], be[4]), ds = WB_SUB(be[4], be[2]);
  const double tfs = WB_FMA(af, sf, WB_MUL(as, ss));
  const double wr = WB_FMA(rho, tfs, be[3]);
  const double afcf = f[R_AFCF], ascs = f[R_ASCS];
  const double wvn = WB_FMA(afcf, df, WB_MUL(ascs, ds));
  const double vb = wb_xsgn(WB_FMA(afcf, ds, -WB_MUL(ascs, df)), S);  // along beta
  const double vp = WB_ADD(be[1], be[5]);                             // along beta-perp
  const double ra = WB_MUL(f[R_SRHO], f[R_A]);
  const double bb = WB_MUL(ra, WB_FMA(as, sf, -WB_MUL(af, ss)));
  const double bp = wb_xsgn(WB_MUL(f[R_SRHO], WB_SUB(be[1], be[5])), S);
  const double wvt1 = WB_FMA(b1, vb, -WB_MUL(b2, vp)), wvt2 = WB_FMA(b2, vb, WB_MUL(b1, vp));
  const double wbt1 = WB_FMA(b1, bb, -WB_MUL(b2, bp)), wbt2 = WB_FMA(b2, bb, WB_MUL(b1, bp));
  // to conserved variables (the pressure row enters the energy as p/(gamma-1))
  const double vn = f[R_VN], vt1 = f[R_VT1], vt2 = f[R_VT2];
  const double u1 = WB_FMA(vn, wr, WB_MUL(rho, wvn));
  const double u2 = WB_FMA(vt1, wr, WB_MUL(rho, wvt1));
  const double u3 = WB_FMA(vt2, wr, WB_MUL(rho, wvt2));
  // energy: B_t . w_Bt + p/(gamma-1) row + K w_rho + rho v . w_v, with
  // rho v . w_v = v . u - v^2 w_rho and the record holding K - v^2, and
  // B_t . w_Bt = |B_t| w_beta: beta is B_t / |B_t|, so the beta-perpendicular
  // part has no component along B_t (where |B_t|^2 is below 1e-24 of the
  // energy scale and beta is set to (1, 1)/sqrt 2 instead, the term is of that
  // size either way)
  const double u6 = WB_FMA(f[R_BTM], bb, WB_FMA(f[R_PG], tfs,
                    WB_FMA(f[R_KX], wr, WB_FMA(vn, u1, WB_FMA(vt1, u2, WB_MUL(vt2, u3))))));
  out[0] = WB_FMA(-dx_2dt, wr, f[R_FAVG + 0]);
  out[1] = WB_FMA(-dx_2dt, u1, f[R_FAVG + 1]);
  out[2] = WB_FMA(-dx_2dt, u2, f[R_FAVG + 2]);
  out[3] = WB_FMA(-dx_2dt, u3, f[R_FAVG + 3]);
  out[4] = WB_FMA(-dx_2dt, wbt1, f[R_FAVG + 4]);
  out[5] = WB_FMA(-dx_2dt, wbt2, f[R_FAVG + 5]);
  out[6] = WB_FMA(-dx_2dt, u6, f[R_FAVG + 6]);
}

// One pencil segment of an MHDTVD sweep along D: fluxes of faces [fa, fb]
// at transverse position (pos[U], pos[W]) of the input fields q (zone B),
// normal face field bn; outputs F.  qo / wo: slot offsets of the input and
// output arrays.  rec: two shared-memory face records of this thread.
// Faces without a Roe state or below the protection floor take the HLL flux
// and give g-tilde = 0 to the limiters of their neighbours.  Returns the
// number of HLL faces among [fa, fb] that are interior faces of the box.
template <int D, bool NC, int EZ = 0, bool PROT = true, class Rc = Rec>
__device__ __forceinline__ int sweep_segment(const WbGeo& g, const double* const* q,
                                             const double* bn, double* const* F, long long qo,
                                             long long wo, int pu, int pw, int fa, int fb,
                                             double dt, const WbPhys& P, const Rc rec[2]) {
  constexpr int T1 = (D + 1) % 3, T2 = (D + 2) % 3;
  constexpr int U = (D == 0) ? 1 : 0;
  constexpr int W = (D == 2) ? 1 : 2;
  int pos[3];
  pos[U] = pu;
  pos[W] = pw;
  pos[D] = fa - 2;
  const long long st = wb_stride<D>(g);
  const long long base = wb_at(g, pos[0], pos[1], pos[2]);
  {
    int last[3] = {pos[0], pos[1], pos[2]};
    last[D] = fb + 1;  // the segment reads zones fa-2 .. fb+1
    WB_CHECK_ZONE(g, last[0], last[1], last[2]);
    (void)last;
  }
  const long long off_in = qo + base;
  const long long off_out = wo + base;
  const double dtdx = WB_MUL(dt, g.idx[D]);
  const double dx_2dt = WB_MUL(wb_half(g.dx[D]), wb_rcp(dt));
  Cell cL, cR;
  load_cell<D, NC>(q, off_in, P, cL);
  double gt_p[7], g_p[7];  // 2 g-tilde of face f-1; 2 g of zone f-2
  int nhll = 0;
  // HLL faces are counted on interior faces only (distinct faces, whatever
  // part of the ghost rings the region covers)
  const bool across = pu >= 0 && pu < g.n[U] && pw >= 0 && pw < g.n[W];
  int cur = 0;
  // faces f = fa-1 .. fb+1; face f lies between zones f-1 and f
  for (int f = fa - 1; f <= fb + 1; ++f) {
    const int c = f - (fa - 2);  // zone f relative to the first zone
    load_cell<D, NC>(q, off_in + c * st, P, cR);
    const double b = ld<NC>(bn + off_in + c * st);
    double gt[7];
    const int code = face_system<EZ, PROT>(cL, cR, b, dtdx, P, rec[cur], gt);
    if (code) {
      const double bnL = ld<NC>(q[F_BX + D] + off_in + (c - 1) * st);
      const double bnR = ld<NC>(q[F_BX + D] + off_in + c * st);
      hll_face(cL, cR, bnL, bnR, code == 1, P, rec[cur]);
#pragma unroll
      for (int k = 0; k < 7; ++k) gt[k] = 0.0;
    }
    if (f >= fa) {
      // 2 g of zone f-1 from 2 g-tilde of faces f (i+1/2) and f-1 (i-1/2)
      double gz[7];
#pragma unroll
      for (int k = 0; k < 7; ++k) gz[k] = wb_sweby(gt[k], gt_p[k], P.sweby, P.minmod);
      if (f >= fa + 1) {
        // flux of face f-1 (zones f-2, f-1): g_{i} = g_p (zone f-2), g_{i+1} = gz
        double out[7];
        const Rc& fr = rec[cur ^ 1];
        if (wb_neg(fr[R_RHO])) {
#pragma unroll
          for (int m = 0; m < 7; ++m) out[m] = fr[R_FAVG + m];
          if (across && f - 1 >= 0 && f - 1 < g.n[D]) ++nhll;
        } else {
          face_flux<EZ>(fr, g_p, gz, dx_2dt, P, out);
        }
        const long long o = off_out + (c - 1) * st;
        F[F_RHO][o] = out[0];
        F[F_MX + D][o] = out[1];
        F[F_MX + T1][o] = out[2];
        F[F_MX + T2][o] = out[3];
        F[F_EN][o] = out[6];
        F[F_BX + T1][o] = out[4];
        F[F_BX + T2][o] = out[5];
      }
#pragma unroll
      for (int k = 0; k < 7; ++k) g_p[k] = gz[k];
    }
#pragma unroll
    for (int k = 0; k < 7; ++k) gt_p[k] = gt[k];
    cur ^= 1;
    cL = cR;
  }
  return nhll;
}

// ---------------------------------------------------------------- stages ---

__device__ __forceinline__ bool in_box(const WbBox& b, int i, int j, int k) {
  return i >= b.lo[0] && i <= b.hi[0] && j >= b.lo[1] && j <= b.hi[1] && k >= b.lo[2] && k <= b.hi[2];
}

// The cheap stages are split into a load of their inputs and a finish that
// computes and stores, so that the batch kernel can load a second item before
// storing the first (two memory requests in flight per thread).  Their
// arithmetic is written with explicit rounding: an item gives the same bits
// whichever inlined copy (first or second of a pair, or alone) handles it.

// Step 2: zone-centred reference EMF E = -v x B from q^n.
struct ErefIn {
  long long w;
  double rho, m[3], B[3];
};

__device__ __forceinline__ void eref_load(const WbView& v, long long qo, long long wo, int i, int j, int k,
                                          ErefIn& in) {
  const long long o = qo + wb_at(v.geo, i, j, k);
  in.w = wo + wb_at(v.geo, i, j, k);
  in.rho = v.q[F_RHO][o];
#pragma unroll
  for (int e = 0; e < 3; ++e) {
    in.m[e] = v.q[F_MX + e][o];
    in.B[e] = v.q[F_BX + e][o];
  }
}

__device__ __forceinline__ void eref_finish(const WbView& v, const ErefIn& in) {
  const double ir = wb_rcp(in.rho);
  const double vx = __dmul_rn(in.m[0], ir), vy = __dmul_rn(in.m[1], ir), vz = __dmul_rn(in.m[2], ir);
  const double bx = in.B[0], by = in.B[1], bz = in.B[2];
  v.Eref[0][in.w] = __fma_rn(vz, by, __dmul_rn(-vy, bz));
  v.Eref[1][in.w] = __fma_rn(vx, bz, __dmul_rn(-vz, bx));
  v.Eref[2][in.w] = __fma_rn(vy, bx, __dmul_rn(-vx, by));
}

__device__ __forceinline__ void eref(const WbView& v, long long qo, long long wo, int i, int j, int k) {
  ErefIn in;
  eref_load(v, qo, wo, i, j, k, in);
  eref_finish(v, in);
}

// The mean of the two one-sided differences, for a zero mass flux.  Not
// inlined: inlined, the compiler if-converts it and every warp issues its
// instructions with every lane predicated off (the FP64 pipe's warp-level
// count exceeded its thread-level count by a third in the corner-EMF kernel).
static __device__ __noinline__ double mean_diff(double xm, double ym, double x0, double y0) {
  return __dmul_rn(0.5, __dadd_rn(__dsub_rn(xm, ym), __dsub_rn(x0, y0)));
}

// Difference x - y upwind of the mass flux m: (xm - ym) from the minus-side
// zone if m > 0, (x0 - y0) from the plus-side zone if m < 0, the mean of both
// if m = 0.  The operands are selected first (integer pipe), so one FP64
// subtraction is spent; the mean is taken only by warps in which some lane
// has a zero mass flux, so the common case carries none of its arithmetic.
__device__ __forceinline__ double upwind_diff(double m, double xm, double ym, double x0, double y0) {
  const bool minus = wb_neg(m);
  double d = __dsub_rn(minus ? x0 : xm, minus ? y0 : ym);
  const bool zero = wb_zero(m);
  if (__any_sync(__activemask(), zero)) {
    const double mean = mean_diff(xm, ym, x0, y0);
    if (zero) d = mean;
  }
  return d;
}

// Steps 3 and 9: upwinded corner EMF (GS05 "CT-contact" form).  Edge along
// axis C at the low faces of axes a = C+1 and b = C+2 (cyclic).  Face EMFs
// E^a = -F_a[B_b], E^b = +F_b[B_a]; the corner value is their average plus
// one quarter of [(dE/db) at -3/4 minus (dE/db) at -1/4] and the same along
// a, each derivative taken from the zone upwind of the mass flux through the
// face it sits on (the mean of both zones when that flux is zero).
struct EdgeIn {
  long long o;
  double Ea_0, Ea_m, Eb_0, Eb_m, ma_0, ma_m, mb_0, mb_m, R00, Rm0, R0m, Rmm;
};

template <int C>
__device__ __forceinline__ void edge_load(const WbView& v, long long wo, bool corr, int i, int j, int k,
                                          EdgeIn& in) {
  constexpr int a = (C + 1) % 3, b = (C + 2) % 3;
  const WbGeo& g = v.geo;
  const long long o = wo + wb_at(g, i, j, k);
  const long long sa = a == 0 ? 1 : (a == 1 ? g.sy : g.sz);
  const long long sb = b == 0 ? 1 : (b == 1 ? g.sy : g.sz);
  WB_CHECK_ZONE(g, i - (a == 0) - (b == 0), j - (a == 1) - (b == 1), k - (a == 2) - (b == 2));
  double* const* Fa = corr ? v.Fc[a] : v.Fp[a];
  double* const* Fb = corr ? v.Fc[b] : v.Fp[b];
  const double* Er = corr ? v.Erefh[C] : v.Eref[C];
  in.o = o;
  in.Ea_0 = wb_flip(Fa[F_BX + b][o]);
  in.Ea_m = wb_flip(Fa[F_BX + b][o - sb]);
  in.Eb_0 = Fb[F_BX + a][o];
  in.Eb_m = Fb[F_BX + a][o - sa];
  in.ma_0 = Fa[F_RHO][o];
  in.ma_m = Fa[F_RHO][o - sb];
  in.mb_0 = Fb[F_RHO][o];
  in.mb_m = Fb[F_RHO][o - sa];
  in.R00 = Er[o];
  in.Rm0 = Er[o - sa];
  in.R0m = Er[o - sb];
  in.Rmm = Er[o - sa - sb];
}

template <int C>
__device__ __forceinline__ void edge_finish(const WbView& v, bool corr, const EdgeIn& in) {
  const double db_hi = upwind_diff(in.ma_0, in.Rm0, in.Eb_m, in.R00, in.Eb_0);
  const double db_lo = upwind_diff(in.ma_m, in.Eb_m, in.Rmm, in.Eb_0, in.R0m);
  const double da_hi = upwind_diff(in.mb_0, in.R0m, in.Ea_m, in.R00, in.Ea_0);
  const double da_lo = upwind_diff(in.mb_m, in.Ea_m, in.Rmm, in.Ea_0, in.Rm0);
  double* out = corr ? v.Eedgeh[C] : v.Eedge[C];
  out[in.o] = wb_quarter((in.Ea_0 + in.Ea_m) + (in.Eb_0 + in.Eb_m) + (db_lo - db_hi) + (da_lo - da_hi));
}

template <int C>
__device__ __forceinline__ void edge(const WbView& v, long long wo, bool corr, int i, int j, int k) {
  EdgeIn in;
  edge_load<C>(v, wo, corr, i, j, k, in);
  edge_finish<C>(v, corr, in);
}

// Steps 4 and 11: b_out = b_in - tau curl E on the faces normal to D.
// Step 4 writes b^{n+1/2} to the workspace, Step 11 updates b in place.
struct CtIn {
  long long w, q;
  double Eb0, Eb1, Ea0, Ea1, b;
};

template <int D>
__device__ __forceinline__ void ct_load(const WbView& v, long long qo, long long wo, bool fin, int i, int j,
                                        int k, CtIn& in) {
  constexpr int a = (D + 1) % 3, b = (D + 2) % 3;
  const WbGeo& g = v.geo;
  in.w = wo + wb_at(g, i, j, k);
  in.q = qo + wb_at(g, i, j, k);
  const long long sa = a == 0 ? 1 : (a == 1 ? g.sy : g.sz);
  const long long sb = b == 0 ? 1 : (b == 1 ? g.sy : g.sz);
  WB_CHECK_ZONE(g, i + (a == 0), j + (a == 1), k + (a == 2));
  WB_CHECK_ZONE(g, i + (b == 0), j + (b == 1), k + (b == 2));
  const double* Eb = fin ? v.Eedgeh[b] : v.Eedge[b];
  const double* Ea = fin ? v.Eedgeh[a] : v.Eedge[a];
  in.Eb0 = Eb[in.w];
  in.Eb1 = Eb[in.w + sa];
  in.Ea0 = Ea[in.w];
  in.Ea1 = Ea[in.w + sb];
  in.b = v.b[D][in.q];
}

template <int D>
__device__ __forceinline__ void ct_finish(const WbView& v, bool fin, double dt, const CtIn& in) {
  constexpr int a = (D + 1) % 3, b = (D + 2) % 3;
  const double tau = fin ? dt : wb_half(dt);
  const double curl = __fma_rn(in.Eb1 - in.Eb0, v.geo.idx[a], __dmul_rn(in.Ea0 - in.Ea1, v.geo.idx[b]));
  const double bn = __fma_rn(-tau, curl, in.b);
  if (fin) v.b[D][in.q] = bn;
  else v.bh[D][in.w] = bn;
}

template <int D>
__device__ __forceinline__ void ct(const WbView& v, long long qo, long long wo, bool fin, double dt,
                                   int i, int j, int k) {
  CtIn in;
  ct_load<D>(v, qo, wo, fin, i, j, k, in);
  ct_finish<D>(v, fin, dt, in);
}

// Steps 5 and 7: q^{n+1/2}_D = q^n - dt/2 (transverse flux divergence)
// + dt/2 S_D, zone B_D := mean of b_D^{n+1/2}, with the GS08-type div B
// source S_D built from face differences of b^n and minmod pairings.
//
// Zone quantities shared by the directions: velocity v, zone field B, B_e v_e,
// the face-field differences scaled by dt/2 (h db_e = dt/2 (b_e+ - b_e)/dx_e;
// minmod commutes with the positive factor dt/2), the flux-difference factors
// c_e = dt/2 / dx_e and the transverse flux differences dF_e = F_e+ - F_e.
// The arithmetic is written with explicit rounding: the same bits in every
// kernel it is inlined into (the grid path, both forms of the batch path).
struct TransZone {
  double qn[8];
  double vv[3], B[3], Bv[3], hdb[3], c[3];
  double dF[3][8];
};

__device__ __forceinline__ void trans_zone(const WbView& v, long long q, long long w, double dt,
                                           int need, TransZone& z) {
  const WbGeo& g = v.geo;
  const long long s[3] = {1, g.sy, g.sz};
  const double hdt = wb_half(dt);
#pragma unroll
  for (int cc = 0; cc < 8; ++cc) z.qn[cc] = v.q[cc][q];
  const double ir = wb_rcp(z.qn[F_RHO]);
#pragma unroll
  for (int e = 0; e < 3; ++e) {
    z.vv[e] = __dmul_rn(z.qn[F_MX + e], ir);
    z.B[e] = z.qn[F_BX + e];
    z.Bv[e] = __dmul_rn(z.B[e], z.vv[e]);
    z.c[e] = __dmul_rn(hdt, g.idx[e]);
    z.hdb[e] = __dmul_rn(__dsub_rn(v.b[e][q + s[e]], v.b[e][q]), z.c[e]);
  }
#pragma unroll
  for (int e = 0; e < 3; ++e) {
#pragma unroll
    for (int cc = 0; cc < 8; ++cc) {
      if (cc == F_BX + e || !(need & (1 << e))) { z.dF[e][cc] = 0.0; continue; }
      z.dF[e][cc] = __dsub_rn(v.Fp[e][cc][w + s[e]], v.Fp[e][cc][w]);
    }
  }
}

// q^{n+1/2}_D of one zone from its shared quantities.  The t1 (t2) field
// component is carried only by the t2 (t1) sweep; density has no source.
template <int D>
__device__ __forceinline__ void trans_dir(const WbView& v, long long w, const TransZone& z) {
  constexpr int t1 = (D + 1) % 3, t2 = (D + 2) % 3;
  const long long sD = D == 0 ? 1 : (D == 1 ? v.geo.sy : v.geo.sz);
  const double hm2 = wb_minmod(z.hdb[D], wb_flip(z.hdb[t1]));  // for the t2 field component
  const double hm1 = wb_minmod(z.hdb[D], wb_flip(z.hdb[t2]));  // for the t1 field component
  const double hSe = __fma_rn(z.Bv[t1], hm1, __dmul_rn(z.Bv[t2], hm2));
  const double c1 = z.c[t1], c2 = z.c[t2];
  double u[8];
#pragma unroll
  for (int cc = F_RHO; cc <= F_EN; ++cc)
    u[cc] = __fma_rn(-c2, z.dF[t2][cc], __fma_rn(-c1, z.dF[t1][cc], z.qn[cc]));
  v.qh[D][F_RHO][w] = u[F_RHO];
#pragma unroll
  for (int e = 0; e < 3; ++e) v.qh[D][F_MX + e][w] = __fma_rn(z.B[e], z.hdb[D], u[F_MX + e]);
  v.qh[D][F_EN][w] = __dadd_rn(u[F_EN], hSe);
  v.qh[D][F_BX + t1][w] = __fma_rn(z.vv[t1], hm1, __fma_rn(-c2, z.dF[t2][F_BX + t1], z.qn[F_BX + t1]));
  v.qh[D][F_BX + t2][w] = __fma_rn(z.vv[t2], hm2, __fma_rn(-c1, z.dF[t1][F_BX + t2], z.qn[F_BX + t2]));
  v.qh[D][F_BX + D][w] = wb_half(__dadd_rn(v.bh[D][w], v.bh[D][w + sD]));
}

// The directions in mask (bit d) at one zone, sharing the zone quantities and
// each transverse flux difference between the two states that use it.
__device__ __forceinline__ void transverse_set(const WbView& v, long long qo, long long wo, double dt,
                                               int mask, int i, int j, int k) {
  const long long q = qo + wb_at(v.geo, i, j, k);
  const long long w = wo + wb_at(v.geo, i, j, k);
  WB_CHECK_ZONE(v.geo, i + 1, j + 1, k + 1);  // the high neighbours of every axis
  // flux differences of every direction some state needs
  int need = 0;
#pragma unroll
  for (int e = 0; e < 3; ++e)
    if (mask & ~(1 << e)) need |= 1 << e;
  TransZone z;
  trans_zone(v, q, w, dt, need, z);
  if (mask & 1) trans_dir<0>(v, w, z);
  if (mask & 2) trans_dir<1>(v, w, z);
  if (mask & 4) trans_dir<2>(v, w, z);
}

// Step 8: reference EMF at n+1/2 from v of q^n - dt/2 div F* and B = mean of
// b^{n+1/2}.
struct ErefHalfIn {
  long long w;
  double q[4];        // rho, M of q^n
  double dF[4][3];    // F*_e+ - F*_e for rho, M
  double bh[3][2];    // b^{n+1/2} on the low and high faces
};

__device__ __forceinline__ void eref_half_load(const WbView& v, long long qo, long long wo, int i, int j,
                                               int k, ErefHalfIn& in) {
  const WbGeo& g = v.geo;
  const long long q = qo + wb_at(g, i, j, k);
  const long long w = wo + wb_at(g, i, j, k);
  const long long s[3] = {1, g.sy, g.sz};
  WB_CHECK_ZONE(g, i + 1, j + 1, k + 1);
  in.w = w;
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    in.q[c] = v.q[c][q];
#pragma unroll
    for (int e = 0; e < 3; ++e) in.dF[c][e] = v.Fc[e][c][w + s[e]] - v.Fc[e][c][w];
  }
#pragma unroll
  for (int e = 0; e < 3; ++e) {
    in.bh[e][0] = v.bh[e][w];
    in.bh[e][1] = v.bh[e][w + s[e]];
  }
}

__device__ __forceinline__ void eref_half_finish(const WbView& v, double dt, const ErefHalfIn& in) {
  const WbGeo& g = v.geo;
  const double hdt = wb_half(dt);
  double u[4];
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    double div = __dmul_rn(in.dF[c][0], g.idx[0]);
    div = __fma_rn(in.dF[c][1], g.idx[1], div);
    div = __fma_rn(in.dF[c][2], g.idx[2], div);
    u[c] = __fma_rn(-hdt, div, in.q[c]);
  }
  const double ir = wb_rcp(u[0]);
  const double vx = __dmul_rn(u[1], ir), vy = __dmul_rn(u[2], ir), vz = __dmul_rn(u[3], ir);
  double B[3];
#pragma unroll
  for (int e = 0; e < 3; ++e) B[e] = wb_half(in.bh[e][0] + in.bh[e][1]);
  v.Erefh[0][in.w] = __fma_rn(vz, B[1], __dmul_rn(-vy, B[2]));
  v.Erefh[1][in.w] = __fma_rn(vx, B[2], __dmul_rn(-vz, B[0]));
  v.Erefh[2][in.w] = __fma_rn(vy, B[0], __dmul_rn(-vx, B[1]));
}

__device__ __forceinline__ void eref_half(const WbView& v, long long qo, long long wo, double dt,
                                          int i, int j, int k) {
  ErefHalfIn in;
  eref_half_load(v, qo, wo, i, j, k, in);
  eref_half_finish(v, dt, in);
}

// sqrt for the CFL rate; inputs below the normal range (or not > 0) give 0
__device__ __forceinline__ double wb_sqrt_fast(double x) {
  return wb_normal_pos(x) ? __dmul_rn(x, wb_rsqrt(x)) : 0.0;
}

// CFL signal rate sum_d (|v_d| + c_f,d)/dx_d of one zone (Sec. 3 fast speed)
// from 1/rho, the velocity, the gas pressure and the zone field.  The fast
// speed along d: c_f^2 = (S + sqrt(disc_d))/2 with S = a^2 + |B|^2/rho and
// disc_d = (a^2 - c_n^2)^2 + c_t^2 (c_t^2 + 2 (a^2 + c_n^2)) (the sum of
// non-negative terms), c_n^2 = B_d^2/rho, c_t^2 = |B|^2/rho - c_n^2.
//
// Written with explicit rounding: the final update (for the next step) and
// the rate of a freshly loaded state are inlined in different kernels and
// must give the same bits, or a resumed run would take a different dt.
__device__ __forceinline__ double signal_rate_core(double ir, const double vv[3], double p,
                                                   const double B[3], const WbPhys& P,
                                                   const WbGeo& g) {
  const double a2 = __dmul_rn(__dmul_rn(P.gamma, p), ir);
  double cn2[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) cn2[d] = __dmul_rn(__dmul_rn(B[d], B[d]), ir);
  const double bbi = __dadd_rn(__dadd_rn(cn2[0], cn2[1]), cn2[2]);
  const double S = __dadd_rn(a2, bbi);
  double w = 0.0;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const double ct2 = __dsub_rn(bbi, cn2[d]);
    const double dd = __dsub_rn(a2, cn2[d]);
    const double disc = __fma_rn(dd, dd, __dmul_rn(ct2, __fma_rn(2.0, __dadd_rn(a2, cn2[d]), ct2)));
    const double cf = wb_sqrt_fast(wb_half(__dadd_rn(S, wb_sqrt_fast(disc))));
    w = __fma_rn(__dadd_rn(wb_fabs(vv[d]), cf), g.idx[d], w);
  }
  return w;
}

// FP32 copy of a double by exponent re-biasing and mantissa truncation on the
// integer pipe (relative error below 2^-23).  Zero maps to zero; magnitudes
// outside [2^-60, 2^61), subnormals, inf and NaN clear *ok.
__device__ __forceinline__ float wb_f32_of(double x, bool* ok) {
  const long long b = __double_as_longlong(x);
  if (wb_zero(x)) return 0.0f;
  const int hi = (int)(b >> 32);
  const int ex = (hi >> 20) & 0x7ff;
  if (ex < 1023 - 60 || ex > 1023 + 60) {
    *ok = false;
    return 0.0f;
  }
  const unsigned sign = (unsigned)hi & 0x80000000u;
  const unsigned mant = (unsigned)((b >> 29) & 0x7fffff);
  return __uint_as_float(sign | ((unsigned)(ex - 1023 + 127) << 23) | mant);
}

// The CFL signal rate in FP32 (same formula as signal_rate_core, relative
// error well below 1e-5 for inputs the conversion accepts; *ok cleared when it
// cannot vouch for one).  p enters already computed in FP64, so the rate has
// no cancellation left: every term of the sum and of the discriminant is
// non-negative except a^2 - c_n^2, which only enters squared.
__device__ __forceinline__ float signal_rate_f32(double ir, const double vv[3], double p, const double B[3],
                                                 const WbPhys& P, const WbGeo& g, bool* ok) {
  const float fir = wb_f32_of(ir, ok), fp = wb_f32_of(p, ok);
  float fv[3], sq[3], fidx[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    fv[d] = fabsf(wb_f32_of(vv[d], ok));
    const float b = wb_f32_of(B[d], ok);
    sq[d] = b * b;
    fidx[d] = wb_f32_of(g.idx[d], ok);
  }
  const float a2 = P.gamma_f * fp * fir;
  float w = 0.0f;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const float cn2 = sq[d] * fir;
    const float ct2 = (sq[(d + 1) % 3] + sq[(d + 2) % 3]) * fir;
    const float dd = a2 - cn2;
    const float disc = dd * dd + ct2 * (ct2 + 2.0f * (a2 + cn2));
    const float cf = sqrtf(0.5f * (a2 + cn2 + ct2 + sqrtf(disc)));
    w += (fv[d] + cf) * fidx[d];
  }
  return w;
}

// The zone's exact (FP64) signal rate when it could be the largest of the
// box, else 0.  The max over zones is all the time step needs: a zone whose
// FP32 screen r32 lies below 0.9999 of the running maximum of the screens
// already seen cannot hold the largest exact rate (with screen errors e < 1e-5,
// the largest exact rate R* has r32 >= R*(1 - e) while the running maximum
// is <= R*(1 + e)), so it skips the FP64 evaluation.  The maximum of the
// returned values is bit-identical to the maximum of signal_rate_core over
// all zones.
__device__ __forceinline__ double screened_rate(double ir, const double vv[3], double p, const double B[3],
                                                const WbPhys& P, const WbGeo& g, WbScalars* scal) {
  bool ok = true;
  const float r32 = signal_rate_f32(ir, vv, p, B, P, g, &ok);
  const float G = __uint_as_float(*(volatile unsigned*)&scal->rate_screen);
  if (ok && r32 < 0.9999f * G) return 0.0;
  if (ok && r32 > G) atomicMax(&scal->rate_screen, __float_as_uint(r32));
  return signal_rate_core(ir, vv, p, B, P, g);
}

// kinetic energy density rho v^2 / 2 from the momentum and the velocity
__device__ __forceinline__ double kinetic(const double m[3], const double vv[3]) {
  return wb_half(__fma_rn(m[2], vv[2], __fma_rn(m[1], vv[1], __dmul_rn(m[0], vv[0]))));
}

// The signal rate of one stored zone (conserved state and zone field), or 0
// when the screen shows it cannot be the box's largest (screened_rate).
__device__ __forceinline__ double signal_rate(double rho, double mx, double my, double mz, double e,
                                              double bx, double by, double bz, const WbPhys& P,
                                              const WbGeo& g, WbScalars* scal) {
  const double ir = wb_rcp(rho);
  const double m[3] = {mx, my, mz};
  const double vv[3] = {mx * ir, my * ir, mz * ir};
  const double B[3] = {bx, by, bz};
  const double me = wb_half(fma(bz, bz, fma(by, by, bx * bx)));
  const double p = P.gm1 * (e - kinetic(m, vv) - me);
  if (!(rho > 0.0)) return __longlong_as_double(0x7ff8000000000000LL);
  return screened_rate(ir, vv, p, B, P, g, scal);
}

// Step 10 (+ the zone field of Step 11, floors and the next step's signal
// rate): U^{n+1} = ((U^n - dt/dx dF*) - dt/dy dG*) - dt/dz dH* at one interior
// zone, zone B = mean of b^{n+1}.  Returns the zone's signal rate (NaN if the
// state is unphysical); floor hits are added to *hits.  The rate is the one
// signal_rate gives for the stored result.  ohi: bit d set when the zone
// row's high end along d is the domain boundary of an outflow axis, whose
// boundary face the ghost fill makes a copy of the last owned face (the
// zero-gradient rule); the last zone's field then averages that copy, so the
// stored state is the one a load of the same faces gives.
__device__ __forceinline__ double final_update(const WbView& v, long long qo, long long wo,
                                               double dt, const WbPhys& P, int i, int j, int k,
                                               int ohi, int* hits, int* bad) {
  const WbGeo& g = v.geo;
  const long long q = qo + wb_at(g, i, j, k);
  const long long wi = wo + wb_at(g, i, j, k);
  WB_CHECK_ZONE(g, i + 1, j + 1, k + 1);
  const long long s[3] = {1, g.sy, g.sz};
  // explicit rounding: the same bits in every kernel this is inlined into
  const double cx = __dmul_rn(dt, g.idx[0]), cy = __dmul_rn(dt, g.idx[1]), cz = __dmul_rn(dt, g.idx[2]);
  double u[5];
#pragma unroll
  for (int c = 0; c < 5; ++c) {
    double x = v.q[c][q];
    x = __fma_rn(-cx, __dsub_rn(v.Fc[0][c][wi + 1], v.Fc[0][c][wi]), x);
    x = __fma_rn(-cy, __dsub_rn(v.Fc[1][c][wi + s[1]], v.Fc[1][c][wi]), x);
    x = __fma_rn(-cz, __dsub_rn(v.Fc[2][c][wi + s[2]], v.Fc[2][c][wi]), x);
    u[c] = x;
  }
  double B[3];
  const int idx[3] = {i, j, k};
#pragma unroll
  for (int e = 0; e < 3; ++e) {
    const bool last = ((ohi >> e) & 1) && idx[e] == g.n[e] - 1;
    const double lo = v.b[e][q];
    const double hi = last ? lo : v.b[e][q + s[e]];
    B[e] = wb_half(__dadd_rn(lo, hi));
    v.q[F_BX + e][q] = B[e];
  }
  // the tests below run on the integer pipe (FP64 compares take FP64 issue)
  if (wb_below_floor(u[0], P.rho_floor)) { u[0] = P.rho_floor; ++*hits; }
  const double ir = wb_rcp(u[0]);
  const double m[3] = {u[1], u[2], u[3]};
  const double vv[3] = {__dmul_rn(u[1], ir), __dmul_rn(u[2], ir), __dmul_rn(u[3], ir)};
  const double ke = kinetic(m, vv);
  const double me = wb_half(__fma_rn(B[2], B[2], __fma_rn(B[1], B[1], __dmul_rn(B[0], B[0]))));
  double p = __dmul_rn(P.gm1, __dsub_rn(__dsub_rn(u[4], ke), me));
  if (wb_below_floor(p, P.p_floor)) {
    u[4] = __dadd_rn(__fma_rn(P.p_floor, P.inv_gm1, ke), me);
    p = __dmul_rn(P.gm1, __dsub_rn(__dsub_rn(u[4], ke), me));
    ++*hits;
  }
  const bool fin = wb_pos(u[0]) && wb_finite(u[1]) && wb_finite(u[2]) && wb_finite(u[3]) &&
                   wb_finite(u[4]) && wb_finite(p);
#pragma unroll
  for (int c = 0; c < 5; ++c) v.q[c][q] = u[c];
  if (!fin) {
    ++*bad;
    return __longlong_as_double(0x7ff8000000000000LL);
  }
  return screened_rate(ir, vv, p, B, P, g, v.scal);
}

// The shell of ghost points within `depth` zones of a box's interior,
// enumerated as the two z slabs of the depth-padded box, then the two y slabs
// and the two x slabs of its interior z (and y) range.  Used for the periodic
// images of intermediates (interior-only stages of a box periodic on every
// axis) and for the ghost fill of a box that is its own domain.
__host__ __device__ __forceinline__ long long shell_count(const WbGeo& g, int depth) {
  const long long w = 2 * depth;
  return (long long)(g.n[0] + w) * (g.n[1] + w) * w + (long long)(g.n[0] + w) * w * g.n[2] +
         w * g.n[1] * (long long)g.n[2];
}

// Shell point t (0 <= t < shell_count) -> its zone index (i, j, k).
__device__ __forceinline__ void shell_point(const WbGeo& g, int depth, long long t, int* pi, int* pj,
                                            int* pk) {
  const int n0 = g.n[0], n1 = g.n[1], n2 = g.n[2];
  const int w = 2 * depth;
  const unsigned e0 = (unsigned)(n0 + w), e1 = (unsigned)(n1 + w);
  const unsigned long long zs = (unsigned long long)e0 * e1 * w;
  const unsigned long long ys = (unsigned long long)e0 * w * n2;
  unsigned long long u = (unsigned long long)t;
  int i, j, k;
  if (u < zs) {
    const unsigned r = (unsigned)(u % ((unsigned long long)e0 * e1));
    const int dz = (int)(u / ((unsigned long long)e0 * e1));
    i = (int)(r % e0) - depth;
    j = (int)(r / e0) - depth;
    k = dz < depth ? dz - depth : n2 + dz - depth;
  } else if ((u -= zs) < ys) {
    const unsigned per = e0 * (unsigned)w;
    k = (int)(u / per);
    const unsigned r = (unsigned)(u % per);
    const int dy = (int)(r / e0);
    i = (int)(r % e0) - depth;
    j = dy < depth ? dy - depth : n1 + dy - depth;
  } else {
    u -= ys;
    const unsigned r = (unsigned)(u / (unsigned)w);
    const int dx = (int)(u % (unsigned)w);
    j = (int)(r % (unsigned)n1);
    k = (int)(r / (unsigned)n1);
    i = dx < depth ? dx - depth : n0 + dx - depth;
  }
  *pi = i;
  *pj = j;
  *pk = k;
}

// Shell point t -> its offset and the offset of the interior point it is a
// periodic image of.
__device__ __forceinline__ void wrap_shell_point(const WbGeo& g, int depth, long long t, long long* dst,
                                                 long long* src) {
  int i, j, k;
  shell_point(g, depth, t, &i, &j, &k);
  const int n0 = g.n[0], n1 = g.n[1], n2 = g.n[2];
  *dst = wb_at(g, i, j, k);
  *src = wb_at(g, ((i % n0) + n0) % n0, ((j % n1) + n1) % n1, ((k % n2) + n2) % n2);
}

// Ghost fill of a box that is its own periodic/outflow domain (no patches):
// ghost point t of the 5-zone shell (shell_point order) copies the wrapped
// (periodic) or clamped (outflow) interior zone of the same box, all 11
// fields; face arrays use the same rule on their face index.
__device__ __forceinline__ void halo_self_offsets(const WbGeo& g, const int bc[3], long long t, long long* dst,
                                                  long long* src_off) {
  int loc[3];
  shell_point(g, WB_NG, t, &loc[0], &loc[1], &loc[2]);
  int src[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    int x = loc[d];
    const int n = g.n[d];
    if (x < 0 || x >= n) {
      if (bc[d] == 0) x = ((x % n) + n) % n;
      else x = x < 0 ? 0 : n - 1;
    }
    src[d] = x;
  }
  *dst = wb_at(g, loc[0], loc[1], loc[2]);
  *src_off = wb_at(g, src[0], src[1], src[2]);
}

__device__ __forceinline__ void halo_self(const WbView& v, long long qo, const int bc[3], long long t) {
  long long dst, so;
  halo_self_offsets(v.geo, bc, t, &dst, &so);
  dst += qo;
  so += qo;
#pragma unroll
  for (int c = 0; c < 8; ++c) v.q[c][dst] = v.q[c][so];
#pragma unroll
  for (int c = 0; c < 3; ++c) v.b[c][dst] = v.b[c][so];
}

}  // namespace wbu
