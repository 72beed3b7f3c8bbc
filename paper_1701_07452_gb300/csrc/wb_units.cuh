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
  c.ir = c.isr * c.isr;
  c.sr = c.rho * c.isr;
  c.vn = c.mn * c.ir;
  c.vt1 = c.mt1 * c.ir;
  c.vt2 = c.mt2 * c.ir;
  const double ke = 0.5 * (c.mn * c.vn + c.mt1 * c.vt1 + c.mt2 * c.vt2);
  const double bt2 = c.bt1 * c.bt1 + c.bt2 * c.bt2;
  const double bn2 = bn * bn;
  const double me = 0.5 * (bn2 + bt2);
  const double p = P.gm1 * (e - ke - me);
  const double pstar = p + me;
  c.eref = e - 0.5 * bn2;
  c.hr = (P.g_over_gm1 * p + ke + bt2) * c.ir;
  // half fluxes: the face needs (F_L + F_R) / 2
  const double hmn = 0.5 * c.mn, hvn = 0.5 * c.vn, hbn = 0.5 * bn;
  c.F[0] = hmn;
  c.F[1] = fma(hmn, c.vn, 0.5 * (pstar - bn2));
  c.F[2] = hmn * c.vt1 - hbn * c.bt1;
  c.F[3] = hmn * c.vt2 - hbn * c.bt2;
  c.F[4] = c.bt1 * hvn - hbn * c.vt1;
  c.F[5] = c.bt2 * hvn - hbn * c.vt2;
  c.F[6] = (e + pstar) * hvn - hbn * (bn * c.vn + c.bt1 * c.vt1 + c.bt2 * c.vt2);
}

// Per-face record (shared memory, structure of arrays over the block).
// R_PG = rho a^2 / (gamma-1); R_KX = v^2/2 + (gamma-2)/(gamma-1) X.
enum {
  R_AL = 0, R_NU = 7, R_RHO = 14, R_SRHO, R_A, R_PG, R_CF, R_CS, R_AF, R_AS, R_B1, R_B2, R_S,
  R_VN, R_VT1, R_VT2, R_BT1, R_BT2, R_KX, R_FAVG, R_WORDS = R_FAVG + 7
};

struct Rec {
  double* p;
  __device__ __forceinline__ double& operator[](int w) const { return p[w * kBlock]; }
};

// Q_k(nu) - nu^2 for the g-tilde of App. A.  Waves in the compile-time mask
// EZ have eps_k = 0, where Q is |nu|; the branch test runs on the integer pipe.
template <int EZ>
__device__ __forceinline__ double Qk_m_nu2(double nu, int k, const WbPhys& P) {
  const double n2 = nu * nu;
  if (EZ & (1 << k)) return fabs(nu) - n2;
  return (wb_abs_less(nu, P.two_eps[k]) ? fma(n2, P.inv4eps[k], P.eps[k]) : fabs(nu)) - n2;
}

// Gas pressure of a zone from its sweep-frame fields (Sec. 3, Eq. totenergy)
__device__ __forceinline__ double zone_pressure(const Cell& c, const WbPhys& P) {
  return P.gm1 * (c.eref - 0.5 * (c.mn * c.vn + c.mt1 * c.vt1 + c.mt2 * c.vt2) -
                  0.5 * (c.bt1 * c.bt1 + c.bt2 * c.bt2));
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
  const double r1 = L.rho + al[0] * (rho * af), p1 = pL + al[0] * (ra2 * af);
  if (r1 < P.prot_rho || p1 < P.prot_p) return true;
  const double r3 = r1 + al[2] * (rho * as), p3 = p1 + al[2] * (ra2 * as);
  if (r3 < P.prot_rho || p3 < P.prot_p) return true;
  const double r4 = r3 + al[3];
  if (r4 < P.prot_rho) return true;
  const double r5 = r4 + al[4] * (rho * as), p5 = p3 + al[4] * (ra2 * as);
  return r5 < P.prot_rho || p5 < P.prot_p;
}

// Fast speed of one zone along the sweep axis with its own zone field (Sec. 3)
__device__ __forceinline__ double zone_fast_speed(const Cell& c, double bn, const WbPhys& P) {
  const double a2 = P.gamma * zone_pressure(c, P) / c.rho;
  const double b2 = (bn * bn + c.bt1 * c.bt1 + c.bt2 * c.bt2) / c.rho;
  const double s = a2 + b2;
  double disc = s * s - 4.0 * a2 * bn * bn / c.rho;
  if (disc < 0.0) disc = 0.0;
  return sqrt(0.5 * (s + sqrt(disc)));
}

// Marker of a face record that holds a finished HLL flux (a Roe density is > 0)
constexpr double kHllFace = -1.0;

// HLL flux of App. A into the record of one face:
//   b+ = max(a_max, vR + cfR, 0), b- = min(a_min, vL - cfL, 0),
//   u = (b+ F_L - b- F_R + b+ b- (q_R - q_L)) / (b+ - b-),
// with a_max, a_min = vn_ +- cf_ of the Roe state when it exists (roe), the
// Einfeldt sign of the F_R term (the printed +b- F_R is not consistent), and
// bounds +-max(|v| + c_f) if both speeds vanish.  Rare path.
__device__ __forceinline__ void hll_face(const Cell& L, const Cell& R, double bnL, double bnR, bool roe,
                                      const WbPhys& P, const Rec& f) {
  const double cfL = zone_fast_speed(L, bnL, P), cfR = zone_fast_speed(R, bnR, P);
  double bp = fmax(R.vn + cfR, 0.0);
  double bm = fmin(L.vn - cfL, 0.0);
  if (roe) {
    bp = fmax(bp, f[R_VN] + f[R_CF]);
    bm = fmin(bm, f[R_VN] - f[R_CF]);
  }
  if (!(bp - bm > 0.0)) {
    const double sp = fmax(fabs(L.vn) + cfL, fabs(R.vn) + cfR);
    bp = sp;
    bm = -sp;
  }
  const double dq[7] = {R.rho - L.rho, R.mn - L.mn, R.mt1 - L.mt1, R.mt2 - L.mt2,
                        R.bt1 - L.bt1, R.bt2 - L.bt2, R.eref - L.eref};
  const double inv = 1.0 / (bp - bm);
#pragma unroll
  for (int m = 0; m < 7; ++m) {
    // the zone fluxes hold F/2
    const double FL = 2.0 * L.F[m], FR = 2.0 * R.F[m];
    f[R_FAVG + m] = (bp * FL - bm * FR + bp * bm * dq[m]) * inv;
  }
  f[R_RHO] = kHllFace;
}

// Roe state, eigen-system, alpha_k, nu_k and g-tilde_k of one interface.
// Returns 0 for an MHDTVD face, 1 when the protection floor asks for the HLL
// flux (the record holds the Roe state), 2 when the Roe state has no real
// sound speed (HLL without Roe speeds).  The protection test is compiled in
// only when PROT is set.
template <int EZ, bool PROT>
__device__ __forceinline__ int face_system(const Cell& L, const Cell& R, double b, double dtdx,
                                           const WbPhys& P, const Rec& f, double gt[7]) {
  const double iD = wb_rcp(L.sr + R.sr);
  const double wL = L.sr * iD, wR = R.sr * iD;
  const double rho = L.sr * R.sr;
  const double irho = L.isr * R.isr;
  const double vn = wL * L.vn + wR * R.vn;
  const double vt1 = wL * L.vt1 + wR * R.vt1;
  const double vt2 = wL * L.vt2 + wR * R.vt2;
  const double bt1 = wR * L.bt1 + wL * R.bt1;
  const double bt2 = wR * L.bt2 + wL * R.bt2;
  const double b2 = b * b;
  // H = wL (h_L + b^2)/rho_L + wR (h_R + b^2)/rho_R, with wL/rho_L + wR/rho_R = 1/rho_
  const double H = fma(b2, irho, wL * L.hr + wR * R.hr);
  const double dbt1 = R.bt1 - L.bt1, dbt2 = R.bt2 - L.bt2;
  const double gX = P.hgm2 * ((dbt1 * dbt1 + dbt2 * dbt2) * (iD * iD));  // (gamma-2) X
  const double hv2 = 0.5 * (vn * vn + vt1 * vt1 + vt2 * vt2);
  const double bt2s = bt1 * bt1 + bt2 * bt2;
  const double a2 = P.gm1 * (H - hv2 - (b2 + bt2s) * irho) - gX;
  if (!wb_normal_pos(a2)) return 2;
  const double isrho = wb_rsqrt(rho);
  const double srho = rho * isrho;
  const double ca2 = b2 * irho, ct2 = bt2s * irho;
  const double dac = a2 - ca2;
  const double disc = dac * dac + ct2 * (ct2 + 2.0 * (a2 + ca2));
  const double sum = a2 + ca2 + ct2;
  double rsd = 0.0, sd = 0.0;
  if (wb_normal_pos(disc)) {  // a subnormal discriminant is degenerate (sd ~ 0)
    rsd = wb_rsqrt(disc);
    sd = disc * rsd;
  }
  const double cf2 = 0.5 * (sum + sd);
  const double icf = wb_rsqrt(cf2);
  const double ia = wb_rsqrt(a2);
  const double a = a2 * ia;
  const double ca = fabs(b) * isrho;
  const double cf = cf2 * icf;
  const double cs = a * ca * icf;  // c_f c_s = a c_a
  double af, as;
  if (wb_le_nonneg(sd, 1e-12 * sum)) {
    const bool fast = wb_le_nonneg(ca2, a2);
    af = fast ? 1.0 : 0.0;
    as = fast ? 0.0 : 1.0;
  } else {
    // cf^2 - a^2 and cf^2 - ca^2 without cancellation; at most one of the
    // two needs a quotient
    const double t1 = ca2 + ct2 - a2;
    const double t2 = a2 - ca2 + ct2;
    const bool n1 = wb_neg(t1), n2 = wb_neg(t2);
    double qd = 0.0;
    if (n1 || n2) {
      const double num = n1 ? 2.0 * a2 * ct2 : 2.0 * ca2 * ct2;
      const double den = n1 ? sd - t1 : sd - t2;
      qd = num * wb_rcp(den);
    }
    const double cf2_a2 = n1 ? qd : 0.5 * (t1 + sd);
    const double cf2_ca2 = n2 ? qd : 0.5 * (t2 + sd);
    const double af2 = wb_clamp01(a2 * cf2_ca2 * (icf * icf) * rsd);
    const double as2 = wb_clamp01(cf2_a2 * rsd);
    // subnormal squares (from underflowing transverse fields) count as 0
    af = wb_normal_pos(af2) ? af2 * wb_rsqrt(af2) : 0.0;
    as = wb_normal_pos(as2) ? as2 * wb_rsqrt(as2) : 0.0;
  }
  const double ra2 = rho * a2;
  double b1n, b2n;
  if (wb_le_nonneg(bt2s, 1e-24 * (ra2 + b2 + bt2s))) {
    b1n = b2n = 0.70710678118654752440;
  } else {
    const double ib = wb_rsqrt(bt2s);
    b1n = bt1 * ib;
    b2n = bt2 * ib;
  }
  const double S = wb_sgn(b);
  // primitive differences of the 7-variable system; the velocity differences
  // are kept times rho_ (dv' = rho_ dv), the 1/rho_ goes into the coefficients
  const double drho = R.rho - L.rho;
  const double dmn = R.mn - L.mn, dmt1 = R.mt1 - L.mt1, dmt2 = R.mt2 - L.mt2;
  const double de = R.eref - L.eref;
  const double dvn = dmn - vn * drho;
  const double dvt1 = dmt1 - vt1 * drho;
  const double dvt2 = dmt2 - vt2 * drho;
  const double dp = P.gm1 * (de - (vn * dmn + vt1 * dmt1 + vt2 * dmt2) + hv2 * drho -
                             (bt1 * dbt1 + bt2 * dbt2)) - gX * drho;
  // projections on the transverse field direction beta and its normal; S = sign(b)
  const double dvbS = wb_xsgn(b1n * dvt1 + b2n * dvt2, S), dvp = -b2n * dvt1 + b1n * dvt2;
  const double dbb = b1n * dbt1 + b2n * dbt2, dbpS = wb_xsgn(-b2n * dbt1 + b1n * dbt2, S);
  const double ia2 = ia * ia;
  const double hir = 0.5 * irho, hisr = 0.5 * isrho;
  const double i2ra = hisr * ia;         // 1 / (2 sqrt(rho) a)
  const double ri2a2 = hir * ia2;        // 1 / (2 rho a^2)
  const double dpr = dp * ri2a2;
  const double afcf = af * cf, ascs = as * cs;
  const double Af = (afcf * dvn - ascs * dvbS) * ri2a2;
  const double Cf = as * dbb * i2ra + af * dpr;
  const double As = (ascs * dvn + afcf * dvbS) * ri2a2;
  const double Cs = -af * dbb * i2ra + as * dpr;
  const double hAa = hisr * dbpS;
  double al[7];
  al[0] = Cf - Af;
  al[6] = Cf + Af;
  al[2] = Cs - As;
  al[4] = Cs + As;
  al[1] = fma(hir, dvp, hAa);
  al[5] = fma(hir, dvp, -hAa);
  al[3] = fma(-dp, ia2, drho);
  // nu_k = (dt/dx) a_k for the eigenvalues a_1..a_7 (Sec. 3)
  const double tvn = dtdx * vn, tcf = dtdx * cf, tca = dtdx * ca, tcs = dtdx * cs;
  const double nuk[7] = {tvn - tcf, tvn - tca, tvn - tcs, tvn, tvn + tcs, tvn + tca, tvn + tcf};
#pragma unroll
  for (int k = 0; k < 7; ++k) {
    const double nu = nuk[k];
    f[R_AL + k] = al[k];
    f[R_NU + k] = nu;
    gt[k] = Qk_m_nu2<EZ>(nu, k, P) * (0.5 * al[k]);
  }
  f[R_RHO] = rho; f[R_SRHO] = srho; f[R_A] = a; f[R_PG] = ra2 * P.inv_gm1; f[R_CF] = cf;
  f[R_CS] = cs; f[R_AF] = af; f[R_AS] = as; f[R_B1] = b1n; f[R_B2] = b2n; f[R_S] = S;
  f[R_VN] = vn; f[R_VT1] = vt1; f[R_VT2] = vt2; f[R_BT1] = bt1; f[R_BT2] = bt2;
  f[R_KX] = fma(gX, P.inv_gm1, hv2);
#pragma unroll
  for (int m = 0; m < 7; ++m) f[R_FAVG + m] = L.F[m] + R.F[m];
  if (PROT && P.prot && protection_hit(L, R, rho, ra2, af, as, al, P)) return 1;
  return 0;
}

// beta_k of App. A without forming gamma_k: Q(nu + gamma) alpha equals
// |nu alpha + dg| sign(alpha) when |nu alpha + dg| >= 2 eps |alpha|, else
// (nu alpha + dg)^2 / (4 eps alpha) + eps alpha
template <int EZ>
__device__ __forceinline__ double beta_k(double al, double nu, double gi, double gi1, int k,
                                         const WbPhys& P) {
  const double w = fma(nu, al, gi1 - gi);             // (nu + gamma) alpha
  double qa;
  if (wb_zero(al)) {
    qa = 0.0;                                           // gamma = 0, Q(nu) 0
  } else if ((EZ & (1 << k)) || !wb_abs_less(w, P.two_eps[k] * al)) {
    qa = wb_copysign_abs(w, al);                        // |nu + gamma| >= 2 eps
  } else if (wb_abs_less(al, 1e-290)) {
    qa = P.eps[k] * al;                                 // w^2/(4 eps alpha) < eps |alpha|
  } else {
    qa = fma(w * w * P.inv4eps[k], wb_rcp(al), P.eps[k] * al);
  }
  return qa - (gi + gi1);
}

// u-bar = (F_L + F_R)/2 - (dx/(2 dt)) sum_k beta_k R_k  (App. A)
template <int EZ>
__device__ __forceinline__ void face_flux(const Rec& f, const double gi[7], const double gi1[7],
                                          double dx_2dt, const WbPhys& P, double out[7]) {
  double be[7];
#pragma unroll
  for (int k = 0; k < 7; ++k) be[k] = beta_k<EZ>(f[R_AL + k], f[R_NU + k], gi[k], gi1[k], k, P);
  const double rho = f[R_RHO], af = f[R_AF], as = f[R_AS], cf = f[R_CF], cs = f[R_CS];
  const double S = f[R_S], b1 = f[R_B1], b2 = f[R_B2];
  // sum_k beta_k r_k in w = (rho, vn, vt, Bt, p)
  const double sf = be[0] + be[6], df = be[6] - be[0];
  const double ss = be[2] + be[4], ds = be[4] - be[2];
  const double tfs = af * sf + as * ss;
  const double wr = rho * tfs + be[3];
  const double afcf = af * cf, ascs = as * cs;
  const double wvn = afcf * df + ascs * ds;
  const double vb = wb_xsgn(afcf * ds - ascs * df, S);   // along beta
  const double vp = be[1] + be[5];                       // along beta-perp
  const double ra = f[R_SRHO] * f[R_A];
  const double bb = ra * (as * sf - af * ss);
  const double bp = wb_xsgn(f[R_SRHO] * (be[1] - be[5]), S);
  const double wvt1 = b1 * vb - b2 * vp, wvt2 = b2 * vb + b1 * vp;
  const double wbt1 = b1 * bb - b2 * bp, wbt2 = b2 * bb + b1 * bp;
  // to conserved variables (the pressure row enters the energy as p/(gamma-1))
  const double vn = f[R_VN], vt1 = f[R_VT1], vt2 = f[R_VT2];
  const double u1 = vn * wr + rho * wvn;
  const double u2 = vt1 * wr + rho * wvt1;
  const double u3 = vt2 * wr + rho * wvt2;
  const double u6 = f[R_PG] * tfs + f[R_KX] * wr + rho * (vn * wvn + vt1 * wvt1 + vt2 * wvt2) +
                    f[R_BT1] * wbt1 + f[R_BT2] * wbt2;
  out[0] = f[R_FAVG + 0] - dx_2dt * wr;
  out[1] = f[R_FAVG + 1] - dx_2dt * u1;
  out[2] = f[R_FAVG + 2] - dx_2dt * u2;
  out[3] = f[R_FAVG + 3] - dx_2dt * u3;
  out[4] = f[R_FAVG + 4] - dx_2dt * wbt1;
  out[5] = f[R_FAVG + 5] - dx_2dt * wbt2;
  out[6] = f[R_FAVG + 6] - dx_2dt * u6;
}

// One pencil segment of an MHDTVD sweep along D: fluxes of faces [fa, fb]
// at transverse position (pos[U], pos[W]) of the input fields q (zone B),
// normal face field bn; outputs F.  qo / wo: slot offsets of the input and
// output arrays.  rec: two shared-memory face records of this thread.
// Faces without a Roe state or below the protection floor take the HLL flux
// and give g-tilde = 0 to the limiters of their neighbours.  Returns the
// number of HLL faces among [fa, fb].
template <int D, bool NC, int EZ = 0, bool PROT = true>
__device__ __forceinline__ int sweep_segment(const WbGeo& g, const double* const* q,
                                             const double* bn, double* const* F, long long qo,
                                             long long wo, int pu, int pw, int fa, int fb,
                                             double dt, const WbPhys& P, const Rec rec[2]) {
  constexpr int T1 = (D + 1) % 3, T2 = (D + 2) % 3;
  constexpr int U = (D == 0) ? 1 : 0;
  constexpr int W = (D == 2) ? 1 : 2;
  int pos[3];
  pos[U] = pu;
  pos[W] = pw;
  pos[D] = fa - 2;
  const long long st = wb_stride<D>(g);
  const long long base = wb_at(g, pos[0], pos[1], pos[2]);
  const long long off_in = qo + base;
  const long long off_out = wo + base;
  const double dtdx = dt * g.idx[D];
  const double dx_2dt = 0.5 * g.dx[D] * wb_rcp(dt);
  Cell cL, cR;
  load_cell<D, NC>(q, off_in, P, cL);
  double gt_p[7], g_p[7];  // g-tilde of face f-1; g of zone f-2
  int nhll = 0;
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
      // g of zone f-1 from g-tilde of faces f (i+1/2) and f-1 (i-1/2)
      double gz[7];
#pragma unroll
      for (int k = 0; k < 7; ++k) gz[k] = wb_sweby(gt[k], gt_p[k], P.sweby, P.minmod);
      if (f >= fa + 1) {
        // flux of face f-1 (zones f-2, f-1): g_{i} = g_p (zone f-2), g_{i+1} = gz
        double out[7];
        const Rec& fr = rec[cur ^ 1];
        if (wb_neg(fr[R_RHO])) {
#pragma unroll
          for (int m = 0; m < 7; ++m) out[m] = fr[R_FAVG + m];
          ++nhll;
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

// Step 2: zone-centred reference EMF E = -v x B from q^n.
__device__ __forceinline__ void eref(const WbView& v, long long qo, long long wo, int i, int j, int k) {
  const long long o = qo + wb_at(v.geo, i, j, k);
  const long long w = wo + wb_at(v.geo, i, j, k);
  const double ir = wb_rcp(v.q[F_RHO][o]);
  const double vx = v.q[F_MX][o] * ir, vy = v.q[F_MY][o] * ir, vz = v.q[F_MZ][o] * ir;
  const double bx = v.q[F_BX][o], by = v.q[F_BY][o], bz = v.q[F_BZ][o];
  v.Eref[0][w] = vz * by - vy * bz;
  v.Eref[1][w] = vx * bz - vz * bx;
  v.Eref[2][w] = vy * bx - vx * by;
}

// value upwind of the mass flux m: from the minus-side zone if m > 0, the
// plus-side zone if m < 0, their mean if m = 0 (rare: a branch, not a select)
__device__ __forceinline__ double upwind(double m, double xm, double x0) {
  double d = wb_neg(m) ? x0 : xm;
  if (wb_zero(m)) d = 0.5 * (xm + x0);
  return d;
}

// Steps 3 and 9: upwinded corner EMF (GS05 "CT-contact" form).  Edge along
// axis C at the low faces of axes a = C+1 and b = C+2 (cyclic).  Face EMFs
// E^a = -F_a[B_b], E^b = +F_b[B_a]; the corner value is their average plus
// one quarter of [(dE/db) at -3/4 minus (dE/db) at -1/4] and the same along
// a, each derivative taken from the zone upwind of the mass flux through the
// face it sits on (the mean of both zones when that flux is zero).
template <int C>
__device__ __forceinline__ void edge(const WbView& v, long long wo, bool corr, int i, int j, int k) {
  constexpr int a = (C + 1) % 3, b = (C + 2) % 3;
  const WbGeo& g = v.geo;
  const long long o = wo + wb_at(g, i, j, k);
  const long long sa = a == 0 ? 1 : (a == 1 ? g.sy : g.sz);
  const long long sb = b == 0 ? 1 : (b == 1 ? g.sy : g.sz);
  double* const* Fa = corr ? v.Fc[a] : v.Fp[a];
  double* const* Fb = corr ? v.Fc[b] : v.Fp[b];
  const double* Er = corr ? v.Erefh[C] : v.Eref[C];
  const double Ea_0 = -Fa[F_BX + b][o];
  const double Ea_m = -Fa[F_BX + b][o - sb];
  const double Eb_0 = Fb[F_BX + a][o];
  const double Eb_m = Fb[F_BX + a][o - sa];
  const double ma_0 = Fa[F_RHO][o], ma_m = Fa[F_RHO][o - sb];
  const double mb_0 = Fb[F_RHO][o], mb_m = Fb[F_RHO][o - sa];
  const double R00 = Er[o], Rm0 = Er[o - sa], R0m = Er[o - sb], Rmm = Er[o - sa - sb];
  const double db_hi = upwind(ma_0, Rm0 - Eb_m, R00 - Eb_0);
  const double db_lo = upwind(ma_m, Eb_m - Rmm, Eb_0 - R0m);
  const double da_hi = upwind(mb_0, R0m - Ea_m, R00 - Ea_0);
  const double da_lo = upwind(mb_m, Ea_m - Rmm, Ea_0 - Rm0);
  double* out = corr ? v.Eedgeh[C] : v.Eedge[C];
  out[o] = 0.25 * ((Ea_0 + Ea_m) + (Eb_0 + Eb_m) + (db_lo - db_hi) + (da_lo - da_hi));
}

// Steps 4 and 11: b_out = b_in - tau curl E on the faces normal to D.
// Step 4 writes b^{n+1/2} to the workspace, Step 11 updates b in place.
template <int D>
__device__ __forceinline__ void ct(const WbView& v, long long qo, long long wo, bool fin, double dt,
                                   int i, int j, int k) {
  constexpr int a = (D + 1) % 3, b = (D + 2) % 3;
  const WbGeo& g = v.geo;
  const long long w = wo + wb_at(g, i, j, k);
  const long long q = qo + wb_at(g, i, j, k);
  const long long sa = a == 0 ? 1 : (a == 1 ? g.sy : g.sz);
  const long long sb = b == 0 ? 1 : (b == 1 ? g.sy : g.sz);
  const double* Eb = fin ? v.Eedgeh[b] : v.Eedge[b];
  const double* Ea = fin ? v.Eedgeh[a] : v.Eedge[a];
  const double tau = fin ? dt : 0.5 * dt;
  const double curl = (Eb[w + sa] - Eb[w]) * g.idx[a] - (Ea[w + sb] - Ea[w]) * g.idx[b];
  const double bn = v.b[D][q] - tau * curl;
  if (fin) v.b[D][q] = bn;
  else v.bh[D][w] = bn;
}

// Steps 5 and 7: q^{n+1/2}_D = q^n - dt/2 (transverse flux divergence)
// + dt/2 S_D, zone B_D := mean of b_D^{n+1/2}, with the GS08-type div B
// source S_D built from face differences of b^n and minmod pairings.
template <int D>
__device__ __forceinline__ void transverse(const WbView& v, long long qo, long long wo, double dt,
                                           int i, int j, int k) {
  constexpr int t1 = (D + 1) % 3, t2 = (D + 2) % 3;
  const WbGeo& g = v.geo;
  const long long q = qo + wb_at(g, i, j, k);
  const long long w = wo + wb_at(g, i, j, k);
  const long long s[3] = {1, g.sy, g.sz};
  const double hdt = 0.5 * dt;
  const double ir = wb_rcp(v.q[F_RHO][q]);
  double vv[3], B[3], db[3];
#pragma unroll
  for (int e = 0; e < 3; ++e) {
    vv[e] = v.q[F_MX + e][q] * ir;
    B[e] = v.q[F_BX + e][q];
    db[e] = (v.b[e][q + s[e]] - v.b[e][q]) * g.idx[e];
  }
  const double m2 = wb_minmod(db[D], -db[t1]);  // for the t2 field component
  const double m1 = wb_minmod(db[D], -db[t2]);  // for the t1 field component
  double S[8];
  S[F_RHO] = 0.0;
#pragma unroll
  for (int e = 0; e < 3; ++e) S[F_MX + e] = B[e] * db[D];
  S[F_EN] = B[D] * vv[D] * db[D] + B[t1] * vv[t1] * m1 + B[t2] * vv[t2] * m2;
  S[F_BX + D] = 0.0;
  S[F_BX + t1] = vv[t1] * m1;
  S[F_BX + t2] = vv[t2] * m2;
  const double c1 = hdt * g.idx[t1], c2 = hdt * g.idx[t2];
  // rho: no source; momentum and energy: both transverse fluxes and the
  // source; B_t1 (B_t2): only the t2 (t1) sweep carries it
  v.qh[D][F_RHO][w] = v.q[F_RHO][q] - ((v.Fp[t1][F_RHO][w + s[t1]] - v.Fp[t1][F_RHO][w]) * c1 +
                                       (v.Fp[t2][F_RHO][w + s[t2]] - v.Fp[t2][F_RHO][w]) * c2);
#pragma unroll
  for (int c = F_MX; c <= F_EN; ++c) {
    const double d1 = (v.Fp[t1][c][w + s[t1]] - v.Fp[t1][c][w]) * c1;
    const double d2 = (v.Fp[t2][c][w + s[t2]] - v.Fp[t2][c][w]) * c2;
    v.qh[D][c][w] = v.q[c][q] - (d1 + d2) + hdt * S[c];
  }
  v.qh[D][F_BX + t1][w] = v.q[F_BX + t1][q] - (v.Fp[t2][F_BX + t1][w + s[t2]] - v.Fp[t2][F_BX + t1][w]) * c2 +
                          hdt * S[F_BX + t1];
  v.qh[D][F_BX + t2][w] = v.q[F_BX + t2][q] - (v.Fp[t1][F_BX + t2][w + s[t1]] - v.Fp[t1][F_BX + t2][w]) * c1 +
                          hdt * S[F_BX + t2];
  v.qh[D][F_BX + D][w] = 0.5 * (v.bh[D][w] + v.bh[D][w + s[D]]);
}

// Steps 5 and 7 for the directions in mask (bit d) at one zone, sharing the
// zone's velocity, field, face differences and each transverse flux
// difference between the two states that use it.  Same arithmetic as
// transverse<D> for every direction.
__device__ __forceinline__ void transverse_set(const WbView& v, long long qo, long long wo, double dt,
                                               int mask, int i, int j, int k) {
  const WbGeo& g = v.geo;
  const long long q = qo + wb_at(g, i, j, k);
  const long long w = wo + wb_at(g, i, j, k);
  const long long s[3] = {1, g.sy, g.sz};
  const double hdt = 0.5 * dt;
  const double ir = wb_rcp(v.q[F_RHO][q]);
  double vv[3], B[3], db[3];
#pragma unroll
  for (int e = 0; e < 3; ++e) {
    vv[e] = v.q[F_MX + e][q] * ir;
    B[e] = v.q[F_BX + e][q];
    db[e] = (v.b[e][q + s[e]] - v.b[e][q]) * g.idx[e];
  }
  // flux differences (times dt/2 / dx_e) of every direction some state needs
  double dF[3][8];
#pragma unroll
  for (int e = 0; e < 3; ++e) {
    const bool need = (mask & ~(1 << e)) != 0;
    const double c = hdt * g.idx[e];
#pragma unroll
    for (int cc = 0; cc < 8; ++cc) {
      if (cc == F_BX + e || !need) { dF[e][cc] = 0.0; continue; }
      dF[e][cc] = (v.Fp[e][cc][w + s[e]] - v.Fp[e][cc][w]) * c;
    }
  }
  double qn[8];
#pragma unroll
  for (int cc = 0; cc < 8; ++cc) qn[cc] = v.q[cc][q];
#pragma unroll
  for (int D = 0; D < 3; ++D) {
    if (!(mask & (1 << D))) continue;
    const int t1 = (D + 1) % 3, t2 = (D + 2) % 3;
    const double m2 = wb_minmod(db[D], -db[t1]);
    const double m1 = wb_minmod(db[D], -db[t2]);
    double S[8];
    S[F_RHO] = 0.0;
#pragma unroll
    for (int e = 0; e < 3; ++e) S[F_MX + e] = B[e] * db[D];
    S[F_EN] = B[D] * vv[D] * db[D] + B[t1] * vv[t1] * m1 + B[t2] * vv[t2] * m2;
    S[F_BX + D] = 0.0;
    S[F_BX + t1] = vv[t1] * m1;
    S[F_BX + t2] = vv[t2] * m2;
    v.qh[D][F_RHO][w] = qn[F_RHO] - (dF[t1][F_RHO] + dF[t2][F_RHO]);
#pragma unroll
    for (int cc = F_MX; cc <= F_EN; ++cc) v.qh[D][cc][w] = qn[cc] - (dF[t1][cc] + dF[t2][cc]) + hdt * S[cc];
    v.qh[D][F_BX + t1][w] = qn[F_BX + t1] - dF[t2][F_BX + t1] + hdt * S[F_BX + t1];
    v.qh[D][F_BX + t2][w] = qn[F_BX + t2] - dF[t1][F_BX + t2] + hdt * S[F_BX + t2];
    v.qh[D][F_BX + D][w] = 0.5 * (v.bh[D][w] + v.bh[D][w + s[D]]);
  }
}

// Step 8: reference EMF at n+1/2 from v of q^n - dt/2 div F* and B = mean of
// b^{n+1/2}.
__device__ __forceinline__ void eref_half(const WbView& v, long long qo, long long wo, double dt,
                                          int i, int j, int k) {
  const WbGeo& g = v.geo;
  const long long q = qo + wb_at(g, i, j, k);
  const long long w = wo + wb_at(g, i, j, k);
  const long long s[3] = {1, g.sy, g.sz};
  const double hdt = 0.5 * dt;
  double u[4];
  const int comps[4] = {F_RHO, F_MX, F_MY, F_MZ};
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    double div = 0.0;
#pragma unroll
    for (int e = 0; e < 3; ++e)
      div += (v.Fc[e][comps[c]][w + s[e]] - v.Fc[e][comps[c]][w]) * g.idx[e];
    u[c] = v.q[comps[c]][q] - hdt * div;
  }
  const double ir = wb_rcp(u[0]);
  const double vx = u[1] * ir, vy = u[2] * ir, vz = u[3] * ir;
  double B[3];
#pragma unroll
  for (int e = 0; e < 3; ++e) B[e] = 0.5 * (v.bh[e][w] + v.bh[e][w + s[e]]);
  v.Erefh[0][w] = vz * B[1] - vy * B[2];
  v.Erefh[1][w] = vx * B[2] - vz * B[0];
  v.Erefh[2][w] = vy * B[0] - vx * B[1];
}

// sqrt for the CFL rate; inputs below the normal range (or not > 0) give 0
__device__ __forceinline__ double wb_sqrt_fast(double x) {
  return wb_normal_pos(x) ? x * wb_rsqrt(x) : 0.0;
}

// CFL signal rate sum_d (|v_d| + c_f,d)/dx_d of one zone (Sec. 3 fast speed).
__device__ __forceinline__ double signal_rate(double rho, double mx, double my, double mz, double e,
                                              double bx, double by, double bz, const WbPhys& P,
                                              const WbGeo& g) {
  const double ir = wb_rcp(rho);
  const double vv[3] = {mx * ir, my * ir, mz * ir};
  const double B[3] = {bx, by, bz};
  const double ke = 0.5 * (mx * vv[0] + my * vv[1] + mz * vv[2]);
  const double bb = bx * bx + by * by + bz * bz;
  const double p = P.gm1 * (e - ke - 0.5 * bb);
  const double a2 = P.gamma * p * ir;
  double w = 0.0;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const double cn2 = B[d] * B[d] * ir;
    const double ct2 = (bb - B[d] * B[d]) * ir;
    const double dd = a2 - cn2;
    const double disc = dd * dd + ct2 * (ct2 + 2.0 * (a2 + cn2));
    const double cf = wb_sqrt_fast(0.5 * (a2 + cn2 + ct2 + wb_sqrt_fast(disc)));
    w += (fabs(vv[d]) + cf) * g.idx[d];
  }
  if (!(rho > 0.0)) w = __longlong_as_double(0x7ff8000000000000LL);
  return w;
}

// Step 10 (+ the zone field of Step 11, floors and the next step's signal
// rate): U^{n+1} = ((U^n - dt/dx dF*) - dt/dy dG*) - dt/dz dH* at one interior
// zone, zone B = mean of b^{n+1}.  Returns the zone's signal rate (NaN if the
// state is unphysical); floor hits are added to *hits.
__device__ __forceinline__ double final_update(const WbView& v, long long qo, long long wo,
                                               double dt, const WbPhys& P, int i, int j, int k,
                                               int* hits, int* bad) {
  const WbGeo& g = v.geo;
  const long long q = qo + wb_at(g, i, j, k);
  const long long wi = wo + wb_at(g, i, j, k);
  const long long s[3] = {1, g.sy, g.sz};
  const double cx = dt * g.idx[0], cy = dt * g.idx[1], cz = dt * g.idx[2];
  double u[5];
#pragma unroll
  for (int c = 0; c < 5; ++c) {
    double x = v.q[c][q];
    x = x - cx * (v.Fc[0][c][wi + 1] - v.Fc[0][c][wi]);
    x = x - cy * (v.Fc[1][c][wi + s[1]] - v.Fc[1][c][wi]);
    x = x - cz * (v.Fc[2][c][wi + s[2]] - v.Fc[2][c][wi]);
    u[c] = x;
  }
  double B[3];
#pragma unroll
  for (int e = 0; e < 3; ++e) {
    B[e] = 0.5 * (v.b[e][q] + v.b[e][q + s[e]]);
    v.q[F_BX + e][q] = B[e];
  }
  if (u[0] < P.rho_floor) { u[0] = P.rho_floor; ++*hits; }
  const double ke = 0.5 * (u[1] * u[1] + u[2] * u[2] + u[3] * u[3]) * wb_rcp(u[0]);
  const double me = 0.5 * (B[0] * B[0] + B[1] * B[1] + B[2] * B[2]);
  const double p = P.gm1 * (u[4] - ke - me);
  if (p < P.p_floor) { u[4] = P.p_floor * P.inv_gm1 + ke + me; ++*hits; }
  const bool fin = isfinite(u[0]) && isfinite(u[1]) && isfinite(u[2]) && isfinite(u[3]) &&
                   isfinite(u[4]) && u[0] > 0.0 && isfinite(p);
#pragma unroll
  for (int c = 0; c < 5; ++c) v.q[c][q] = u[c];
  if (!fin) {
    ++*bad;
    return __longlong_as_double(0x7ff8000000000000LL);
  }
  return signal_rate(u[0], u[1], u[2], u[3], u[4], B[0], B[1], B[2], P, g);
}

// Ghost fill of a box that is its own periodic/outflow domain (no patches):
// padded index t outside the interior copies the wrapped/clamped interior
// zone of the same box (all 11 fields).
__device__ __forceinline__ void halo_self(const WbView& v, long long qo, const int bc[3], long long t) {
  const WbGeo& g = v.geo;
  const int i = (int)(t % g.pd[0]) - WB_NG;
  const long long r = t / g.pd[0];
  const int j = (int)(r % g.pd[1]) - WB_NG;
  const int k = (int)(r / g.pd[1]) - WB_NG;
  if (i >= 0 && i < g.n[0] && j >= 0 && j < g.n[1] && k >= 0 && k < g.n[2]) return;
  int loc[3] = {i, j, k};
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
  const long long dst = qo + t;
  const long long so = qo + wb_at(g, src[0], src[1], src[2]);
#pragma unroll
  for (int c = 0; c < 8; ++c) v.q[c][dst] = v.q[c][so];
#pragma unroll
  for (int c = 0; c < 3; ++c) v.b[c][dst] = v.b[c][so];
}

}  // namespace wbu
