// TEST INFRASTRUCTURE ONLY -- plain, slow FP64 CPU oracle of the WOMBAT
// per-patch ideal-MHD step (Mendygral et al. 2017, arXiv:1701.07452).
// Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may
// load it; it shares no code with the CUDA path.  Built with
// -O2 -ffp-contract=off so that no multiply-add is fused.
//
// What each part follows (paper section / equation):
//   cell_prim, cell_flux      Sec. 3, Eqs. for q, F, P* (totpressure), E (totenergy)
//   roe_state, eigen_*        Sec. 3 (eigenvalues a_1..a_7, c_f, c_s, c_a) and
//                             App. A (R_k, alpha_k "from Cargo & Gallice"; see
//                             the derivation notes at roe_state)
//   pencil_flux               App. A, Eqs. mhdtvd_flux2 (u-bar), f, beta, alpha,
//                             gamma, g (SWEBY limiter), g-tilde, Q_k
//   step (Steps 1-11)         Sec. "MHD in Three Dimensions", Steps 1-11
//   edge_emf                  Steps 3 and 9: GS05 upwinded corner EMF
//   transverse_state          Steps 5 and 7 incl. the div B source term
//   ghost fill                Sec. "MHD in Two Dimensions": 5 boundary zones,
//                             one exchange per step
//   hll_flux, protection      App. A, the protection floor and the HLL flux
//                             (Eqs. for u-bar of the HLL scheme, b+ and b-)
// Readings where the paper is silent are tagged R1..R27; the comment at each
// tag states the reading taken.
//
// The div B source of Steps 5 and 7 (reading R13, after GS08, which is not
// available) is pinned to the flux derivative it supplies in every row
// (momentum, energy, induction) where its limiter is inactive, and its minmod
// pairing to the planar problem.  Parity unpinned: the limiter itself (GS08's
// choice to limit the induction and energy rows by minmod) where it is active,
// and the free constants eps_k and beta_s (readings R7, R8).

#include "mhd_oracle.h"

#include <cmath>
#include <cstdint>
#include <cstring>
#include <limits>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

// The arithmetic type: plain double, or, in the separate operation-counting
// build (-DORACLE_COUNT_FLOPS, single-threaded), an instrumented scalar with
// the same IEEE results (flop_count.h).  Parameters (gamma, eps_k, dt, dx)
// stay plain double.
#ifdef ORACLE_COUNT_FLOPS
#include "flop_count.h"
using flopcount::real;
using flopcount::r_sqrt;
using flopcount::r_fabs;
using flopcount::r_fmin;
using flopcount::r_fmax;
using flopcount::r_isfinite;
using flopcount::to_d;
namespace flopcount {
long long flops[SEC_COUNT];
long long units[SEC_COUNT];
int section = SEC_NONE;
}  // namespace flopcount
#define FLOP_SECTION(s) flopcount::enter(flopcount::s)
#define FLOP_UNIT(s) flopcount::unit(flopcount::s)
#else
typedef double real;
inline double r_sqrt(double x) { return std::sqrt(x); }
inline double r_fabs(double x) { return std::fabs(x); }
inline double r_fmin(double a, double b) { return std::fmin(a, b); }
inline double r_fmax(double a, double b) { return std::fmax(a, b); }
inline bool r_isfinite(double x) { return std::isfinite(x); }
inline double to_d(double x) { return x; }
#define FLOP_SECTION(s) ((void)0)
#define FLOP_UNIT(s) ((void)0)
#endif

namespace {

const int NG = 5;  // boundary zones (Sec. "MHD in Two Dimensions")
const double NaN = std::numeric_limits<double>::quiet_NaN();

struct Params {
  double gamma, cfl, eps[7], sweby, rho_floor, p_floor;
  double prot_rho = 0.0, prot_p = 0.0;  // protection floors (App. A)
  double source_scale = 1.0;            // factor on the div B source (test ablation only)
};

// 3D array over the padded box [-NG, n+NG) per dimension, x fastest.
struct Arr {
  int nx = 0, ny = 0, nz = 0, px = 0, py = 0;
  std::vector<real> d;
  void init(int nx_, int ny_, int nz_) {
    nx = nx_; ny = ny_; nz = nz_;
    px = nx + 2 * NG; py = ny + 2 * NG;
    d.assign((size_t)px * py * (nz + 2 * NG), NaN);
  }
  real& operator()(int i, int j, int k) {
    return d[((size_t)(k + NG) * py + (j + NG)) * px + (i + NG)];
  }
  real operator()(int i, int j, int k) const {
    return d[((size_t)(k + NG) * py + (j + NG)) * px + (i + NG)];
  }
};

enum { RHO = 0, MX = 1, MY = 2, MZ = 3, EN = 4, BX = 5, BY = 6, BZ = 7 };

// ---------------------------------------------------------------------------
// Single-cell quantities in a sweep frame (n = sweep normal, t1, t2 cyclic).
// ---------------------------------------------------------------------------
struct Cell {  // conserved, zone-centred B
  real rho, mn, mt1, mt2, e, bn, bt1, bt2;
};
struct Prim {
  real rho, vn, vt1, vt2, p, bn, bt1, bt2;
};

// Sec. 3, Eqs. totpressure / totenergy solved for P.
inline Prim cell_prim(const Cell& c, double gamma) {
  Prim p;
  p.rho = c.rho;
  p.vn = c.mn / c.rho;
  p.vt1 = c.mt1 / c.rho;
  p.vt2 = c.mt2 / c.rho;
  p.bn = c.bn; p.bt1 = c.bt1; p.bt2 = c.bt2;
  real ke = 0.5 * c.rho * (p.vn * p.vn + p.vt1 * p.vt1 + p.vt2 * p.vt2);
  real me = 0.5 * (c.bn * c.bn + c.bt1 * c.bt1 + c.bt2 * c.bt2);
  p.p = (gamma - 1.0) * (c.e - ke - me);
  return p;
}

// Sec. 3, flux vector F of the 1D conservative form (7 non-trivial
// components, ordered rho, Mn, Mt1, Mt2, Bt1, Bt2, E; F[Bn] = 0).
inline void cell_flux(const Cell& c, const Prim& p, real F[7]) {
  real me = 0.5 * (c.bn * c.bn + c.bt1 * c.bt1 + c.bt2 * c.bt2);
  real pstar = p.p + me;
  F[0] = c.mn;
  F[1] = c.mn * p.vn + pstar - c.bn * c.bn;
  F[2] = c.mn * p.vt1 - c.bn * c.bt1;
  F[3] = c.mn * p.vt2 - c.bn * c.bt2;
  F[4] = c.bt1 * p.vn - c.bn * p.vt1;
  F[5] = c.bt2 * p.vn - c.bn * p.vt2;
  F[6] = (c.e + pstar) * p.vn - c.bn * (c.bn * p.vn + c.bt1 * p.vt1 + c.bt2 * p.vt2);
}

// ---------------------------------------------------------------------------
// Interface eigen-system (App. A: R_k and alpha_k from Cargo & Gallice).
//
// Roe linearisation (our derivation of a Cargo-Gallice type average; reading R5):
// with s = sqrt(rho), the interface state is rho_ = sL sR, v_ and H_ weighted by
// s, transverse B weighted by the opposite s, normal field = face value b.
// The exact identity d(B_t^2/2) = B_t_ . dB_t + X d rho, with
// X = |dB_t|^2 / (2 (sL+sR)^2), makes the linearised system the ideal-MHD
// Jacobian at (rho_, v_, B_t_, b) with the sound speed
//   a_^2 = (gamma-1)(H_ - v_^2/2 - (b^2+B_t_^2)/rho_) - (gamma-2) X,
// so that dF = A_roe dU holds exactly (Roe property, pinned in tests).  The
// eigenvectors are the ideal-MHD ones in primitive variables
// w = (rho, vn, vt1, vt2, Bt1, Bt2, p) mapped to conserved variables by the
// exact linear map T (and its inverse W) of this linearisation.
// ---------------------------------------------------------------------------
struct Eigen {
  // Roe state
  real rho, srho, vn, vt1, vt2, b, bt1, bt2, X;
  real a2, a, ca2, ct2, cf2, cs2, cf, cs, ca, af, as, beta1, beta2, S;
  real lam[7];
  real R[7][7];  // R[m][k]: conserved component m of right eigenvector k
  real L[7][7];  // L[k][m]: left eigenvector k
  real rrho[7], rp[7];  // density and pressure rows of the primitive r_k
  bool bad;
};

inline real sgn_pos(real x) { return x >= 0.0 ? 1.0 : -1.0; }

// Roe state + eigenvalues + eigenvectors for one interface.
// L, R in the sweep frame with zone-centred B; b = face normal field.
void roe_state(const Prim& pL, const Prim& pR, real b, double gamma, Eigen* e) {
  e->bad = false;
  real sL = r_sqrt(pL.rho), sR = r_sqrt(pR.rho);
  real D = sL + sR;
  e->rho = sL * sR;
  e->vn = (sL * pL.vn + sR * pR.vn) / D;
  e->vt1 = (sL * pL.vt1 + sR * pR.vt1) / D;
  e->vt2 = (sL * pL.vt2 + sR * pR.vt2) / D;
  // enthalpy with the face normal field: H = (gamma/(gamma-1) P + rho v^2/2 + b^2 + Bt^2)/rho
  real keL = 0.5 * pL.rho * (pL.vn * pL.vn + pL.vt1 * pL.vt1 + pL.vt2 * pL.vt2);
  real keR = 0.5 * pR.rho * (pR.vn * pR.vn + pR.vt1 * pR.vt1 + pR.vt2 * pR.vt2);
  real HL = (gamma / (gamma - 1.0) * pL.p + keL + b * b + pL.bt1 * pL.bt1 + pL.bt2 * pL.bt2) / pL.rho;
  real HR = (gamma / (gamma - 1.0) * pR.p + keR + b * b + pR.bt1 * pR.bt1 + pR.bt2 * pR.bt2) / pR.rho;
  real H = (sL * HL + sR * HR) / D;
  e->b = b;
  e->bt1 = (sR * pL.bt1 + sL * pR.bt1) / D;
  e->bt2 = (sR * pL.bt2 + sL * pR.bt2) / D;
  real dbt1 = pR.bt1 - pL.bt1, dbt2 = pR.bt2 - pL.bt2;
  e->X = 0.5 * (dbt1 * dbt1 + dbt2 * dbt2) / (D * D);
  real v2 = e->vn * e->vn + e->vt1 * e->vt1 + e->vt2 * e->vt2;
  real bt2sum = e->bt1 * e->bt1 + e->bt2 * e->bt2;
  e->a2 = (gamma - 1.0) * (H - 0.5 * v2 - (b * b + bt2sum) / e->rho) - (gamma - 2.0) * e->X;
  // No usable sound speed: a^2 <= 0, or a^2 below the smallest normal double,
  // where it has lost significant bits and the 1/(2 a^2) factors of the left
  // eigenvectors (App. A) lose them too or overflow (below ~5.6e-309).
  if (!(e->a2 >= std::numeric_limits<double>::min())) {
    e->bad = true;
    return;
  }
  e->srho = r_sqrt(e->rho);
  // characteristic speeds (Sec. 3) at the Roe state; the discriminant is
  // written as a sum of non-negative terms (reading R2).
  real a2 = e->a2;
  e->ca2 = b * b / e->rho;
  e->ct2 = bt2sum / e->rho;
  real ca2 = e->ca2, ct2 = e->ct2;
  real disc = (a2 - ca2) * (a2 - ca2) + ct2 * (ct2 + 2.0 * a2 + 2.0 * ca2);
  real sd = r_sqrt(disc);  // = cf^2 - cs^2
  e->cf2 = 0.5 * (a2 + ca2 + ct2 + sd);
  e->cs2 = a2 * ca2 / e->cf2;   // cf^2 cs^2 = a^2 ca^2 (product of the two roots)
  e->cf = r_sqrt(e->cf2);
  e->cs = r_sqrt(e->cs2);
  e->ca = r_sqrt(ca2);
  e->a = r_sqrt(a2);
  // normalisation factors alpha_f, alpha_s (reading R6 for degeneracies)
  if (sd <= 1e-12 * (a2 + ca2 + ct2)) {
    if (a2 >= ca2) { e->af = 1.0; e->as = 0.0; }
    else { e->af = 0.0; e->as = 1.0; }
  } else {
    // cf^2 - a^2 and a^2 - cs^2 without cancellation (ca^2 - a^2 first: the
    // difference of two nearly equal squares is exact, a sum rounded before
    // it is not)
    real t1 = (ca2 - a2) + ct2;
    real cf2_a2 = (t1 >= 0.0) ? 0.5 * (t1 + sd) : 2.0 * a2 * ct2 / (sd - t1);
    real t2 = a2 - ca2 + ct2;
    real cf2_ca2 = (t2 >= 0.0) ? 0.5 * (t2 + sd) : 2.0 * ca2 * ct2 / (sd - t2);
    real a2_cs2 = a2 * cf2_ca2 / e->cf2;
    real af2 = a2_cs2 / sd, as2 = cf2_a2 / sd;
    if (af2 > 1.0) af2 = 1.0;
    if (af2 < 0.0) af2 = 0.0;
    if (as2 > 1.0) as2 = 1.0;
    if (as2 < 0.0) as2 = 0.0;
    e->af = r_sqrt(af2);
    e->as = r_sqrt(as2);
  }
  real btm2 = bt2sum;
  if (btm2 <= 1e-24 * (e->rho * a2 + b * b + bt2sum)) {
    e->beta1 = e->beta2 = 1.0 / std::sqrt(2.0);
  } else {
    real btm = r_sqrt(btm2);
    e->beta1 = e->bt1 / btm;
    e->beta2 = e->bt2 / btm;
  }
  e->S = sgn_pos(b);
  // eigenvalues a_1..a_7 (Sec. 3)
  e->lam[0] = e->vn - e->cf;
  e->lam[1] = e->vn - e->ca;
  e->lam[2] = e->vn - e->cs;
  e->lam[3] = e->vn;
  e->lam[4] = e->vn + e->cs;
  e->lam[5] = e->vn + e->ca;
  e->lam[6] = e->vn + e->cf;

  // primitive right (columns r[.][k]) and left (rows l[k][.]) eigenvectors in
  // w = (rho, vn, vt1, vt2, Bt1, Bt2, p)
  real r[7][7], l[7][7];
  for (int m = 0; m < 7; ++m)
    for (int k = 0; k < 7; ++k) { r[m][k] = 0.0; l[k][m] = 0.0; }
  real af = e->af, as = e->as, cf = e->cf, cs = e->cs, S = e->S;
  real b1 = e->beta1, b2 = e->beta2, rho = e->rho, sr = e->srho, a = e->a;
  // fast k=0 (v-cf) and k=6 (v+cf)
  for (int s = 0; s < 2; ++s) {
    int k = s == 0 ? 0 : 6;
    real sg = s == 0 ? -1.0 : 1.0;  // sign of u = lambda - vn
    r[0][k] = rho * af;
    r[1][k] = sg * af * cf;
    r[2][k] = -sg * as * cs * S * b1;
    r[3][k] = -sg * as * cs * S * b2;
    r[4][k] = as * sr * a * b1;
    r[5][k] = as * sr * a * b2;
    r[6][k] = rho * a2 * af;
    l[k][1] = sg * af * cf / (2.0 * a2);
    l[k][2] = -sg * as * cs * S * b1 / (2.0 * a2);
    l[k][3] = -sg * as * cs * S * b2 / (2.0 * a2);
    l[k][4] = as * b1 / (2.0 * sr * a);
    l[k][5] = as * b2 / (2.0 * sr * a);
    l[k][6] = af / (2.0 * rho * a2);
  }
  // slow k=2 (v-cs) and k=4 (v+cs)
  for (int s = 0; s < 2; ++s) {
    int k = s == 0 ? 2 : 4;
    real sg = s == 0 ? -1.0 : 1.0;
    r[0][k] = rho * as;
    r[1][k] = sg * as * cs;
    r[2][k] = sg * af * cf * S * b1;
    r[3][k] = sg * af * cf * S * b2;
    r[4][k] = -af * sr * a * b1;
    r[5][k] = -af * sr * a * b2;
    r[6][k] = rho * a2 * as;
    l[k][1] = sg * as * cs / (2.0 * a2);
    l[k][2] = sg * af * cf * S * b1 / (2.0 * a2);
    l[k][3] = sg * af * cf * S * b2 / (2.0 * a2);
    l[k][4] = -af * b1 / (2.0 * sr * a);
    l[k][5] = -af * b2 / (2.0 * sr * a);
    l[k][6] = as / (2.0 * rho * a2);
  }
  // Alfven k=1 (v-ca) and k=5 (v+ca)
  for (int s = 0; s < 2; ++s) {
    int k = s == 0 ? 1 : 5;
    real sg = s == 0 ? 1.0 : -1.0;
    r[2][k] = -b2;
    r[3][k] = b1;
    r[4][k] = -sg * S * sr * b2;
    r[5][k] = sg * S * sr * b1;
    l[k][2] = -0.5 * b2;
    l[k][3] = 0.5 * b1;
    l[k][4] = -0.5 * sg * S * b2 / sr;
    l[k][5] = 0.5 * sg * S * b1 / sr;
  }
  // entropy k=3
  r[0][3] = 1.0;
  l[3][0] = 1.0;
  l[3][6] = -1.0 / a2;

  for (int k = 0; k < 7; ++k) {
    e->rrho[k] = r[0][k];
    e->rp[k] = r[6][k];
  }
  // W: conserved (rho, Mn, Mt1, Mt2, Bt1, Bt2, E) -> w
  real W[7][7];
  for (int m = 0; m < 7; ++m)
    for (int n = 0; n < 7; ++n) W[m][n] = 0.0;
  W[0][0] = 1.0;
  W[1][0] = -e->vn / rho;  W[1][1] = 1.0 / rho;
  W[2][0] = -e->vt1 / rho; W[2][2] = 1.0 / rho;
  W[3][0] = -e->vt2 / rho; W[3][3] = 1.0 / rho;
  W[4][4] = 1.0;
  W[5][5] = 1.0;
  W[6][0] = (gamma - 1.0) * 0.5 * v2 - (gamma - 2.0) * e->X;
  W[6][1] = -(gamma - 1.0) * e->vn;
  W[6][2] = -(gamma - 1.0) * e->vt1;
  W[6][3] = -(gamma - 1.0) * e->vt2;
  W[6][4] = -(gamma - 1.0) * e->bt1;
  W[6][5] = -(gamma - 1.0) * e->bt2;
  W[6][6] = gamma - 1.0;
  // T = W^-1: w -> conserved
  real T[7][7];
  for (int m = 0; m < 7; ++m)
    for (int n = 0; n < 7; ++n) T[m][n] = 0.0;
  T[0][0] = 1.0;
  T[1][0] = e->vn;  T[1][1] = rho;
  T[2][0] = e->vt1; T[2][2] = rho;
  T[3][0] = e->vt2; T[3][3] = rho;
  T[4][4] = 1.0;
  T[5][5] = 1.0;
  T[6][0] = 0.5 * v2 + (gamma - 2.0) / (gamma - 1.0) * e->X;
  T[6][1] = rho * e->vn;
  T[6][2] = rho * e->vt1;
  T[6][3] = rho * e->vt2;
  T[6][4] = e->bt1;
  T[6][5] = e->bt2;
  T[6][6] = 1.0 / (gamma - 1.0);
  // R = T r, L = l W
  for (int m = 0; m < 7; ++m)
    for (int k = 0; k < 7; ++k) {
      real s = 0.0;
      for (int n = 0; n < 7; ++n) s += T[m][n] * r[n][k];
      e->R[m][k] = s;
    }
  for (int k = 0; k < 7; ++k)
    for (int m = 0; m < 7; ++m) {
      real s = 0.0;
      for (int n = 0; n < 7; ++n) s += l[k][n] * W[n][m];
      e->L[k][m] = s;
    }
}

// conserved 7-vector difference qR - qL in system order
// (rho, Mn, Mt1, Mt2, Bt1, Bt2, E); the energy of each cell is referred to the
// face normal field (the 7-variable system treats Bn as a parameter; its
// zone-centred value differs from b between the two cells), reading R4.
inline void cons_diff(const Cell& L, const Cell& R, real dq[7]) {
  dq[0] = R.rho - L.rho;
  dq[1] = R.mn - L.mn;
  dq[2] = R.mt1 - L.mt1;
  dq[3] = R.mt2 - L.mt2;
  dq[4] = R.bt1 - L.bt1;
  dq[5] = R.bt2 - L.bt2;
  dq[6] = (R.e - 0.5 * R.bn * R.bn) - (L.e - 0.5 * L.bn * L.bn);
}

// App. A: Q_k(chi)
inline real Qk(real chi, double eps) {
  real ac = r_fabs(chi);
  if (ac < 2.0 * eps) return chi * chi / (4.0 * eps) + eps;
  return ac;
}

// App. A: g_{k,i} = SIGN(gt_{i+1/2}) SWEBY(gt_{i+1/2}, gt_{i-1/2}) (reading R8)
inline real sweby(real gp, real gm, double beta) {
  real s = gp >= 0.0 ? 1.0 : -1.0;
  real ap = r_fabs(gp);
  real m1 = r_fmin(beta * ap, s * gm);
  real m2 = r_fmin(ap, beta * s * gm);
  real m = r_fmax(0.0, r_fmax(m1, m2));
  return s * m;
}

// Fast magnetosonic speed of one zone along the sweep normal (Sec. 3):
// c_f^2 = [a^2 + B^2/rho + sqrt((a^2 + B^2/rho)^2 - 4 a^2 Bn^2/rho)] / 2,
// a^2 = gamma P / rho, zone-centred B.
inline real fast_speed(const Prim& p, double gamma) {
  real a2 = gamma * p.p / p.rho;
  real b2 = (p.bn * p.bn + p.bt1 * p.bt1 + p.bt2 * p.bt2) / p.rho;
  real s = a2 + b2;
  real disc = s * s - 4.0 * a2 * p.bn * p.bn / p.rho;
  if (disc < 0.0) disc = 0.0;  // reading R2
  return r_sqrt(0.5 * (s + r_sqrt(disc)));
}

// Protection floor (App. A, reading R22): active when a floor is > 0.  A face
// takes the HLL flux when one of the states of its linearised (Roe) Riemann
// problem has a density or pressure below the floors: the two zone states
// and the intermediate states w_L + sum_{j<=k} alpha_j r_j, k = 1..6, in the
// primitive variables of the linearisation (Roe-type fluxes fail exactly when
// these states are unphysical).
inline bool protection_active(const Params& P) { return P.prot_rho > 0.0 || P.prot_p > 0.0; }

bool protection_hit(const Prim& pL, const Prim& pR, const Eigen& e, const real alpha[7],
                    const Params& P) {
  if (pL.rho < P.prot_rho || pL.p < P.prot_p) return true;
  if (pR.rho < P.prot_rho || pR.p < P.prot_p) return true;
  real rho = pL.rho, p = pL.p;
  for (int k = 0; k < 6; ++k) {
    rho += alpha[k] * e.rrho[k];
    p += alpha[k] * e.rp[k];
    if (rho < P.prot_rho || p < P.prot_p) return true;
  }
  return false;
}

// HLL flux of App. A between zones L = i and R = i+1 (reading R22):
//   b+ = max(a_max, v_R + c_f,R, 0),  b- = min(a_min, v_L - c_f,L, 0),
//   u = (b+ F(q_L) - b- F(q_R) + b+ b- (q_R - q_L)) / (b+ - b-),
// a_max, a_min the largest and smallest Roe eigenvalues when the Roe state
// exists (roe == nullptr otherwise).  The printed numerator has +b- F(q_R),
// which is not consistent (u != F for q_L = q_R); the Einfeldt form used here
// is.  If both speeds vanish (no Roe state and both zones moving
// supersonically into the face) the bounds are +-max(|v| + c_f).
void hll_flux(const Cell& L, const Cell& R, const Prim& pL, const Prim& pR, const real FL[7],
              const real FR[7], const Eigen* roe, double gamma, real out[7]) {
  real cfL = fast_speed(pL, gamma), cfR = fast_speed(pR, gamma);
  real bp = r_fmax(pR.vn + cfR, 0.0);
  real bm = r_fmin(pL.vn - cfL, 0.0);
  if (roe) {
    bp = r_fmax(bp, roe->lam[6]);
    bm = r_fmin(bm, roe->lam[0]);
  }
  if (!(bp - bm > 0.0)) {
    real s = r_fmax(r_fabs(pL.vn) + cfL, r_fabs(pR.vn) + cfR);
    bp = s;
    bm = -s;
  }
  real dq[7];
  cons_diff(L, R, dq);
  for (int m = 0; m < 7; ++m)
    out[m] = (bp * FL[m] - bm * FR[m] + bp * bm * dq[m]) / (bp - bm);
}

struct Face {
  Eigen e;
  real alpha[7], nu[7], gt[7], Favg[7];
  bool hll;
  real Fhll[7];
};

// MHDTVD flux on one pencil.  cells[c] for c in [0, ncell), face f between
// cells f-1 and f, bface[f] for f in [0, ncell].  Faces f in [2, ncell-2] get
// a flux (they need g at cells f-1 and f, i.e. g-tilde at faces f-1..f+1,
// i.e. cells f-2..f+1).  A face whose Roe state has no real sound speed, or
// next to a zone below the protection floor, takes the HLL flux instead and
// contributes g-tilde = 0 to the limiter of its neighbours (reading R22).
// Returns the number of output faces that took the HLL flux; if hll_flag is
// given, hll_flag[f] = 1 marks those faces (0 elsewhere).
int pencil_flux(int ncell, const Cell* cells, const real* bface, double dtdx,
                double dx_2dt, const Params& P, real (*out)[7],
                unsigned char* hll_flag = nullptr) {
  if (hll_flag)
    for (int f = 0; f <= ncell; ++f) hll_flag[f] = 0;
  int nhll = 0;
  std::vector<Prim> prim(ncell);
  std::vector<real> Fc((size_t)ncell * 7);
  FLOP_SECTION(SEC_CELL);
  for (int c = 0; c < ncell; ++c) {
    FLOP_UNIT(SEC_CELL);
    prim[c] = cell_prim(cells[c], P.gamma);
    cell_flux(cells[c], prim[c], &Fc[(size_t)c * 7]);
  }
  std::vector<Face> face(ncell + 1);
  for (int f = 1; f <= ncell - 1; ++f) {
    Face& F = face[f];
    const Cell& L = cells[f - 1];
    const Cell& R = cells[f];
    FLOP_SECTION(SEC_FACE);
    FLOP_UNIT(SEC_FACE);
    roe_state(prim[f - 1], prim[f], bface[f], P.gamma, &F.e);
    F.hll = F.e.bad;
    if (!F.hll) {
      real dq[7];
      cons_diff(L, R, dq);
      for (int k = 0; k < 7; ++k) {
        real s = 0.0;
        for (int m = 0; m < 7; ++m) s += F.e.L[k][m] * dq[m];
        F.alpha[k] = s;                       // alpha_k = L_k . (q_{i+1} - q_i)
      }
      if (protection_active(P)) F.hll = protection_hit(prim[f - 1], prim[f], F.e, F.alpha, P);
    }
    if (F.hll) {
      for (int k = 0; k < 7; ++k) {
        F.alpha[k] = F.nu[k] = NaN;
        F.gt[k] = 0.0;
      }
      FLOP_SECTION(SEC_HLL);
      FLOP_UNIT(SEC_HLL);
      hll_flux(L, R, prim[f - 1], prim[f], &Fc[(size_t)(f - 1) * 7], &Fc[(size_t)f * 7],
               F.e.bad ? nullptr : &F.e, P.gamma, F.Fhll);
      continue;
    }
    for (int k = 0; k < 7; ++k) {
      F.nu[k] = dtdx * F.e.lam[k];          // (dt/dx) a_k
      F.gt[k] = 0.5 * (Qk(F.nu[k], P.eps[k]) - F.nu[k] * F.nu[k]) * F.alpha[k];
    }
    for (int m = 0; m < 7; ++m)
      F.Favg[m] = 0.5 * (Fc[(size_t)(f - 1) * 7 + m] + Fc[(size_t)f * 7 + m]);
  }
  // g_{k,c} for cells c in [1, ncell-2]: faces c (i-1/2) and c+1 (i+1/2)
  std::vector<real> g((size_t)ncell * 7, NaN);
  FLOP_SECTION(SEC_LIMIT);
  for (int c = 1; c <= ncell - 2; ++c) {
    FLOP_UNIT(SEC_LIMIT);
    for (int k = 0; k < 7; ++k)
      g[(size_t)c * 7 + k] = sweby(face[c + 1].gt[k], face[c].gt[k], P.sweby);
  }
  FLOP_SECTION(SEC_EMIT);
  for (int f = 2; f <= ncell - 2; ++f) {
    const Face& F = face[f];
    FLOP_UNIT(SEC_EMIT);
    if (F.hll) {
      ++nhll;
      if (hll_flag) hll_flag[f] = 1;
      for (int m = 0; m < 7; ++m) out[f][m] = F.Fhll[m];
      continue;
    }
    real fsum[7] = {0, 0, 0, 0, 0, 0, 0};
    for (int k = 0; k < 7; ++k) {
      real gi = g[(size_t)(f - 1) * 7 + k];   // g_{k,i}, i = left cell
      real gi1 = g[(size_t)f * 7 + k];        // g_{k,i+1}
      real gam = (F.alpha[k] != 0.0) ? (gi1 - gi) / F.alpha[k] : 0.0;
      real beta = Qk(F.nu[k] + gam, P.eps[k]) * F.alpha[k] - (gi + gi1);
      for (int m = 0; m < 7; ++m) fsum[m] += beta * F.e.R[m][k];
    }
    for (int m = 0; m < 7; ++m) out[f][m] = F.Favg[m] - dx_2dt * fsum[m];
  }
  FLOP_SECTION(SEC_NONE);
  return nhll;
}

// ---------------------------------------------------------------------------
struct Range {  // inclusive ranges per dimension, relative to the interior
  int lo[3], hi[3];
};

}  // namespace

struct or_grid {
  int n[3];
  double dxv[3], len[3];
  int bc[3];
  Params P;
  Arr q[8];                       // zone-centred state q^n (rho, M, E, B)
  Arr b[3];                       // face fields (index = low face of the cell)
  // intermediates of one step
  Arr Fp[3][8], Fc[3][8];         // predictor / corrector fluxes (8 global comps)
  Arr Eref[3], Eedge[3];          // reference and edge EMFs
  Arr bh[3];                      // b^{n+1/2}
  Arr qh[3][8];                   // q^{n+1/2}_d
  Arr Erefh[3], Eedgeh[3];        // half-step reference, corrector edge EMFs
  long long floor_hits = 0, unphysical = 0, hll_faces = 0;
};

namespace {

void alloc_like(or_grid* g, Arr& a) { a.init(g->n[0], g->n[1], g->n[2]); }

inline int wrap(int i, int n) { return ((i % n) + n) % n; }

// Ghost fill (one exchange per step).  Periodic: wrap; outflow: copy the
// nearest interior zone; for the normal face field on an outflow side copy the
// boundary face (low side) or the last owned face (high side), reading R16.
// Face arrays: face index f is the low face of cell f; faces [0, n) are owned
// (reading R17), face n and beyond are ghosts.
void fill_array(or_grid* g, Arr& a, int face_dim) {
  const int* n = g->n;
#pragma omp parallel for schedule(static)
  for (int k = -NG; k < n[2] + NG; ++k)
    for (int j = -NG; j < n[1] + NG; ++j)
      for (int i = -NG; i < n[0] + NG; ++i) {
        int idx[3] = {i, j, k};
        bool inside = true;
        for (int d = 0; d < 3; ++d)
          if (idx[d] < 0 || idx[d] >= n[d]) inside = false;
        if (inside) continue;
        int src[3];
        for (int d = 0; d < 3; ++d) {
          int x = idx[d];
          if (x >= 0 && x < n[d]) { src[d] = x; continue; }
          if (g->bc[d] == 0) src[d] = wrap(x, n[d]);
          else src[d] = x < 0 ? 0 : n[d] - 1;
        }
        (void)face_dim;
        a(i, j, k) = a(src[0], src[1], src[2]);
      }
}

void ghost_fill(or_grid* g) {
  for (int v = 0; v < 8; ++v) fill_array(g, g->q[v], -1);
  for (int d = 0; d < 3; ++d) fill_array(g, g->b[d], d);
}

inline void load_cell(const or_grid* g, const Arr* q, int d, int i, int j, int k, Cell* c) {
  int n = d, t1 = (d + 1) % 3, t2 = (d + 2) % 3;
  c->rho = q[RHO](i, j, k);
  c->mn = q[MX + n](i, j, k);
  c->mt1 = q[MX + t1](i, j, k);
  c->mt2 = q[MX + t2](i, j, k);
  c->e = q[EN](i, j, k);
  c->bn = q[BX + n](i, j, k);
  c->bt1 = q[BX + t1](i, j, k);
  c->bt2 = q[BX + t2](i, j, k);
  (void)g;
}

// Sweep along d over faces [r.lo[d], r.hi[d]] and transverse cells r (other
// dims).  Input state qin (8 comps, zone-centred B), normal face field bn.
// Output flux arrays out[8] (global component order, normal-B flux = 0).
// Returns the number of interior faces (faces [0, n_d) along d, zones [0, n)
// across) that took the HLL flux: the count of distinct faces, independent of
// how far the region reaches into the ghost zones.
int sweep(or_grid* g, int d, const Arr* qin, const Arr& bn, double dt, const Range& r, Arr* out) {
  int t1 = (d + 1) % 3, t2 = (d + 2) % 3;
  double dtdx = dt / g->dxv[d];
  double dx_2dt = g->dxv[d] / (2.0 * dt);
  int f0 = r.lo[d], f1 = r.hi[d];
  int c0 = f0 - 2, c1 = f1 + 1;  // cells of the pencil
  int ncell = c1 - c0 + 1;
  int bad = 0;
  int na = r.hi[t1] - r.lo[t1] + 1, nb = r.hi[t2] - r.lo[t2] + 1;
#pragma omp parallel for collapse(2) schedule(static) reduction(+ : bad)
  for (int ib = 0; ib < nb; ++ib)
    for (int ia = 0; ia < na; ++ia) {
      int a = r.lo[t1] + ia, bb = r.lo[t2] + ib;
      std::vector<Cell> cells(ncell);
      std::vector<real> bface(ncell + 1);
      std::vector<real> flux((size_t)(ncell + 1) * 7, NaN);
      std::vector<unsigned char> hflag(ncell + 1);
      for (int c = 0; c < ncell; ++c) {
        int idx[3];
        idx[d] = c0 + c; idx[t1] = a; idx[t2] = bb;
        load_cell(g, qin, d, idx[0], idx[1], idx[2], &cells[c]);
      }
      for (int f = 1; f <= ncell - 1; ++f) {
        int idx[3];
        idx[d] = c0 + f; idx[t1] = a; idx[t2] = bb;
        bface[f] = bn(idx[0], idx[1], idx[2]);
      }
      bface[0] = NaN;
      pencil_flux(ncell, cells.data(), bface.data(), dtdx, dx_2dt, g->P,
                  reinterpret_cast<real(*)[7]>(flux.data()), hflag.data());
      const bool across = a >= 0 && a < g->n[t1] && bb >= 0 && bb < g->n[t2];
      for (int f = 2; f <= ncell - 2; ++f)
        if (hflag[f] && across && c0 + f >= 0 && c0 + f < g->n[d]) ++bad;
      for (int f = 2; f <= ncell - 2; ++f) {
        int idx[3];
        idx[d] = c0 + f; idx[t1] = a; idx[t2] = bb;
        const real* F = &flux[(size_t)f * 7];
        int i = idx[0], j = idx[1], k = idx[2];
        out[RHO](i, j, k) = F[0];
        out[MX + d](i, j, k) = F[1];
        out[MX + t1](i, j, k) = F[2];
        out[MX + t2](i, j, k) = F[3];
        out[EN](i, j, k) = F[6];
        out[BX + d](i, j, k) = 0.0;
        out[BX + t1](i, j, k) = F[4];
        out[BX + t2](i, j, k) = F[5];
      }
    }
  return bad;
}

// Steps 2 and 8: zone-centred reference EMF E = -v x B.
void reference_emf(const Arr* rho, const Arr* m, const Arr* B, Arr* E, const Range& r) {
  FLOP_SECTION(SEC_EREF);
#pragma omp parallel for schedule(static)
  for (int k = r.lo[2]; k <= r.hi[2]; ++k)
    for (int j = r.lo[1]; j <= r.hi[1]; ++j)
      for (int i = r.lo[0]; i <= r.hi[0]; ++i) {
        FLOP_UNIT(SEC_EREF);
        real vx = m[0](i, j, k) / rho[0](i, j, k);
        real vy = m[1](i, j, k) / rho[0](i, j, k);
        real vz = m[2](i, j, k) / rho[0](i, j, k);
        real bx = B[0](i, j, k), by = B[1](i, j, k), bz = B[2](i, j, k);
        E[0](i, j, k) = vz * by - vy * bz;
        E[1](i, j, k) = vx * bz - vz * bx;
        E[2](i, j, k) = vy * bx - vx * by;
      }
}

// Steps 3 and 9: GS05 upwinded corner EMF (reading R11).  Edge along axis c,
// a -> b -> c cyclic; the edge (fa, fb) sits at a-face fa and b-face fb.
// Face EMFs from the fluxes: Ea = -F_a[B_b] on a-faces, Eb = +F_b[B_a] on
// b-faces; upwinding by the mass fluxes F_a[rho], F_b[rho]; the corner value
// is the face average plus (1/4)[(dE/db)_{-3/4} - (dE/db)_{-1/4}] and the same
// in a, each derivative taken from the upwind zone (average if the mass flux
// is zero).
void edge_emf(or_grid* g, int c, Arr F[3][8], const Arr& Er, Arr& Eout, const Range& r) {
  int a = (c + 1) % 3, b = (c + 2) % 3;
  Arr* Fa = F[a];
  Arr* Fb = F[b];
  (void)g;
  FLOP_SECTION(SEC_EDGE);
#pragma omp parallel for schedule(static)
  for (int k = r.lo[2]; k <= r.hi[2]; ++k)
    for (int j = r.lo[1]; j <= r.hi[1]; ++j)
      for (int i = r.lo[0]; i <= r.hi[0]; ++i) {
        FLOP_UNIT(SEC_EDGE);
        int p[3] = {i, j, k};
        // neighbour offsets: ma = one step back along a, mb = back along b
        int pa[3] = {i, j, k}; pa[a] -= 1;           // (fa-1, fb)
        int pb[3] = {i, j, k}; pb[b] -= 1;           // (fa, fb-1)
        int pab[3] = {i, j, k}; pab[a] -= 1; pab[b] -= 1;
        // a-face EMF at (fa, jb) and (fa, jb-1)
        real Ea_0 = -Fa[BX + b](p[0], p[1], p[2]);      // (fa, fb)   -> a-face fa, b-cell fb
        real Ea_m = -Fa[BX + b](pb[0], pb[1], pb[2]);   // (fa, fb-1)
        // b-face EMF at (ia, fb) and (ia-1, fb)
        real Eb_0 = Fb[BX + a](p[0], p[1], p[2]);       // a-cell fa, b-face fb
        real Eb_m = Fb[BX + a](pa[0], pa[1], pa[2]);    // a-cell fa-1
        real ma_0 = Fa[RHO](p[0], p[1], p[2]);
        real ma_m = Fa[RHO](pb[0], pb[1], pb[2]);
        real mb_0 = Fb[RHO](p[0], p[1], p[2]);
        real mb_m = Fb[RHO](pa[0], pa[1], pa[2]);
        // reference EMF at the four zones around the edge
        real R00 = Er(p[0], p[1], p[2]);          // zone (fa, fb)
        real Rm0 = Er(pa[0], pa[1], pa[2]);       // zone (fa-1, fb)
        real R0m = Er(pb[0], pb[1], pb[2]);       // zone (fa, fb-1)
        real Rmm = Er(pab[0], pab[1], pab[2]);    // zone (fa-1, fb-1)
        // d/db at b-position fb-1/4 (between b-face fb and zone fb), upwind in a by ma_0
        real db_hi_m = Rm0 - Eb_m, db_hi_0 = R00 - Eb_0;
        real db_hi = ma_0 > 0.0 ? db_hi_m : (ma_0 < 0.0 ? db_hi_0 : 0.5 * (db_hi_m + db_hi_0));
        // d/db at fb-3/4 (between zone fb-1 and b-face fb), upwind by ma_m
        real db_lo_m = Eb_m - Rmm, db_lo_0 = Eb_0 - R0m;
        real db_lo = ma_m > 0.0 ? db_lo_m : (ma_m < 0.0 ? db_lo_0 : 0.5 * (db_lo_m + db_lo_0));
        // d/da at a-position fa-1/4 (between a-face fa and zone fa), upwind in b by mb_0
        real da_hi_m = R0m - Ea_m, da_hi_0 = R00 - Ea_0;
        real da_hi = mb_0 > 0.0 ? da_hi_m : (mb_0 < 0.0 ? da_hi_0 : 0.5 * (da_hi_m + da_hi_0));
        // d/da at fa-3/4 (between zone fa-1 and a-face fa), upwind by mb_m
        real da_lo_m = Ea_m - Rmm, da_lo_0 = Ea_0 - Rm0;
        real da_lo = mb_m > 0.0 ? da_lo_m : (mb_m < 0.0 ? da_lo_0 : 0.5 * (da_lo_m + da_lo_0));
        Eout(i, j, k) = 0.25 * (Ea_0 + Ea_m + Eb_0 + Eb_m) + 0.25 * (db_lo - db_hi) +
                        0.25 * (da_lo - da_hi);
      }
}

// Steps 4 and 11: constrained transport b_out = b_in - tau curl E on faces.
// E[c] indexed by the low faces of the two other axes.
void ct_update(or_grid* g, const Arr* bin, Arr* E, double tau, Arr* bout, const Range rr[3]) {
  for (int d = 0; d < 3; ++d) {
    int a = (d + 1) % 3, b = (d + 2) % 3;
    // (curl E)_d = dE_b/da - dE_a/db
    const Range& r = rr[d];
    double da = g->dxv[a], db = g->dxv[b];
    FLOP_SECTION(SEC_CT);
#pragma omp parallel for schedule(static)
    for (int k = r.lo[2]; k <= r.hi[2]; ++k)
      for (int j = r.lo[1]; j <= r.hi[1]; ++j)
        for (int i = r.lo[0]; i <= r.hi[0]; ++i) {
          FLOP_UNIT(SEC_CT);
          int pa[3] = {i, j, k}; pa[a] += 1;
          int pb[3] = {i, j, k}; pb[b] += 1;
          real curl = (E[b](pa[0], pa[1], pa[2]) - E[b](i, j, k)) / da -
                        (E[a](pb[0], pb[1], pb[2]) - E[a](i, j, k)) / db;
          bout[d](i, j, k) = bin[d](i, j, k) - tau * curl;
        }
  }
}

inline real minmod(real x, real y) {
  if (x > 0.0 && y > 0.0) return r_fmin(x, y);
  if (x < 0.0 && y < 0.0) return r_fmax(x, y);
  return 0.0;
}

// Steps 5 and 7: q^{n+1/2}_d = q^n - dt/2 (transverse flux divergence) + dt/2 S_d,
// zone-centred B_d := average of b_d^{n+1/2} (reading R12), with the GS08
// div B source term S_d (reading R13).  S_d supplies the part of the d-flux
// gradient that a d-sweep leaves out because it holds B_d fixed (with the
// energy referred to the normal field, reading R4):
// -(dF_d/dB_d) db_d/dx_d at fixed (rho, M, E - B_d^2/2, B_t), i.e.
// (0, B db_d, (B_t . v_t) db_d, v_t db_d) for (rho, M, E, B_t).  Following
// GS08, each transverse field component and its energy share are limited by
// minmod(db_d, -db_t) against the other transverse axis, whose difference
// carries the same divergence in the transverse flux of that component.
void transverse_state(or_grid* g, int d, double dt, const Range& r) {
  int t1 = (d + 1) % 3, t2 = (d + 2) % 3;
  double hdt = 0.5 * dt;
  Arr* out = g->qh[d];
  FLOP_SECTION(SEC_TRANS);
#pragma omp parallel for schedule(static)
  for (int k = r.lo[2]; k <= r.hi[2]; ++k)
    for (int j = r.lo[1]; j <= r.hi[1]; ++j)
      for (int i = r.lo[0]; i <= r.hi[0]; ++i) {
        FLOP_UNIT(SEC_TRANS);
        int p[3] = {i, j, k};
        int p1[3] = {i, j, k}; p1[t1] += 1;
        int p2[3] = {i, j, k}; p2[t2] += 1;
        int pd[3] = {i, j, k}; pd[d] += 1;
        real rho = g->q[RHO](i, j, k);
        real v[3], B[3], db[3];
        for (int e = 0; e < 3; ++e) {
          v[e] = g->q[MX + e](i, j, k) / rho;
          B[e] = g->q[BX + e](i, j, k);
          int pe[3] = {i, j, k}; pe[e] += 1;
          db[e] = (g->b[e](pe[0], pe[1], pe[2]) - g->b[e](i, j, k)) / g->dxv[e];
        }
        // GS08 source: m_t1 pairs d with t2, m_t2 pairs d with t1
        real m2 = minmod(db[d], -db[t1]);   // used for the t2 field component
        real m1 = minmod(db[d], -db[t2]);   // used for the t1 field component
        real S[8];
        S[RHO] = 0.0;
        for (int e = 0; e < 3; ++e) S[MX + e] = B[e] * db[d];
        S[EN] = B[t1] * v[t1] * m1 + B[t2] * v[t2] * m2;
        S[BX + d] = 0.0;
        S[BX + t1] = v[t1] * m1;
        S[BX + t2] = v[t2] * m2;
        for (int c = 0; c < 8; ++c) {
          if (c == BX + d) continue;
          real div = (g->Fp[t1][c](p1[0], p1[1], p1[2]) - g->Fp[t1][c](p[0], p[1], p[2])) / g->dxv[t1] +
                       (g->Fp[t2][c](p2[0], p2[1], p2[2]) - g->Fp[t2][c](p[0], p[1], p[2])) / g->dxv[t2];
          out[c](i, j, k) = g->q[c](i, j, k) - hdt * div + hdt * (g->P.source_scale * S[c]);
        }
        out[BX + d](i, j, k) = 0.5 * (g->bh[d](i, j, k) + g->bh[d](pd[0], pd[1], pd[2]));
      }
}

// Step 8: reference EMF at n+1/2 from v of q^n - dt/2 div F* and B from the
// averages of b^{n+1/2} (reading R14).
void half_reference_emf(or_grid* g, double dt, const Range& r) {
  double hdt = 0.5 * dt;
  FLOP_SECTION(SEC_EREFH);
#pragma omp parallel for schedule(static)
  for (int k = r.lo[2]; k <= r.hi[2]; ++k)
    for (int j = r.lo[1]; j <= r.hi[1]; ++j)
      for (int i = r.lo[0]; i <= r.hi[0]; ++i) {
        FLOP_UNIT(SEC_EREFH);
        real u[4];
        int comps[4] = {RHO, MX, MY, MZ};
        for (int c = 0; c < 4; ++c) {
          real div = 0.0;
          for (int e = 0; e < 3; ++e) {
            int pe[3] = {i, j, k}; pe[e] += 1;
            div += (g->Fc[e][comps[c]](pe[0], pe[1], pe[2]) - g->Fc[e][comps[c]](i, j, k)) / g->dxv[e];
          }
          u[c] = g->q[comps[c]](i, j, k) - hdt * div;
        }
        real vx = u[1] / u[0], vy = u[2] / u[0], vz = u[3] / u[0];
        real B[3];
        for (int e = 0; e < 3; ++e) {
          int pe[3] = {i, j, k}; pe[e] += 1;
          B[e] = 0.5 * (g->bh[e](i, j, k) + g->bh[e](pe[0], pe[1], pe[2]));
        }
        g->Erefh[0](i, j, k) = vz * B[1] - vy * B[2];
        g->Erefh[1](i, j, k) = vx * B[2] - vz * B[0];
        g->Erefh[2](i, j, k) = vy * B[0] - vx * B[1];
      }
}

Range box(int l0, int h0, int l1, int h1, int l2, int h2) {
  Range r;
  r.lo[0] = l0; r.hi[0] = h0; r.lo[1] = l1; r.hi[1] = h1; r.lo[2] = l2; r.hi[2] = h2;
  return r;
}

void apply_floors_and_ccb(or_grid* g) {
  const int* n = g->n;
  double gam = g->P.gamma;
  long long hits = 0, bad = 0;
  FLOP_SECTION(SEC_FINAL);
#pragma omp parallel for schedule(static) reduction(+ : hits, bad)
  for (int k = 0; k < n[2]; ++k)
    for (int j = 0; j < n[1]; ++j)
      for (int i = 0; i < n[0]; ++i) {
        FLOP_UNIT(SEC_FINAL);
        g->q[BX](i, j, k) = 0.5 * (g->b[0](i, j, k) + g->b[0](i + 1, j, k));
        g->q[BY](i, j, k) = 0.5 * (g->b[1](i, j, k) + g->b[1](i, j + 1, k));
        g->q[BZ](i, j, k) = 0.5 * (g->b[2](i, j, k) + g->b[2](i, j, k + 1));
        // density and pressure floors (reading R1)
        real rho = g->q[RHO](i, j, k);
        if (rho < g->P.rho_floor) { rho = g->P.rho_floor; g->q[RHO](i, j, k) = rho; ++hits; }
        real mx = g->q[MX](i, j, k), my = g->q[MY](i, j, k), mz = g->q[MZ](i, j, k);
        real ke = 0.5 * (mx * mx + my * my + mz * mz) / rho;
        real bx = g->q[BX](i, j, k), by = g->q[BY](i, j, k), bz = g->q[BZ](i, j, k);
        real me = 0.5 * (bx * bx + by * by + bz * bz);
        real p = (gam - 1.0) * (g->q[EN](i, j, k) - ke - me);
        if (p < g->P.p_floor) {
          g->q[EN](i, j, k) = g->P.p_floor / (gam - 1.0) + ke + me;
          ++hits;
        }
        bool ok = r_isfinite(rho) && r_isfinite(p) && r_isfinite(g->q[EN](i, j, k)) &&
                  r_isfinite(mx) && r_isfinite(my) && r_isfinite(mz) && rho > 0.0;
        if (!ok) ++bad;
      }
  FLOP_SECTION(SEC_NONE);
  g->floor_hits += hits;
  g->unphysical += bad;
}

}  // namespace

extern "C" {

or_grid* or_create(int nx, int ny, int nz, double lx, double ly, double lz, double gamma,
                   double cfl, const int bc[3], const double eps[7], double sweby,
                   double rho_floor, double p_floor) {
  if (nx < 1 || ny < 1 || nz < 1 || !(lx > 0) || !(ly > 0) || !(lz > 0)) return nullptr;
  if (!(gamma > 1.0) || gamma > 2.0) return nullptr;
  or_grid* g = new or_grid();
  g->n[0] = nx; g->n[1] = ny; g->n[2] = nz;
  g->len[0] = lx; g->len[1] = ly; g->len[2] = lz;
  for (int d = 0; d < 3; ++d) {
    g->dxv[d] = g->len[d] / g->n[d];
    g->bc[d] = bc ? bc[d] : 0;
  }
  g->P.gamma = gamma;
  g->P.cfl = cfl;
  for (int k = 0; k < 7; ++k) g->P.eps[k] = eps[k];
  g->P.sweby = sweby;
  g->P.rho_floor = rho_floor;
  g->P.p_floor = p_floor;
  for (int v = 0; v < 8; ++v) alloc_like(g, g->q[v]);
  for (int d = 0; d < 3; ++d) alloc_like(g, g->b[d]);
  for (int d = 0; d < 3; ++d) {
    for (int v = 0; v < 8; ++v) {
      alloc_like(g, g->Fp[d][v]);
      alloc_like(g, g->Fc[d][v]);
      alloc_like(g, g->qh[d][v]);
    }
    alloc_like(g, g->Eref[d]);
    alloc_like(g, g->Eedge[d]);
    alloc_like(g, g->bh[d]);
    alloc_like(g, g->Erefh[d]);
    alloc_like(g, g->Eedgeh[d]);
  }
  return g;
}

void or_destroy(or_grid* g) { delete g; }

int or_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
  return omp_get_max_threads();
#else
  (void)n;
  return 1;
#endif
}

int or_load(or_grid* g, const double* U, const double* bx, const double* by, const double* bz) {
  if (!g || !U || !bx || !by || !bz) return 1;
  FLOP_SECTION(SEC_NONE);
  int nx = g->n[0], ny = g->n[1], nz = g->n[2];
  size_t nc = (size_t)nx * ny * nz;
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        size_t c = ((size_t)k * ny + j) * nx + i;
        for (int v = 0; v < 5; ++v) g->q[v](i, j, k) = U[v * nc + c];
        g->b[0](i, j, k) = bx[((size_t)k * ny + j) * (nx + 1) + i];
        g->b[1](i, j, k) = by[((size_t)k * (ny + 1) + j) * nx + i];
        g->b[2](i, j, k) = bz[((size_t)k * ny + j) * nx + i];
      }
  for (int d = 0; d < 3; ++d) fill_array(g, g->b[d], d);
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        g->q[BX](i, j, k) = 0.5 * (g->b[0](i, j, k) + g->b[0](i + 1, j, k));
        g->q[BY](i, j, k) = 0.5 * (g->b[1](i, j, k) + g->b[1](i, j + 1, k));
        g->q[BZ](i, j, k) = 0.5 * (g->b[2](i, j, k) + g->b[2](i, j, k + 1));
      }
  ghost_fill(g);
  return 0;
}

int or_load_primitive(or_grid* g, const double* W, const double* bx, const double* by,
                      const double* bz) {
  if (!g || !W) return 1;
  int nx = g->n[0], ny = g->n[1], nz = g->n[2];
  size_t nc = (size_t)nx * ny * nz;
  std::vector<double> U(5 * nc, 0.0);
  for (size_t c = 0; c < nc; ++c) U[c] = W[c];
  int rc = or_load(g, U.data(), bx, by, bz);  // loads faces, zone B = face averages
  if (rc) return rc;
  double gam = g->P.gamma;
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        size_t c = ((size_t)k * ny + j) * nx + i;
        real rho = W[c], vx = W[nc + c], vy = W[2 * nc + c], vz = W[3 * nc + c], p = W[4 * nc + c];
        real bxc = g->q[BX](i, j, k), byc = g->q[BY](i, j, k), bzc = g->q[BZ](i, j, k);
        g->q[MX](i, j, k) = rho * vx;
        g->q[MY](i, j, k) = rho * vy;
        g->q[MZ](i, j, k) = rho * vz;
        // Eq. totenergy
        g->q[EN](i, j, k) = p / (gam - 1.0) + 0.5 * rho * (vx * vx + vy * vy + vz * vz) +
                            0.5 * (bxc * bxc + byc * byc + bzc * bzc);
      }
  ghost_fill(g);
  return 0;
}

int or_read(const or_grid* g, double* U, double* bx, double* by, double* bz, double* B) {
  if (!g) return 1;
  int nx = g->n[0], ny = g->n[1], nz = g->n[2];
  size_t nc = (size_t)nx * ny * nz;
  for (int k = 0; k <= nz; ++k)
    for (int j = 0; j <= ny; ++j)
      for (int i = 0; i <= nx; ++i) {
        bool ci = i < nx, cj = j < ny, ck = k < nz;
        if (ci && cj && ck) {
          size_t c = ((size_t)k * ny + j) * nx + i;
          if (U)
            for (int v = 0; v < 5; ++v) U[v * nc + c] = to_d(g->q[v](i, j, k));
          if (B)
            for (int v = 0; v < 3; ++v) B[v * nc + c] = to_d(g->q[BX + v](i, j, k));
        }
        if (bx && cj && ck) bx[((size_t)k * ny + j) * (nx + 1) + i] = to_d(g->b[0](i, j, k));
        if (by && ci && ck) by[((size_t)k * (ny + 1) + j) * nx + i] = to_d(g->b[1](i, j, k));
        if (bz && ci && cj) bz[((size_t)k * ny + j) * nx + i] = to_d(g->b[2](i, j, k));
      }
  return 0;
}

// Reading R3: dt = C / max over interior zones of sum_d (|v_d| + c_f,d) / dx_d,
// with c_f,d the fast speed along d (Sec. 3).
double or_compute_dt(const or_grid* g) {
  const int* n = g->n;
  double gam = g->P.gamma;
  double wmax = 0.0;
  FLOP_SECTION(SEC_DT);
#pragma omp parallel for schedule(static) reduction(max : wmax)
  for (int k = 0; k < n[2]; ++k)
    for (int j = 0; j < n[1]; ++j)
      for (int i = 0; i < n[0]; ++i) {
        FLOP_UNIT(SEC_DT);
        real rho = g->q[RHO](i, j, k);
        real v[3], B[3];
        for (int e = 0; e < 3; ++e) {
          v[e] = g->q[MX + e](i, j, k) / rho;
          B[e] = g->q[BX + e](i, j, k);
        }
        real ke = 0.5 * rho * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
        real me = 0.5 * (B[0] * B[0] + B[1] * B[1] + B[2] * B[2]);
        real p = (gam - 1.0) * (g->q[EN](i, j, k) - ke - me);
        real a2 = gam * p / rho;
        real w = 0.0;
        for (int d = 0; d < 3; ++d) {
          int t1 = (d + 1) % 3, t2 = (d + 2) % 3;
          real cn2 = B[d] * B[d] / rho;
          real ct2 = (B[t1] * B[t1] + B[t2] * B[t2]) / rho;
          real disc = (a2 - cn2) * (a2 - cn2) + ct2 * (ct2 + 2.0 * a2 + 2.0 * cn2);
          real cf = r_sqrt(0.5 * (a2 + cn2 + ct2 + r_sqrt(disc)));
          w += (r_fabs(v[d]) + cf) / g->dxv[d];
        }
        if (to_d(w) > wmax) wmax = to_d(w);
      }
  FLOP_SECTION(SEC_DT);
  real rate = wmax;
  real out = g->P.cfl / rate;   // one division per box
  FLOP_SECTION(SEC_NONE);
  return to_d(out);
}

int or_step(or_grid* g, double dt) {
  if (!g || !(dt > 0.0)) return 1;
  const int* n = g->n;
  const int N0 = n[0], N1 = n[1], N2 = n[2];
  long long nhll = 0;
  // Step 1: predictor fluxes from q^n over the regions the later steps read.
  {
    Range rx = box(-3, N0 + 3, -4, N1 + 3, -4, N2 + 3);
    Range ry = box(-4, N0 + 3, -3, N1 + 3, -4, N2 + 3);
    Range rz = box(-4, N0 + 3, -4, N1 + 3, -3, N2 + 3);
    nhll += sweep(g, 0, g->q, g->b[0], dt, rx, g->Fp[0]);
    nhll += sweep(g, 1, g->q, g->b[1], dt, ry, g->Fp[1]);
    nhll += sweep(g, 2, g->q, g->b[2], dt, rz, g->Fp[2]);
  }
  // Step 2: reference EMF from q^n
  reference_emf(&g->q[RHO], &g->q[MX], &g->q[BX], g->Eref,
                box(-4, N0 + 3, -4, N1 + 3, -4, N2 + 3));
  // Step 3: corner EMFs (edge along c at the low faces of the two other axes)
  edge_emf(g, 2, g->Fp, g->Eref[2], g->Eedge[2], box(-3, N0 + 3, -3, N1 + 3, -1, N2));
  edge_emf(g, 1, g->Fp, g->Eref[1], g->Eedge[1], box(-3, N0 + 3, -1, N1, -3, N2 + 3));
  edge_emf(g, 0, g->Fp, g->Eref[0], g->Eedge[0], box(-1, N0, -3, N1 + 3, -3, N2 + 3));
  // Step 4: b^{n+1/2} = b^n - dt/2 curl E
  {
    Range rr[3] = {box(-3, N0 + 3, -1, N1, -1, N2), box(-1, N0, -3, N1 + 3, -1, N2),
                   box(-1, N0, -1, N1, -3, N2 + 3)};
    ct_update(g, g->b, g->Eedge, 0.5 * dt, g->bh, rr);
  }
  // Steps 5 and 7 (transverse-flux preconditioned states)
  transverse_state(g, 0, dt, box(-3, N0 + 2, -1, N1, -1, N2));
  transverse_state(g, 1, dt, box(-1, N0, -3, N1 + 2, -1, N2));
  transverse_state(g, 2, dt, box(-1, N0, -1, N1, -3, N2 + 2));
  // Steps 6 and 7: corrector fluxes, normal Roe field = b^{n+1/2}
  nhll += sweep(g, 0, g->qh[0], g->bh[0], dt, box(-1, N0 + 1, -1, N1, -1, N2), g->Fc[0]);
  nhll += sweep(g, 1, g->qh[1], g->bh[1], dt, box(-1, N0, -1, N1 + 1, -1, N2), g->Fc[1]);
  nhll += sweep(g, 2, g->qh[2], g->bh[2], dt, box(-1, N0, -1, N1, -1, N2 + 1), g->Fc[2]);
  // Step 8: half-step reference EMF
  half_reference_emf(g, dt, box(-1, N0, -1, N1, -1, N2));
  // Step 9: corner EMFs from the corrector fluxes
  edge_emf(g, 2, g->Fc, g->Erefh[2], g->Eedgeh[2], box(0, N0, 0, N1, 0, N2 - 1));
  edge_emf(g, 1, g->Fc, g->Erefh[1], g->Eedgeh[1], box(0, N0, 0, N1 - 1, 0, N2));
  edge_emf(g, 0, g->Fc, g->Erefh[0], g->Eedgeh[0], box(0, N0 - 1, 0, N1, 0, N2));
  // Step 10: un-split conservative update (reading R15: x, then y, then z)
  {
    double cx = dt / g->dxv[0], cy = dt / g->dxv[1], cz = dt / g->dxv[2];
    int comps[5] = {RHO, MX, MY, MZ, EN};
    FLOP_SECTION(SEC_UPDATE);
#pragma omp parallel for schedule(static)
    for (int k = 0; k < N2; ++k)
      for (int j = 0; j < N1; ++j)
        for (int i = 0; i < N0; ++i) {
          FLOP_UNIT(SEC_UPDATE);
          for (int c5 = 0; c5 < 5; ++c5) {
            int c = comps[c5];
            real u = g->q[c](i, j, k);
            u = u - cx * (g->Fc[0][c](i + 1, j, k) - g->Fc[0][c](i, j, k));
            u = u - cy * (g->Fc[1][c](i, j + 1, k) - g->Fc[1][c](i, j, k));
            u = u - cz * (g->Fc[2][c](i, j, k + 1) - g->Fc[2][c](i, j, k));
            g->q[c](i, j, k) = u;
          }
        }
    FLOP_SECTION(SEC_NONE);
  }
  // Step 11: b^{n+1} = b^n - dt curl E^{n+1/2}; zone B from face averages
  {
    Range rr[3] = {box(0, N0, 0, N1 - 1, 0, N2 - 1), box(0, N0 - 1, 0, N1, 0, N2 - 1),
                   box(0, N0 - 1, 0, N1 - 1, 0, N2)};
    // write into bh (no longer needed) then copy, so that b^n stays intact
    // while the update reads it
    Arr tmp[3];
    for (int d = 0; d < 3; ++d) tmp[d] = g->b[d];
    ct_update(g, g->b, g->Eedgeh, dt, tmp, rr);
    for (int d = 0; d < 3; ++d) g->b[d].d.swap(tmp[d].d);
  }
  long long unph0 = g->unphysical;
  // Step 11: the zone field is the average of the face field as the boundary
  // condition leaves it, so the face ghosts are filled first (on an outflow
  // axis the high boundary face becomes a copy of the last owned face,
  // reading R16); then the zone fields and their ghosts
  for (int d = 0; d < 3; ++d) fill_array(g, g->b[d], d);
  apply_floors_and_ccb(g);
  g->hll_faces += nhll;
  for (int v = 0; v < 8; ++v) fill_array(g, g->q[v], -1);
  return g->unphysical > unph0 ? 4 : 0;
}

int or_totals(const or_grid* g, double tot[8]) {
  const int* n = g->n;
  double vol = g->dxv[0] * g->dxv[1] * g->dxv[2];
  for (int c = 0; c < 8; ++c) {
    // Neumaier compensated sum over owned zones / faces
    double s = 0.0, comp = 0.0;
    for (int k = 0; k < n[2]; ++k)
      for (int j = 0; j < n[1]; ++j)
        for (int i = 0; i < n[0]; ++i) {
          double x = to_d(c < 5 ? g->q[c](i, j, k) : g->b[c - 5](i, j, k));
          double t = s + x;
          if (std::fabs(s) >= std::fabs(x)) comp += (s - t) + x;
          else comp += (x - t) + s;
          s = t;
        }
    tot[c] = (s + comp) * vol;
  }
  return 0;
}

double or_divb_max(const or_grid* g) {
  const int* n = g->n;
  double m = 0.0;
  for (int k = 0; k < n[2]; ++k)
    for (int j = 0; j < n[1]; ++j)
      for (int i = 0; i < n[0]; ++i) {
        double dv = (to_d(g->b[0](i + 1, j, k)) - to_d(g->b[0](i, j, k))) / g->dxv[0] +
                    (to_d(g->b[1](i, j + 1, k)) - to_d(g->b[1](i, j, k))) / g->dxv[1] +
                    (to_d(g->b[2](i, j, k + 1)) - to_d(g->b[2](i, j, k))) / g->dxv[2];
        if (std::fabs(dv) > m) m = std::fabs(dv);
      }
  return m;
}

int or_counters(const or_grid* g, long long out[3]) {
  out[0] = g->floor_hits;
  out[1] = g->unphysical;
  out[2] = g->hll_faces;
  return 0;
}

int or_set_source_scale(or_grid* g, double s) {
  if (!g || !std::isfinite(s)) return 1;
  g->P.source_scale = s;
  return 0;
}

int or_set_protection(or_grid* g, double prot_rho, double prot_p) {
  if (!g || !(prot_rho >= 0.0) || !(prot_p >= 0.0)) return 1;
  g->P.prot_rho = prot_rho;
  g->P.prot_p = prot_p;
  return 0;
}

long long or_stage(const or_grid* g, int which, double* out, long long cap) {
  const int* n = g->n;
  long long w = 0;
  auto put = [&](real x) { if (w < cap) out[w] = to_d(x); ++w; };
  if (which >= 0 && which < 6) {
    int d = which % 3;
    const Arr* F = which < 3 ? g->Fp[d] : g->Fc[d];
    int hi[3] = {n[0], n[1], n[2]};
    hi[d] += 1;
    for (int c = 0; c < 8; ++c)
      for (int k = 0; k < hi[2]; ++k)
        for (int j = 0; j < hi[1]; ++j)
          for (int i = 0; i < hi[0]; ++i) put(F[c](i, j, k));
  } else if (which >= 6 && which < 9) {
    int d = which - 6;
    // b^{n+1/2} is computed on [-1, n] transverse and faces [-3, n+3]; dump faces [0, n]
    int hi[3] = {n[0], n[1], n[2]};
    hi[d] += 1;
    for (int k = 0; k < hi[2]; ++k)
      for (int j = 0; j < hi[1]; ++j)
        for (int i = 0; i < hi[0]; ++i) put(g->bh[d](i, j, k));
  } else if (which >= 9 && which < 12) {
    int d = which - 9;
    for (int c = 0; c < 8; ++c)
      for (int k = 0; k < n[2]; ++k)
        for (int j = 0; j < n[1]; ++j)
          for (int i = 0; i < n[0]; ++i) put(g->qh[d][c](i, j, k));
  }
  return w;
}

int or_face_eigen(const double qL[8], const double qR[8], double b, double gamma,
                  double lam[7], double alpha[7], double R[49], double L[49]) {
  Cell cl = {qL[0], qL[1], qL[2], qL[3], qL[4], qL[5], qL[6], qL[7]};
  Cell cr = {qR[0], qR[1], qR[2], qR[3], qR[4], qR[5], qR[6], qR[7]};
  Prim pl = cell_prim(cl, gamma), pr = cell_prim(cr, gamma);
  Eigen e;
  roe_state(pl, pr, b, gamma, &e);
  if (e.bad) return 4;
  real dq[7];
  cons_diff(cl, cr, dq);
  for (int k = 0; k < 7; ++k) {
    lam[k] = to_d(e.lam[k]);
    real s = 0.0;
    for (int m = 0; m < 7; ++m) s += e.L[k][m] * dq[m];
    alpha[k] = to_d(s);
    for (int m = 0; m < 7; ++m) {
      R[m * 7 + k] = to_d(e.R[m][k]);
      L[k * 7 + m] = to_d(e.L[k][m]);
    }
  }
  return 0;
}

int or_flux_pencil(int ncell, const double* cells, const double* bface, double dtdx,
                   double dx_over_2dt, double gamma, const double eps[7], double sweby,
                   double prot_rho, double prot_p, double* out) {
  if (ncell < 4) return -1;
  Params P;
  P.gamma = gamma;
  P.cfl = 0.0;
  for (int k = 0; k < 7; ++k) P.eps[k] = eps[k];
  P.sweby = sweby;
  P.rho_floor = P.p_floor = 0.0;
  P.prot_rho = prot_rho;
  P.prot_p = prot_p;
  std::vector<Cell> c(ncell);
  for (int i = 0; i < ncell; ++i) {
    const double* q = cells + (size_t)i * 8;
    c[i] = Cell{q[0], q[1], q[2], q[3], q[4], q[5], q[6], q[7]};
  }
  std::vector<real> bf(bface, bface + ncell + 1);
  std::vector<real> fl((size_t)(ncell + 1) * 7);
  for (size_t m = 0; m < fl.size(); ++m) fl[m] = out[m];
  int nh = pencil_flux(ncell, c.data(), bf.data(), dtdx, dx_over_2dt, P,
                       reinterpret_cast<real(*)[7]>(fl.data()));
  for (size_t m = 0; m < fl.size(); ++m) out[m] = to_d(fl[m]);
  return nh;
}

// Operation counts of the counting build, per section (flop_count.h): the
// FP64 operations and the units (zones, faces, edges) evaluated since the last
// reset.  Returns the number of sections, or -1 in the ordinary build.
int or_flop_report(long long* flops, long long* units, int cap) {
#ifdef ORACLE_COUNT_FLOPS
  for (int s = 0; s < flopcount::SEC_COUNT && s < cap; ++s) {
    flops[s] = flopcount::flops[s];
    units[s] = flopcount::units[s];
  }
  return flopcount::SEC_COUNT;
#else
  (void)flops; (void)units; (void)cap;
  return -1;
#endif
}

void or_flop_reset() {
#ifdef ORACLE_COUNT_FLOPS
  for (int s = 0; s < flopcount::SEC_COUNT; ++s) flopcount::flops[s] = flopcount::units[s] = 0;
#endif
}

// Independent 1D driver (the RJ95 one-dimensional scheme, App. A Eq.
// mhd_finite): periodic ghosts, the same interface flux, q -= dt/dx du.
int or_step_1d(int n, double* q, double b, double dt, double dx, double gamma,
               const double eps[7], double sweby, double prot_rho, double prot_p, int outflow) {
  if (n < 1) return -1;
  const int G = 3;  // a face flux needs two zones on each side
  int ncell = n + 2 * G;
  std::vector<double> cells((size_t)ncell * 8), bface(ncell + 1, b);
  for (int c = 0; c < ncell; ++c) {
    int src = outflow ? std::min(std::max(c - G, 0), n - 1) : wrap(c - G, n);
    for (int v = 0; v < 8; ++v) cells[(size_t)c * 8 + v] = q[(size_t)src * 8 + v];
  }
  std::vector<double> flux((size_t)(ncell + 1) * 7, NaN);
  int rc = or_flux_pencil(ncell, cells.data(), bface.data(), dt / dx, dx / (2.0 * dt), gamma,
                          eps, sweby, prot_rho, prot_p, flux.data());
  // system order (rho, Mn, Mt1, Mt2, Bt1, Bt2, E) -> cell order (rho, Mn, Mt1, Mt2, E, Bn, Bt1, Bt2)
  const int map[7] = {0, 1, 2, 3, 6, 7, 4};
  for (int i = 0; i < n; ++i) {
    int f = i + G;  // low face of cell i in pencil numbering
    for (int m = 0; m < 7; ++m) {
      double du = flux[(size_t)(f + 1) * 7 + m] - flux[(size_t)f * 7 + m];
      q[(size_t)i * 8 + map[m]] = q[(size_t)i * 8 + map[m]] - dt / dx * du;
    }
  }
  return rc;
}

}  // extern "C"
