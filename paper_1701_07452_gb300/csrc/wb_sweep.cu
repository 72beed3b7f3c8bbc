// MHDTVD sweep kernel: the modified flux of App. A (Eq. mhdtvd_flux2 and the
// definitions of f, beta, alpha, gamma, g, g-tilde and Q) along one axis, used
// for the predictor fluxes of Step 1 and the corrector fluxes of Steps 6-7 of
// the 3D CTU+CT integrator (Sec. "MHD in Three Dimensions").
//
// One thread marches along one pencil of faces.  For each face it builds the
// Roe-averaged interface state (a Cargo-Gallice type average, App. A), the
// characteristic amplitudes alpha_k, nu_k = (dt/dx) a_k and g-tilde_k; the
// flux of face f is emitted once g-tilde of face f+1 is known, so every
// eigen-system is computed exactly once and only g-tilde of three faces plus
// the eigen-data of one face are carried in registers.
//
// Eigen-structure (derived for this implementation): the linearisation
// dF = A dU with rho_ = sL sR, s-weighted v and H, opposite-weighted B_t and
// the face normal field b is the ideal-MHD Jacobian at that state with sound
// speed a_^2 = (gamma-1)(H_ - v_^2/2 - (b^2+B_t^2)/rho_) - (gamma-2) X,
// X = |dB_t|^2 / (2 (sL+sR)^2).  The waves are projected in primitive
// variables w = (rho, vn, vt, Bt, p) and sum_k beta_k R_k is accumulated in w
// and mapped to conserved variables once (the map is linear).
#include "wb_device.cuh"
#include "wb_internal.h"

namespace {

struct Cell {
  double rho, ir, sr, isr;        // rho, 1/rho, sqrt(rho), 1/sqrt(rho)
  double vn, vt1, vt2, p;
  double bn, bt1, bt2;
  double eref;                    // E - bn^2/2 (energy referred to the face field)
  double h;                       // gamma/(gamma-1) P + rho v^2/2 + |Bt|^2
  double F[7];                    // Sec. 3 flux (rho, Mn, Mt1, Mt2, Bt1, Bt2, E)
  double mn, mt1, mt2;
};

template <int D>
__device__ __forceinline__ void load_cell(const SweepArgs& A, long long off, Cell& c) {
  constexpr int T1 = (D + 1) % 3, T2 = (D + 2) % 3;
  const WbPhys& P = A.phys;
  c.rho = __ldg(A.q[F_RHO] + off);
  c.mn = __ldg(A.q[F_MX + D] + off);
  c.mt1 = __ldg(A.q[F_MX + T1] + off);
  c.mt2 = __ldg(A.q[F_MX + T2] + off);
  double e = __ldg(A.q[F_EN] + off);
  c.bn = __ldg(A.q[F_BX + D] + off);
  c.bt1 = __ldg(A.q[F_BX + T1] + off);
  c.bt2 = __ldg(A.q[F_BX + T2] + off);
  c.isr = rsqrt(c.rho);
  c.ir = c.isr * c.isr;
  c.sr = c.rho * c.isr;
  c.vn = c.mn * c.ir;
  c.vt1 = c.mt1 * c.ir;
  c.vt2 = c.mt2 * c.ir;
  double ke = 0.5 * (c.mn * c.vn + c.mt1 * c.vt1 + c.mt2 * c.vt2);
  double bt2 = c.bt1 * c.bt1 + c.bt2 * c.bt2;
  double me = 0.5 * (c.bn * c.bn + bt2);
  c.p = P.gm1 * (e - ke - me);
  double pstar = c.p + me;
  c.eref = e - 0.5 * c.bn * c.bn;
  c.h = P.g_over_gm1 * c.p + ke + bt2;
  c.F[0] = c.mn;
  c.F[1] = c.mn * c.vn + pstar - c.bn * c.bn;
  c.F[2] = c.mn * c.vt1 - c.bn * c.bt1;
  c.F[3] = c.mn * c.vt2 - c.bn * c.bt2;
  c.F[4] = c.bt1 * c.vn - c.bn * c.vt1;
  c.F[5] = c.bt2 * c.vn - c.bn * c.vt2;
  c.F[6] = (e + pstar) * c.vn - c.bn * (c.bn * c.vn + c.bt1 * c.vt1 + c.bt2 * c.vt2);
}

// Per-face data kept until the face's flux is emitted.
struct Face {
  double alpha[7], nu[7];
  double rho, srho, a, a2, cf, cs, af, as, b1, b2, S;
  double vn, vt1, vt2, bt1, bt2, X;
  double Favg[7];
};

// Q_k(chi) of App. A
__device__ __forceinline__ double Qk(double chi, int k, const WbPhys& P) {
  double ac = fabs(chi);
  return (ac < P.two_eps[k]) ? chi * chi * P.inv4eps[k] + P.eps[k] : ac;
}

__device__ __forceinline__ bool face_system(const Cell& L, const Cell& R, double b, double dtdx,
                                            const WbPhys& P, Face& f, double gt[7]) {
  double iD = 1.0 / (L.sr + R.sr);
  double wL = L.sr * iD, wR = R.sr * iD;
  double rho = L.sr * R.sr;
  double irho = L.isr * R.isr;
  f.vn = wL * L.vn + wR * R.vn;
  f.vt1 = wL * L.vt1 + wR * R.vt1;
  f.vt2 = wL * L.vt2 + wR * R.vt2;
  f.bt1 = wR * L.bt1 + wL * R.bt1;
  f.bt2 = wR * L.bt2 + wL * R.bt2;
  double b2 = b * b;
  double H = wL * ((L.h + b2) * L.ir) + wR * ((R.h + b2) * R.ir);
  double dbt1 = R.bt1 - L.bt1, dbt2 = R.bt2 - L.bt2;
  f.X = 0.5 * (dbt1 * dbt1 + dbt2 * dbt2) * (iD * iD);
  double v2 = f.vn * f.vn + f.vt1 * f.vt1 + f.vt2 * f.vt2;
  double bt2s = f.bt1 * f.bt1 + f.bt2 * f.bt2;
  double a2 = P.gm1 * (H - 0.5 * v2 - (b2 + bt2s) * irho) - P.gm2 * f.X;
  if (!(a2 > 0.0)) return false;
  f.rho = rho;
  double isrho = rsqrt(rho);
  f.srho = rho * isrho;
  double ca2 = b2 * irho, ct2 = bt2s * irho;
  double dac = a2 - ca2;
  double disc = dac * dac + ct2 * (ct2 + 2.0 * (a2 + ca2));
  double sum = a2 + ca2 + ct2;
  double cf2, icf, rsd = 0.0, sd;
  if (disc > 0.0) {
    rsd = rsqrt(disc);
    sd = disc * rsd;
  } else {
    sd = 0.0;
  }
  cf2 = 0.5 * (sum + sd);
  icf = rsqrt(cf2);
  double ia = rsqrt(a2);
  double a = a2 * ia;
  double ca = fabs(b) * isrho;
  f.a = a;
  f.a2 = a2;
  f.cf = cf2 * icf;
  f.cs = a * ca * icf;  // c_f c_s = a c_a
  if (sd <= 1e-12 * sum) {
    if (a2 >= ca2) { f.af = 1.0; f.as = 0.0; }
    else { f.af = 0.0; f.as = 1.0; }
  } else {
    // cf^2 - a^2 and cf^2 - ca^2 without cancellation; at most one of the
    // two needs a division
    double t1 = ca2 + ct2 - a2;
    double t2 = a2 - ca2 + ct2;
    double num = (t1 < 0.0) ? 2.0 * a2 * ct2 : 2.0 * ca2 * ct2;
    double den = (t1 < 0.0) ? sd - t1 : sd - t2;
    double qd = (t1 < 0.0 || t2 < 0.0) ? num / den : 0.0;
    double cf2_a2 = (t1 >= 0.0) ? 0.5 * (t1 + sd) : qd;
    double cf2_ca2 = (t2 >= 0.0) ? 0.5 * (t2 + sd) : qd;
    double a2_cs2 = a2 * cf2_ca2 * (icf * icf);
    double af2 = fmin(fmax(a2_cs2 * rsd, 0.0), 1.0);
    double as2 = fmin(fmax(cf2_a2 * rsd, 0.0), 1.0);
    f.af = sqrt(af2);
    f.as = sqrt(as2);
  }
  if (bt2s <= 1e-24 * (rho * a2 + b2 + bt2s)) {
    f.b1 = f.b2 = 0.70710678118654752440;
  } else {
    double ib = rsqrt(bt2s);
    f.b1 = f.bt1 * ib;
    f.b2 = f.bt2 * ib;
  }
  f.S = wb_sgn(b);
  // eigenvalues a_1..a_7 (Sec. 3)
  double lam[7] = {f.vn - f.cf, f.vn - ca, f.vn - f.cs, f.vn, f.vn + f.cs, f.vn + ca, f.vn + f.cf};
  // primitive differences of the 7-variable system
  double drho = R.rho - L.rho;
  double dmn = R.mn - L.mn, dmt1 = R.mt1 - L.mt1, dmt2 = R.mt2 - L.mt2;
  double dbt1c = dbt1, dbt2c = dbt2;
  double de = R.eref - L.eref;
  double dvn = (dmn - f.vn * drho) * irho;
  double dvt1 = (dmt1 - f.vt1 * drho) * irho;
  double dvt2 = (dmt2 - f.vt2 * drho) * irho;
  double dp = P.gm1 * (de - (f.vn * dmn + f.vt1 * dmt1 + f.vt2 * dmt2) + 0.5 * v2 * drho -
                       (f.bt1 * dbt1c + f.bt2 * dbt2c)) - P.gm2 * f.X * drho;
  // projections on the transverse field direction beta and its normal
  double dvb = f.b1 * dvt1 + f.b2 * dvt2, dvp = -f.b2 * dvt1 + f.b1 * dvt2;
  double dbb = f.b1 * dbt1c + f.b2 * dbt2c, dbp = -f.b2 * dbt1c + f.b1 * dbt2c;
  double i2a2 = 0.5 * ia * ia;
  double i2ra = 0.5 * isrho * ia;
  double dpr = dp * irho * i2a2;  // dp / (2 rho a^2)
  double Af = (f.af * f.cf * dvn - f.as * f.cs * f.S * dvb) * i2a2;
  double Cf = f.as * dbb * i2ra + f.af * dpr;
  double As = (f.as * f.cs * dvn + f.af * f.cf * f.S * dvb) * i2a2;
  double Cs = -f.af * dbb * i2ra + f.as * dpr;
  double Aa = f.S * dbp * isrho;
  f.alpha[0] = Cf - Af;
  f.alpha[6] = Cf + Af;
  f.alpha[2] = Cs - As;
  f.alpha[4] = Cs + As;
  f.alpha[1] = 0.5 * (dvp + Aa);
  f.alpha[5] = 0.5 * (dvp - Aa);
  f.alpha[3] = drho - dp * (2.0 * i2a2);
#pragma unroll
  for (int k = 0; k < 7; ++k) {
    double nu = dtdx * lam[k];
    f.nu[k] = nu;
    gt[k] = 0.5 * (Qk(nu, k, P) - nu * nu) * f.alpha[k];
  }
#pragma unroll
  for (int m = 0; m < 7; ++m) f.Favg[m] = 0.5 * (L.F[m] + R.F[m]);
  return true;
}

// u-bar = (F_L + F_R)/2 - (dx/(2 dt)) sum_k beta_k R_k  (App. A)
__device__ __forceinline__ void face_flux(const Face& f, const double gi[7], const double gi1[7],
                                          double dx_2dt, const WbPhys& P, double out[7]) {
  double be[7];
#pragma unroll
  for (int k = 0; k < 7; ++k) {
    double al = f.alpha[k];
    double gam = (al != 0.0) ? (gi1[k] - gi[k]) / al : 0.0;
    be[k] = Qk(f.nu[k] + gam, k, P) * al - (gi[k] + gi1[k]);
  }
  // sum_k beta_k r_k in w = (rho, vn, vt, Bt, p)
  double sf = be[0] + be[6], df = be[6] - be[0];
  double ss = be[2] + be[4], ds = be[4] - be[2];
  double wr = f.rho * (f.af * sf + f.as * ss) + be[3];
  double wvn = f.af * f.cf * df + f.as * f.cs * ds;
  double vb = f.S * (f.af * f.cf * ds - f.as * f.cs * df);   // along beta
  double vp = be[1] + be[5];                                // along beta-perp
  double ra = f.srho * f.a;
  double bb = ra * (f.as * sf - f.af * ss);
  double bp = f.S * f.srho * (be[1] - be[5]);
  double wp = f.rho * f.a2 * (f.af * sf + f.as * ss);
  double wvt1 = f.b1 * vb - f.b2 * vp, wvt2 = f.b2 * vb + f.b1 * vp;
  double wbt1 = f.b1 * bb - f.b2 * bp, wbt2 = f.b2 * bb + f.b1 * bp;
  // to conserved variables
  double v2 = f.vn * f.vn + f.vt1 * f.vt1 + f.vt2 * f.vt2;
  double u0 = wr;
  double u1 = f.vn * wr + f.rho * wvn;
  double u2 = f.vt1 * wr + f.rho * wvt1;
  double u3 = f.vt2 * wr + f.rho * wvt2;
  double u6 = wp * P.inv_gm1 + (0.5 * v2 + P.gm2_over_gm1 * f.X) * wr +
              f.rho * (f.vn * wvn + f.vt1 * wvt1 + f.vt2 * wvt2) + f.bt1 * wbt1 + f.bt2 * wbt2;
  out[0] = f.Favg[0] - dx_2dt * u0;
  out[1] = f.Favg[1] - dx_2dt * u1;
  out[2] = f.Favg[2] - dx_2dt * u2;
  out[3] = f.Favg[3] - dx_2dt * u3;
  out[4] = f.Favg[4] - dx_2dt * wbt1;
  out[5] = f.Favg[5] - dx_2dt * wbt2;
  out[6] = f.Favg[6] - dx_2dt * u6;
}

template <int D>
__global__ void __launch_bounds__(128) k_sweep(SweepArgs A) {
  constexpr int T1 = (D + 1) % 3, T2 = (D + 2) % 3;
  constexpr int U = (D == 0) ? 1 : 0;  // fastest transverse axis of the thread map
  constexpr int W = (D == 2) ? 1 : 2;
  const WbGeo& g = A.geo;
  const double dt = *A.dt;
  if (!(dt > 0.0)) return;
  const int nu_ = A.box.hi[U] - A.box.lo[U] + 1;
  const int nw_ = A.box.hi[W] - A.box.lo[W] + 1;
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= nu_ * nw_) return;
  const long long slot = blockIdx.y;
  int pos[3];
  pos[U] = A.box.lo[U] + tid % nu_;
  pos[W] = A.box.lo[W] + tid / nu_;
  const int f0 = A.box.lo[D], f1 = A.box.hi[D];
  pos[D] = f0 - 2;
  const long long st = wb_stride<D>(g);
  const long long off_in = slot * A.slot_in + wb_at(g, pos[0], pos[1], pos[2]);
  const long long off_out = slot * A.slot_out + wb_at(g, pos[0], pos[1], pos[2]);
  const double dtdx = dt * g.idx[D];
  const double dx_2dt = 0.5 * g.dx[D] / dt;
  const WbPhys& P = A.phys;

  Cell cL, cR;
  load_cell<D>(A, off_in, cL);
  Face fprev;
  double gt_p[7], g_p[7];  // g-tilde of face f-1; g of zone f-2
  int bad = 0;
  // faces f = f0-1 .. f1+1; face f lies between zones f-1 and f
  for (int f = f0 - 1; f <= f1 + 1; ++f) {
    const int c = f - (f0 - 2);  // zone f relative to the first zone
    load_cell<D>(A, off_in + c * st, cR);
    double b = __ldg(A.bn + off_in + c * st);
    Face fc;
    double gt[7];
    if (!face_system(cL, cR, b, dtdx, P, fc, gt)) {
      // unphysical Roe state: counted, and the flux is poisoned with NaN
      ++bad;
      const double nan = __longlong_as_double(0x7ff8000000000000LL);
#pragma unroll
      for (int k = 0; k < 7; ++k) { gt[k] = nan; fc.alpha[k] = nan; fc.nu[k] = nan; fc.Favg[k] = nan; }
      fc.rho = fc.srho = fc.a = fc.a2 = fc.cf = fc.cs = fc.af = fc.as = fc.b1 = fc.b2 = fc.S = nan;
      fc.vn = fc.vt1 = fc.vt2 = fc.bt1 = fc.bt2 = fc.X = nan;
    }
    if (f >= f0) {
      // g of zone f-1 from g-tilde of faces f (i+1/2) and f-1 (i-1/2)
      double gz[7];
#pragma unroll
      for (int k = 0; k < 7; ++k) gz[k] = wb_sweby(gt[k], gt_p[k], P.sweby, P.minmod);
      if (f >= f0 + 1) {
        // flux of face f-1 (zones f-2, f-1): g_{i} = g_p (zone f-2), g_{i+1} = gz
        double out[7];
        face_flux(fprev, g_p, gz, dx_2dt, P, out);
        const long long o = off_out + (c - 1) * st;
        A.F[F_RHO][o] = out[0];
        A.F[F_MX + D][o] = out[1];
        A.F[F_MX + T1][o] = out[2];
        A.F[F_MX + T2][o] = out[3];
        A.F[F_EN][o] = out[6];
        A.F[F_BX + T1][o] = out[4];
        A.F[F_BX + T2][o] = out[5];
      }
#pragma unroll
      for (int k = 0; k < 7; ++k) g_p[k] = gz[k];
    }
#pragma unroll
    for (int k = 0; k < 7; ++k) gt_p[k] = gt[k];
    fprev = fc;
    cL = cR;
  }
  if (bad) atomicAdd((unsigned long long*)&A.scal->unphysical, (unsigned long long)bad);
}

}  // namespace

template <int D>
static void launch_sweep(const SweepArgs& a, int nslots, cudaStream_t s) {
  constexpr int U = (D == 0) ? 1 : 0;
  constexpr int W = (D == 2) ? 1 : 2;
  long long npen = (long long)(a.box.hi[U] - a.box.lo[U] + 1) * (a.box.hi[W] - a.box.lo[W] + 1);
  dim3 grid((unsigned)((npen + 127) / 128), (unsigned)nslots);
  k_sweep<D><<<grid, 128, 0, s>>>(a);
}

void wb_launch_sweep(int dir, const SweepArgs& a, int nslots, cudaStream_t s) {
  if (dir == 0) launch_sweep<0>(a, nslots, s);
  else if (dir == 1) launch_sweep<1>(a, nslots, s);
  else launch_sweep<2>(a, nslots, s);
}
