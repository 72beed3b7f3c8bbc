// MHDTVD sweep kernel: the modified flux of App. A (Eq. mhdtvd_flux2 and the
// definitions of f, beta, alpha, gamma, g, g-tilde and Q) along one axis, used
// for the predictor fluxes of Step 1 and the corrector fluxes of Steps 6-7 of
// the 3D CTU+CT integrator (Sec. "MHD in Three Dimensions").
//
// One thread marches along one segment of a pencil of faces.  For each face it
// builds the Roe-averaged interface state (a Cargo-Gallice type average,
// App. A), the characteristic amplitudes alpha_k, nu_k = (dt/dx) a_k and
// g-tilde_k; the flux of face f is emitted once g-tilde of face f+1 is known,
// so every eigen-system is computed once per segment (segments overlap by the
// two faces whose g-tilde the limiter needs).  The per-face eigen-data wait
// for one iteration in a double-buffered shared-memory record.
//
// Eigen-structure (derived for this implementation): the linearisation
// dF = A dU with rho_ = sL sR, s-weighted v and H, opposite-weighted B_t and
// the face normal field b is the ideal-MHD Jacobian at that state with sound
// speed a_^2 = (gamma-1)(H_ - v_^2/2 - (b^2+B_t^2)/rho_) - (gamma-2) X,
// X = |dB_t|^2 / (2 (sL+sR)^2).  The waves are projected in primitive
// variables w = (rho, vn, vt, Bt, p) and sum_k beta_k R_k is accumulated in w
// and mapped to conserved variables once (the map is linear).
//
// FP64 is the scarce unit on this GPU, so the arithmetic avoids the library
// divide and square-root sequences (wb_rcp / wb_rsqrt), and gamma_k = dg/alpha
// is never formed: Q(nu + gamma) alpha = |nu alpha + dg| sign(alpha) when
// |nu alpha + dg| >= 2 eps |alpha|, else (nu alpha + dg)^2 / (4 eps alpha) +
// eps alpha, which is the same quantity with one reciprocal, needed only for
// waves with eps > 0.
#include "wb_device.cuh"
#include "wb_internal.h"

namespace {

constexpr int kBlock = 64;

struct Cell {
  double rho, ir, sr, isr;        // rho, 1/rho, sqrt(rho), 1/sqrt(rho)
  double vn, vt1, vt2;
  double bt1, bt2;
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
  const double e = __ldg(A.q[F_EN] + off);
  const double bn = __ldg(A.q[F_BX + D] + off);
  c.bt1 = __ldg(A.q[F_BX + T1] + off);
  c.bt2 = __ldg(A.q[F_BX + T2] + off);
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
  c.h = P.g_over_gm1 * p + ke + bt2;
  c.F[0] = c.mn;
  c.F[1] = c.mn * c.vn + pstar - bn2;
  c.F[2] = c.mn * c.vt1 - bn * c.bt1;
  c.F[3] = c.mn * c.vt2 - bn * c.bt2;
  c.F[4] = c.bt1 * c.vn - bn * c.vt1;
  c.F[5] = c.bt2 * c.vn - bn * c.vt2;
  c.F[6] = (e + pstar) * c.vn - bn * (bn * c.vn + c.bt1 * c.vt1 + c.bt2 * c.vt2);
}

// Per-face record (shared memory, structure of arrays over the block)
enum {
  R_AL = 0, R_NU = 7, R_RHO = 14, R_SRHO, R_A, R_A2, R_CF, R_CS, R_AF, R_AS, R_B1, R_B2, R_S,
  R_VN, R_VT1, R_VT2, R_BT1, R_BT2, R_X, R_FAVG, R_WORDS = R_FAVG + 7
};

struct Rec {
  double* p;
  __device__ __forceinline__ double& operator[](int w) const { return p[w * kBlock]; }
};

// Q_k(chi) of App. A; the branch test runs on the integer pipe
__device__ __forceinline__ double Qk(double chi, int k, const WbPhys& P) {
  return wb_abs_less(chi, P.two_eps[k]) ? fma(chi * chi, P.inv4eps[k], P.eps[k]) : fabs(chi);
}

__device__ __forceinline__ bool face_system(const Cell& L, const Cell& R, double b, double dtdx,
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
  const double H = wL * ((L.h + b2) * L.ir) + wR * ((R.h + b2) * R.ir);
  const double dbt1 = R.bt1 - L.bt1, dbt2 = R.bt2 - L.bt2;
  const double X = 0.5 * (dbt1 * dbt1 + dbt2 * dbt2) * (iD * iD);
  const double v2 = vn * vn + vt1 * vt1 + vt2 * vt2;
  const double bt2s = bt1 * bt1 + bt2 * bt2;
  const double a2 = P.gm1 * (H - 0.5 * v2 - (b2 + bt2s) * irho) - P.gm2 * X;
  if (!(a2 > 0.0)) return false;
  const double isrho = wb_rsqrt(rho);
  const double srho = rho * isrho;
  const double ca2 = b2 * irho, ct2 = bt2s * irho;
  const double dac = a2 - ca2;
  const double disc = dac * dac + ct2 * (ct2 + 2.0 * (a2 + ca2));
  const double sum = a2 + ca2 + ct2;
  double rsd = 0.0, sd = 0.0;
  if (disc > 0.0) {
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
  if (sd <= 1e-12 * sum) {
    const bool fast = a2 >= ca2;
    af = fast ? 1.0 : 0.0;
    as = fast ? 0.0 : 1.0;
  } else {
    // cf^2 - a^2 and cf^2 - ca^2 without cancellation; at most one of the
    // two needs a quotient
    const double t1 = ca2 + ct2 - a2;
    const double t2 = a2 - ca2 + ct2;
    const bool n1 = t1 < 0.0, n2 = t2 < 0.0;
    double qd = 0.0;
    if (n1 || n2) {
      const double num = n1 ? 2.0 * a2 * ct2 : 2.0 * ca2 * ct2;
      const double den = n1 ? sd - t1 : sd - t2;
      qd = num * wb_rcp(den);
    }
    const double cf2_a2 = n1 ? qd : 0.5 * (t1 + sd);
    const double cf2_ca2 = n2 ? qd : 0.5 * (t2 + sd);
    const double af2 = fmin(fmax(a2 * cf2_ca2 * (icf * icf) * rsd, 0.0), 1.0);
    const double as2 = fmin(fmax(cf2_a2 * rsd, 0.0), 1.0);
    af = (af2 > 0.0) ? af2 * wb_rsqrt(af2) : 0.0;
    as = (as2 > 0.0) ? as2 * wb_rsqrt(as2) : 0.0;
  }
  double b1n, b2n;
  if (bt2s <= 1e-24 * (rho * a2 + b2 + bt2s)) {
    b1n = b2n = 0.70710678118654752440;
  } else {
    const double ib = wb_rsqrt(bt2s);
    b1n = bt1 * ib;
    b2n = bt2 * ib;
  }
  const double S = wb_sgn(b);
  // primitive differences of the 7-variable system
  const double drho = R.rho - L.rho;
  const double dmn = R.mn - L.mn, dmt1 = R.mt1 - L.mt1, dmt2 = R.mt2 - L.mt2;
  const double de = R.eref - L.eref;
  const double dvn = (dmn - vn * drho) * irho;
  const double dvt1 = (dmt1 - vt1 * drho) * irho;
  const double dvt2 = (dmt2 - vt2 * drho) * irho;
  const double dp = P.gm1 * (de - (vn * dmn + vt1 * dmt1 + vt2 * dmt2) + 0.5 * v2 * drho -
                             (bt1 * dbt1 + bt2 * dbt2)) - P.gm2 * X * drho;
  // projections on the transverse field direction beta and its normal
  const double dvb = b1n * dvt1 + b2n * dvt2, dvp = -b2n * dvt1 + b1n * dvt2;
  const double dbb = b1n * dbt1 + b2n * dbt2, dbp = -b2n * dbt1 + b1n * dbt2;
  const double i2a2 = 0.5 * ia * ia;
  const double i2ra = 0.5 * isrho * ia;
  const double dpr = dp * irho * i2a2;  // dp / (2 rho a^2)
  const double afcf = af * cf, ascs = as * cs;
  const double Af = (afcf * dvn - ascs * S * dvb) * i2a2;
  const double Cf = as * dbb * i2ra + af * dpr;
  const double As = (ascs * dvn + afcf * S * dvb) * i2a2;
  const double Cs = -af * dbb * i2ra + as * dpr;
  const double Aa = S * dbp * isrho;
  double al[7];
  al[0] = Cf - Af;
  al[6] = Cf + Af;
  al[2] = Cs - As;
  al[4] = Cs + As;
  al[1] = 0.5 * (dvp + Aa);
  al[5] = 0.5 * (dvp - Aa);
  al[3] = drho - dp * (2.0 * i2a2);
  // eigenvalues a_1..a_7 (Sec. 3)
  const double lam[7] = {vn - cf, vn - ca, vn - cs, vn, vn + cs, vn + ca, vn + cf};
#pragma unroll
  for (int k = 0; k < 7; ++k) {
    const double nu = dtdx * lam[k];
    f[R_AL + k] = al[k];
    f[R_NU + k] = nu;
    gt[k] = (Qk(nu, k, P) - nu * nu) * (0.5 * al[k]);
  }
  f[R_RHO] = rho; f[R_SRHO] = srho; f[R_A] = a; f[R_A2] = a2; f[R_CF] = cf; f[R_CS] = cs;
  f[R_AF] = af; f[R_AS] = as; f[R_B1] = b1n; f[R_B2] = b2n; f[R_S] = S;
  f[R_VN] = vn; f[R_VT1] = vt1; f[R_VT2] = vt2; f[R_BT1] = bt1; f[R_BT2] = bt2; f[R_X] = X;
#pragma unroll
  for (int m = 0; m < 7; ++m) f[R_FAVG + m] = 0.5 * (L.F[m] + R.F[m]);
  return true;
}

// beta_k of App. A without forming gamma_k (see the file comment)
__device__ __forceinline__ double beta_k(double al, double nu, double gi, double gi1, int k,
                                         const WbPhys& P) {
  const double w = fma(nu, al, gi1 - gi);             // (nu + gamma) alpha
  double qa;
  if (al == 0.0) {
    qa = 0.0;                                           // gamma = 0, Q(nu) 0
  } else if (!wb_abs_less(w, P.two_eps[k] * al)) {
    qa = wb_copysign_abs(w, al);                        // |nu + gamma| >= 2 eps
  } else if (wb_abs_less(al, 1e-290)) {
    qa = P.eps[k] * al;                                 // w^2/(4 eps alpha) < eps |alpha|
  } else {
    qa = fma(w * w * P.inv4eps[k], wb_rcp(al), P.eps[k] * al);
  }
  return qa - (gi + gi1);
}

// u-bar = (F_L + F_R)/2 - (dx/(2 dt)) sum_k beta_k R_k  (App. A)
__device__ __forceinline__ void face_flux(const Rec& f, const double gi[7], const double gi1[7],
                                          double dx_2dt, const WbPhys& P, double out[7]) {
  double be[7];
#pragma unroll
  for (int k = 0; k < 7; ++k) be[k] = beta_k(f[R_AL + k], f[R_NU + k], gi[k], gi1[k], k, P);
  const double rho = f[R_RHO], af = f[R_AF], as = f[R_AS], cf = f[R_CF], cs = f[R_CS];
  const double S = f[R_S], b1 = f[R_B1], b2 = f[R_B2];
  // sum_k beta_k r_k in w = (rho, vn, vt, Bt, p)
  const double sf = be[0] + be[6], df = be[6] - be[0];
  const double ss = be[2] + be[4], ds = be[4] - be[2];
  const double tfs = af * sf + as * ss;
  const double wr = rho * tfs + be[3];
  const double afcf = af * cf, ascs = as * cs;
  const double wvn = afcf * df + ascs * ds;
  const double vb = S * (afcf * ds - ascs * df);   // along beta
  const double vp = be[1] + be[5];                 // along beta-perp
  const double ra = f[R_SRHO] * f[R_A];
  const double bb = ra * (as * sf - af * ss);
  const double bp = S * f[R_SRHO] * (be[1] - be[5]);
  const double wp = rho * f[R_A2] * tfs;
  const double wvt1 = b1 * vb - b2 * vp, wvt2 = b2 * vb + b1 * vp;
  const double wbt1 = b1 * bb - b2 * bp, wbt2 = b2 * bb + b1 * bp;
  // to conserved variables
  const double vn = f[R_VN], vt1 = f[R_VT1], vt2 = f[R_VT2];
  const double v2 = vn * vn + vt1 * vt1 + vt2 * vt2;
  const double u1 = vn * wr + rho * wvn;
  const double u2 = vt1 * wr + rho * wvt1;
  const double u3 = vt2 * wr + rho * wvt2;
  const double u6 = wp * P.inv_gm1 + (0.5 * v2 + P.gm2_over_gm1 * f[R_X]) * wr +
                    rho * (vn * wvn + vt1 * wvt1 + vt2 * wvt2) + f[R_BT1] * wbt1 + f[R_BT2] * wbt2;
  out[0] = f[R_FAVG + 0] - dx_2dt * wr;
  out[1] = f[R_FAVG + 1] - dx_2dt * u1;
  out[2] = f[R_FAVG + 2] - dx_2dt * u2;
  out[3] = f[R_FAVG + 3] - dx_2dt * u3;
  out[4] = f[R_FAVG + 4] - dx_2dt * wbt1;
  out[5] = f[R_FAVG + 5] - dx_2dt * wbt2;
  out[6] = f[R_FAVG + 6] - dx_2dt * u6;
}

__device__ __forceinline__ void poison(const Rec& f, double gt[7]) {
  const double nan = __longlong_as_double(0x7ff8000000000000LL);
#pragma unroll
  for (int k = 0; k < 7; ++k) gt[k] = nan;
  for (int w = 0; w < R_WORDS; ++w) f[w] = nan;
}

template <int D>
__global__ void __launch_bounds__(kBlock, 4) k_sweep(SweepArgs A) {
  constexpr int T1 = (D + 1) % 3, T2 = (D + 2) % 3;
  constexpr int U = (D == 0) ? 1 : 0;  // fastest transverse axis of the thread map
  constexpr int W = (D == 2) ? 1 : 2;
  __shared__ double srec[2][R_WORDS][kBlock];
  const WbGeo& g = A.geo;
  const double dt = *A.dt;
  if (!(dt > 0.0)) return;
  const int nu_ = A.box.hi[U] - A.box.lo[U] + 1;
  const int nw_ = A.box.hi[W] - A.box.lo[W] + 1;
  const long long npen = (long long)nu_ * nw_;
  const long long item = blockIdx.x * (long long)kBlock + threadIdx.x;
  if (item >= npen * A.nseg) return;
  const int seg = (int)(item / npen);
  const long long pen = item - seg * npen;
  const long long slot = blockIdx.y;
  // faces of this segment: [fa, fb] within [box.lo[D], box.hi[D]]
  const int fa = A.box.lo[D] + seg * A.seg_len;
  int fb = fa + A.seg_len - 1;
  if (fb > A.box.hi[D]) fb = A.box.hi[D];
  if (fa > fb) return;
  int pos[3];
  pos[U] = A.box.lo[U] + (int)(pen % nu_);
  pos[W] = A.box.lo[W] + (int)(pen / nu_);
  pos[D] = fa - 2;
  const long long st = wb_stride<D>(g);
  const long long off_in = slot * A.slot_in + wb_at(g, pos[0], pos[1], pos[2]);
  const long long off_out = slot * A.slot_out + wb_at(g, pos[0], pos[1], pos[2]);
  const double dtdx = dt * g.idx[D];
  const double dx_2dt = 0.5 * g.dx[D] * wb_rcp(dt);
  const WbPhys& P = A.phys;
  Rec rec[2] = {{&srec[0][0][threadIdx.x]}, {&srec[1][0][threadIdx.x]}};

  Cell cL, cR;
  load_cell<D>(A, off_in, cL);
  double gt_p[7], g_p[7];  // g-tilde of face f-1; g of zone f-2
  int bad = 0;
  int cur = 0;
  // faces f = fa-1 .. fb+1; face f lies between zones f-1 and f
  for (int f = fa - 1; f <= fb + 1; ++f) {
    const int c = f - (fa - 2);  // zone f relative to the first zone
    load_cell<D>(A, off_in + c * st, cR);
    const double b = __ldg(A.bn + off_in + c * st);
    double gt[7];
    if (!face_system(cL, cR, b, dtdx, P, rec[cur], gt)) {
      // unphysical Roe state: counted, and the flux is poisoned with NaN
      ++bad;
      poison(rec[cur], gt);
    }
    if (f >= fa) {
      // g of zone f-1 from g-tilde of faces f (i+1/2) and f-1 (i-1/2)
      double gz[7];
#pragma unroll
      for (int k = 0; k < 7; ++k) gz[k] = wb_sweby(gt[k], gt_p[k], P.sweby, P.minmod);
      if (f >= fa + 1) {
        // flux of face f-1 (zones f-2, f-1): g_{i} = g_p (zone f-2), g_{i+1} = gz
        double out[7];
        face_flux(rec[cur ^ 1], g_p, gz, dx_2dt, P, out);
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
    cur ^= 1;
    cL = cR;
  }
  if (bad) atomicAdd((unsigned long long*)&A.scal->unphysical, (unsigned long long)bad);
}

template <int D>
int blocks_per_sm() {
  static int cached = -1;
  if (cached < 0) {
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_sweep<D>, kBlock, 0) != cudaSuccess || nb < 1)
      nb = 1;
    cached = nb;
  }
  return cached;
}

int sm_count() {
  static int cached = -1;
  if (cached < 0) {
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) n = 1;
    cached = n;
  }
  return cached;
}

// Segments per pencil: balance waves of resident threads against the two
// extra interfaces each segment recomputes.
int choose_segments(long long pencils, int len, int resident) {
  int best = 1;
  double best_cost = 1e300;
  for (int s = 1; s <= 16; ++s) {
    int seg_len = (len + s - 1) / s;
    if (seg_len < 4 && s > 1) break;
    long long items = pencils * s;
    long long waves = (items + resident - 1) / resident;
    double cost = (double)waves * (seg_len + 2);
    if (cost < best_cost * 0.999) { best_cost = cost; best = s; }
  }
  return best;
}

}  // namespace

template <int D>
static void launch_sweep(SweepArgs a, int nslots, cudaStream_t s) {
  constexpr int U = (D == 0) ? 1 : 0;
  constexpr int W = (D == 2) ? 1 : 2;
  long long npen = (long long)(a.box.hi[U] - a.box.lo[U] + 1) * (a.box.hi[W] - a.box.lo[W] + 1);
  int len = a.box.hi[D] - a.box.lo[D] + 1;
  int resident = blocks_per_sm<D>() * sm_count() * kBlock;
  int nseg = a.nseg > 0 ? a.nseg : choose_segments(npen * nslots, len, resident);
  a.nseg = nseg;
  a.seg_len = (len + nseg - 1) / nseg;
  dim3 grid((unsigned)((npen * nseg + kBlock - 1) / kBlock), (unsigned)nslots);
  k_sweep<D><<<grid, kBlock, 0, s>>>(a);
}

void wb_launch_sweep(int dir, const SweepArgs& a, int nslots, cudaStream_t s) {
  if (dir == 0) launch_sweep<0>(a, nslots, s);
  else if (dir == 1) launch_sweep<1>(a, nslots, s);
  else launch_sweep<2>(a, nslots, s);
}

// Self-test of the FP64 reciprocal helpers against the library division and
// reciprocal square root on n inputs spread over [1e-40, 1e40].
namespace {
__global__ void k_math_selftest(int n, unsigned long long seed, unsigned long long* worst) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  double e_rcp = 0.0, e_rsq = 0.0;
  if (i < n) {
    unsigned long long z = seed + 0x9e3779b97f4a7c15ULL * (unsigned long long)(i + 1);
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    z ^= z >> 31;
    double u = (double)(z >> 11) * (1.0 / 9007199254740992.0);
    double x = exp((u - 0.5) * 184.2);
    e_rcp = fabs(wb_rcp(x) * x - 1.0);
    e_rsq = fabs(wb_rsqrt(x) / rsqrt(x) - 1.0);
  }
  atomicMax(&worst[0], (unsigned long long)__double_as_longlong(e_rcp));
  atomicMax(&worst[1], (unsigned long long)__double_as_longlong(e_rsq));
}
}  // namespace

void wb_launch_math_selftest(int n, unsigned long long* worst, cudaStream_t s) {
  k_math_selftest<<<(n + 255) / 256, 256, 0, s>>>(n, 0x1234567ULL, worst);
}
