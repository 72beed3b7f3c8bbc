// Stage kernels of the 3D CTU+CT step (Sec. "MHD in Three Dimensions",
// Steps 2-5 and 7-11) plus the ghost fill, time step and diagnostics.
// Every kernel maps one thread to one zone, face or edge of an index box and
// one patch slot (blockIdx.y); all arrays share the padded patch geometry.
#include "wb_device.cuh"
#include "wb_internal.h"

namespace {

__device__ __forceinline__ bool box_index(const WbBox& b, long long t, int& i, int& j, int& k) {
  const int nx = b.hi[0] - b.lo[0] + 1, ny = b.hi[1] - b.lo[1] + 1, nz = b.hi[2] - b.lo[2] + 1;
  if (t >= (long long)nx * ny * nz) return false;
  i = b.lo[0] + (int)(t % nx);
  long long r = t / nx;
  j = b.lo[1] + (int)(r % ny);
  k = b.lo[2] + (int)(r / ny);
  return true;
}

inline long long box_count(const WbBox& b) {
  return (long long)(b.hi[0] - b.lo[0] + 1) * (b.hi[1] - b.lo[1] + 1) * (b.hi[2] - b.lo[2] + 1);
}

inline dim3 grid_for(long long n, int nslots, int bs) {
  return dim3((unsigned)((n + bs - 1) / bs), (unsigned)nslots);
}

// Step 2: zone-centred reference EMF E = -v x B from q^n.
__global__ void k_eref(StageArgs A, WbBox box) {
  if (!(A.scal->dt > 0.0)) return;
  int i, j, k;
  if (!box_index(box, blockIdx.x * (long long)blockDim.x + threadIdx.x, i, j, k)) return;
  const long long o = blockIdx.y * A.slot_q + wb_at(A.geo, i, j, k);
  const long long w = blockIdx.y * A.slot_w + wb_at(A.geo, i, j, k);
  double ir = 1.0 / A.q[F_RHO][o];
  double vx = A.q[F_MX][o] * ir, vy = A.q[F_MY][o] * ir, vz = A.q[F_MZ][o] * ir;
  double bx = A.q[F_BX][o], by = A.q[F_BY][o], bz = A.q[F_BZ][o];
  A.Eref[0][w] = vz * by - vy * bz;
  A.Eref[1][w] = vx * bz - vz * bx;
  A.Eref[2][w] = vy * bx - vx * by;
}

// Steps 3 and 9: upwinded corner EMF (GS05 "CT-contact" form).  Edge along
// axis C at the low faces of axes a = C+1 and b = C+2 (cyclic).  Face EMFs
// E^a = -F_a[B_b], E^b = +F_b[B_a]; the corner value is their average plus
// one quarter of [(dE/db) at -3/4 minus (dE/db) at -1/4] and the same along
// a, each derivative taken from the zone upwind of the mass flux through the
// face it sits on (the mean of both zones when that flux is zero).
template <int C>
__global__ void k_edge(StageArgs A, bool corr, WbBox box) {
  if (!(A.scal->dt > 0.0)) return;
  constexpr int a = (C + 1) % 3, b = (C + 2) % 3;
  int i, j, k;
  if (!box_index(box, blockIdx.x * (long long)blockDim.x + threadIdx.x, i, j, k)) return;
  const WbGeo& g = A.geo;
  const long long o = blockIdx.y * A.slot_w + wb_at(g, i, j, k);
  const long long sa = a == 0 ? 1 : (a == 1 ? g.sy : g.sz);
  const long long sb = b == 0 ? 1 : (b == 1 ? g.sy : g.sz);
  double* const* Fa = corr ? A.Fc[a] : A.Fp[a];
  double* const* Fb = corr ? A.Fc[b] : A.Fp[b];
  const double* Er = corr ? A.Erefh[C] : A.Eref[C];
  const double Ea_0 = -Fa[F_BX + b][o];
  const double Ea_m = -Fa[F_BX + b][o - sb];
  const double Eb_0 = Fb[F_BX + a][o];
  const double Eb_m = Fb[F_BX + a][o - sa];
  const double ma_0 = Fa[F_RHO][o], ma_m = Fa[F_RHO][o - sb];
  const double mb_0 = Fb[F_RHO][o], mb_m = Fb[F_RHO][o - sa];
  const double R00 = Er[o], Rm0 = Er[o - sa], R0m = Er[o - sb], Rmm = Er[o - sa - sb];
  double db_hi_m = Rm0 - Eb_m, db_hi_0 = R00 - Eb_0;
  double db_hi = ma_0 > 0.0 ? db_hi_m : (ma_0 < 0.0 ? db_hi_0 : 0.5 * (db_hi_m + db_hi_0));
  double db_lo_m = Eb_m - Rmm, db_lo_0 = Eb_0 - R0m;
  double db_lo = ma_m > 0.0 ? db_lo_m : (ma_m < 0.0 ? db_lo_0 : 0.5 * (db_lo_m + db_lo_0));
  double da_hi_m = R0m - Ea_m, da_hi_0 = R00 - Ea_0;
  double da_hi = mb_0 > 0.0 ? da_hi_m : (mb_0 < 0.0 ? da_hi_0 : 0.5 * (da_hi_m + da_hi_0));
  double da_lo_m = Ea_m - Rmm, da_lo_0 = Ea_0 - Rm0;
  double da_lo = mb_m > 0.0 ? da_lo_m : (mb_m < 0.0 ? da_lo_0 : 0.5 * (da_lo_m + da_lo_0));
  double* out = corr ? A.Eedgeh[C] : A.Eedge[C];
  out[o] = 0.25 * (Ea_0 + Ea_m + Eb_0 + Eb_m) + 0.25 * (db_lo - db_hi) + 0.25 * (da_lo - da_hi);
}

// Steps 4 and 11: b_out = b_in - tau curl E on the faces normal to D.
template <int D>
__global__ void k_ct(StageArgs A, bool fin, WbBox box) {
  const double dt = A.scal->dt;
  if (!(dt > 0.0)) return;
  constexpr int a = (D + 1) % 3, b = (D + 2) % 3;
  int i, j, k;
  if (!box_index(box, blockIdx.x * (long long)blockDim.x + threadIdx.x, i, j, k)) return;
  const WbGeo& g = A.geo;
  const long long w = blockIdx.y * A.slot_w + wb_at(g, i, j, k);
  const long long q = blockIdx.y * A.slot_q + wb_at(g, i, j, k);
  const long long sa = a == 0 ? 1 : (a == 1 ? g.sy : g.sz);
  const long long sb = b == 0 ? 1 : (b == 1 ? g.sy : g.sz);
  const double* Eb = fin ? A.Eedgeh[b] : A.Eedge[b];
  const double* Ea = fin ? A.Eedgeh[a] : A.Eedge[a];
  const double tau = fin ? dt : 0.5 * dt;
  double curl = (Eb[w + sa] - Eb[w]) * g.idx[a] - (Ea[w + sb] - Ea[w]) * g.idx[b];
  double bn = A.b[D][q] - tau * curl;
  if (fin) A.b[D][q] = bn;
  else A.bh[D][w] = bn;
}

__device__ __forceinline__ double minmod_src(double x, double y) {
  if (x > 0.0 && y > 0.0) return fmin(x, y);
  if (x < 0.0 && y < 0.0) return fmax(x, y);
  return 0.0;
}

// Steps 5 and 7: q^{n+1/2}_D = q^n - dt/2 (transverse flux divergence)
// + dt/2 S_D, zone B_D := mean of b_D^{n+1/2}, with the GS08-type div B
// source S_D built from face differences of b^n and minmod pairings.
template <int D>
__global__ void k_transverse(StageArgs A, WbBox box) {
  const double dt = A.scal->dt;
  if (!(dt > 0.0)) return;
  constexpr int t1 = (D + 1) % 3, t2 = (D + 2) % 3;
  int i, j, k;
  if (!box_index(box, blockIdx.x * (long long)blockDim.x + threadIdx.x, i, j, k)) return;
  const WbGeo& g = A.geo;
  const long long q = blockIdx.y * A.slot_q + wb_at(g, i, j, k);
  const long long w = blockIdx.y * A.slot_w + wb_at(g, i, j, k);
  const long long s[3] = {1, g.sy, g.sz};
  const double hdt = 0.5 * dt;
  double ir = 1.0 / A.q[F_RHO][q];
  double v[3], B[3], db[3];
#pragma unroll
  for (int e = 0; e < 3; ++e) {
    v[e] = A.q[F_MX + e][q] * ir;
    B[e] = A.q[F_BX + e][q];
    db[e] = (A.b[e][q + s[e]] - A.b[e][q]) * g.idx[e];
  }
  double m2 = minmod_src(db[D], -db[t1]);  // for the t2 field component
  double m1 = minmod_src(db[D], -db[t2]);  // for the t1 field component
  double S[8];
  S[F_RHO] = 0.0;
#pragma unroll
  for (int e = 0; e < 3; ++e) S[F_MX + e] = B[e] * db[D];
  S[F_EN] = B[D] * v[D] * db[D] + B[t1] * v[t1] * m1 + B[t2] * v[t2] * m2;
  S[F_BX + D] = 0.0;
  S[F_BX + t1] = v[t1] * m1;
  S[F_BX + t2] = v[t2] * m2;
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    if (c == F_BX + D) continue;
    // normal-field fluxes of a sweep vanish (F_d[B_d] = 0)
    double d1 = (c == F_BX + t1) ? 0.0 : (A.Fp[t1][c][w + s[t1]] - A.Fp[t1][c][w]) * g.idx[t1];
    double d2 = (c == F_BX + t2) ? 0.0 : (A.Fp[t2][c][w + s[t2]] - A.Fp[t2][c][w]) * g.idx[t2];
    A.qh[D][c][w] = A.q[c][q] - hdt * (d1 + d2) + hdt * S[c];
  }
  A.qh[D][F_BX + D][w] = 0.5 * (A.bh[D][w] + A.bh[D][w + s[D]]);
}

// Step 8: reference EMF at n+1/2 from v of q^n - dt/2 div F* and B = mean of
// b^{n+1/2}.
__global__ void k_eref_half(StageArgs A, WbBox box) {
  const double dt = A.scal->dt;
  if (!(dt > 0.0)) return;
  int i, j, k;
  if (!box_index(box, blockIdx.x * (long long)blockDim.x + threadIdx.x, i, j, k)) return;
  const WbGeo& g = A.geo;
  const long long q = blockIdx.y * A.slot_q + wb_at(g, i, j, k);
  const long long w = blockIdx.y * A.slot_w + wb_at(g, i, j, k);
  const long long s[3] = {1, g.sy, g.sz};
  const double hdt = 0.5 * dt;
  double u[4];
  const int comps[4] = {F_RHO, F_MX, F_MY, F_MZ};
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    double div = 0.0;
#pragma unroll
    for (int e = 0; e < 3; ++e)
      div += (A.Fc[e][comps[c]][w + s[e]] - A.Fc[e][comps[c]][w]) * g.idx[e];
    u[c] = A.q[comps[c]][q] - hdt * div;
  }
  double ir = 1.0 / u[0];
  double vx = u[1] * ir, vy = u[2] * ir, vz = u[3] * ir;
  double B[3];
#pragma unroll
  for (int e = 0; e < 3; ++e) B[e] = 0.5 * (A.bh[e][w] + A.bh[e][w + s[e]]);
  A.Erefh[0][w] = vz * B[1] - vy * B[2];
  A.Erefh[1][w] = vx * B[2] - vz * B[0];
  A.Erefh[2][w] = vy * B[0] - vx * B[1];
}

// CFL signal rate sum_d (|v_d| + c_f,d)/dx_d of one zone (Sec. 3 fast speed).
__device__ __forceinline__ double signal_rate(double rho, double mx, double my, double mz, double e,
                                              double bx, double by, double bz, const WbPhys& P,
                                              const WbGeo& g) {
  double ir = 1.0 / rho;
  double v[3] = {mx * ir, my * ir, mz * ir};
  double B[3] = {bx, by, bz};
  double ke = 0.5 * (mx * v[0] + my * v[1] + mz * v[2]);
  double bb = bx * bx + by * by + bz * bz;
  double p = P.gm1 * (e - ke - 0.5 * bb);
  double a2 = P.gamma * p * ir;
  double w = 0.0;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    double cn2 = B[d] * B[d] * ir;
    double ct2 = (bb - B[d] * B[d]) * ir;
    double dd = a2 - cn2;
    double disc = dd * dd + ct2 * (ct2 + 2.0 * (a2 + cn2));
    double cf = sqrt(0.5 * (a2 + cn2 + ct2 + sqrt(disc)));
    w += (fabs(v[d]) + cf) * g.idx[d];
  }
  return w;
}

__device__ __forceinline__ void block_max_atomic(double w, unsigned long long* dst) {
  // warp-shuffle max, then one atomic per warp (exact, order independent)
  unsigned long long bits = (w >= 0.0) ? (unsigned long long)__double_as_longlong(w)
                                       : (w != w ? 0x7ff8000000000000ULL : 0ULL);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    unsigned long long other = __shfl_xor_sync(0xffffffffu, bits, o);
    bits = other > bits ? other : bits;
  }
  if ((threadIdx.x & 31) == 0 && bits) atomicMax(dst, bits);
}

// Step 10 (+ the zone field of Step 11, floors and the next step's signal
// rate): U^{n+1} = ((U^n - dt/dx dF*) - dt/dy dG*) - dt/dz dH* on interior
// zones, zone B = mean of b^{n+1}.
__global__ void k_final(StageArgs A) {
  const double dt = A.scal->dt;
  if (!(dt > 0.0)) return;
  const WbGeo& g = A.geo;
  WbBox box = {{0, 0, 0}, {g.n[0] - 1, g.n[1] - 1, g.n[2] - 1}};
  int i, j, k;
  bool ok = box_index(box, blockIdx.x * (long long)blockDim.x + threadIdx.x, i, j, k);
  double w = 0.0;
  if (ok) {
    const long long q = blockIdx.y * A.slot_q + wb_at(g, i, j, k);
    const long long wi = blockIdx.y * A.slot_w + wb_at(g, i, j, k);
    const long long s[3] = {1, g.sy, g.sz};
    const WbPhys& P = A.phys;
    double cx = dt * g.idx[0], cy = dt * g.idx[1], cz = dt * g.idx[2];
    double u[5];
#pragma unroll
    for (int c = 0; c < 5; ++c) {
      double x = A.q[c][q];
      x = x - cx * (A.Fc[0][c][wi + 1] - A.Fc[0][c][wi]);
      x = x - cy * (A.Fc[1][c][wi + s[1]] - A.Fc[1][c][wi]);
      x = x - cz * (A.Fc[2][c][wi + s[2]] - A.Fc[2][c][wi]);
      u[c] = x;
    }
    double B[3];
#pragma unroll
    for (int e = 0; e < 3; ++e) {
      B[e] = 0.5 * (A.b[e][q] + A.b[e][q + s[e]]);
      A.q[F_BX + e][q] = B[e];
    }
    long long hits = 0;
    if (u[0] < P.rho_floor) { u[0] = P.rho_floor; ++hits; }
    double ke = 0.5 * (u[1] * u[1] + u[2] * u[2] + u[3] * u[3]) / u[0];
    double me = 0.5 * (B[0] * B[0] + B[1] * B[1] + B[2] * B[2]);
    double p = P.gm1 * (u[4] - ke - me);
    if (p < P.p_floor) { u[4] = P.p_floor * P.inv_gm1 + ke + me; ++hits; }
    bool fin = isfinite(u[0]) && isfinite(u[1]) && isfinite(u[2]) && isfinite(u[3]) &&
               isfinite(u[4]) && u[0] > 0.0 && isfinite(p);
#pragma unroll
    for (int c = 0; c < 5; ++c) A.q[c][q] = u[c];
    if (hits) atomicAdd((unsigned long long*)&A.scal->floor_hits, (unsigned long long)hits);
    if (!fin) atomicAdd((unsigned long long*)&A.scal->unphysical, 1ULL);
    w = signal_rate(u[0], u[1], u[2], u[3], u[4], B[0], B[1], B[2], P, g);
    if (!fin) w = __longlong_as_double(0x7ff8000000000000LL);
  }
  block_max_atomic(w, &A.scal->wmax_next);
}

// Ghost fill of every patch: zone (i,j,k) outside the interior copies the
// zone of the same global position wrapped (periodic) or clamped (outflow)
// into the domain; face arrays use the same rule on their face index.
__global__ void k_halo(StageArgs A, GridMap m) {
  const WbGeo& g = A.geo;
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= g.V) return;
  long long p = blockIdx.y;
  int i = (int)(t % g.pd[0]) - WB_NG;
  long long r = t / g.pd[0];
  int j = (int)(r % g.pd[1]) - WB_NG;
  int k = (int)(r / g.pd[1]) - WB_NG;
  int loc[3] = {i, j, k};
  if (i >= 0 && i < g.n[0] && j >= 0 && j < g.n[1] && k >= 0 && k < g.n[2]) return;
  long long pc[3];
  pc[0] = p % m.np[0];
  pc[1] = (p / m.np[0]) % m.np[1];
  pc[2] = p / ((long long)m.np[0] * m.np[1]);
  long long src_patch = 0;
  int sl[3];
  long long mul = 1;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    long long G = pc[d] * g.n[d] + loc[d];
    if (G < 0 || G >= m.N[d]) {
      if (m.bc[d] == 0) G = ((G % m.N[d]) + m.N[d]) % m.N[d];
      else G = G < 0 ? 0 : m.N[d] - 1;
    }
    long long sp = G / g.n[d];
    sl[d] = (int)(G - sp * g.n[d]);
    src_patch += sp * mul;
    mul *= m.np[d];
  }
  const long long dst = p * g.V + t;
  const long long src = src_patch * g.V + wb_at(g, sl[0], sl[1], sl[2]);
#pragma unroll
  for (int c = 0; c < 8; ++c) A.q[c][dst] = A.q[c][src];
#pragma unroll
  for (int c = 0; c < 3; ++c) A.b[c][dst] = A.b[c][src];
}

__global__ void k_dt_init(StageArgs A, long long npatch) {
  const WbGeo& g = A.geo;
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  long long nint = (long long)g.n[0] * g.n[1] * g.n[2];
  double w = 0.0;
  if (t < nint * npatch) {
    long long p = t / nint, r = t % nint;
    int i = (int)(r % g.n[0]);
    int j = (int)((r / g.n[0]) % g.n[1]);
    int k = (int)(r / ((long long)g.n[0] * g.n[1]));
    long long o = p * g.V + wb_at(g, i, j, k);
    w = signal_rate(A.q[0][o], A.q[1][o], A.q[2][o], A.q[3][o], A.q[4][o], A.q[5][o], A.q[6][o],
                    A.q[7][o], A.phys, g);
    if (!(w >= 0.0)) w = __longlong_as_double(0x7ff8000000000000LL);
  }
  block_max_atomic(w, &A.scal->wmax_next);
}

// dt of the next step from the signal rate of its start state (reading R3)
__global__ void k_dt_step(WbScalars* s, double cfl, double t_end) {
  double w = __longlong_as_double((long long)s->wmax_next);
  double dt = cfl / w;
  bool ok = (w > 0.0) && isfinite(w) && isfinite(dt) && dt > 0.0;
  if (t_end > 0.0) {
    double rem = t_end - s->t;
    if (!(rem > 0.0)) { s->dt = 0.0; return; }  // past t_end: skip, keep the rate
    if (ok && dt > rem) dt = rem;
  }
  if (!ok) {
    s->dt = 0.0;
    s->unphysical += 1;
    return;
  }
  s->dt = dt;
  s->t += dt;
  s->steps += 1;
  s->wmax_next = 0ULL;
}

__global__ void k_ccb(StageArgs A, long long npatch) {
  const WbGeo& g = A.geo;
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  long long nint = (long long)g.n[0] * g.n[1] * g.n[2];
  if (t >= nint * npatch) return;
  long long p = t / nint, r = t % nint;
  int i = (int)(r % g.n[0]);
  int j = (int)((r / g.n[0]) % g.n[1]);
  int k = (int)(r / ((long long)g.n[0] * g.n[1]));
  long long o = p * g.V + wb_at(g, i, j, k);
  const long long s[3] = {1, g.sy, g.sz};
#pragma unroll
  for (int e = 0; e < 3; ++e) A.q[F_BX + e][o] = 0.5 * (A.b[e][o] + A.b[e][o + s[e]]);
}

// primitive (rho, v, P) in fields 0..4 -> conserved, with the zone field (Eq. totenergy)
__global__ void k_prim_to_cons(StageArgs A, long long npatch) {
  const WbGeo& g = A.geo;
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  long long nint = (long long)g.n[0] * g.n[1] * g.n[2];
  if (t >= nint * npatch) return;
  long long p = t / nint, r = t % nint;
  int i = (int)(r % g.n[0]);
  int j = (int)((r / g.n[0]) % g.n[1]);
  int k = (int)(r / ((long long)g.n[0] * g.n[1]));
  long long o = p * g.V + wb_at(g, i, j, k);
  double rho = A.q[0][o], vx = A.q[1][o], vy = A.q[2][o], vz = A.q[3][o], pr = A.q[4][o];
  double bx = A.q[5][o], by = A.q[6][o], bz = A.q[7][o];
  A.q[1][o] = rho * vx;
  A.q[2][o] = rho * vy;
  A.q[3][o] = rho * vz;
  A.q[4][o] = pr * A.phys.inv_gm1 + 0.5 * rho * (vx * vx + vy * vy + vz * vz) +
              0.5 * (bx * bx + by * by + bz * bz);
}

// global array (host layout) <-> patch interiors
template <bool SCATTER>
__global__ void k_move(const double* src, double* dst, int comp, WbGeo g, GridMap m) {
  int ext[3] = {m.N[0], m.N[1], m.N[2]};
  if (comp >= 5) ext[comp - 5] += 1;
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  long long tot = (long long)ext[0] * ext[1] * ext[2];
  if (t >= tot) return;
  int G[3];
  G[0] = (int)(t % ext[0]);
  G[1] = (int)((t / ext[0]) % ext[1]);
  G[2] = (int)(t / ((long long)ext[0] * ext[1]));
  long long patch = 0, mul = 1;
  int loc[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    int pc = G[d] / g.n[d];
    if (pc >= m.np[d]) pc = m.np[d] - 1;  // the high boundary face of the last patch
    loc[d] = G[d] - pc * g.n[d];
    patch += pc * mul;
    mul *= m.np[d];
  }
  long long o = patch * g.V + wb_at(g, loc[0], loc[1], loc[2]);
  if (SCATTER) {
    // faces at the high boundary are ghosts: filled by the halo fill instead
    if (comp >= 5 && loc[comp - 5] >= g.n[comp - 5]) return;
    dst[o] = src[t];
  } else {
    dst[t] = src[o];
  }
}

__global__ void k_divb(StageArgs A, long long npatch, unsigned long long* out) {
  const WbGeo& g = A.geo;
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  long long nint = (long long)g.n[0] * g.n[1] * g.n[2];
  double w = 0.0;
  if (t < nint * npatch) {
    long long p = t / nint, r = t % nint;
    int i = (int)(r % g.n[0]);
    int j = (int)((r / g.n[0]) % g.n[1]);
    int k = (int)(r / ((long long)g.n[0] * g.n[1]));
    long long o = p * g.V + wb_at(g, i, j, k);
    double dv = (A.b[0][o + 1] - A.b[0][o]) * g.idx[0] + (A.b[1][o + g.sy] - A.b[1][o]) * g.idx[1] +
                (A.b[2][o + g.sz] - A.b[2][o]) * g.idx[2];
    w = fabs(dv);
  }
  block_max_atomic(w, out);
}

__global__ void k_copy_box(const double* src, long long slot, WbGeo g, WbBox box, double* dst) {
  int i, j, k;
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (!box_index(box, t, i, j, k)) return;
  dst[t] = src[slot * g.V + wb_at(g, i, j, k)];
}

__global__ void k_fp64_probe(double* out, int iters) {
  double a = 0.9999999, c = 1e-9;
  double x0 = threadIdx.x * 1e-7, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3;
  double x4 = x0 + 4, x5 = x0 + 5, x6 = x0 + 6, x7 = x0 + 7;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < 16; ++u) {
      x0 = fma(x0, a, c); x1 = fma(x1, a, c); x2 = fma(x2, a, c); x3 = fma(x3, a, c);
      x4 = fma(x4, a, c); x5 = fma(x5, a, c); x6 = fma(x6, a, c); x7 = fma(x7, a, c);
    }
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
}

StageArgs mini_args(double* const q[8], double* const b[3], const WbGeo& geo) {
  StageArgs a = {};
  for (int c = 0; c < 8; ++c) a.q[c] = q[c];
  if (b)
    for (int c = 0; c < 3; ++c) a.b[c] = b[c];
  a.geo = geo;
  return a;
}

}  // namespace

void wb_launch_eref(const StageArgs& a, const WbBox& box, cudaStream_t s) {
  k_eref<<<grid_for(box_count(box), a.nslots, 256), 256, 0, s>>>(a, box);
}

void wb_launch_edge(const StageArgs& a, int axis, bool corr, const WbBox& box, cudaStream_t s) {
  dim3 gr = grid_for(box_count(box), a.nslots, 256);
  if (axis == 0) k_edge<0><<<gr, 256, 0, s>>>(a, corr, box);
  else if (axis == 1) k_edge<1><<<gr, 256, 0, s>>>(a, corr, box);
  else k_edge<2><<<gr, 256, 0, s>>>(a, corr, box);
}

void wb_launch_ct(const StageArgs& a, bool fin, const WbBox box[3], cudaStream_t s) {
  k_ct<0><<<grid_for(box_count(box[0]), a.nslots, 256), 256, 0, s>>>(a, fin, box[0]);
  k_ct<1><<<grid_for(box_count(box[1]), a.nslots, 256), 256, 0, s>>>(a, fin, box[1]);
  k_ct<2><<<grid_for(box_count(box[2]), a.nslots, 256), 256, 0, s>>>(a, fin, box[2]);
}

void wb_launch_transverse(const StageArgs& a, int dir, const WbBox& box, cudaStream_t s) {
  dim3 gr = grid_for(box_count(box), a.nslots, 128);
  if (dir == 0) k_transverse<0><<<gr, 128, 0, s>>>(a, box);
  else if (dir == 1) k_transverse<1><<<gr, 128, 0, s>>>(a, box);
  else k_transverse<2><<<gr, 128, 0, s>>>(a, box);
}

void wb_launch_eref_half(const StageArgs& a, const WbBox& box, cudaStream_t s) {
  k_eref_half<<<grid_for(box_count(box), a.nslots, 256), 256, 0, s>>>(a, box);
}

void wb_launch_final(const StageArgs& a, cudaStream_t s) {
  long long n = (long long)a.geo.n[0] * a.geo.n[1] * a.geo.n[2];
  k_final<<<grid_for(n, a.nslots, 256), 256, 0, s>>>(a);
}

void wb_launch_halo(double* const q[8], double* const b[3], const WbGeo& geo, const GridMap& m,
                    cudaStream_t s) {
  StageArgs a = mini_args(q, b, geo);
  k_halo<<<grid_for(geo.V, (int)m.npatch, 256), 256, 0, s>>>(a, m);
}

void wb_launch_dt_init(double* const q[8], const WbGeo& geo, long long npatch, const WbPhys& ph,
                       WbScalars* scal, cudaStream_t s) {
  StageArgs a = mini_args(q, nullptr, geo);
  a.phys = ph;
  a.scal = scal;
  long long n = (long long)geo.n[0] * geo.n[1] * geo.n[2] * npatch;
  k_dt_init<<<grid_for(n, 1, 256), 256, 0, s>>>(a, npatch);
}

void wb_launch_dt_step(WbScalars* scal, double cfl, double t_end, cudaStream_t s) {
  k_dt_step<<<1, 1, 0, s>>>(scal, cfl, t_end);
}

void wb_launch_ccb(double* const q[8], double* const b[3], const WbGeo& geo, long long npatch,
                   cudaStream_t s) {
  StageArgs a = mini_args(q, b, geo);
  long long n = (long long)geo.n[0] * geo.n[1] * geo.n[2] * npatch;
  k_ccb<<<grid_for(n, 1, 256), 256, 0, s>>>(a, npatch);
}

void wb_launch_prim_to_cons(double* const q[8], const WbGeo& geo, long long npatch,
                            const WbPhys& ph, cudaStream_t s) {
  StageArgs a = mini_args(q, nullptr, geo);
  a.phys = ph;
  long long n = (long long)geo.n[0] * geo.n[1] * geo.n[2] * npatch;
  k_prim_to_cons<<<grid_for(n, 1, 256), 256, 0, s>>>(a, npatch);
}

void wb_launch_scatter(const double* src, double* dst_field, int comp, const WbGeo& geo,
                       const GridMap& m, cudaStream_t s) {
  long long ext[3] = {m.N[0], m.N[1], m.N[2]};
  if (comp >= 5) ext[comp - 5] += 1;
  long long n = ext[0] * ext[1] * ext[2];
  k_move<true><<<grid_for(n, 1, 256), 256, 0, s>>>(src, dst_field, comp, geo, m);
}

void wb_launch_gather(const double* src_field, double* dst, int comp, const WbGeo& geo,
                      const GridMap& m, cudaStream_t s) {
  long long ext[3] = {m.N[0], m.N[1], m.N[2]};
  if (comp >= 5) ext[comp - 5] += 1;
  long long n = ext[0] * ext[1] * ext[2];
  k_move<false><<<grid_for(n, 1, 256), 256, 0, s>>>(src_field, dst, comp, geo, m);
}

void wb_launch_divb(double* const b[3], const WbGeo& geo, long long npatch,
                    unsigned long long* out_bits, cudaStream_t s) {
  double* q[8] = {};
  StageArgs a = mini_args(q, b, geo);
  long long n = (long long)geo.n[0] * geo.n[1] * geo.n[2] * npatch;
  k_divb<<<grid_for(n, 1, 256), 256, 0, s>>>(a, npatch, out_bits);
}

void wb_launch_copy_box(const double* src, long long slot, const WbGeo& geo, const WbBox& box,
                        double* dst, cudaStream_t s) {
  k_copy_box<<<grid_for(box_count(box), 1, 256), 256, 0, s>>>(src, slot, geo, box, dst);
}

void wb_launch_fp64_probe(double* out, int blocks, int iters, cudaStream_t s) {
  k_fp64_probe<<<blocks, 256, 0, s>>>(out, iters);
}
