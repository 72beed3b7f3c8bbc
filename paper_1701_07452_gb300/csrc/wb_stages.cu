// Stage kernels of the 3D CTU+CT step (Sec. "MHD in Three Dimensions",
// Steps 2-5 and 7-11) plus the ghost fill, time step and diagnostics.
// Every kernel maps one thread to one zone, face or edge of an index box and
// one patch slot (blockIdx.y); all arrays share the padded patch geometry.
#include "../../include/wombat.h"
#include "wb_device.cuh"
#include "wb_internal.h"
#include <cstring>

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

// Step 2: zone-centred reference EMF from q^n.
__global__ void k_eref(StageArgs A, WbBox box) {
  if (!wb_pos(A.v.scal->dt)) return;
  int i, j, k;
  if (!box_index(box, blockIdx.x * (long long)blockDim.x + threadIdx.x, i, j, k)) return;
  wbu::eref(A.v, blockIdx.y * A.slot_q, blockIdx.y * A.slot_w, i, j, k);
}

inline WbBox box_union(const WbBox b[3]) {
  WbBox u = b[0];
  for (int n = 1; n < 3; ++n)
    for (int d = 0; d < 3; ++d) {
      u.lo[d] = b[n].lo[d] < u.lo[d] ? b[n].lo[d] : u.lo[d];
      u.hi[d] = b[n].hi[d] > u.hi[d] ? b[n].hi[d] : u.hi[d];
    }
  return u;
}

struct Boxes3 {
  WbBox b[3];
  WbBox u;
};

// Steps 3 and 9: the three corner-EMF components, one thread per index of
// the union of their boxes.
__global__ void k_edges(StageArgs A, bool corr, Boxes3 B) {
  if (!wb_pos(A.v.scal->dt)) return;
  int i, j, k;
  if (!box_index(B.u, blockIdx.x * (long long)blockDim.x + threadIdx.x, i, j, k)) return;
  const long long wo = blockIdx.y * A.slot_w;
  if (wbu::in_box(B.b[0], i, j, k)) wbu::edge<0>(A.v, wo, corr, i, j, k);
  if (wbu::in_box(B.b[1], i, j, k)) wbu::edge<1>(A.v, wo, corr, i, j, k);
  if (wbu::in_box(B.b[2], i, j, k)) wbu::edge<2>(A.v, wo, corr, i, j, k);
}

// Steps 4 and 11: constrained transport of the three face components.
__global__ void k_ct(StageArgs A, bool fin, Boxes3 B) {
  const double dt = A.v.scal->dt;
  if (!wb_pos(dt)) return;
  int i, j, k;
  if (!box_index(B.u, blockIdx.x * (long long)blockDim.x + threadIdx.x, i, j, k)) return;
  const long long qo = blockIdx.y * A.slot_q, wo = blockIdx.y * A.slot_w;
  if (wbu::in_box(B.b[0], i, j, k)) wbu::ct<0>(A.v, qo, wo, fin, dt, i, j, k);
  if (wbu::in_box(B.b[1], i, j, k)) wbu::ct<1>(A.v, qo, wo, fin, dt, i, j, k);
  if (wbu::in_box(B.b[2], i, j, k)) wbu::ct<2>(A.v, qo, wo, fin, dt, i, j, k);
}

// Steps 5 and 7: the three transverse-flux preconditioned states, all
// directions of a zone in one thread.
__global__ void k_transverse(StageArgs A, Boxes3 B) {
  const double dt = A.v.scal->dt;
  if (!wb_pos(dt)) return;
  int i, j, k;
  if (!box_index(B.u, blockIdx.x * (long long)blockDim.x + threadIdx.x, i, j, k)) return;
  const int mask = (wbu::in_box(B.b[0], i, j, k) ? 1 : 0) | (wbu::in_box(B.b[1], i, j, k) ? 2 : 0) |
                   (wbu::in_box(B.b[2], i, j, k) ? 4 : 0);
  // zones that need every direction take the mask as a constant: with a run-time
  // mask the compiler recomputes shared zone terms (13 FP64 instructions a zone)
  if (mask == 7) wbu::transverse_set(A.v, blockIdx.y * A.slot_q, blockIdx.y * A.slot_w, dt, 7, i, j, k);
  else if (mask) wbu::transverse_set(A.v, blockIdx.y * A.slot_q, blockIdx.y * A.slot_w, dt, mask, i, j, k);
}

// Step 8: half-step reference EMF.
__global__ void k_eref_half(StageArgs A, WbBox box) {
  const double dt = A.v.scal->dt;
  if (!wb_pos(dt)) return;
  int i, j, k;
  if (!box_index(box, blockIdx.x * (long long)blockDim.x + threadIdx.x, i, j, k)) return;
  wbu::eref_half(A.v, blockIdx.y * A.slot_q, blockIdx.y * A.slot_w, dt, i, j, k);
}

// Periodic images of intermediate arrays of a single-patch box that is
// periodic on every axis: each ghost point within `depth` zones of the
// interior takes the value computed at the interior point it is an image of
// (the same function of the same inputs, so the copy equals a recomputation
// bit for bit).  One thread per shell point.
__global__ void k_wrap(WrapList L, WbGeo g, int depth, long long n) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= n) return;
  long long dst, src;
  wbu::wrap_shell_point(g, depth, t, &dst, &src);
  for (int a = 0; a < L.n; ++a) L.a[a][dst] = L.a[a][src];
}

// The same for a grid of patches periodic on every axis, all patches resident
// (slot = patch): a ghost point of patch blockIdx.y takes the value the
// neighbouring patch (periodic across the domain) holds at that global
// position.
__global__ void k_wrap_patches(WrapList L, WbGeo g, GridMap m, int depth, long long n) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= n) return;
  const long long p = blockIdx.y;
  int loc[3];
  wbu::shell_point(g, depth, t, &loc[0], &loc[1], &loc[2]);
  long long pc[3];
  pc[0] = p % m.np[0];
  pc[1] = (p / m.np[0]) % m.np[1];
  pc[2] = p / ((long long)m.np[0] * m.np[1]);
  long long sp = 0, mul = 1;
  int sl[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    long long G = pc[d] * g.n[d] + loc[d];
    G = ((G % m.N[d]) + m.N[d]) % m.N[d];
    const long long q = G / g.n[d];
    sl[d] = (int)(G - q * g.n[d]);
    sp += q * mul;
    mul *= m.np[d];
  }
  const long long dst = p * g.V + wb_at(g, loc[0], loc[1], loc[2]);
  const long long src = sp * g.V + wb_at(g, sl[0], sl[1], sl[2]);
  for (int a = 0; a < L.n; ++a) L.a[a][dst] = L.a[a][src];
}

__device__ __forceinline__ void block_max_atomic(double w, unsigned long long* dst) {
  // warp-shuffle max, then one atomic per warp (exact, order independent);
  // the bits of w >= 0, 0 for w < 0, the canonical NaN for any NaN (tests on
  // the bit pattern: an FP64 compare takes an FP64-pipe instruction)
  unsigned long long bits = wb_rate_bits(w);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    unsigned long long other = __shfl_xor_sync(0xffffffffu, bits, o);
    bits = other > bits ? other : bits;
  }
  if ((threadIdx.x & 31) == 0 && bits) atomicMax(dst, bits);
}

// Step 10 (+ zone field of Step 11, floors, next signal rate) on interior zones.
__global__ void k_final(StageArgs A) {
  const double dt = A.v.scal->dt;
  if (!wb_pos(dt)) return;
  const WbGeo& g = A.v.geo;
  WbBox box = {{0, 0, 0}, {g.n[0] - 1, g.n[1] - 1, g.n[2] - 1}};
  int i, j, k;
  const bool ok = box_index(box, blockIdx.x * (long long)blockDim.x + threadIdx.x, i, j, k);
  double w = 0.0;
  int hits = 0, bad = 0;
  // axes along which this slot's patch is the last one of an outflow axis
  const long long p = A.p0 + blockIdx.y;
  const long long pc[3] = {p % A.np[0], (p / A.np[0]) % A.np[1], p / ((long long)A.np[0] * A.np[1])};
  int ohi = 0;
#pragma unroll
  for (int d = 0; d < 3; ++d)
    if (((A.ohi_bc >> d) & 1) && pc[d] == A.np[d] - 1) ohi |= 1 << d;
  if (ok) w = wbu::final_update(A.v, blockIdx.y * A.slot_q, blockIdx.y * A.slot_w, dt, A.phys, i, j, k,
                                ohi, &hits, &bad);
  if (hits) atomicAdd((unsigned long long*)&A.v.scal->floor_hits, (unsigned long long)hits);
  if (bad) atomicAdd((unsigned long long*)&A.v.scal->unphysical, (unsigned long long)bad);
  block_max_atomic(w, &A.v.scal->wmax_next);
}

// Ghost fill of every patch: zone (i,j,k) outside the interior copies the
// zone of the same global position wrapped (periodic) or clamped (outflow)
// into the domain; face arrays use the same rule on their face index.
__global__ void k_halo(StageArgs A, GridMap m) {
  const WbGeo& g = A.v.geo;
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= g.V) return;
  long long p = blockIdx.y;
  int i = (int)(t % g.pd[0]) - WB_NG;
  long long r = t / g.pd[0];
  int j = (int)(r % g.pd[1]) - WB_NG;
  int k = g.sz == 0 ? 0 : (int)(r / g.pd[1]) - WB_NG;  // a flat-z box has one plane
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
  for (int c = 0; c < 8; ++c) A.v.q[c][dst] = A.v.q[c][src];
#pragma unroll
  for (int c = 0; c < 3; ++c) A.v.b[c][dst] = A.v.b[c][src];
}

__global__ void k_dt_init(StageArgs A, long long npatch) {
  const WbGeo& g = A.v.geo;
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  long long nint = (long long)g.n[0] * g.n[1] * g.n[2];
  double w = 0.0;
  if (t < nint * npatch) {
    long long p = t / nint, r = t % nint;
    int i = (int)(r % g.n[0]);
    int j = (int)((r / g.n[0]) % g.n[1]);
    int k = (int)(r / ((long long)g.n[0] * g.n[1]));
    long long o = p * g.V + wb_at(g, i, j, k);
    w = wbu::signal_rate(A.v.q[0][o], A.v.q[1][o], A.v.q[2][o], A.v.q[3][o], A.v.q[4][o], A.v.q[5][o], A.v.q[6][o],
                    A.v.q[7][o], A.phys, g, A.v.scal);
    if (!(w >= 0.0)) w = __longlong_as_double(0x7ff8000000000000LL);
  }
  block_max_atomic(w, &A.v.scal->wmax_next);
}

// dt of the next step from the signal rate of its start state (reading R3),
// or with lag from the rate of the previous step's start state (the paper
// delays the dt reduction by one step to overlap it with work; the first two
// steps both use the loaded state's rate)
__global__ void k_dt_step(WbScalars* s, double cfl, double t_end, int lag) {
  const double w_now = __longlong_as_double((long long)s->wmax_next);
  double w = w_now;
  if (lag) {
    const double wl = __longlong_as_double((long long)s->wmax_lag);
    if (wl > 0.0) w = wl;
  }
  double dt = cfl / w;
  bool ok = (w > 0.0) && isfinite(w) && isfinite(dt) && dt > 0.0 && (w_now > 0.0) && isfinite(w_now);
  bool last = false;
  if (t_end > 0.0) {
    double rem = t_end - s->t;
    if (!(rem > 0.0)) { s->dt = 0.0; return; }  // past t_end: skip, keep the rate
    // the step that reaches t_end lands on it exactly and leaves no sliver
    // below 1e-10 of a step (a near-zero dt still carries the eps_k
    // dissipation of Q_k and dx/(2 dt) overflows the flux scale)
    if (ok && dt >= rem * (1.0 - 1e-10)) { dt = rem; last = true; }
  }
  if (!ok) {
    s->dt = 0.0;
    s->unphysical += 1;
    return;
  }
  s->dt = dt;
  s->t = last ? t_end : s->t + dt;
  if (lag) s->wmax_lag = s->wmax_next;
  s->steps += 1;
  s->wmax_next = 0ULL;
  s->rate_screen = 0u;
}

__global__ void k_ccb(StageArgs A, long long npatch) {
  const WbGeo& g = A.v.geo;
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
  for (int e = 0; e < 3; ++e) A.v.q[F_BX + e][o] = 0.5 * (A.v.b[e][o] + A.v.b[e][o + s[e]]);
}

// primitive (rho, v, P) in fields 0..4 -> conserved, with the zone field (Eq. totenergy)
__global__ void k_prim_to_cons(StageArgs A, long long npatch) {
  const WbGeo& g = A.v.geo;
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  long long nint = (long long)g.n[0] * g.n[1] * g.n[2];
  if (t >= nint * npatch) return;
  long long p = t / nint, r = t % nint;
  int i = (int)(r % g.n[0]);
  int j = (int)((r / g.n[0]) % g.n[1]);
  int k = (int)(r / ((long long)g.n[0] * g.n[1]));
  long long o = p * g.V + wb_at(g, i, j, k);
  double rho = A.v.q[0][o], vx = A.v.q[1][o], vy = A.v.q[2][o], vz = A.v.q[3][o], pr = A.v.q[4][o];
  double bx = A.v.q[5][o], by = A.v.q[6][o], bz = A.v.q[7][o];
  A.v.q[1][o] = rho * vx;
  A.v.q[2][o] = rho * vy;
  A.v.q[3][o] = rho * vz;
  A.v.q[4][o] = pr * A.phys.inv_gm1 + 0.5 * rho * (vx * vx + vy * vy + vz * vz) +
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
  const WbGeo& g = A.v.geo;
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  long long nint = (long long)g.n[0] * g.n[1] * g.n[2];
  double w = 0.0;
  if (t < nint * npatch) {
    long long p = t / nint, r = t % nint;
    int i = (int)(r % g.n[0]);
    int j = (int)((r / g.n[0]) % g.n[1]);
    int k = (int)(r / ((long long)g.n[0] * g.n[1]));
    long long o = p * g.V + wb_at(g, i, j, k);
    double dv = (A.v.b[0][o + 1] - A.v.b[0][o]) * g.idx[0] + (A.v.b[1][o + g.sy] - A.v.b[1][o]) * g.idx[1] +
                (A.v.b[2][o + g.sz] - A.v.b[2][o]) * g.idx[2];
    w = fabs(dv);
  }
  block_max_atomic(w, out);
}

// Conserved totals (diagnostic): compensated sums over the interior zones of
// every patch of rho, M, E and of the owned faces of b (the low face of each
// zone).  Each thread keeps a Neumaier pair (sum, compensation) per quantity
// over a strided range of zones; a block combines its pairs in a fixed tree
// and writes one partial per quantity; k_totals_final combines the partials
// in block order.  The grid size is fixed, so the result does not depend on
// timing.
constexpr int kTotBlock = 256;

__device__ __forceinline__ void neumaier_add(double& s, double& c, double x) {
  const double t = s + x;
  const bool big = !wb_abs_less(s, x);  // |s| >= |x|
  const double a = big ? s : x, b = big ? x : s;
  c += (a - t) + b;
  s = t;
}

__global__ void __launch_bounds__(kTotBlock) k_totals(StageArgs A, long long npatch, double* part) {
  __shared__ double ss[8][kTotBlock], sc[8][kTotBlock];
  const WbGeo& g = A.v.geo;
  const long long nint = (long long)g.n[0] * g.n[1] * g.n[2];
  double s[8], c[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) s[q] = c[q] = 0.0;
  const long long stride = (long long)gridDim.x * kTotBlock;
  for (long long t = blockIdx.x * (long long)kTotBlock + threadIdx.x; t < nint * npatch; t += stride) {
    const long long p = t / nint, r = t % nint;
    const int i = (int)(r % g.n[0]);
    const int j = (int)((r / g.n[0]) % g.n[1]);
    const int k = (int)(r / ((long long)g.n[0] * g.n[1]));
    const long long o = p * g.V + wb_at(g, i, j, k);
#pragma unroll
    for (int q = 0; q < 5; ++q) neumaier_add(s[q], c[q], A.v.q[q][o]);
#pragma unroll
    for (int q = 0; q < 3; ++q) neumaier_add(s[5 + q], c[5 + q], A.v.b[q][o]);
  }
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    ss[q][threadIdx.x] = s[q];
    sc[q][threadIdx.x] = c[q];
  }
  __syncthreads();
  for (int h = kTotBlock / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) {
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        double a = ss[q][threadIdx.x], ca = sc[q][threadIdx.x] + sc[q][threadIdx.x + h];
        neumaier_add(a, ca, ss[q][threadIdx.x + h]);
        ss[q][threadIdx.x] = a;
        sc[q][threadIdx.x] = ca;
      }
    }
    __syncthreads();
  }
  if (threadIdx.x < 8) {
    part[(size_t)blockIdx.x * 16 + threadIdx.x] = ss[threadIdx.x][0];
    part[(size_t)blockIdx.x * 16 + 8 + threadIdx.x] = sc[threadIdx.x][0];
  }
}

__global__ void k_totals_final(const double* part, int nblocks, double vol, double* out) {
  const int q = threadIdx.x;
  if (q >= 8) return;
  double s = 0.0, c = 0.0;
  for (int b = 0; b < nblocks; ++b) {
    c += part[(size_t)b * 16 + 8 + q];
    neumaier_add(s, c, part[(size_t)b * 16 + q]);
  }
  out[q] = (s + c) * vol;
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
  StageArgs a;
  memset(&a, 0, sizeof(a));
  for (int c = 0; c < 8; ++c) a.v.q[c] = q[c];
  if (b)
    for (int c = 0; c < 3; ++c) a.v.b[c] = b[c];
  a.v.geo = geo;
  return a;
}

Boxes3 boxes3(const WbBox b[3]) {
  Boxes3 B;
  for (int n = 0; n < 3; ++n) B.b[n] = b[n];
  B.u = box_union(b);
  return B;
}

}  // namespace

void wb_launch_eref(const StageArgs& a, const WbBox& box, cudaStream_t s) {
  k_eref<<<grid_for(box_count(box), a.nslots, 256), 256, 0, s>>>(a, box);
}

void wb_launch_edges(const StageArgs& a, bool corr, const WbBox box[3], cudaStream_t s) {
  Boxes3 B = boxes3(box);
  k_edges<<<grid_for(box_count(B.u), a.nslots, 256), 256, 0, s>>>(a, corr, B);
}

void wb_launch_ct(const StageArgs& a, bool fin, const WbBox box[3], cudaStream_t s) {
  Boxes3 B = boxes3(box);
  k_ct<<<grid_for(box_count(B.u), a.nslots, 256), 256, 0, s>>>(a, fin, B);
}

void wb_launch_transverse(const StageArgs& a, const WbBox box[3], cudaStream_t s) {
  Boxes3 B = boxes3(box);
  k_transverse<<<grid_for(box_count(B.u), a.nslots, 128), 128, 0, s>>>(a, B);
}

void wb_launch_eref_half(const StageArgs& a, const WbBox& box, cudaStream_t s) {
  k_eref_half<<<grid_for(box_count(box), a.nslots, 256), 256, 0, s>>>(a, box);
}

void wb_launch_final(const StageArgs& a, cudaStream_t s) {
  long long n = (long long)a.v.geo.n[0] * a.v.geo.n[1] * a.v.geo.n[2];
  k_final<<<grid_for(n, a.nslots, 256), 256, 0, s>>>(a);
}

void wb_launch_halo(double* const q[8], double* const b[3], const WbGeo& geo, const GridMap& m,
                    cudaStream_t s) {
  StageArgs a = mini_args(q, b, geo);
  k_halo<<<grid_for(geo.V, (int)m.npatch, 256), 256, 0, s>>>(a, m);
}

void wb_launch_wrap(const WrapList& L, const WbGeo& geo, const GridMap& m, int depth, cudaStream_t s) {
  if (L.n <= 0) return;
  const long long n = wbu::shell_count(geo, depth);
  if (m.npatch == 1) k_wrap<<<grid_for(n, 1, 256), 256, 0, s>>>(L, geo, depth, n);
  else k_wrap_patches<<<grid_for(n, (int)m.npatch, 256), 256, 0, s>>>(L, geo, m, depth, n);
}

void wb_launch_dt_init(double* const q[8], const WbGeo& geo, long long npatch, const WbPhys& ph,
                       WbScalars* scal, cudaStream_t s) {
  StageArgs a = mini_args(q, nullptr, geo);
  a.phys = ph;
  a.v.scal = scal;
  long long n = (long long)geo.n[0] * geo.n[1] * geo.n[2] * npatch;
  k_dt_init<<<grid_for(n, 1, 256), 256, 0, s>>>(a, npatch);
}

void wb_launch_dt_step(WbScalars* scal, double cfl, double t_end, int lag, cudaStream_t s) {
  k_dt_step<<<1, 1, 0, s>>>(scal, cfl, t_end, lag);
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

void wb_launch_totals(double* const q[8], double* const b[3], const WbGeo& geo, long long npatch, double vol,
                      double* part, int nblocks, double* out, cudaStream_t s) {
  StageArgs a = mini_args(q, b, geo);
  k_totals<<<nblocks, kTotBlock, 0, s>>>(a, npatch, part);
  k_totals_final<<<1, 32, 0, s>>>(part, nblocks, vol, out);
}

void wb_launch_copy_box(const double* src, long long slot, const WbGeo& geo, const WbBox& box,
                        double* dst, cudaStream_t s) {
  k_copy_box<<<grid_for(box_count(box), 1, 256), 256, 0, s>>>(src, slot, geo, box, dst);
}

void wb_launch_fp64_probe(double* out, int blocks, int iters, cudaStream_t s) {
  k_fp64_probe<<<blocks, 256, 0, s>>>(out, iters);
}

WB_CHECK_ACCESSOR(wb_check_take_stages)

// Self-test of the integer-pipe helpers against their FP64 definitions: for
// each helper, the number of inputs on which the two disagree (counts[h],
// h < WB_BITS_TESTS).  Inputs: a table of special values (signed zeros,
// subnormals, the normal range's ends, infinities, NaN) paired with each
// other, then random bit patterns (every class of double, NaN included) and
// pairs of nearby or opposite values.
namespace {
constexpr int kSpecials = 16;
__device__ double special_value(int k) {
  const double tiny = __longlong_as_double(1LL);                      // smallest subnormal
  const double sub = __longlong_as_double(0x000fffffffffffffLL);      // largest subnormal
  const double v[kSpecials] = {0.0, -0.0, tiny, -tiny, sub, -sub, 2.2250738585072014e-308,
                               -2.2250738585072014e-308, 1.0, -1.0, 1.7976931348623157e308,
                               -1.7976931348623157e308, __longlong_as_double(0x7ff0000000000000LL),
                               __longlong_as_double((long long)0xfff0000000000000ULL),
                               __longlong_as_double(0x7ff8000000000000LL), 4.4501477170144028e-308};
  return v[k];
}
__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
  return z ^ (z >> 31);
}
__device__ __forceinline__ bool same_bits(double a, double b) {
  return __double_as_longlong(a) == __double_as_longlong(b);
}

__global__ void k_bits_selftest(int n, unsigned long long* counts) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double a, b;
  if (i < kSpecials * kSpecials) {
    a = special_value(i / kSpecials);
    b = special_value(i % kSpecials);
  } else {
    const unsigned long long za = mix64(0x9e3779b97f4a7c15ULL * (unsigned long long)i);
    const unsigned long long zb = mix64(za + 0x632be59bd9b4e019ULL);
    a = __longlong_as_double((long long)za);
    switch (i & 3) {
      case 0: b = __longlong_as_double((long long)zb); break;            // independent pattern
      case 1: b = __longlong_as_double((long long)za + 1 - (long long)(zb & 2)); break;  // one ulp away
      case 2: b = -a; break;
      default: b = a; break;
    }
  }
  const bool na = isnan(a), nb = isnan(b);
  unsigned bad = 0;
  // 0 zero test
  if (wb_zero(a) != (a == 0.0)) bad |= 1u << 0;
  // 1 exact doubling
  { const double t = wb_twice(a), r = a + a;
    if (na ? !isnan(t) : !same_bits(t, r)) bad |= 1u << 1; }
  // 2 order of the values (signed zeros and NaN excluded)
  if (!na && !nb && !(a == 0.0 && b == 0.0) && wb_order_less(a, b) != (a < b)) bad |= 1u << 2;
  // 3 signal-rate key
  { const unsigned long long want = na ? 0x7ff8000000000000ULL
                                       : (a > 0.0 ? (unsigned long long)__double_as_longlong(a) : 0ULL);
    if (wb_rate_bits(a) != want) bad |= 1u << 3; }
  // 4 positive and finite, 5 negative, 6 positive normal, 14 finite
  if (wb_pos(a) != (a > 0.0 && isfinite(a))) bad |= 1u << 4;
  if (wb_neg(a) != (a < 0.0)) bad |= 1u << 5;
  if (wb_normal_pos(a) != (a >= 2.2250738585072014e-308 && isfinite(a))) bad |= 1u << 6;
  if (wb_finite(a) != (bool)isfinite(a)) bad |= 1u << 14;
  // 7 magnitude order, 8 minmod (values; NaN excluded)
  if (!na && !nb) {
    if (wb_abs_less(a, b) != (fabs(a) < fabs(b))) bad |= 1u << 7;
    const bool same_sign = (a > 0.0 && b > 0.0) || (a < 0.0 && b < 0.0);
    const double mm = same_sign ? (fabs(a) < fabs(b) ? a : b) : 0.0;
    if (!(wb_minmod(a, b) == mm)) bad |= 1u << 8;
  }
  // 9 halving, exact for |a| >= 2^-1021 and for inf / NaN (documented domain)
  if (na ? !isnan(wb_half(a)) : (fabs(a) >= 4.4501477170144028e-308 && !same_bits(wb_half(a), a * 0.5)))
    bad |= 1u << 9;
  // 10 absolute value, 11 negation (bit patterns; NaN excluded: the FP64
  // abs and neg the references compile to need not keep a NaN's payload)
  if (!na && !same_bits(wb_fabs(a), fabs(a))) bad |= 1u << 10;
  if (!na && !same_bits(wb_flip(a), -a)) bad |= 1u << 11;
  // 12 a <= b for non-negative operands
  { const double x = fabs(a), y = fabs(b);
    if (!isnan(x) && !isnan(y) && wb_le_nonneg(x, y) != (x <= y)) bad |= 1u << 12; }
  // 13 below a finite, non-negative floor
  { const double f = fabs(b);
    if (isfinite(f) && wb_below_floor(a, f) != (a < f)) bad |= 1u << 13; }
  for (int h = 0; h < WB_BITS_TESTS; ++h)
    if (bad & (1u << h)) atomicAdd(&counts[h], 1ULL);
}
}  // namespace

void wb_launch_bits_selftest(int n, unsigned long long* counts, cudaStream_t s) {
  k_bits_selftest<<<(n + 255) / 256, 256, 0, s>>>(n, counts);
}
