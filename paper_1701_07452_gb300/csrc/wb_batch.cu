// Batched advance of many independent boxes of uneven sizes in one persistent
// kernel (the batching pattern built around the paper's Patch update engine,
// Sec. "Update Engine": a work list of patch updates drained by all threads,
// with dynamic -- GUIDED-like -- scheduling, Sec. "Thread Scheduling at Scale").
//
// One launch advances every active box by up to nsteps CTU+CT steps (Sec. "MHD
// in Three Dimensions", Steps 1-11), each box with its own CFL dt.  Inside the
// launch the stages of a step run one after another over all boxes of a
// workspace group; within a stage, thread blocks take chunks of work items
// (pencil segments, zones, faces, edges of some box) from an atomic counter,
// and a grid-wide barrier separates stages.  The barrier waits are bounded:
// a block that waits longer than the budget sets an error word and every
// block returns, so a stalled launch ends with WB_ERR_TIMEOUT instead of a
// hang.  The stage bodies are the same device functions the per-stage kernels
// of a grid use (wb_units.cuh).
//
// The staged form runs the same stages as one ordinary launch each (the
// sweeps in a kernel that holds only the sweep, the zone stages in kernels
// compiled per stage class with their own occupancy), all captured in one
// CUDA graph; the stage arithmetic is explicitly rounded, so both forms (and
// the single-grid path) give the same bits.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "../../include/wombat.h"
#include "wb_device.cuh"
#include "wb_internal.h"

namespace {

// Stages of a step.  BS_W* fill the periodic images of intermediates for
// boxes periodic on every axis, whose other stages then run on the interior
// only (the grid path's enqueue_pass_wrap); they have no work for other boxes.
enum {
  BS_DT = 0, BS_PRED, BS_EREF, BS_W_FP, BS_EDGE_P, BS_W_EE, BS_CT_H, BS_W_BH, BS_TRANS, BS_W_QH,
  BS_CORR, BS_W_FC, BS_EREF_H, BS_W_ERH, BS_EDGE_C, BS_W_EEH, BS_CT_F, BS_FINAL, BS_HALO, BS_COUNT
};

__host__ __device__ inline bool stage_is_wrap(int s) {
  return s == BS_W_FP || s == BS_W_EE || s == BS_W_BH || s == BS_W_QH || s == BS_W_FC ||
         s == BS_W_ERH || s == BS_W_EEH;
}

constexpr int kB = wbu::kBlock;        // threads per block
constexpr int kItemsPerThread = 8;     // items per thread in a chunk of a cheap stage

__host__ __device__ inline WbBox bxx(int l0, int h0, int l1, int h1, int l2, int h2) {
  WbBox b;
  b.lo[0] = l0; b.hi[0] = h0; b.lo[1] = l1; b.hi[1] = h1; b.lo[2] = l2; b.hi[2] = h2;
  return b;
}

__host__ __device__ inline int stage_nsub(int s) {
  return (s == BS_PRED || s == BS_CORR || s == BS_EDGE_P || s == BS_EDGE_C || s == BS_CT_H ||
          s == BS_CT_F) ? 3 : 1;
}

__host__ __device__ inline bool stage_is_sweep(int s) { return s == BS_PRED || s == BS_CORR; }

// Index boxes of every stage (the same regions as the grid path, wb_capi.cu);
// wrap: the box is periodic on every axis (interior-only regions).
__host__ __device__ inline WbBox stage_box(int s, int d, const int* n, bool wrap) {
  const int N0 = n[0], N1 = n[1], N2 = n[2];
  if (wrap && s != BS_CT_F && s != BS_HALO) return bxx(0, N0 - 1, 0, N1 - 1, 0, N2 - 1);
  switch (s) {
    case BS_PRED:
      if (d == 0) return bxx(-3, N0 + 3, -4, N1 + 3, -4, N2 + 3);
      if (d == 1) return bxx(-4, N0 + 3, -3, N1 + 3, -4, N2 + 3);
      return bxx(-4, N0 + 3, -4, N1 + 3, -3, N2 + 3);
    case BS_EREF: return bxx(-4, N0 + 3, -4, N1 + 3, -4, N2 + 3);
    case BS_EDGE_P:
      if (d == 0) return bxx(-1, N0, -3, N1 + 3, -3, N2 + 3);
      if (d == 1) return bxx(-3, N0 + 3, -1, N1, -3, N2 + 3);
      return bxx(-3, N0 + 3, -3, N1 + 3, -1, N2);
    case BS_CT_H:
      if (d == 0) return bxx(-3, N0 + 3, -1, N1, -1, N2);
      if (d == 1) return bxx(-1, N0, -3, N1 + 3, -1, N2);
      return bxx(-1, N0, -1, N1, -3, N2 + 3);
    case BS_TRANS:  // union of the three directions' boxes; trans_mask picks per zone
      return bxx(-3, N0 + 2, -3, N1 + 2, -3, N2 + 2);
    case BS_CORR:
      if (d == 0) return bxx(-1, N0 + 1, -1, N1, -1, N2);
      if (d == 1) return bxx(-1, N0, -1, N1 + 1, -1, N2);
      return bxx(-1, N0, -1, N1, -1, N2 + 1);
    case BS_EREF_H: return bxx(-1, N0, -1, N1, -1, N2);
    case BS_EDGE_C:
      if (d == 0) return bxx(0, N0 - 1, 0, N1, 0, N2);
      if (d == 1) return bxx(0, N0, 0, N1 - 1, 0, N2);
      return bxx(0, N0, 0, N1, 0, N2 - 1);
    case BS_CT_F:
      if (d == 0) return bxx(0, N0, 0, N1 - 1, 0, N2 - 1);
      if (d == 1) return bxx(0, N0 - 1, 0, N1, 0, N2 - 1);
      return bxx(0, N0 - 1, 0, N1 - 1, 0, N2);
    case BS_FINAL: return bxx(0, N0 - 1, 0, N1 - 1, 0, N2 - 1);
    default: return bxx(0, 0, 0, 0, 0, 0);
  }
}

// Directions whose transverse-predictor state (Steps 5, 7) zone (i,j,k)
// needs: bit d when the zone lies in [-3, N_d + 2] along d and [-1, N_e] along
// the other axes e (the grid path's boxes).
__host__ __device__ inline int trans_mask(const int* n, int i, int j, int k) {
  const int x[3] = {i, j, k};
  bool core[3], wide[3];
  for (int a = 0; a < 3; ++a) {
    core[a] = x[a] >= -1 && x[a] <= n[a];
    wide[a] = x[a] >= -3 && x[a] <= n[a] + 2;
  }
  return ((wide[0] && core[1] && core[2]) ? 1 : 0) | ((core[0] && wide[1] && core[2]) ? 2 : 0) |
         ((core[0] && core[1] && wide[2]) ? 4 : 0);
}

__host__ __device__ inline long long box_cnt(const WbBox& b) {
  return (long long)(b.hi[0] - b.lo[0] + 1) * (b.hi[1] - b.lo[1] + 1) * (b.hi[2] - b.lo[2] + 1);
}

// sweep items: pencils x segments.  seg_len is the longest segment wanted;
// a pencil is cut into nseg segments of nearly equal length (*len_out each,
// the last one shorter by less than nseg faces) so that no item is left far
// shorter than the others.
__host__ __device__ inline void sweep_shape(const WbBox& b, int d, int seg_len, long long* npen,
                                            int* nseg, int* len_out = nullptr) {
  const int U = (d == 0) ? 1 : 0, W = (d == 2) ? 1 : 2;
  *npen = (long long)(b.hi[U] - b.lo[U] + 1) * (b.hi[W] - b.lo[W] + 1);
  const int len = b.hi[d] - b.lo[d] + 1;
  *nseg = (len + seg_len - 1) / seg_len;
  if (len_out) *len_out = (len + *nseg - 1) / *nseg;
}

__host__ __device__ inline long long stage_items(int s, int d, const WbGeo& g, bool wrap, int seg_len) {
  if (s == BS_DT) return 1;
  if (stage_is_wrap(s)) return wrap ? wbu::shell_count(g, s == BS_W_QH ? 2 : 1) : 0;
  if (s == BS_HALO) return wbu::shell_count(g, WB_NG);
  WbBox b = stage_box(s, d, g.n, wrap);
  if (stage_is_sweep(s)) {
    long long np;
    int ns;
    sweep_shape(b, d, seg_len, &np, &ns);
    return np * ns;
  }
  return box_cnt(b);
}

__host__ __device__ inline int items_per_chunk(int s) {
  return (stage_is_sweep(s) || s == BS_DT) ? kB : kB * kItemsPerThread;
}

struct BoxInfo {
  WbView v;
  int bc[3];
  int wrap;  // periodic on every axis: interior-only stages + periodic images
};

// Axes whose high boundary face is an outflow copy of the last owned face
// (every box is its own domain): the final update's zone-field rule there.
__device__ __forceinline__ int outflow_mask(const BoxInfo& bi) {
  return (bi.bc[0] == WB_BC_OUTFLOW ? 1 : 0) | (bi.bc[1] == WB_BC_OUTFLOW ? 2 : 0) |
         (bi.bc[2] == WB_BC_OUTFLOW ? 4 : 0);
}

struct BatchParams {
  const BoxInfo* boxes;
  WbScalars* scal;            // per box
  int* steps_left;            // per box
  const int* gbox;            // box ids of each group, concatenated
  const int* gfirst;          // [ngroups + 1]
  const long long* pre;       // chunk prefix sums per (group, stage): entries (box, sub)
  const long long* pre_off;   // [ngroups * BS_COUNT] start of each prefix array in pre
  int ngroups;
  unsigned* sync;             // [0] arrivals, [1] generation, [2] error, [3..4] chunk counters
  unsigned long long* prof;   // per-stage nanoseconds, or null (stage timer off)
  WbPhys phys;
  double cfl;
  int dt_lag;                 // dt from the previous step's start state
  int seg_len;
  long long budget;           // barrier wait budget in SM clock cycles
};

// Grid-wide barrier with a bounded wait.  Returns false when the error word is
// set (timeout here or elsewhere); every block then leaves the kernel.
__device__ bool grid_barrier(const BatchParams& B, unsigned nblocks) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* gen = B.sync + 1;
    volatile unsigned* err = B.sync + 2;
    __threadfence();
    const unsigned g = *gen;
    const unsigned arrived = atomicAdd(B.sync, 1u);
    if (arrived == nblocks - 1) {
      atomicExch(B.sync, 0u);
      __threadfence();
      atomicAdd((unsigned*)gen, 1u);
    } else {
      const long long t0 = clock64();
      while (*gen == g) {
        if (*err) break;
        if (clock64() - t0 > B.budget) {
          atomicExch((unsigned*)err, 1u);
          break;
        }
        __nanosleep(100);
      }
    }
    __threadfence();
    s_ok = (*err == 0);
  }
  __syncthreads();
  return s_ok != 0;
}

// Warp max of signal-rate keys (wb_rate_bits), one atomicMax per warp.
__device__ __forceinline__ void warp_max_key(unsigned long long bits, unsigned long long* dst) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    unsigned long long other = __shfl_xor_sync(0xffffffffu, bits, o);
    bits = other > bits ? other : bits;
  }
  if ((threadIdx.x & 31) == 0 && bits) atomicMax(dst, bits);
}

__device__ __forceinline__ void warp_max_atomic(double w, unsigned long long* dst) {
  warp_max_key(wb_rate_bits(w), dst);
}

template <int D, int EZ, bool PROT>
__device__ __forceinline__ int sweep_item(const BoxInfo& bi, bool corr, const WbBox& b, long long item,
                                          int seg_len, double dt, const WbPhys& P,
                                          const wbu::Rec rec[2]) {
  constexpr int U = (D == 0) ? 1 : 0, W = (D == 2) ? 1 : 2;
  long long npen;
  int nseg, slen;
  sweep_shape(b, D, seg_len, &npen, &nseg, &slen);
  const int seg = (int)(item / npen);
  const long long pen = item - seg * npen;
  const int nu = b.hi[U] - b.lo[U] + 1;
  const int fa = b.lo[D] + seg * slen;
  int fb = fa + slen - 1;
  if (fb > b.hi[D]) fb = b.hi[D];
  const WbView& v = bi.v;
  const double* const* q = corr ? v.qh[D] : v.q;
  const double* bn = corr ? v.bh[D] : v.b[D];
  double* const* F = corr ? v.Fc[D] : v.Fp[D];
  return wbu::sweep_segment<D, false, EZ, PROT>(v.geo, q, bn, F, 0, 0, b.lo[U] + (int)(pen % nu), b.lo[W] + (int)(pen / nu),
                               fa, fb, dt, P, rec);
}

template <int EZ, bool PROT>
__device__ __forceinline__ void unit_item(const BatchParams& B, int s, int d, int box,
                                          const BoxInfo& bi, long long item, double dt,
                                          const wbu::Rec rec[2], unsigned long long* wkey, int* hits, int* bad,
                                          int* hll) {
  const WbView& v = bi.v;
  const int* n = v.geo.n;
  const bool wrap = bi.wrap != 0;
  if (stage_is_sweep(s)) {
    const WbBox b = stage_box(s, d, n, wrap);
    const bool corr = s == BS_CORR;
    if (d == 0) *hll += sweep_item<0, EZ, PROT>(bi, corr, b, item, B.seg_len, dt, B.phys, rec);
    else if (d == 1) *hll += sweep_item<1, EZ, PROT>(bi, corr, b, item, B.seg_len, dt, B.phys, rec);
    else *hll += sweep_item<2, EZ, PROT>(bi, corr, b, item, B.seg_len, dt, B.phys, rec);
    return;
  }
  // the remaining stages (transverse states, half-step EMF, update); the
  // cheap ones go through unit_pair
  const WbBox b = stage_box(s, d, n, wrap);
  const int nx = b.hi[0] - b.lo[0] + 1, ny = b.hi[1] - b.lo[1] + 1;
  const int i = b.lo[0] + (int)(item % nx);
  const long long r = item / nx;
  const int j = b.lo[1] + (int)(r % ny);
  const int k = b.lo[2] + (int)(r / ny);
  switch (s) {
    case BS_TRANS: {
      const int mask = trans_mask(n, i, j, k);
      if (mask == 7) wbu::transverse_set(v, 0, 0, dt, 7, i, j, k);  // constant mask: see k_transverse
      else if (mask) wbu::transverse_set(v, 0, 0, dt, mask, i, j, k);
      break;
    }
    case BS_EREF_H: wbu::eref_half(v, 0, 0, dt, i, j, k); break;
    case BS_FINAL: {
      const double w = wbu::final_update(v, 0, 0, dt, B.phys, i, j, k, outflow_mask(bi), hits, bad);
      // running max of the rate keys: integer compares, and a NaN stays
      const unsigned long long kw = wb_rate_bits(w);
      if (kw > *wkey) *wkey = kw;
      break;
    }
    default: break;
  }
  (void)box;
}

// Stages whose items are cheap and mostly waiting on memory: a thread takes
// two items per pass and loads both before storing either (the grid path's
// per-stage kernels hide that latency with many resident warps instead).
__host__ __device__ inline bool stage_pairs(int s) {
  return s == BS_EREF || s == BS_EDGE_P || s == BS_EDGE_C || s == BS_CT_H || s == BS_CT_F ||
         s == BS_HALO || stage_is_wrap(s);
}

__device__ __forceinline__ void item_ijk(const WbBox& b, long long item, int* i, int* j, int* k) {
  const int nx = b.hi[0] - b.lo[0] + 1, ny = b.hi[1] - b.lo[1] + 1;
  *i = b.lo[0] + (int)(item % nx);
  const long long r = item / nx;
  *j = b.lo[1] + (int)(r % ny);
  *k = b.lo[2] + (int)(r / ny);
}

// Copy of one array for two shell points: both loads issue before either
// store.
__device__ __forceinline__ void copy2(double* a, long long d0, long long s0, long long d1, long long s1,
                                      bool two) {
  const double x0 = a[s0];
  const double x1 = two ? a[s1] : 0.0;
  a[d0] = x0;
  if (two) a[d1] = x1;
}

// The arrays of a copy stage (state for the ghost fill, intermediates for
// the periodic-image stages), moved for two shell points at a time.
__device__ __forceinline__ void copy_stage(const WbView& v, int s, long long d0, long long s0, long long d1,
                                           long long s1, bool two) {
  switch (s) {
    case BS_HALO:
#pragma unroll
      for (int c = 0; c < 8; ++c) copy2(v.q[c], d0, s0, d1, s1, two);
#pragma unroll
      for (int c = 0; c < 3; ++c) copy2(v.b[c], d0, s0, d1, s1, two);
      return;
    case BS_W_FP:
    case BS_W_FC: {
      double* const(*F)[8] = s == BS_W_FP ? v.Fp : v.Fc;
#pragma unroll
      for (int e = 0; e < 3; ++e)
#pragma unroll
        for (int c = 0; c < 8; ++c)
          if (c != F_BX + e) copy2(F[e][c], d0, s0, d1, s1, two);
      if (s == BS_W_FP) {
#pragma unroll
        for (int e = 0; e < 3; ++e) copy2(v.Eref[e], d0, s0, d1, s1, two);
      }
      return;
    }
    case BS_W_QH:
#pragma unroll
      for (int e = 0; e < 3; ++e)
#pragma unroll
        for (int c = 0; c < 8; ++c) copy2(v.qh[e][c], d0, s0, d1, s1, two);
      return;
    default: {
      double* const* a3 = s == BS_W_EE ? v.Eedge : (s == BS_W_BH ? v.bh : (s == BS_W_ERH ? v.Erefh : v.Eedgeh));
#pragma unroll
      for (int e = 0; e < 3; ++e) copy2(a3[e], d0, s0, d1, s1, two);
    }
  }
}

// Items it0 and it1 (it1 < 0: none) of a copy stage (ghost fill, periodic
// images) for one box.
__device__ __forceinline__ void unit_pair_copy(int s, const BoxInfo& bi, long long it0, long long it1) {
  const WbView& v = bi.v;
  const bool two = it1 >= 0;
  long long d0, s0, d1 = 0, s1 = 0;
  if (s == BS_HALO) {
    wbu::halo_self_offsets(v.geo, bi.bc, it0, &d0, &s0);
    if (two) wbu::halo_self_offsets(v.geo, bi.bc, it1, &d1, &s1);
  } else {
    const int depth = s == BS_W_QH ? 2 : 1;
    wbu::wrap_shell_point(v.geo, depth, it0, &d0, &s0);
    if (two) wbu::wrap_shell_point(v.geo, depth, it1, &d1, &s1);
  }
  copy_stage(v, s, d0, s0, d1, s1, two);
}

// Items it0 and it1 (it1 < 0: none) of the reference EMF, corner EMF or CT
// stages for one box.
__device__ __forceinline__ void unit_pair_emf(int s, int d, const BoxInfo& bi, long long it0, long long it1,
                                              double dt) {
  const WbView& v = bi.v;
  const bool two = it1 >= 0;
  const WbBox b = stage_box(s, d, v.geo.n, bi.wrap != 0);
  int i0, j0, k0, i1 = 0, j1 = 0, k1 = 0;
  item_ijk(b, it0, &i0, &j0, &k0);
  if (two) item_ijk(b, it1, &i1, &j1, &k1);
  switch (s) {
    case BS_EREF: {
      wbu::ErefIn a0, a1;
      wbu::eref_load(v, 0, 0, i0, j0, k0, a0);
      if (two) wbu::eref_load(v, 0, 0, i1, j1, k1, a1);
      wbu::eref_finish(v, a0);
      if (two) wbu::eref_finish(v, a1);
      return;
    }
    case BS_EDGE_P:
    case BS_EDGE_C: {
      const bool corr = s == BS_EDGE_C;
      wbu::EdgeIn a0, a1;
#define WB_EDGE_PAIR(C)                                             \
  wbu::edge_load<C>(v, 0, corr, i0, j0, k0, a0);                    \
  if (two) wbu::edge_load<C>(v, 0, corr, i1, j1, k1, a1);           \
  wbu::edge_finish<C>(v, corr, a0);                                 \
  if (two) wbu::edge_finish<C>(v, corr, a1);
      if (d == 0) { WB_EDGE_PAIR(0) } else if (d == 1) { WB_EDGE_PAIR(1) } else { WB_EDGE_PAIR(2) }
#undef WB_EDGE_PAIR
      return;
    }
    default: {  // BS_CT_H, BS_CT_F
      const bool fin = s == BS_CT_F;
      wbu::CtIn a0, a1;
#define WB_CT_PAIR(D)                                               \
  wbu::ct_load<D>(v, 0, 0, fin, i0, j0, k0, a0);                    \
  if (two) wbu::ct_load<D>(v, 0, 0, fin, i1, j1, k1, a1);           \
  wbu::ct_finish<D>(v, fin, dt, a0);                                \
  if (two) wbu::ct_finish<D>(v, fin, dt, a1);
      if (d == 0) { WB_CT_PAIR(0) } else if (d == 1) { WB_CT_PAIR(1) } else { WB_CT_PAIR(2) }
#undef WB_CT_PAIR
      return;
    }
  }
}

// One item of the reference EMF, corner EMF or CT stages (staged form: the
// latency is hidden by resident warps rather than by pairs of items).
__device__ __forceinline__ void unit_emf(int s, int d, const BoxInfo& bi, long long it, double dt) {
  const WbView& v = bi.v;
  const WbBox b = stage_box(s, d, v.geo.n, bi.wrap != 0);
  int i, j, k;
  item_ijk(b, it, &i, &j, &k);
  if (s == BS_EREF) {
    wbu::eref(v, 0, 0, i, j, k);
  } else if (s == BS_EDGE_P || s == BS_EDGE_C) {
    const bool corr = s == BS_EDGE_C;
    if (d == 0) wbu::edge<0>(v, 0, corr, i, j, k);
    else if (d == 1) wbu::edge<1>(v, 0, corr, i, j, k);
    else wbu::edge<2>(v, 0, corr, i, j, k);
  } else {
    const bool fin = s == BS_CT_F;
    if (d == 0) wbu::ct<0>(v, 0, 0, fin, dt, i, j, k);
    else if (d == 1) wbu::ct<1>(v, 0, 0, fin, dt, i, j, k);
    else wbu::ct<2>(v, 0, 0, fin, dt, i, j, k);
  }
}

// Items it0 and it1 (it1 < 0: none) of a pairing stage for one box.
__device__ __forceinline__ void unit_pair(int s, int d, const BoxInfo& bi, long long it0, long long it1,
                                          double dt) {
  if (s == BS_HALO || stage_is_wrap(s)) unit_pair_copy(s, bi, it0, it1);
  else unit_pair_emf(s, d, bi, it0, it1, dt);
}

// dt of one box for the coming step: C_cfl / max zone signal rate, the rate
// sum_d (|v_d| + c_f,d) / dx_d (reading R3)
__device__ void box_dt(const BatchParams& B, int box) {
  WbScalars* s = B.scal + box;
  if (B.steps_left[box] <= 0) { s->dt = 0.0; return; }
  const double w_now = __longlong_as_double((long long)s->wmax_next);
  double w = w_now;
  if (B.dt_lag) {
    const double wl = __longlong_as_double((long long)s->wmax_lag);
    if (wl > 0.0) w = wl;
  }
  const double dt = B.cfl / w;
  if (!((w > 0.0) && isfinite(w) && isfinite(dt) && dt > 0.0 && w_now > 0.0 && isfinite(w_now))) {
    s->dt = 0.0;
    s->unphysical += 1;
    B.steps_left[box] = 0;
    return;
  }
  s->dt = dt;
  s->t += dt;
  s->steps += 1;
  if (B.dt_lag) s->wmax_lag = s->wmax_next;
  s->wmax_next = 0ULL;
  s->rate_screen = 0u;
  B.steps_left[box] -= 1;
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// EZ: compile-time mask of waves with eps_k = 0 (their Q-branch arithmetic is
// dropped); PROT: the protection-floor test is compiled in.  The launch picks
// the variant from the physics, as the grid path's sweep launches do.
// Launch seq of a sequence uses chunk counter seq & 1 (and done counter
// 5 + (seq & 1) when timing); its block 0 clears the other pair, which the
// launch before it (complete by stream order) used.
__device__ __forceinline__ unsigned* stage_counter(const BatchParams& B, unsigned seq) {
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    atomicExch(B.sync + 3 + ((seq + 1) & 1u), 0u);
    atomicExch(B.sync + 5 + ((seq + 1) & 1u), 0u);
  }
  return B.sync + 3 + (seq & 1u);
}

// Stage timer of the staged form: the last block to finish a launch adds the
// time since the previous launch's end to the stage (the dt launch only sets
// the mark, so time between advances is not counted).
__device__ __forceinline__ void stage_stamp(const BatchParams& B, int s, unsigned seq) {
  if (!B.prof) return;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned done = atomicAdd(B.sync + 5 + (seq & 1u), 1u);
    if (done == gridDim.x - 1) {
      const unsigned long long t = global_ns();
      unsigned long long* mark = B.prof + BS_COUNT;
      if (s != BS_DT && *mark) B.prof[s] += t - *mark;
      *mark = t;
    }
  }
}

template <int EZ, bool PROT>
__global__ void __launch_bounds__(wbu::kBlock, 4) k_batch(BatchParams B, int nsteps) {
  __shared__ double srec[2][wbu::R_WORDS][wbu::kBlock];
  __shared__ long long s_chunk;
  const wbu::Rec rec[2] = {{&srec[0][0][threadIdx.x]}, {&srec[1][0][threadIdx.x]}};
  const unsigned nblocks = gridDim.x;
  unsigned stage_seq = 0;
  // stage timer: block 0 stamps the end of every stage (after its barrier)
  const bool timer = B.prof != nullptr && blockIdx.x == 0 && threadIdx.x == 0;
  unsigned long long t_prev = timer ? global_ns() : 0ULL;
  for (int step = 0; step < nsteps; ++step) {
    for (int grp = 0; grp < B.ngroups; ++grp) {
      const int gb0 = B.gfirst[grp];
      const int nbox = B.gfirst[grp + 1] - gb0;
      for (int s = 0; s < BS_COUNT; ++s, ++stage_seq) {
        unsigned* ctr = B.sync + 3 + (stage_seq & 1u);
        // the other counter is idle during this stage: block 0 clears it
        if (blockIdx.x == 0 && threadIdx.x == 0) atomicExch(B.sync + 3 + ((stage_seq + 1) & 1u), 0u);
        const long long* pre = B.pre + B.pre_off[grp * BS_COUNT + s];
        const int nsub = stage_nsub(s);
        const int nent = nbox * nsub;
        const long long nchunks = pre[nent];
        const int ipc = items_per_chunk(s);
        for (;;) {
          if (threadIdx.x == 0) s_chunk = (long long)atomicAdd(ctr, 1u);
          __syncthreads();
          const long long c = s_chunk;
          __syncthreads();
          if (c >= nchunks) break;
          // (box, sub) entry holding chunk c
          int lo = 0, hi = nent - 1;
          while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (pre[mid] <= c) lo = mid; else hi = mid - 1;
          }
          const int box = B.gbox[gb0 + lo / nsub];
          const int sub = lo % nsub;
          if (s == BS_DT) {
            if (threadIdx.x == 0) box_dt(B, box);
            continue;
          }
          const double dt = *(volatile const double*)&B.scal[box].dt;
          if (!wb_pos(dt)) continue;
          const BoxInfo& bi = B.boxes[box];
          const long long nitems = stage_items(s, sub, bi.v.geo, bi.wrap != 0, B.seg_len);
          const long long i0 = (c - pre[lo]) * ipc;
          long long i1 = i0 + ipc;
          if (i1 > nitems) i1 = nitems;
          unsigned long long wkey = 0ULL;
          int hits = 0, bad = 0, hll = 0;
          if (stage_pairs(s)) {
            for (long long it = i0 + threadIdx.x; it < i1; it += 2 * kB)
              unit_pair(s, sub, bi, it, it + kB < i1 ? it + kB : -1, dt);
          } else {
            for (long long it = i0 + threadIdx.x; it < i1; it += kB)
              unit_item<EZ, PROT>(B, s, sub, box, bi, it, dt, rec, &wkey, &hits, &bad, &hll);
          }
          if (s == BS_FINAL) warp_max_key(wkey, &B.scal[box].wmax_next);
          if (hits) atomicAdd((unsigned long long*)&B.scal[box].floor_hits, (unsigned long long)hits);
          if (bad) atomicAdd((unsigned long long*)&B.scal[box].unphysical, (unsigned long long)bad);
          if (hll) atomicAdd((unsigned long long*)&B.scal[box].hll_faces, (unsigned long long)hll);
        }
        if (!grid_barrier(B, nblocks)) return;
        if (timer) {
          const unsigned long long t = global_ns();
          B.prof[s] += t - t_prev;
          t_prev = t;
        }
      }
    }
  }
}

// ------------------------------------------------------------ staged form
// The same stages as separate launches, one per stage and workspace group: a
// kernel boundary takes the place of each grid barrier, and blocks drain the
// same chunk lists from the stage's counter.  The sweeps run in a kernel that
// holds only the sweep; the zone stages run in kernels compiled per stage
// class, with as many resident warps as their own registers allow (inside the
// persistent kernel every stage keeps the sweep's 4 blocks of 64 threads per
// SM).  All stage arithmetic is written with explicit rounding, so both forms
// compute the same bits.
enum { SC_SWEEP = 0, SC_COPY, SC_EMF, SC_TRANS, SC_EREF_H, SC_FINAL, SC_DT, SC_COUNT };

__host__ __device__ inline int stage_class(int s) {
  if (stage_is_sweep(s)) return SC_SWEEP;
  if (s == BS_HALO || stage_is_wrap(s)) return SC_COPY;  // copies of up to 24 arrays
  if (stage_pairs(s)) return SC_EMF;                    // reference EMF, corner EMFs, CT (one item a thread)
  if (s == BS_TRANS) return SC_TRANS;
  if (s == BS_EREF_H) return SC_EREF_H;
  if (s == BS_FINAL) return SC_FINAL;
  return SC_DT;
}

constexpr int kNtZone = 256;  // threads per block of the zone-stage kernels

// resident blocks per SM each zone-stage kernel is compiled for (its register
// budget: 64 registers a thread at 4 blocks of 256 threads)
__host__ __device__ constexpr int zone_min_blocks(int cls) {
  return cls == SC_TRANS ? 2 : ((cls == SC_EREF_H || cls == SC_FINAL) ? 3 : 4);
}

// Chunks of stage s for the boxes of group grp, claimed by whole blocks:
// body(box, sub, chunk index within the (box, sub) entry).
template <class Body>
__device__ __forceinline__ void drain_stage(const BatchParams& B, int grp, int s, unsigned* ctr,
                                            Body&& body) {
  __shared__ long long s_chunk;
  const int gb0 = B.gfirst[grp];
  const int nbox = B.gfirst[grp + 1] - gb0;
  const long long* pre = B.pre + B.pre_off[grp * BS_COUNT + s];
  const int nsub = stage_nsub(s);
  const int nent = nbox * nsub;
  const long long nchunks = pre[nent];
  for (;;) {
    if (threadIdx.x == 0) s_chunk = (long long)atomicAdd(ctr, 1u);
    __syncthreads();
    const long long c = s_chunk;
    __syncthreads();
    if (c >= nchunks) break;
    int lo = 0, hi = nent - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (pre[mid] <= c) lo = mid; else hi = mid - 1;
    }
    body(B.gbox[gb0 + lo / nsub], lo % nsub, c - pre[lo]);
  }
}

// The sweep stages of the staged form: the same chunks and per-item code as
// the persistent kernel's sweep stage, in a kernel that holds nothing else
// (the flux arithmetic is explicitly rounded, so the bits do not depend on
// which kernel runs it).
template <int EZ, bool PROT>
__global__ void __launch_bounds__(kB, 4) k_bstage_sweep(BatchParams B, int grp, int s, unsigned seq) {
  __shared__ double srec[2][wbu::R_WORDS][kB];
  const wbu::Rec rec[2] = {{&srec[0][0][threadIdx.x]}, {&srec[1][0][threadIdx.x]}};
  unsigned* ctr = stage_counter(B, seq);
  const bool corr = s == BS_CORR;
  drain_stage(B, grp, s, ctr, [&](int box, int d, long long cc) {
    const double dt = B.scal[box].dt;
    if (!wb_pos(dt)) return;
    const BoxInfo& bi = B.boxes[box];
    const long long nitems = stage_items(s, d, bi.v.geo, bi.wrap != 0, B.seg_len);
    const long long it = cc * kB + threadIdx.x;
    if (it >= nitems) return;
    const WbBox b = stage_box(s, d, bi.v.geo.n, bi.wrap != 0);
    int hll;
    if (d == 0) hll = sweep_item<0, EZ, PROT>(bi, corr, b, it, B.seg_len, dt, B.phys, rec);
    else if (d == 1) hll = sweep_item<1, EZ, PROT>(bi, corr, b, it, B.seg_len, dt, B.phys, rec);
    else hll = sweep_item<2, EZ, PROT>(bi, corr, b, it, B.seg_len, dt, B.phys, rec);
    if (hll) atomicAdd((unsigned long long*)&B.scal[box].hll_faces, (unsigned long long)hll);
  });
  stage_stamp(B, s, seq);
}

template <int CLS>
__global__ void __launch_bounds__(kNtZone, zone_min_blocks(CLS))
    k_bstage_zone(BatchParams B, int grp, int s, unsigned seq) {
  constexpr int NT = kNtZone;
  unsigned* ctr = stage_counter(B, seq);
  const int ipc = items_per_chunk(s);
  drain_stage(B, grp, s, ctr, [&](int box, int d, long long cc) {
    if (CLS == SC_DT) {
      if (threadIdx.x == 0) box_dt(B, box);
      return;
    }
    const double dt = B.scal[box].dt;
    if (!wb_pos(dt)) return;
    const BoxInfo& bi = B.boxes[box];
    const long long nitems = stage_items(s, d, bi.v.geo, bi.wrap != 0, B.seg_len);
    const long long i0 = cc * ipc;
    const long long i1 = i0 + ipc < nitems ? i0 + ipc : nitems;
    if (CLS == SC_COPY) {
      for (long long it = i0 + threadIdx.x; it < i1; it += 2 * NT)
        unit_pair_copy(s, bi, it, it + NT < i1 ? it + NT : -1);
      return;
    }
    if (CLS == SC_EMF) {
      for (long long it = i0 + threadIdx.x; it < i1; it += NT) unit_emf(s, d, bi, it, dt);
      return;
    }
    const WbView& v = bi.v;
    const WbBox b = stage_box(s, d, v.geo.n, bi.wrap != 0);
    unsigned long long wkey = 0ULL;
    int hits = 0, bad = 0;
    for (long long it = i0 + threadIdx.x; it < i1; it += NT) {
      int i, j, k;
      item_ijk(b, it, &i, &j, &k);
      if (CLS == SC_TRANS) {
        const int mask = trans_mask(v.geo.n, i, j, k);
        if (mask == 7) wbu::transverse_set(v, 0, 0, dt, 7, i, j, k);  // constant mask: see k_transverse
        else if (mask) wbu::transverse_set(v, 0, 0, dt, mask, i, j, k);
      } else if (CLS == SC_EREF_H) {
        wbu::eref_half(v, 0, 0, dt, i, j, k);
      } else {
        const double w = wbu::final_update(v, 0, 0, dt, B.phys, i, j, k, outflow_mask(bi), &hits, &bad);
        const unsigned long long kw = wb_rate_bits(w);
        if (kw > wkey) wkey = kw;
      }
    }
    if (CLS == SC_FINAL) {
      warp_max_key(wkey, &B.scal[box].wmax_next);
      if (hits) atomicAdd((unsigned long long*)&B.scal[box].floor_hits, (unsigned long long)hits);
      if (bad) atomicAdd((unsigned long long*)&B.scal[box].unphysical, (unsigned long long)bad);
    }
  });
  stage_stamp(B, s, seq);
}

// initial signal rate of one box (the view is passed by value: the device box
// table is only uploaded before the next launch of k_batch)
__global__ void k_box_rate(WbView v, WbScalars* scal, WbPhys P) {
  const WbGeo& g = v.geo;
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long nint = (long long)g.n[0] * g.n[1] * g.n[2];
  double w = 0.0;
  if (t < nint) {
    const int i = (int)(t % g.n[0]);
    const int j = (int)((t / g.n[0]) % g.n[1]);
    const int k = (int)(t / ((long long)g.n[0] * g.n[1]));
    const long long o = wb_at(g, i, j, k);
    w = wbu::signal_rate(v.q[0][o], v.q[1][o], v.q[2][o], v.q[3][o], v.q[4][o], v.q[5][o], v.q[6][o],
                         v.q[7][o], P, g, scal);
  }
  warp_max_atomic(w, &scal->wmax_next);
}

const int kWorkB = 3 * 7 + 3 + 3 + 3 + 3 * 8;  // 54: corrector fluxes, half-step EMFs alias

struct TuneKey {
  std::vector<int> sizes;
  bool operator<(const TuneKey& o) const { return sizes < o.sizes; }
};
std::mutex g_tune_mu;
struct TuneVal {
  int seg_len, blocks_per_sm, form;
};
std::map<TuneKey, TuneVal> g_tune_cache;

}  // namespace

// A batch is a pool: a state region shared by the resident boxes (first-fit
// allocation on the host side), a workspace region shared by workspace groups
// of the resident boxes, and device tables sized for max_boxes slots.
struct wb_batch {
  int cap;
  std::vector<char> alive;
  // steps granted by the last wb_batch_set_steps per box (host mirror), and
  // whether the box sits in the current workspace groups: only boxes with
  // steps granted are grouped, so a pool whose policy runs a few of its
  // resident runs per launch does not pay for the others' stage work lists
  std::vector<int> granted;
  std::vector<char> grouped;
  std::vector<wb_desc> d;
  std::vector<WbGeo> geo;
  std::vector<BoxInfo> info;
  std::vector<size_t> state_off;              // doubles from the state base
  std::map<size_t, size_t> free_;             // free state blocks: offset -> length (doubles)
  size_t state_cap, work_cap, staging_elems;  // doubles
  int max_n;
  wb_desc phys_desc;
  WbPhys phys;
  double cfl;
  int dt_lag = 0;
  cudaStream_t stream;
  char* mem;
  size_t bytes;
  double* state_base;
  double* work_base;
  std::vector<int> gbox, gfirst;
  bool dirty;
  // device tables
  BoxInfo* d_info;
  WbScalars* d_scal;
  int* d_steps;
  int* d_gbox;
  int* d_gfirst;
  long long* d_pre;
  long long* d_pre_off;
  unsigned* d_sync;
  unsigned long long* d_prof;  // per-stage nanoseconds (stage timer)
  bool prof = false;
  double* staging;
  size_t pre_cap;
  // launch configuration
  int form = WB_BATCH_PERSISTENT;
  int zone_blocks[SC_COUNT];  // resident blocks per SM of each zone-stage kernel (staged form)
  int sweep_blocks = 1;       // resident blocks per SM of the staged form's sweep kernel
  int seg_len;
  int blocks_per_sm;
  int max_blocks_per_sm;
  int sms;
  long long budget;
  // graph
  cudaGraphExec_t graph;
  int graph_steps;
  bool graph_ok;
  std::string err;
  int nbox;  // slots in use (highest alive slot + 1)
};

namespace {

int bfail(wb_batch* b, int code, const std::string& m) {
  if (b) b->err = m;
  return code;
}

int bcuda(wb_batch* b, cudaError_t e, const char* where) {
  if (e == cudaSuccess) return WB_OK;
  return bfail(b, WB_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

size_t al(size_t x) { return (x + 255) / 256 * 256; }

WbGeo geo_of(const wb_desc& d) {
  WbGeo g;
  for (int a = 0; a < 3; ++a) {
    g.n[a] = d.n[a];
    g.pd[a] = g.n[a] + 2 * WB_NG;
    g.dx[a] = d.length[a] / d.n[a];
    g.idx[a] = 1.0 / g.dx[a];
  }
  g.sy = g.pd[0];
  g.sz = (long long)g.pd[0] * g.pd[1];
  g.V = g.sz * g.pd[2];
  return g;
}

bool same_physics(const wb_desc& a, const wb_desc& b) {
  if (a.gamma != b.gamma || a.cfl != b.cfl || a.sweby_beta != b.sweby_beta ||
      a.rho_floor != b.rho_floor || a.p_floor != b.p_floor)
    return false;
  for (int k = 0; k < 7; ++k)
    if (a.eps[k] != b.eps[k]) return false;
  return true;
}

bool box_ok(const wb_desc& d) {
  for (int a = 0; a < 3; ++a)
    if (d.n[a] < 1 || d.patches[a] != 1 || !(d.length[a] > 0.0) ||
        (d.bc[a] != WB_BC_PERIODIC && d.bc[a] != WB_BC_OUTFLOW))
      return false;
  return true;
}

// state doubles of a box (rounded to 256 bytes so every field stays aligned)
size_t state_doubles(const WbGeo& g) { return al((size_t)g.V * 11 * sizeof(double)) / sizeof(double); }
size_t work_doubles(const WbGeo& g) { return al((size_t)g.V * kWorkB * sizeof(double)) / sizeof(double); }

struct PoolSizes {
  size_t state, work, tables, staging, total, pre_cap;
};

PoolSizes pool_sizes(size_t state_bytes, size_t work_bytes, int cap, int max_n) {
  PoolSizes P;
  P.state = al(state_bytes);
  P.work = al(work_bytes);
  P.pre_cap = (size_t)BS_COUNT * (4 * (size_t)cap + 2) + 16;
  P.tables = al(sizeof(BoxInfo) * cap) + al(sizeof(WbScalars) * cap) + al(sizeof(int) * cap) +
             al(sizeof(int) * cap) + al(sizeof(int) * (cap + 1)) + al(sizeof(long long) * P.pre_cap) +
             al(sizeof(long long) * (size_t)cap * BS_COUNT) + al(sizeof(unsigned) * 8) +
             al(sizeof(unsigned long long) * (BS_COUNT + 1));
  P.staging = al(sizeof(double) * (size_t)(max_n + 1) * (max_n + 1) * (max_n + 1));
  P.total = P.state + P.work + P.tables + P.staging;
  return P;
}

// chunk prefix tables for the current groups and seg_len
void build_prefix(const wb_batch* b, std::vector<long long>& pre, std::vector<long long>& off) {
  const int ngroups = (int)b->gfirst.size() - 1;
  pre.clear();
  off.assign((size_t)ngroups * BS_COUNT, 0);
  for (int gi = 0; gi < ngroups; ++gi)
    for (int s = 0; s < BS_COUNT; ++s) {
      off[gi * BS_COUNT + s] = (long long)pre.size();
      const int nsub = stage_nsub(s);
      long long acc = 0;
      for (int e = b->gfirst[gi]; e < b->gfirst[gi + 1]; ++e) {
        const int box = b->gbox[e];
        for (int sub = 0; sub < nsub; ++sub) {
          pre.push_back(acc);
          const long long items = stage_items(s, sub, b->geo[box], b->info[box].wrap != 0, b->seg_len);
          acc += (items + items_per_chunk(s) - 1) / items_per_chunk(s);
        }
      }
      pre.push_back(acc);
    }
}

// Whether box i belongs in the workspace groups: a resident box with steps
// granted; when no box has steps granted, every resident box (a batch before
// its first wb_batch_set_steps is grouped as a whole).
bool any_granted(const wb_batch* b) {
  for (int j = 0; j < b->cap; ++j)
    if (b->alive[j] && b->granted[j] > 0) return true;
  return false;
}

bool wants_group(const wb_batch* b, int i, bool any) {
  return b->alive[i] && (!any || b->granted[i] > 0);
}

// Regroup the resident boxes (in slot order) into workspace groups, point
// their workspace views into the shared region and upload every table.
int rebuild(wb_batch* b) {
  b->gbox.clear();
  b->gfirst.assign(1, 0);
  size_t cur = 0;
  double* work = b->work_base;
  b->nbox = 0;
  // boxes in decreasing size: within a stage the work list then starts with
  // the longest items (the big boxes' pencil segments) and ends with the
  // shortest, so the blocks that finish last leave little idle time
  std::vector<int> order;
  std::vector<char> want(b->cap);
  const bool any = any_granted(b);
  for (int i = 0; i < b->cap; ++i) want[i] = wants_group(b, i, any);
  for (int i = 0; i < b->cap; ++i) {
    b->grouped[i] = want[i];
    if (b->alive[i]) b->nbox = i + 1;
    if (b->grouped[i]) order.push_back(i);
  }
  std::stable_sort(order.begin(), order.end(), [b](int x, int y) { return b->geo[x].V > b->geo[y].V; });
  for (int i : order) {
    const WbGeo& g = b->geo[i];
    const size_t w = work_doubles(g);
    if (cur > 0 && cur + w > b->work_cap) {
      b->gfirst.push_back((int)b->gbox.size());
      cur = 0;
    }
    BoxInfo& bi = b->info[i];
    double* base = work + cur;
    size_t k = 0;
    for (int dd = 0; dd < 3; ++dd)
      for (int c = 0; c < 8; ++c) {
        double* f = (c == F_BX + dd) ? nullptr : base + (size_t)g.V * k++;
        bi.v.Fp[dd][c] = f;
        bi.v.Fc[dd][c] = f;  // corrector fluxes reuse the predictor flux arrays
      }
    for (int dd = 0; dd < 3; ++dd) { bi.v.Eref[dd] = base + (size_t)g.V * k; bi.v.Erefh[dd] = bi.v.Eref[dd]; ++k; }
    for (int dd = 0; dd < 3; ++dd) { bi.v.Eedge[dd] = base + (size_t)g.V * k; bi.v.Eedgeh[dd] = bi.v.Eedge[dd]; ++k; }
    for (int dd = 0; dd < 3; ++dd) bi.v.bh[dd] = base + (size_t)g.V * k++;
    for (int dd = 0; dd < 3; ++dd)
      for (int c = 0; c < 8; ++c) bi.v.qh[dd][c] = base + (size_t)g.V * k++;
    cur += w;
    b->gbox.push_back(i);
  }
  if (b->gbox.empty()) b->gfirst.clear();
  b->gfirst.push_back((int)b->gbox.size());
  if (b->gfirst.size() >= 2 && b->gfirst[b->gfirst.size() - 2] == b->gfirst.back() && b->gbox.size() > 0)
    b->gfirst.pop_back();
  if (b->gbox.empty()) b->gfirst.assign(1, 0);
  std::vector<long long> pre, off;
  build_prefix(b, pre, off);
  if (pre.size() > b->pre_cap) return bfail(b, WB_ERR_INVALID, "prefix table overflow");
  cudaStream_t s = b->stream;
  cudaError_t e = cudaMemcpyAsync(b->d_info, b->info.data(), sizeof(BoxInfo) * b->cap, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && !b->gbox.empty())
    e = cudaMemcpyAsync(b->d_gbox, b->gbox.data(), sizeof(int) * b->gbox.size(), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->d_gfirst, b->gfirst.data(), sizeof(int) * b->gfirst.size(), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && !pre.empty())
    e = cudaMemcpyAsync(b->d_pre, pre.data(), sizeof(long long) * pre.size(), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && !off.empty())
    e = cudaMemcpyAsync(b->d_pre_off, off.data(), sizeof(long long) * off.size(), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return bcuda(b, e, "batch tables");
  b->dirty = false;
  return WB_OK;
}

int ensure_built(wb_batch* b) {
  if (!b->dirty) return WB_OK;
  if (b->graph) cudaGraphExecDestroy(b->graph);
  b->graph = nullptr;
  b->graph_steps = 0;
  return rebuild(b);
}

BatchParams params(const wb_batch* b) {
  BatchParams p;
  p.boxes = b->d_info;
  p.scal = b->d_scal;
  p.steps_left = b->d_steps;
  p.gbox = b->d_gbox;
  p.gfirst = b->d_gfirst;
  p.pre = b->d_pre;
  p.pre_off = b->d_pre_off;
  p.ngroups = (int)b->gfirst.size() - 1;
  p.sync = b->d_sync;
  p.prof = b->prof ? b->d_prof : nullptr;
  p.phys = b->phys;
  p.cfl = b->cfl;
  p.dt_lag = b->dt_lag;
  p.seg_len = b->seg_len;
  p.budget = b->budget;
  return p;
}

// The k_batch variant for the physics: the default eps_k (zero on the Alfven
// and entropy waves) without protection floors takes the specialised sweep;
// anything else the general one (protection tested at run time).
const void* batch_kernel(const WbPhys& ph) {
  const bool ez = (ph.eps_zero & wbu::kEpsZeroLD) == wbu::kEpsZeroLD;
  if (ez && !ph.prot) return (const void*)k_batch<wbu::kEpsZeroLD, false>;
  return (const void*)k_batch<0, true>;
}

const void* bstage_sweep_kernel(const WbPhys& ph) {
  const bool ez = (ph.eps_zero & wbu::kEpsZeroLD) == wbu::kEpsZeroLD;
  if (ez && !ph.prot) return (const void*)k_bstage_sweep<wbu::kEpsZeroLD, false>;
  return (const void*)k_bstage_sweep<0, true>;
}

const void* bstage_zone_kernel(int cls) {
  switch (cls) {
    case SC_COPY: return (const void*)k_bstage_zone<SC_COPY>;
    case SC_EMF: return (const void*)k_bstage_zone<SC_EMF>;
    case SC_TRANS: return (const void*)k_bstage_zone<SC_TRANS>;
    case SC_EREF_H: return (const void*)k_bstage_zone<SC_EREF_H>;
    case SC_FINAL: return (const void*)k_bstage_zone<SC_FINAL>;
    default: return (const void*)k_bstage_zone<SC_DT>;
  }
}

// enqueue the staged form of nsteps steps: one launch per (step, group,
// stage), no synchronisation
cudaError_t enqueue_staged(wb_batch* b, int nsteps) {
  cudaError_t e = cudaMemsetAsync(b->d_sync, 0, sizeof(unsigned) * 8, b->stream);
  if (e != cudaSuccess) return e;
  BatchParams p = params(b);
  unsigned seq = 0;
  for (int step = 0; step < nsteps; ++step)
    for (int grp = 0; grp < p.ngroups; ++grp)
      for (int s = 0; s < BS_COUNT; ++s, ++seq) {
        const int cls = stage_class(s);
        const void* fn;
        unsigned nt, nblocks;
        if (cls == SC_SWEEP) {
          fn = bstage_sweep_kernel(b->phys);
          nt = kB;
          nblocks = (unsigned)(std::min(b->blocks_per_sm, b->sweep_blocks) * b->sms);
        } else {
          fn = bstage_zone_kernel(cls);
          nt = kNtZone;
          nblocks = (unsigned)((cls == SC_DT ? 1 : b->zone_blocks[cls]) * b->sms);
        }
        void* args[] = {&p, &grp, &s, &seq};
        e = cudaLaunchKernel(fn, dim3(nblocks), dim3(nt), args, 0, b->stream);
        if (e != cudaSuccess) return e;
      }
  return cudaSuccess;
}

// enqueue nsteps steps in the batch's form (no synchronisation); the
// persistent form is one cooperative launch
cudaError_t enqueue_advance(wb_batch* b, int nsteps) {
  if (b->form == WB_BATCH_STAGED) return enqueue_staged(b, nsteps);
  cudaError_t e = cudaMemsetAsync(b->d_sync, 0, sizeof(unsigned) * 8, b->stream);
  if (e != cudaSuccess) return e;
  BatchParams p = params(b);
  if (p.ngroups <= 0) return cudaSuccess;
  int nblocks = b->blocks_per_sm * b->sms;
  void* args[] = {&p, &nsteps};
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(nblocks);
  cfg.blockDim = dim3(kB);
  cfg.stream = b->stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelExC(&cfg, batch_kernel(b->phys), args);
}

int read_sync_error(wb_batch* b) {
  unsigned err = 0;
  cudaError_t e = cudaMemcpyAsync(&err, b->d_sync + 2, sizeof(unsigned), cudaMemcpyDeviceToHost, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return bcuda(b, e, "batch sync");
  if (err) return bfail(b, WB_ERR_TIMEOUT, "a grid barrier wait ran out of its budget");
  return WB_OK;
}

void drop_graph(wb_batch* b) {
  if (b->graph) cudaGraphExecDestroy(b->graph);
  b->graph = nullptr;
  b->graph_steps = 0;
}


bool phys_ok(const wb_desc& d) {
  if (!(d.gamma > 1.0) || d.gamma > 2.0 || !(d.cfl > 0.0)) return false;
  for (int k = 0; k < 7; ++k)
    if (!(d.eps[k] >= 0.0) || !(d.eps[k] < 0.5)) return false;
  if (!(d.prot_rho >= 0.0) || !(d.prot_p >= 0.0)) return false;
  if (!(d.rho_floor >= 0.0) || !(d.p_floor >= 0.0) || !std::isfinite(d.rho_floor) || !std::isfinite(d.p_floor))
    return false;
  return d.sweby_beta >= 1.0 && d.sweby_beta <= 2.0;
}

void apply_tune_cache(wb_batch* b) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  TuneKey key;
  for (int i = 0; i < b->cap; ++i)
    if (b->alive[i]) key.sizes.push_back(b->d[i].n[0] * 1000000 + b->d[i].n[1] * 1000 + b->d[i].n[2]);
  std::sort(key.sizes.begin(), key.sizes.end());
  auto it = g_tune_cache.find(key);
  if (it != g_tune_cache.end()) {
    b->seg_len = it->second.seg_len;
    b->blocks_per_sm = std::min(it->second.blocks_per_sm, b->max_blocks_per_sm);
    b->form = it->second.form;
  }
}

}  // namespace

extern "C" {

int wb_pool_bytes(size_t state_bytes, size_t work_bytes, int max_boxes, int max_n, size_t* bytes) {
  if (!bytes || max_boxes < 1 || max_n < 1 || state_bytes == 0 || work_bytes == 0) return WB_ERR_INVALID;
  *bytes = pool_sizes(state_bytes, work_bytes, max_boxes, max_n).total;
  return WB_OK;
}

int wb_pool_create(const wb_desc* physics, size_t state_bytes, size_t work_bytes, int max_boxes,
                   int max_n, void* dev_mem, size_t bytes, void* stream, wb_batch** out) {
  if (!out || !physics) return WB_ERR_INVALID;
  *out = nullptr;
  size_t need = 0;
  int rc = wb_pool_bytes(state_bytes, work_bytes, max_boxes, max_n, &need);
  if (rc) return rc;
  if (!phys_ok(*physics)) return WB_ERR_INVALID;
  if (!dev_mem || (reinterpret_cast<uintptr_t>(dev_mem) & 255u)) return WB_ERR_INVALID;
  if (bytes < need) return WB_ERR_NOMEM;
  wb_batch* b = new (std::nothrow) wb_batch();
  if (!b) return WB_ERR_NOMEM;
  PoolSizes P = pool_sizes(state_bytes, work_bytes, max_boxes, max_n);
  b->cap = max_boxes;
  b->alive.assign(max_boxes, 0);
  b->granted.assign(max_boxes, 0);
  b->grouped.assign(max_boxes, 0);
  b->d.resize(max_boxes);
  b->geo.resize(max_boxes);
  b->info.resize(max_boxes);
  std::memset(b->info.data(), 0, sizeof(BoxInfo) * max_boxes);
  b->state_off.assign(max_boxes, 0);
  b->state_cap = P.state / sizeof(double);
  b->work_cap = P.work / sizeof(double);
  b->free_[0] = b->state_cap;
  b->max_n = max_n;
  b->phys_desc = *physics;
  b->phys = wb_phys_of(physics);
  b->cfl = physics->cfl;
  b->dt_lag = physics->dt_lag ? 1 : 0;
  b->stream = reinterpret_cast<cudaStream_t>(stream);
  b->mem = reinterpret_cast<char*>(dev_mem);
  b->bytes = bytes;
  b->state_base = reinterpret_cast<double*>(b->mem);
  b->work_base = reinterpret_cast<double*>(b->mem + P.state);
  char* t = b->mem + P.state + P.work;
  b->d_info = reinterpret_cast<BoxInfo*>(t); t += al(sizeof(BoxInfo) * max_boxes);
  b->d_scal = reinterpret_cast<WbScalars*>(t); t += al(sizeof(WbScalars) * max_boxes);
  b->d_steps = reinterpret_cast<int*>(t); t += al(sizeof(int) * max_boxes);
  b->d_gbox = reinterpret_cast<int*>(t); t += al(sizeof(int) * max_boxes);
  b->d_gfirst = reinterpret_cast<int*>(t); t += al(sizeof(int) * (max_boxes + 1));
  b->pre_cap = P.pre_cap;
  b->d_pre = reinterpret_cast<long long*>(t); t += al(sizeof(long long) * P.pre_cap);
  b->d_pre_off = reinterpret_cast<long long*>(t); t += al(sizeof(long long) * (size_t)max_boxes * BS_COUNT);
  b->d_sync = reinterpret_cast<unsigned*>(t); t += al(sizeof(unsigned) * 8);
  b->d_prof = reinterpret_cast<unsigned long long*>(t); t += al(sizeof(unsigned long long) * (BS_COUNT + 1));
  b->staging = reinterpret_cast<double*>(b->mem + P.state + P.work + P.tables);
  b->staging_elems = P.staging / sizeof(double);
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev);
  int nb = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, batch_kernel(b->phys), kB, 0);
  b->max_blocks_per_sm = nb > 0 ? nb : 1;
  b->blocks_per_sm = b->max_blocks_per_sm;
  nb = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, bstage_sweep_kernel(b->phys), kB, 0);
  b->sweep_blocks = nb > 0 ? nb : 1;
  for (int c = 0; c < SC_COUNT; ++c) {
    nb = 0;
    if (c != SC_SWEEP) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, bstage_zone_kernel(c), kNtZone, 0);
    b->zone_blocks[c] = nb > 0 ? nb : 1;
  }
  b->seg_len = 32;
  int clk_khz = 0;
  cudaDeviceGetAttribute(&clk_khz, cudaDevAttrClockRate, dev);
  b->budget = (long long)(clk_khz > 0 ? clk_khz : 2000000) * 1000LL * 20;  // 20 s of cycles
  b->graph = nullptr;
  b->graph_steps = 0;
  b->graph_ok = true;
  b->dirty = true;
  b->nbox = 0;
  cudaStream_t s = b->stream;
  cudaError_t e = cudaMemsetAsync(b->mem, 0xff, P.state + P.work, s);  // NaN poison
  if (e == cudaSuccess) e = cudaMemsetAsync(b->d_scal, 0, sizeof(WbScalars) * max_boxes, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->d_steps, 0, sizeof(int) * max_boxes, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    delete b;
    return WB_ERR_CUDA;
  }
  *out = b;
  return WB_OK;
}

int wb_pool_admit(wb_batch* b, const wb_desc* d, int* box) {
  if (!b || !d || !box) return bfail(b, WB_ERR_INVALID, "null argument");
  *box = -1;
  if (!box_ok(*d)) return bfail(b, WB_ERR_INVALID, "a batch box needs patches = 1 and valid sizes");
  if (!same_physics(*d, b->phys_desc)) return bfail(b, WB_ERR_INVALID, "physics differ from the pool's");
  if (d->n[0] > b->max_n || d->n[1] > b->max_n || d->n[2] > b->max_n)
    return bfail(b, WB_ERR_INVALID, "box larger than the pool's max_n");
  const WbGeo g = geo_of(*d);
  if (work_doubles(g) > b->work_cap) return bfail(b, WB_ERR_NOMEM, "box workspace exceeds the pool workspace");
  int slot = -1;
  for (int i = 0; i < b->cap; ++i)
    if (!b->alive[i]) { slot = i; break; }
  if (slot < 0) return bfail(b, WB_ERR_NOMEM, "no free box slot");
  const size_t need = state_doubles(g);
  auto it = b->free_.begin();
  for (; it != b->free_.end(); ++it)
    if (it->second >= need) break;
  if (it == b->free_.end()) return bfail(b, WB_ERR_NOMEM, "state region full");
  const size_t off = it->first, len = it->second;
  b->free_.erase(it);
  if (len > need) b->free_[off + need] = len - need;
  b->alive[slot] = 1;
  b->granted[slot] = 0;
  b->d[slot] = *d;
  b->geo[slot] = g;
  b->state_off[slot] = off;
  BoxInfo& bi = b->info[slot];
  std::memset(&bi, 0, sizeof(bi));
  bi.v.geo = g;
  for (int a = 0; a < 3; ++a) bi.bc[a] = d->bc[a];
  bi.wrap = d->bc[0] == WB_BC_PERIODIC && d->bc[1] == WB_BC_PERIODIC && d->bc[2] == WB_BC_PERIODIC;
  double* st = b->state_base + off;
  for (int c = 0; c < 8; ++c) bi.v.q[c] = st + (size_t)c * g.V;
  for (int c = 0; c < 3; ++c) bi.v.b[c] = st + (size_t)(8 + c) * g.V;
  bi.v.scal = b->d_scal + slot;
  b->dirty = true;
  cudaError_t e = cudaMemsetAsync(b->d_scal + slot, 0, sizeof(WbScalars), b->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->d_steps + slot, 0, sizeof(int), b->stream);
  if (e != cudaSuccess) return bcuda(b, e, "admit");
  *box = slot;
  return WB_OK;
}

int wb_pool_release(wb_batch* b, int box) {
  if (!b || box < 0 || box >= b->cap || !b->alive[box]) return bfail(b, WB_ERR_INVALID, "bad box");
  size_t off = b->state_off[box], len = state_doubles(b->geo[box]);
  // coalesce with neighbours
  auto next = b->free_.lower_bound(off);
  if (next != b->free_.end() && off + len == next->first) {
    len += next->second;
    next = b->free_.erase(next);
  }
  if (next != b->free_.begin()) {
    auto prev = std::prev(next);
    if (prev->first + prev->second == off) {
      off = prev->first;
      len += prev->second;
      b->free_.erase(prev);
    }
  }
  b->free_[off] = len;
  b->alive[box] = 0;
  b->granted[box] = 0;
  b->dirty = true;
  cudaError_t e = cudaMemsetAsync(b->d_steps + box, 0, sizeof(int), b->stream);
  return bcuda(b, e, "release");
}

int wb_pool_free_bytes(wb_batch* b, size_t* largest, size_t* total) {
  if (!b) return WB_ERR_INVALID;
  size_t lg = 0, tot = 0;
  for (auto& kv : b->free_) {
    lg = std::max(lg, kv.second);
    tot += kv.second;
  }
  if (largest) *largest = lg * sizeof(double);
  if (total) *total = tot * sizeof(double);
  return WB_OK;
}

int wb_batch_steps_left(wb_batch* b, int* out) {
  if (!b || !out) return bfail(b, WB_ERR_INVALID, "null argument");
  cudaError_t e = cudaMemcpyAsync(out, b->d_steps, sizeof(int) * b->cap, cudaMemcpyDeviceToHost, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  return bcuda(b, e, "steps left");
}

int wb_batch_bytes(int nbox, const wb_desc* descs, size_t work_budget, size_t* bytes) {
  if (nbox < 1 || !descs || !bytes) return WB_ERR_INVALID;
  size_t st = 0, wmax = 0, wsum = 0;
  int maxn = 1;
  for (int i = 0; i < nbox; ++i) {
    if (!box_ok(descs[i]) || !same_physics(descs[i], descs[0])) return WB_ERR_INVALID;
    WbGeo g = geo_of(descs[i]);
    st += state_doubles(g);
    wmax = std::max(wmax, work_doubles(g));
    wsum += work_doubles(g);
    for (int a = 0; a < 3; ++a) maxn = std::max(maxn, descs[i].n[a]);
  }
  size_t budget = work_budget > 0 ? work_budget : ((size_t)64 << 30);
  size_t work = std::max(wmax * sizeof(double), std::min(budget, wsum * sizeof(double)));
  *bytes = pool_sizes(st * sizeof(double), work, nbox, maxn).total;
  return WB_OK;
}

int wb_batch_create(int nbox, const wb_desc* descs, size_t work_budget, void* dev_mem, size_t bytes,
                    void* stream, wb_batch** out) {
  if (!out) return WB_ERR_INVALID;
  *out = nullptr;
  size_t need = 0;
  int rc = wb_batch_bytes(nbox, descs, work_budget, &need);
  if (rc) return rc;
  if (bytes < need) return WB_ERR_NOMEM;
  size_t st = 0, wmax = 0, wsum = 0;
  int maxn = 1;
  for (int i = 0; i < nbox; ++i) {
    WbGeo g = geo_of(descs[i]);
    st += state_doubles(g);
    wmax = std::max(wmax, work_doubles(g));
    wsum += work_doubles(g);
    for (int a = 0; a < 3; ++a) maxn = std::max(maxn, descs[i].n[a]);
  }
  size_t budget = work_budget > 0 ? work_budget : ((size_t)64 << 30);
  size_t work = std::max(wmax * sizeof(double), std::min(budget, wsum * sizeof(double)));
  wb_batch* b = nullptr;
  rc = wb_pool_create(&descs[0], st * sizeof(double), work, nbox, maxn, dev_mem, bytes, stream, &b);
  if (rc) return rc;
  for (int i = 0; i < nbox; ++i) {
    int slot = -1;
    rc = wb_pool_admit(b, &descs[i], &slot);
    if (rc) {
      delete b;
      return rc;
    }
  }
  apply_tune_cache(b);
  rc = rebuild(b);
  if (rc) {
    delete b;
    return rc;
  }
  *out = b;
  return WB_OK;
}

int wb_batch_destroy(wb_batch* b) {
  if (!b) return WB_OK;
  drop_graph(b);
  delete b;
  return WB_OK;
}

int wb_batch_load(wb_batch* b, int box, const double* U, const double* bx, const double* by,
                  const double* bz, int on_device, int primitive) {
  if (!b || box < 0 || box >= b->cap || !b->alive[box] || !U || !bx || !by || !bz)
    return bfail(b, WB_ERR_INVALID, "bad argument");
  const wb_desc& d = b->d[box];
  const WbGeo& g = b->geo[box];
  GridMap m;
  for (int a = 0; a < 3; ++a) { m.N[a] = d.n[a]; m.np[a] = 1; m.bc[a] = d.bc[a]; }
  m.npatch = 1;
  const BoxInfo& bi = b->info[box];
  cudaStream_t s = b->stream;
  const long long nc = (long long)d.n[0] * d.n[1] * d.n[2];
  const double* faces[3] = {bx, by, bz};
  for (int comp = 0; comp < 8; ++comp) {
    long long ext[3] = {d.n[0], d.n[1], d.n[2]};
    const double* src;
    if (comp < 5) src = U + comp * nc;
    else { ext[comp - 5] += 1; src = faces[comp - 5]; }
    const double* dsrc = src;
    if (!on_device) {
      cudaError_t e = cudaMemcpyAsync(b->staging, src, sizeof(double) * ext[0] * ext[1] * ext[2],
                                      cudaMemcpyHostToDevice, s);
      if (e != cudaSuccess) return bcuda(b, e, "batch load");
      dsrc = b->staging;
    }
    double* dst = comp < 5 ? bi.v.q[comp] : bi.v.b[comp - 5];
    wb_launch_scatter(dsrc, dst, comp, g, m, s);
    if (!on_device) {
      cudaError_t e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) return bcuda(b, e, "batch load");
    }
  }
  double* q[8];
  double* bb[3];
  for (int c = 0; c < 8; ++c) q[c] = bi.v.q[c];
  for (int c = 0; c < 3; ++c) bb[c] = bi.v.b[c];
  wb_launch_halo(q, bb, g, m, s);
  wb_launch_ccb(q, bb, g, 1, s);
  if (primitive) wb_launch_prim_to_cons(q, g, 1, b->phys, s);
  wb_launch_halo(q, bb, g, m, s);
  cudaError_t e = cudaMemsetAsync(b->d_scal + box, 0, sizeof(WbScalars), s);
  if (e != cudaSuccess) return bcuda(b, e, "batch load");
  const long long nint = (long long)g.n[0] * g.n[1] * g.n[2];
  k_box_rate<<<(unsigned)((nint + 255) / 256), 256, 0, s>>>(bi.v, b->d_scal + box, b->phys);
  e = cudaStreamSynchronize(s);
  if (e == cudaSuccess) e = cudaGetLastError();
  return bcuda(b, e, "batch load");
}

int wb_batch_set_steps(wb_batch* b, int box, int nsteps) {
  if (!b || box < -1 || box >= b->cap || nsteps < 0) return bfail(b, WB_ERR_INVALID, "bad argument");
  if (box >= 0 && !b->alive[box]) return bfail(b, WB_ERR_INVALID, "box not resident");
  std::vector<int> v;
  int first = box < 0 ? 0 : box, count = box < 0 ? b->cap : 1;
  v.assign(count, nsteps);
  if (box < 0)
    for (int i = 0; i < b->cap; ++i)
      if (!b->alive[i]) v[i] = 0;
  for (int i = 0; i < count; ++i) b->granted[first + i] = v[i];
  const bool any = any_granted(b);
  for (int i = 0; i < b->cap; ++i)
    if (wants_group(b, i, any) != (b->grouped[i] != 0)) {
      b->dirty = true;
      break;
    }
  cudaError_t e = cudaMemcpyAsync(b->d_steps + first, v.data(), sizeof(int) * count, cudaMemcpyHostToDevice,
                                  b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  return bcuda(b, e, "set steps");
}

int wb_batch_advance(wb_batch* b, int nsteps, int use_graph) {
  if (!b || nsteps < 0) return bfail(b, WB_ERR_INVALID, "bad argument");
  if (nsteps == 0) return WB_OK;
  int brc = ensure_built(b);
  if (brc) return brc;
  cudaError_t e;
  if (use_graph && b->graph_ok) {
    if (!b->graph || b->graph_steps != nsteps) {
      drop_graph(b);
      cudaGraph_t graph = nullptr;
      e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
      if (e == cudaSuccess) {
        cudaError_t le = enqueue_advance(b, nsteps);
        e = cudaStreamEndCapture(b->stream, &graph);
        if (le != cudaSuccess) e = le;
      }
      if (e == cudaSuccess) e = cudaGraphInstantiate(&b->graph, graph, 0);
      if (graph) cudaGraphDestroy(graph);
      if (e != cudaSuccess) {
        cudaGetLastError();
        b->graph = nullptr;
        b->graph_ok = false;  // fall back to direct launches
      } else {
        b->graph_steps = nsteps;
      }
    }
    if (b->graph) {
      e = cudaGraphLaunch(b->graph, b->stream);
      if (e != cudaSuccess) return bcuda(b, e, "graph launch");
      return read_sync_error(b);
    }
  }
  e = enqueue_advance(b, nsteps);
  if (e != cudaSuccess) return bcuda(b, e, "batch launch");
  return read_sync_error(b);
}

int wb_batch_read(wb_batch* b, int box, double* U, double* bx, double* by, double* bz, double* B,
                  int on_device) {
  if (!b || box < 0 || box >= b->cap || !b->alive[box]) return bfail(b, WB_ERR_INVALID, "bad argument");
  const wb_desc& d = b->d[box];
  const WbGeo& g = b->geo[box];
  GridMap m;
  for (int a = 0; a < 3; ++a) { m.N[a] = d.n[a]; m.np[a] = 1; m.bc[a] = d.bc[a]; }
  m.npatch = 1;
  const BoxInfo& bi = b->info[box];
  cudaStream_t s = b->stream;
  const long long nc = (long long)d.n[0] * d.n[1] * d.n[2];
  double* faces[3] = {bx, by, bz};
  for (int comp = 0; comp < 11; ++comp) {
    double* dst;
    const double* src;
    int mcomp = comp;
    long long ext[3] = {d.n[0], d.n[1], d.n[2]};
    if (comp < 5) { if (!U) continue; dst = U + comp * nc; src = bi.v.q[comp]; }
    else if (comp < 8) {
      if (!faces[comp - 5]) continue;
      dst = faces[comp - 5]; src = bi.v.b[comp - 5]; ext[comp - 5] += 1;
    } else {
      if (!B) continue;
      dst = B + (comp - 8) * nc; src = bi.v.q[F_BX + comp - 8]; mcomp = 0;
    }
    double* ddst = on_device ? dst : b->staging;
    wb_launch_gather(src, ddst, mcomp, g, m, s);
    if (!on_device) {
      cudaError_t e = cudaMemcpyAsync(dst, b->staging, sizeof(double) * ext[0] * ext[1] * ext[2],
                                      cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) return bcuda(b, e, "batch read");
    }
  }
  return bcuda(b, cudaGetLastError(), "batch read");
}

int wb_batch_counters(wb_batch* b, int box, wb_counters_t* c) {
  if (!b || !c || box < 0 || box >= b->cap) return bfail(b, WB_ERR_INVALID, "bad argument");
  WbScalars sc;
  cudaError_t e = cudaMemcpyAsync(&sc, b->d_scal + box, sizeof(sc), cudaMemcpyDeviceToHost, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return bcuda(b, e, "batch counters");
  c->steps = sc.steps;
  c->floor_hits = sc.floor_hits;
  c->unphysical = sc.unphysical;
  c->hll_faces = sc.hll_faces;
  c->t = sc.t;
  c->last_dt = sc.dt;
  return WB_OK;
}

int wb_batch_config(wb_batch* b, int seg_len, int blocks_per_sm, long long barrier_budget_cycles) {
  if (!b) return WB_ERR_INVALID;
  if (seg_len > 0) b->seg_len = seg_len;
  if (blocks_per_sm > 0) b->blocks_per_sm = std::min(blocks_per_sm, b->max_blocks_per_sm);
  if (barrier_budget_cycles > 0) b->budget = barrier_budget_cycles;
  drop_graph(b);
  b->dirty = true;
  return ensure_built(b);
}

int wb_batch_stage_timer(wb_batch* b, int on) {
  if (!b) return WB_ERR_INVALID;
  drop_graph(b);
  b->prof = on != 0;
  if (b->prof) {
    cudaError_t e = cudaMemsetAsync(b->d_prof, 0, sizeof(unsigned long long) * (BS_COUNT + 1), b->stream);
    if (e != cudaSuccess) return bcuda(b, e, "stage timer");
  }
  return WB_OK;
}

int wb_batch_stage_times(wb_batch* b, double* ms, int n, int* count) {
  if (!b || (!ms && n > 0)) return WB_ERR_INVALID;
  if (count) *count = BS_COUNT;
  unsigned long long ns[BS_COUNT];
  cudaError_t e = cudaMemcpyAsync(ns, b->d_prof, sizeof(ns), cudaMemcpyDeviceToHost, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return bcuda(b, e, "stage times");
  for (int i = 0; i < n && i < BS_COUNT; ++i) ms[i] = 1e-6 * (double)ns[i];
  return WB_OK;
}

int wb_batch_set_form(wb_batch* b, int form) {
  if (!b || (form != WB_BATCH_PERSISTENT && form != WB_BATCH_STAGED))
    return bfail(b, WB_ERR_INVALID, "unknown batch form");
  if (form != b->form) drop_graph(b);
  b->form = form;
  return WB_OK;
}

int wb_batch_get_form(wb_batch* b, int* form) {
  if (!b || !form) return WB_ERR_INVALID;
  *form = b->form;
  return WB_OK;
}

int wb_batch_get_config(wb_batch* b, int* seg_len, int* blocks_per_sm, int* groups) {
  if (!b) return WB_ERR_INVALID;
  if (seg_len) *seg_len = b->seg_len;
  if (blocks_per_sm) *blocks_per_sm = b->blocks_per_sm;
  if (groups) *groups = (int)b->gfirst.size() - 1;
  if (b->dirty) {
    int rc = ensure_built(b);
    if (rc) return rc;
    if (groups) *groups = (int)b->gfirst.size() - 1;
  }
  return WB_OK;
}

// Online autotuner: time trial_steps steps under each candidate segment
// length, then each block count, keep the fastest.  The candidates change
// only the work decomposition, so the trial steps are ordinary steps of the
// simulation (results do not depend on the configuration).
int wb_batch_autotune(wb_batch* b, int trial_steps, double* best_ms) {
  if (!b || trial_steps < 1) return bfail(b, WB_ERR_INVALID, "bad argument");
  int brc = ensure_built(b);
  if (brc) return brc;
  const int segs[] = {16, 24, 32, 48, 64, 96, 136};
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  auto trial = [&](int seg, int bps, float* ms) -> int {
    int rc = wb_batch_config(b, seg, bps, 0);
    if (rc) return rc;
    cudaEventRecord(e0, b->stream);
    cudaError_t e = enqueue_advance(b, trial_steps);
    if (e != cudaSuccess) return bcuda(b, e, "autotune");
    cudaEventRecord(e1, b->stream);
    rc = read_sync_error(b);
    if (rc) return rc;
    cudaEventElapsedTime(ms, e0, e1);
    return WB_OK;
  };
  int best_seg = b->seg_len, best_b = b->max_blocks_per_sm, best_form = b->form;
  float best = 1e30f, ms = 0.f;
  int rc = WB_OK;
  for (int form = WB_BATCH_PERSISTENT; rc == WB_OK && form <= WB_BATCH_STAGED; ++form) {
    b->form = form;
    int fseg = b->seg_len, fb = b->max_blocks_per_sm;
    float fbest = 1e30f;
    for (int seg : segs) {
      rc = trial(seg, b->max_blocks_per_sm, &ms);
      if (rc) break;
      if (ms < fbest) { fbest = ms; fseg = seg; }
    }
    for (int bps = 1; rc == WB_OK && bps < b->max_blocks_per_sm; ++bps) {
      rc = trial(fseg, bps, &ms);
      if (rc) break;
      if (ms < fbest) { fbest = ms; fb = bps; }
    }
    if (rc == WB_OK && fbest < best) { best = fbest; best_seg = fseg; best_b = fb; best_form = form; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  b->form = best_form;
  if (rc) return rc;
  rc = wb_batch_config(b, best_seg, best_b, 0);
  if (rc) return rc;
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    TuneKey key;
    for (int i = 0; i < b->cap; ++i)
      if (b->alive[i]) key.sizes.push_back(b->d[i].n[0] * 1000000 + b->d[i].n[1] * 1000 + b->d[i].n[2]);
    std::sort(key.sizes.begin(), key.sizes.end());
    g_tune_cache[key] = {best_seg, best_b, best_form};
  }
  if (best_ms) *best_ms = best;
  return WB_OK;
}

const char* wb_batch_last_error(const wb_batch* b) { return b ? b->err.c_str() : "null batch"; }

}  // extern "C"

WB_CHECK_ACCESSOR(wb_check_take_batch)
