// C ABI and grid manager of the GB300-native WOMBAT step (include/wombat.h).
// Host code: carves the caller's device workspace into the patch state and the
// per-batch intermediates, and enqueues the stage kernels of one CTU+CT step
// (Sec. "MHD in Three Dimensions", Steps 1-11) on the caller's stream.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <initializer_list>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "../../include/wombat.h"
#include "wb_device.cuh"
#include "wb_internal.h"

struct wb_grid {
  wb_desc d;
  WbGeo geo;
  GridMap map;
  WbPhys phys;
  cudaStream_t stream;
  char* mem;
  size_t bytes;
  long long npatch;
  int S;  // patch slots per pipeline pass
  double* q[8];
  double* b[3];
  // workspace, slot 0 bases (stride geo.V)
  double* Fp[3][8];
  double* Fc[3][8];
  double* Eref[3];
  double* Eedge[3];
  double* bh[3];
  double* qh[3][8];
  double* Erefh[3];
  double* Eedgeh[3];
  double* staging;
  WbScalars* scal;
  unsigned long long* red;
  std::string err;
  bool loaded;
  // interior-only stages with periodic images of the intermediates: periodic
  // on every axis, 3D storage, every patch in one pass
  bool wrap = false;
  // sweep timing (wb_profile_sweeps)
  bool prof;
  std::vector<cudaEvent_t> ev;
  size_t ev_used;
};

namespace {

const size_t kAlign = 256;

size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

struct Layout {
  size_t state, work, staging, scalars, total;
  long long npatch, V;
  int S;
};

bool valid_desc(const wb_desc* d, std::string* why) {
  if (!d) { *why = "null descriptor"; return false; }
  for (int a = 0; a < 3; ++a) {
    if (d->n[a] < 1 || d->patches[a] < 1 || d->n[a] % d->patches[a] != 0) {
      *why = "n must be a positive multiple of patches on every axis";
      return false;
    }
    if (!(d->length[a] > 0.0)) { *why = "length must be positive"; return false; }
    if (d->bc[a] != WB_BC_PERIODIC && d->bc[a] != WB_BC_OUTFLOW) { *why = "bad bc"; return false; }
  }
  if (!(d->gamma > 1.0) || d->gamma > 2.0) { *why = "gamma must be in (1, 2]"; return false; }
  if (!(d->cfl > 0.0)) { *why = "cfl must be positive"; return false; }
  for (int k = 0; k < 7; ++k)
    if (!(d->eps[k] >= 0.0) || !(d->eps[k] < 0.5)) { *why = "eps_k must be in [0, 0.5)"; return false; }
  if (!(d->sweby_beta >= 1.0) || d->sweby_beta > 2.0) { *why = "sweby_beta must be in [1, 2]"; return false; }
  if (d->batch_patches < 0) { *why = "batch_patches must be >= 0"; return false; }
  if (d->keep_stages != 0 && d->keep_stages != 1) { *why = "keep_stages must be 0 or 1"; return false; }
  {
    // padded zones of all patches (sizes beyond any device are refused before
    // a byte count could overflow)
    double vol = 1.0;
    for (int a = 0; a < 3; ++a) vol *= (double)(d->n[a] / d->patches[a] + 2 * WB_NG) * d->patches[a];
    if (vol > 1.0e12) { *why = "grid too large (more than 1e12 padded zones)"; return false; }
  }
  if (!(d->prot_rho >= 0.0) || !(d->prot_p >= 0.0)) {
    *why = "protection floors must be >= 0";
    return false;
  }
  if (!(d->rho_floor >= 0.0) || !(d->p_floor >= 0.0) || !std::isfinite(d->rho_floor) ||
      !std::isfinite(d->p_floor)) {
    *why = "floors must be finite and >= 0";
    return false;
  }
  return true;
}

// A box one zone thick along z with periodic z is the 2D problem of
// Sec. "MHD in Two Dimensions": every z layer, ghosts included, holds the
// same values, so it is stored as one plane with z stride 0.  Reads at
// k +- 1 then see that plane, z flux and EMF differences vanish exactly, and
// the z sweep reduces to one face per pencil (the flux of a z-uniform state).
bool flat_z(const wb_desc* d) {
  return d->n[2] == 1 && d->patches[2] == 1 && d->bc[2] == WB_BC_PERIODIC;
}

WbGeo make_geo(const wb_desc* d) {
  WbGeo g;
  for (int a = 0; a < 3; ++a) {
    g.n[a] = d->n[a] / d->patches[a];
    g.pd[a] = g.n[a] + 2 * WB_NG;
    g.dx[a] = d->length[a] / d->n[a];
    g.idx[a] = 1.0 / g.dx[a];
  }
  g.sy = g.pd[0];
  g.sz = (long long)g.pd[0] * g.pd[1];
  if (flat_z(d)) {
    g.pd[2] = 1;
    g.sz = 0;
  }
  g.V = (long long)g.pd[0] * g.pd[1] * g.pd[2];
  return g;
}

// workspace arrays per padded zone and patch slot: predictor fluxes (3 x 7),
// reference EMF, corner EMFs, b^{n+1/2} (3 each), q^{n+1/2} (3 x 8), and with
// keep_stages the corrector fluxes, half-step EMF and corrector corner EMFs in
// arrays of their own (3 x 7 + 3 + 3) instead of their predictor counterparts'
int work_arrays(const wb_desc* d) { return 3 * 7 + 3 + 3 + 3 + 3 * 8 + (d->keep_stages ? 3 * 7 + 3 + 3 : 0); }

// blocks of the conserved-totals reduction (a fixed count: the summation
// order, and so the result, do not depend on the device)
constexpr int kTotalsBlocks = 256;

// Point a grid's intermediates into the workspace w (slab doubles per array).
// Without keep, the corrector fluxes, the half-step reference EMF and the
// corrector corner EMFs take the arrays of the predictor fluxes, the reference
// EMF and the predictor corner EMFs: each is written (Steps 6, 8, 9) after the
// last stage that reads its counterpart (Steps 7, 3, 4).
void carve_work(wb_grid* g, double* w, size_t slab, bool keep) {
  size_t k = 0;
  for (int dd = 0; dd < 3; ++dd)
    for (int c = 0; c < 8; ++c) g->Fp[dd][c] = (c == F_BX + dd) ? nullptr : w + slab * k++;
  for (int dd = 0; dd < 3; ++dd) g->Eref[dd] = w + slab * k++;
  for (int dd = 0; dd < 3; ++dd) g->Eedge[dd] = w + slab * k++;
  for (int dd = 0; dd < 3; ++dd) g->bh[dd] = w + slab * k++;
  for (int dd = 0; dd < 3; ++dd)
    for (int c = 0; c < 8; ++c) g->qh[dd][c] = w + slab * k++;
  for (int dd = 0; dd < 3; ++dd)
    for (int c = 0; c < 8; ++c)
      g->Fc[dd][c] = !keep ? g->Fp[dd][c] : ((c == F_BX + dd) ? nullptr : w + slab * k++);
  for (int dd = 0; dd < 3; ++dd) g->Erefh[dd] = keep ? w + slab * k++ : g->Eref[dd];
  for (int dd = 0; dd < 3; ++dd) g->Eedgeh[dd] = keep ? w + slab * k++ : g->Eedge[dd];
}

Layout layout(const wb_desc* d) {
  Layout L;
  WbGeo g = make_geo(d);
  L.V = g.V;
  L.npatch = (long long)d->patches[0] * d->patches[1] * d->patches[2];
  long long S = d->batch_patches > 0 ? d->batch_patches : L.npatch;
  if (S > L.npatch) S = L.npatch;
  L.S = (int)S;
  L.state = align_up(sizeof(double) * (size_t)L.V * L.npatch * 11);
  L.work = align_up(sizeof(double) * (size_t)L.V * S * work_arrays(d));
  size_t gmax = (size_t)(d->n[0] + 1) * (d->n[1] + 1) * (d->n[2] + 1);
  L.staging = align_up(sizeof(double) * gmax);
  // device scalars, 64 reduction words, the 8 totals and the totals' partials
  L.scalars = align_up(sizeof(WbScalars) + 64 * sizeof(unsigned long long) +
                       sizeof(double) * (8 + 16 * kTotalsBlocks));
  L.total = L.state + L.work + L.staging + L.scalars;
  return L;
}

}  // namespace

WbPhys wb_phys_of(const wb_desc* d) {
  WbPhys p;
  p.gamma = d->gamma;
  p.gamma_f = (float)d->gamma;
  p.gm1 = d->gamma - 1.0;
  p.gm2 = d->gamma - 2.0;
  p.hgm2 = 0.5 * (d->gamma - 2.0);
  p.g_over_gm1 = d->gamma / (d->gamma - 1.0);
  p.inv_gm1 = 1.0 / (d->gamma - 1.0);
  p.gm2_over_gm1 = (d->gamma - 2.0) / (d->gamma - 1.0);
  p.cfl = d->cfl;
  p.eps_zero = 0;
  for (int k = 0; k < 7; ++k) {
    p.eps[k] = d->eps[k];
    p.two_eps[k] = 2.0 * d->eps[k];
    p.four_eps[k] = 4.0 * d->eps[k];
    p.inv16eps[k] = d->eps[k] > 0.0 ? 1.0 / (16.0 * d->eps[k]) : 0.0;
    p.inv4eps_m1[k] = d->eps[k] > 0.0 ? 1.0 / (4.0 * d->eps[k]) - 1.0 : 0.0;
    if (d->eps[k] == 0.0) p.eps_zero |= 1 << k;
  }
  p.sweby = d->sweby_beta;
  p.minmod = d->sweby_beta == 1.0 ? 1 : 0;
  p.rho_floor = d->rho_floor;
  p.p_floor = d->p_floor;
  p.prot_rho = d->prot_rho;
  p.prot_p = d->prot_p;
  p.prot = (d->prot_rho > 0.0 || d->prot_p > 0.0) ? 1 : 0;
  return p;
}

namespace {

int fail(wb_grid* g, int code, const std::string& msg) {
  if (g) g->err = msg;
  return code;
}

int check_cuda(wb_grid* g, cudaError_t e, const char* where) {
  if (e == cudaSuccess) return WB_OK;
  return fail(g, WB_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

WbBox box(int l0, int h0, int l1, int h1, int l2, int h2) {
  WbBox b;
  b.lo[0] = l0; b.hi[0] = h0; b.lo[1] = l1; b.hi[1] = h1; b.lo[2] = l2; b.hi[2] = h2;
  return b;
}

StageArgs stage_args(wb_grid* g, long long p0, int nslots) {
  StageArgs a;
  std::memset(&a, 0, sizeof(a));
  WbView& v = a.v;
  for (int c = 0; c < 8; ++c) v.q[c] = g->q[c] + p0 * g->geo.V;
  for (int c = 0; c < 3; ++c) v.b[c] = g->b[c] + p0 * g->geo.V;
  a.slot_q = g->geo.V;
  for (int d = 0; d < 3; ++d) {
    for (int c = 0; c < 8; ++c) {
      v.Fp[d][c] = g->Fp[d][c];
      v.Fc[d][c] = g->Fc[d][c];
      v.qh[d][c] = g->qh[d][c];
    }
    v.Eref[d] = g->Eref[d];
    v.Eedge[d] = g->Eedge[d];
    v.bh[d] = g->bh[d];
    v.Erefh[d] = g->Erefh[d];
    v.Eedgeh[d] = g->Eedgeh[d];
  }
  a.slot_w = g->geo.V;
  v.geo = g->geo;
  v.scal = g->scal;
  a.phys = g->phys;
  a.nslots = nslots;
  a.p0 = p0;
  a.ohi_bc = 0;
  for (int d = 0; d < 3; ++d) {
    a.np[d] = g->map.np[d];
    if (g->map.bc[d] == WB_BC_OUTFLOW) a.ohi_bc |= 1 << d;
  }
  return a;
}

SweepArgs sweep_args(wb_grid* g, const StageArgs& s, int dir, bool corr, const WbBox& bx) {
  SweepArgs a;
  std::memset(&a, 0, sizeof(a));
  for (int c = 0; c < 8; ++c) a.q[c] = corr ? s.v.qh[dir][c] : s.v.q[c];
  a.bn = corr ? s.v.bh[dir] : s.v.b[dir];
  for (int c = 0; c < 8; ++c) a.F[c] = corr ? s.v.Fc[dir][c] : s.v.Fp[dir][c];
  a.slot_in = corr ? s.slot_w : s.slot_q;
  a.slot_out = s.slot_w;
  a.geo = g->geo;
  a.box = bx;
  a.dt = &g->scal->dt;
  a.phys = g->phys;
  a.scal = g->scal;
  return a;
}

const size_t kMaxProfiled = 8192;

void sweep(wb_grid* g, int dir, const SweepArgs& a, int nslots) {
  bool rec = g->prof && g->ev_used + 2 <= g->ev.size();
  if (rec) cudaEventRecord(g->ev[g->ev_used], g->stream);
  wb_launch_sweep(dir, a, nslots, g->stream);
  if (rec) {
    cudaEventRecord(g->ev[g->ev_used + 1], g->stream);
    g->ev_used += 2;
  }
}

WrapList wrap_list(std::initializer_list<double*> arrays) {
  WrapList L;
  std::memset(&L, 0, sizeof(L));
  for (double* a : arrays)
    if (a && L.n < 24) L.a[L.n++] = a;
  return L;
}

// One step of a grid periodic on every axis whose patches all sit in one
// pass (a single patch, or every patch resident: slot = patch).  Every stage
// runs on the interior index range of each patch only; between stages the
// ghost points a later stage reads (1 deep, 2 for the preconditioned states
// the corrector sweeps read) are filled with periodic images, from the
// neighbouring patch where there is one.  On one GPU the copies cost a small
// fraction of recomputing the ghost rings, which the 5-zone scheme (one
// exchange per step) otherwise does at every stage.
void enqueue_pass_wrap(wb_grid* g) {
  cudaStream_t s = g->stream;
  const int ns = (int)g->npatch;
  StageArgs A = stage_args(g, 0, ns);
  const WbGeo& G = g->geo;
  const int N0 = G.n[0], N1 = G.n[1], N2 = G.n[2];
  const WbBox in = box(0, N0 - 1, 0, N1 - 1, 0, N2 - 1);
  const WbBox in3[3] = {in, in, in};
  // Step 1: predictor fluxes on the interior faces (face N_d is face 0)
  for (int d = 0; d < 3; ++d) sweep(g, d, sweep_args(g, A, d, false, in), ns);
  // Step 2: reference EMF; then the images of both
  wb_launch_eref(A, in, s);
  wb_launch_wrap(wrap_list({g->Fp[0][0], g->Fp[0][1], g->Fp[0][2], g->Fp[0][3], g->Fp[0][4], g->Fp[0][6],
                            g->Fp[0][7], g->Fp[1][0], g->Fp[1][1], g->Fp[1][2], g->Fp[1][3], g->Fp[1][4],
                            g->Fp[1][5], g->Fp[1][7], g->Fp[2][0], g->Fp[2][1], g->Fp[2][2], g->Fp[2][3],
                            g->Fp[2][4], g->Fp[2][5], g->Fp[2][6], g->Eref[0], g->Eref[1], g->Eref[2]}),
                 G, g->map, 1, s);
  // Step 3: corner EMFs; Step 4: b^{n+1/2}
  wb_launch_edges(A, false, in3, s);
  wb_launch_wrap(wrap_list({g->Eedge[0], g->Eedge[1], g->Eedge[2]}), G, g->map, 1, s);
  wb_launch_ct(A, false, in3, s);
  wb_launch_wrap(wrap_list({g->bh[0], g->bh[1], g->bh[2]}), G, g->map, 1, s);
  // Steps 5, 7: preconditioned states (the corrector sweeps read 2 zones out)
  wb_launch_transverse(A, in3, s);
  {
    WrapList L = wrap_list({});
    for (int d = 0; d < 3; ++d)
      for (int c = 0; c < 8; ++c)
        if (g->qh[d][c]) L.a[L.n++] = g->qh[d][c];
    wb_launch_wrap(L, G, g->map, 2, s);
  }
  // Steps 6, 7: corrector fluxes
  for (int d = 0; d < 3; ++d) sweep(g, d, sweep_args(g, A, d, true, in), ns);
  wb_launch_wrap(wrap_list({g->Fc[0][0], g->Fc[0][1], g->Fc[0][2], g->Fc[0][3], g->Fc[0][4], g->Fc[0][6],
                            g->Fc[0][7], g->Fc[1][0], g->Fc[1][1], g->Fc[1][2], g->Fc[1][3], g->Fc[1][4],
                            g->Fc[1][5], g->Fc[1][7], g->Fc[2][0], g->Fc[2][1], g->Fc[2][2], g->Fc[2][3],
                            g->Fc[2][4], g->Fc[2][5], g->Fc[2][6]}),
                 G, g->map, 1, s);
  // Step 8: half-step reference EMF; Step 9: corner EMFs
  wb_launch_eref_half(A, in, s);
  wb_launch_wrap(wrap_list({g->Erefh[0], g->Erefh[1], g->Erefh[2]}), G, g->map, 1, s);
  wb_launch_edges(A, true, in3, s);
  wb_launch_wrap(wrap_list({g->Eedgeh[0], g->Eedgeh[1], g->Eedgeh[2]}), G, g->map, 1, s);
  // Step 11 (faces, the high boundary face included), then Step 10
  {
    WbBox bb[3] = {box(0, N0, 0, N1 - 1, 0, N2 - 1), box(0, N0 - 1, 0, N1, 0, N2 - 1),
                   box(0, N0 - 1, 0, N1 - 1, 0, N2)};
    wb_launch_ct(A, true, bb, s);
  }
  wb_launch_final(A, s);
}

// One pipeline pass (Steps 1-11) over patches [p0, p0 + nslots).
void enqueue_pass(wb_grid* g, long long p0, int nslots) {
  if (g->wrap) {
    enqueue_pass_wrap(g);
    return;
  }
  cudaStream_t s = g->stream;
  StageArgs A = stage_args(g, p0, nslots);
  const int N0 = g->geo.n[0], N1 = g->geo.n[1], N2 = g->geo.n[2];
  // one plane for a flat-z (2D) box: every region's z range is layer 0
  const bool flat = g->geo.sz == 0;
  auto box = [flat](int l0, int h0, int l1, int h1, int l2, int h2) {
    return flat ? ::box(l0, h0, l1, h1, 0, 0) : ::box(l0, h0, l1, h1, l2, h2);
  };
  // Step 1: predictor fluxes from q^n
  sweep(g, 0, sweep_args(g, A, 0, false, box(-3, N0 + 3, -4, N1 + 3, -4, N2 + 3)), nslots);
  sweep(g, 1, sweep_args(g, A, 1, false, box(-4, N0 + 3, -3, N1 + 3, -4, N2 + 3)), nslots);
  sweep(g, 2, sweep_args(g, A, 2, false, box(-4, N0 + 3, -4, N1 + 3, -3, N2 + 3)), nslots);
  // Step 2: reference EMF; Step 3: corner EMFs
  wb_launch_eref(A, box(-4, N0 + 3, -4, N1 + 3, -4, N2 + 3), s);
  {
    WbBox eb[3] = {box(-1, N0, -3, N1 + 3, -3, N2 + 3), box(-3, N0 + 3, -1, N1, -3, N2 + 3),
                   box(-3, N0 + 3, -3, N1 + 3, -1, N2)};
    wb_launch_edges(A, false, eb, s);
  }
  // Step 4: b^{n+1/2}
  {
    WbBox bb[3] = {box(-3, N0 + 3, -1, N1, -1, N2), box(-1, N0, -3, N1 + 3, -1, N2),
                   box(-1, N0, -1, N1, -3, N2 + 3)};
    wb_launch_ct(A, false, bb, s);
  }
  // Steps 5, 7: transverse-flux preconditioned states
  {
    WbBox tb[3] = {box(-3, N0 + 2, -1, N1, -1, N2), box(-1, N0, -3, N1 + 2, -1, N2),
                   box(-1, N0, -1, N1, -3, N2 + 2)};
    wb_launch_transverse(A, tb, s);
  }
  // Steps 6, 7: corrector fluxes
  sweep(g, 0, sweep_args(g, A, 0, true, box(-1, N0 + 1, -1, N1, -1, N2)), nslots);
  sweep(g, 1, sweep_args(g, A, 1, true, box(-1, N0, -1, N1 + 1, -1, N2)), nslots);
  sweep(g, 2, sweep_args(g, A, 2, true, box(-1, N0, -1, N1, -1, N2 + 1)), nslots);
  // Step 8: half-step reference EMF; Step 9: corner EMFs
  wb_launch_eref_half(A, box(-1, N0, -1, N1, -1, N2), s);
  {
    WbBox eb[3] = {box(0, N0 - 1, 0, N1, 0, N2), box(0, N0, 0, N1 - 1, 0, N2),
                   box(0, N0, 0, N1, 0, N2 - 1)};
    wb_launch_edges(A, true, eb, s);
  }
  // Step 11 (faces), then Step 10 + zone field + floors + next signal rate
  {
    WbBox bb[3] = {box(0, N0, 0, N1 - 1, 0, N2 - 1), box(0, N0 - 1, 0, N1, 0, N2 - 1),
                   box(0, N0 - 1, 0, N1 - 1, 0, N2)};
    wb_launch_ct(A, true, bb, s);
  }
  wb_launch_final(A, s);
}

int sync(wb_grid* g, const char* where) {
  return check_cuda(g, cudaStreamSynchronize(g->stream), where);
}

// Device address of a host array of n doubles that lives in page-locked host
// memory the GPU can address (cudaHostAlloc / cudaHostRegister), or null.
// Kernels then read or write it in place over the CPU-GPU link instead of
// going through a staging copy; both ends of the array are checked.
const void* host_mapped(const void* p, long long n) {
  if (!p || n <= 0) return nullptr;
  cudaPointerAttributes a0, a1;
  if (cudaPointerGetAttributes(&a0, p) != cudaSuccess) { cudaGetLastError(); return nullptr; }
  const char* last = static_cast<const char*>(p) + sizeof(double) * (size_t)(n - 1);
  if (cudaPointerGetAttributes(&a1, last) != cudaSuccess) { cudaGetLastError(); return nullptr; }
  if (a0.type != cudaMemoryTypeHost || a1.type != cudaMemoryTypeHost) return nullptr;
  if (!a0.devicePointer || !a1.devicePointer) return nullptr;
  const char* d0 = static_cast<const char*>(a0.devicePointer);
  const char* d1 = static_cast<const char*>(a1.devicePointer);
  if (d1 - d0 != last - static_cast<const char*>(p)) return nullptr;
  return a0.devicePointer;
}

int load_common(wb_grid* g, const double* U, const double* bx, const double* by,
                const double* bz, int on_device, bool primitive) {
  if (!g || !U || !bx || !by || !bz) return fail(g, WB_ERR_INVALID, "null argument");
  cudaStream_t s = g->stream;
  const long long nc = (long long)g->d.n[0] * g->d.n[1] * g->d.n[2];
  const double* faces[3] = {bx, by, bz};
  for (int comp = 0; comp < 8; ++comp) {
    long long ext[3] = {g->d.n[0], g->d.n[1], g->d.n[2]};
    const double* src;
    if (comp < 5) src = U + comp * nc;
    else { ext[comp - 5] += 1; src = faces[comp - 5]; }
    long long n = ext[0] * ext[1] * ext[2];
    const double* dsrc = src;
    const void* mapped = on_device ? nullptr : host_mapped(src, n);
    const bool staged = !on_device && !mapped;
    if (mapped) dsrc = static_cast<const double*>(mapped);
    if (staged) {
      cudaError_t e = cudaMemcpyAsync(g->staging, src, sizeof(double) * n, cudaMemcpyHostToDevice, s);
      if (e != cudaSuccess) return check_cuda(g, e, "load copy");
      dsrc = g->staging;
    }
    double* dst = comp < 5 ? g->q[comp] : g->b[comp - 5];
    wb_launch_scatter(dsrc, dst, comp, g->geo, g->map, s);
    if (staged) {
      // staging is reused by the next component
      int rc = sync(g, "load");
      if (rc) return rc;
    }
  }
  wb_launch_halo(g->q, g->b, g->geo, g->map, s);
  wb_launch_ccb(g->q, g->b, g->geo, g->npatch, s);
  if (primitive) wb_launch_prim_to_cons(g->q, g->geo, g->npatch, g->phys, s);
  wb_launch_halo(g->q, g->b, g->geo, g->map, s);
  WbScalars z;
  std::memset(&z, 0, sizeof(z));
  cudaError_t e = cudaMemcpyAsync(g->scal, &z, sizeof(z), cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return check_cuda(g, e, "load scalars");
  wb_launch_dt_init(g->q, g->geo, g->npatch, g->phys, g->scal, s);
  int rc = sync(g, "load");
  if (rc) return rc;
  g->loaded = true;
  return check_cuda(g, cudaGetLastError(), "load kernels");
}

}  // namespace

extern "C" {

void wb_desc_default(wb_desc* d, int nx, int ny, int nz) {
  if (!d) return;
  std::memset(d, 0, sizeof(*d));
  d->n[0] = nx; d->n[1] = ny; d->n[2] = nz;
  d->patches[0] = d->patches[1] = d->patches[2] = 1;
  d->length[0] = nx; d->length[1] = ny; d->length[2] = nz;
  d->gamma = 5.0 / 3.0;
  d->cfl = 0.8;
  const double eps[7] = {0.1, 0.0, 0.1, 0.0, 0.1, 0.0, 0.1};
  for (int k = 0; k < 7; ++k) d->eps[k] = eps[k];
  d->sweby_beta = 1.0;
  d->rho_floor = 1e-20;
  d->p_floor = 1e-20;
  d->batch_patches = 0;
}

int wb_grid_bytes(const wb_desc* d, size_t* bytes) {
  std::string why;
  if (!bytes || !valid_desc(d, &why)) return WB_ERR_INVALID;
  *bytes = layout(d).total;
  return WB_OK;
}

int wb_grid_create(const wb_desc* d, void* dev_mem, size_t bytes, void* stream, wb_grid** out) {
  std::string why;
  if (!out) return WB_ERR_INVALID;
  *out = nullptr;
  if (!valid_desc(d, &why)) return WB_ERR_INVALID;
  if (!dev_mem || (reinterpret_cast<uintptr_t>(dev_mem) % kAlign) != 0) return WB_ERR_INVALID;
  Layout L = layout(d);
  if (bytes < L.total) return WB_ERR_NOMEM;
  wb_grid* g = new (std::nothrow) wb_grid();
  if (!g) return WB_ERR_NOMEM;
  g->d = *d;
  g->geo = make_geo(d);
  for (int a = 0; a < 3; ++a) {
    g->map.N[a] = d->n[a];
    g->map.np[a] = d->patches[a];
    g->map.bc[a] = d->bc[a];
  }
  g->map.npatch = L.npatch;
  g->npatch = L.npatch;
  g->wrap = L.S == L.npatch && !flat_z(d) && d->bc[0] == WB_BC_PERIODIC && d->bc[1] == WB_BC_PERIODIC &&
            d->bc[2] == WB_BC_PERIODIC;
  g->S = L.S;
  g->phys = wb_phys_of(d);
  g->stream = reinterpret_cast<cudaStream_t>(stream);
  g->mem = reinterpret_cast<char*>(dev_mem);
  g->bytes = bytes;
  const size_t V = (size_t)g->geo.V;
  double* st = reinterpret_cast<double*>(g->mem);
  for (int c = 0; c < 8; ++c) g->q[c] = st + (size_t)c * V * L.npatch;
  for (int c = 0; c < 3; ++c) g->b[c] = st + (size_t)(8 + c) * V * L.npatch;
  double* w = reinterpret_cast<double*>(g->mem + L.state);
  size_t slab = V * (size_t)L.S;
  carve_work(g, w, slab, d->keep_stages != 0);
  g->staging = reinterpret_cast<double*>(g->mem + L.state + L.work);
  g->scal = reinterpret_cast<WbScalars*>(g->mem + L.state + L.work + L.staging);
  g->red = reinterpret_cast<unsigned long long*>(g->scal + 1);
  g->loaded = false;
  g->prof = false;
  g->ev_used = 0;
  // NaN-poison the workspace so that any read of an uncomputed value shows
  cudaError_t e = cudaMemsetAsync(g->mem, 0xff, L.state + L.work, g->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(g->scal, 0, L.scalars, g->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
  if (e != cudaSuccess) {
    delete g;
    return WB_ERR_CUDA;
  }
  *out = g;
  return WB_OK;
}

int wb_grid_destroy(wb_grid* g) {
  if (!g) return WB_OK;
  for (cudaEvent_t e : g->ev) cudaEventDestroy(e);
  delete g;
  return WB_OK;
}

int wb_profile_sweeps(wb_grid* g, int enable) {
  if (!g) return WB_ERR_INVALID;
  if (enable) {
    if (g->ev.empty()) {
      g->ev.resize(2 * kMaxProfiled);
      for (auto& e : g->ev)
        if (cudaEventCreate(&e) != cudaSuccess) return fail(g, WB_ERR_CUDA, "event create");
    }
    g->ev_used = 0;
  }
  g->prof = enable != 0;
  return WB_OK;
}

int wb_profile_read(wb_grid* g, double* sweep_ms, long long* launches) {
  if (!g || !sweep_ms || !launches) return fail(g, WB_ERR_INVALID, "null argument");
  cudaError_t e = cudaStreamSynchronize(g->stream);
  if (e != cudaSuccess) return check_cuda(g, e, "profile");
  double tot = 0.0;
  for (size_t i = 0; i + 1 < g->ev_used; i += 2) {
    float ms = 0.0f;
    e = cudaEventElapsedTime(&ms, g->ev[i], g->ev[i + 1]);
    if (e != cudaSuccess) return check_cuda(g, e, "profile");
    tot += ms;
  }
  *sweep_ms = tot;
  *launches = (long long)(g->ev_used / 2);
  return WB_OK;
}

int wb_load_state(wb_grid* g, const double* U, const double* bx, const double* by,
                  const double* bz, int on_device) {
  return load_common(g, U, bx, by, bz, on_device, false);
}

int wb_load_primitive(wb_grid* g, const double* W, const double* bx, const double* by,
                      const double* bz, int on_device) {
  return load_common(g, W, bx, by, bz, on_device, true);
}

int wb_compute_dt(wb_grid* g, double* dt) {
  if (!g || !dt) return fail(g, WB_ERR_INVALID, "null argument");
  if (!g->loaded) return fail(g, WB_ERR_INVALID, "no state loaded");
  unsigned long long bits = 0;
  cudaError_t e = cudaMemcpyAsync(&bits, &g->scal->wmax_next, sizeof(bits), cudaMemcpyDeviceToHost,
                                  g->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
  if (e != cudaSuccess) return check_cuda(g, e, "compute_dt");
  double w;
  std::memcpy(&w, &bits, sizeof(w));
  if (!(w > 0.0) || !std::isfinite(w)) return fail(g, WB_ERR_UNPHYSICAL, "no finite signal speed");
  *dt = g->d.cfl / w;
  return WB_OK;
}

int wb_advance(wb_grid* g, int nsteps, double t_end, double* t_out) {
  if (!g || nsteps < 0) return fail(g, WB_ERR_INVALID, "bad argument");
  if (!g->loaded) return fail(g, WB_ERR_INVALID, "no state loaded");
  cudaStream_t s = g->stream;
  cudaError_t e;
  long long unph0 = 0;
  if (t_out) {
    e = cudaMemcpyAsync(&unph0, &g->scal->unphysical, sizeof(unph0), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return check_cuda(g, e, "advance");
  }
  // With a time limit, the device clock is read back every kStepsPerCheck
  // steps and the remaining steps (which would do nothing) are not launched.
  constexpr int kStepsPerCheck = 64;
  for (int st = 0; st < nsteps; ++st) {
    if (t_end > 0.0 && st > 0 && st % kStepsPerCheck == 0) {
      double t_now = 0.0;
      e = cudaMemcpyAsync(&t_now, &g->scal->t, sizeof(t_now), cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) return check_cuda(g, e, "advance");
      if (t_now >= t_end) break;
    }
    wb_launch_dt_step(g->scal, g->d.cfl, t_end, g->d.dt_lag, s);
    for (long long p0 = 0; p0 < g->npatch; p0 += g->S) {
      int ns = (int)std::min<long long>(g->S, g->npatch - p0);
      enqueue_pass(g, p0, ns);
    }
    wb_launch_halo(g->q, g->b, g->geo, g->map, s);
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return check_cuda(g, e, "advance launch");
  if (t_out) {
    WbScalars sc;
    e = cudaMemcpyAsync(&sc, g->scal, sizeof(sc), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return check_cuda(g, e, "advance");
    *t_out = sc.t;
    if (sc.unphysical > unph0) return fail(g, WB_ERR_UNPHYSICAL, "unphysical state met");
  }
  return WB_OK;
}

int wb_read_state(wb_grid* g, double* U, double* bx, double* by, double* bz, double* B,
                  int on_device) {
  if (!g) return WB_ERR_INVALID;
  if (!g->loaded) return fail(g, WB_ERR_INVALID, "no state loaded");
  cudaStream_t s = g->stream;
  const long long nc = (long long)g->d.n[0] * g->d.n[1] * g->d.n[2];
  double* faces[3] = {bx, by, bz};
  for (int comp = 0; comp < 11; ++comp) {
    double* dst;
    int mcomp = comp;
    const double* src;
    long long ext[3] = {g->d.n[0], g->d.n[1], g->d.n[2]};
    if (comp < 5) { if (!U) continue; dst = U + comp * nc; src = g->q[comp]; }
    else if (comp < 8) {
      if (!faces[comp - 5]) continue;
      dst = faces[comp - 5]; src = g->b[comp - 5]; ext[comp - 5] += 1;
    } else {
      if (!B) continue;
      dst = B + (comp - 8) * nc; src = g->q[F_BX + comp - 8]; mcomp = 0;
    }
    long long n = ext[0] * ext[1] * ext[2];
    const void* mapped = on_device ? nullptr : host_mapped(dst, n);
    const bool staged = !on_device && !mapped;
    double* ddst = on_device ? dst : (mapped ? static_cast<double*>(const_cast<void*>(mapped)) : g->staging);
    wb_launch_gather(src, ddst, mcomp, g->geo, g->map, s);
    if (staged) {
      cudaError_t e = cudaMemcpyAsync(dst, g->staging, sizeof(double) * n, cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) return check_cuda(g, e, "read");
    }
  }
  // host arrays written in place by the kernels are complete once the stream is
  if (!on_device) {
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return check_cuda(g, e, "read");
  }
  return check_cuda(g, cudaGetLastError(), "read");
}

int wb_conserved_totals(wb_grid* g, double tot[8]) {
  if (!g || !tot) return fail(g, WB_ERR_INVALID, "null argument");
  if (!g->loaded) return fail(g, WB_ERR_INVALID, "no state loaded");
  const int nx = g->d.n[0], ny = g->d.n[1], nz = g->d.n[2];
  const double vol = (g->d.length[0] / nx) * (g->d.length[1] / ny) * (g->d.length[2] / nz);
  double* out = reinterpret_cast<double*>(g->red + 64);
  double* part = out + 8;
  cudaStream_t s = g->stream;
  wb_launch_totals(g->q, g->b, g->geo, g->npatch, vol, part, kTotalsBlocks, out, s);
  cudaError_t e = cudaMemcpyAsync(tot, out, sizeof(double) * 8, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return check_cuda(g, e, "totals");
  return check_cuda(g, cudaGetLastError(), "totals");
}

int wb_divb_max(wb_grid* g, double* divb) {
  if (!g || !divb) return fail(g, WB_ERR_INVALID, "null argument");
  cudaStream_t s = g->stream;
  cudaError_t e = cudaMemsetAsync(g->red, 0, sizeof(unsigned long long), s);
  if (e != cudaSuccess) return check_cuda(g, e, "divb");
  wb_launch_divb(g->b, g->geo, g->npatch, g->red, s);
  unsigned long long bits = 0;
  e = cudaMemcpyAsync(&bits, g->red, sizeof(bits), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return check_cuda(g, e, "divb");
  std::memcpy(divb, &bits, sizeof(double));
  return WB_OK;
}

int wb_counters(wb_grid* g, wb_counters_t* c) {
  if (!g || !c) return fail(g, WB_ERR_INVALID, "null argument");
  WbScalars sc;
  cudaError_t e = cudaMemcpyAsync(&sc, g->scal, sizeof(sc), cudaMemcpyDeviceToHost, g->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
  if (e != cudaSuccess) return check_cuda(g, e, "counters");
  c->steps = sc.steps;
  c->floor_hits = sc.floor_hits;
  c->unphysical = sc.unphysical;
  c->hll_faces = sc.hll_faces;
  c->t = sc.t;
  c->last_dt = sc.dt;
  return WB_OK;
}

const char* wb_last_error(const wb_grid* g) {
  if (!g) return "null grid";
  return g->err.c_str();
}

int wb_debug_stage(wb_grid* g, int which, double* out, long long cap, long long* written) {
  if (!g || !out || !written) return fail(g, WB_ERR_INVALID, "null argument");
  if (g->npatch != 1) return fail(g, WB_ERR_INVALID, "stage dump needs a single patch");
  const int* n = g->geo.n;
  std::vector<const double*> arrays;
  WbBox bx = box(0, n[0] - 1, 0, n[1] - 1, 0, n[2] - 1);
  if (which >= 0 && which < 3 && !g->d.keep_stages)
    return fail(g, WB_ERR_INVALID, "predictor fluxes are overwritten by the corrector; "
                                   "create the grid with keep_stages = 1");
  if (which >= 0 && which < 6) {
    int d = which % 3;
    for (int c = 0; c < 8; ++c) arrays.push_back(which < 3 ? g->Fp[d][c] : g->Fc[d][c]);
    bx.hi[d] += 1;
  } else if (which >= 6 && which < 9) {
    int d = which - 6;
    arrays.push_back(g->bh[d]);
    bx.hi[d] += 1;
  } else if (which >= 9 && which < 12) {
    for (int c = 0; c < 8; ++c) arrays.push_back(g->qh[which - 9][c]);
  } else {
    return fail(g, WB_ERR_INVALID, "bad stage");
  }
  long long per = (long long)(bx.hi[0] + 1) * (bx.hi[1] + 1) * (bx.hi[2] + 1);
  long long need = per * (long long)arrays.size();
  if (cap < need) return fail(g, WB_ERR_INVALID, "output too small");
  const double nanv = std::nan("");
  for (size_t a = 0; a < arrays.size(); ++a) {
    if (!arrays[a]) {
      for (long long i = 0; i < per; ++i) out[a * per + i] = (which < 6) ? 0.0 : nanv;
      continue;
    }
    wb_launch_copy_box(arrays[a], 0, g->geo, bx, g->staging, g->stream);
    cudaError_t e = cudaMemcpyAsync(out + a * per, g->staging, sizeof(double) * per,
                                    cudaMemcpyDeviceToHost, g->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
    if (e != cudaSuccess) return check_cuda(g, e, "stage");
  }
  *written = need;
  return WB_OK;
}

int wb_selftest_math(wb_grid* g, int n, double worst[2]) {
  if (!g || !worst || n < 1) return fail(g, WB_ERR_INVALID, "bad argument");
  cudaError_t e = cudaMemsetAsync(g->red, 0, 2 * sizeof(unsigned long long), g->stream);
  if (e != cudaSuccess) return check_cuda(g, e, "selftest");
  wb_launch_math_selftest(n, g->red, g->stream);
  unsigned long long bits[2] = {0, 0};
  e = cudaMemcpyAsync(bits, g->red, sizeof(bits), cudaMemcpyDeviceToHost, g->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
  if (e != cudaSuccess) return check_cuda(g, e, "selftest");
  std::memcpy(worst, bits, sizeof(bits));
  return WB_OK;
}

int wb_selftest_bits(wb_grid* g, int n, long long counts[WB_BITS_TESTS]) {
  if (!g || !counts || n < 1) return fail(g, WB_ERR_INVALID, "bad argument");
  cudaError_t e = cudaMemsetAsync(g->red, 0, WB_BITS_TESTS * sizeof(unsigned long long), g->stream);
  if (e != cudaSuccess) return check_cuda(g, e, "selftest");
  wb_launch_bits_selftest(n, g->red, g->stream);
  e = cudaMemcpyAsync(counts, g->red, WB_BITS_TESTS * sizeof(long long), cudaMemcpyDeviceToHost, g->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
  if (e != cudaSuccess) return check_cuda(g, e, "selftest");
  return WB_OK;
}

int wb_measure_fp64_peak(void* stream, double* flops) {
  if (!flops) return WB_ERR_INVALID;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return WB_ERR_CUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return WB_ERR_CUDA;
  // the probe is a diagnostic outside any grid: it uses a small buffer of its own
  const int blocks = sms * 4, iters = 1500;
  double* buf = nullptr;
  if (cudaMalloc(&buf, sizeof(double) * blocks * 256) != cudaSuccess) return WB_ERR_CUDA;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  wb_launch_fp64_probe(buf, blocks, 20, s);
  float best = 1e30f;
  for (int r = 0; r < 3; ++r) {
    cudaEventRecord(e0, s);
    wb_launch_fp64_probe(buf, blocks, iters, s);
    cudaEventRecord(e1, s);
    cudaEventSynchronize(e1);
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best) best = ms;
  }
  cudaError_t err = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(buf);
  if (err != cudaSuccess) return WB_ERR_CUDA;
  *flops = 2.0 * 8 * 16 * (double)iters * blocks * 256 / (best * 1e-3);
  return WB_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// wb_step_noalloc: one step of a small single box with every intermediate in
// a file-scope device array, for callers that cannot allocate device memory.
// ---------------------------------------------------------------------------
namespace {

const size_t kNoallocBytes = 24u << 20;  // 24 MiB
static __device__ __align__(256) double wb_noalloc_scratch[kNoallocBytes / sizeof(double)];

std::mutex g_noalloc_mu;
void* g_noalloc_addr[256];  // device address of the array, per device ordinal
thread_local std::string g_noalloc_err;  // the calling thread's last failure

int noalloc_fail(int code, const std::string& msg) {
  g_noalloc_err = msg;
  return code;
}

}  // namespace

extern "C" {

const char* wb_noalloc_last_error(void) { return g_noalloc_err.c_str(); }

int wb_step_noalloc(const wb_desc* d, const double* U, const double* bx, const double* by,
                    const double* bz, double* U_out, double* bx_out, double* by_out,
                    double* bz_out, double* dt_out, void* stream) {
  std::string why;
  if (!valid_desc(d, &why)) return noalloc_fail(WB_ERR_INVALID, "invalid descriptor: " + why);
  if (d->patches[0] != 1 || d->patches[1] != 1 || d->patches[2] != 1)
    return noalloc_fail(WB_ERR_INVALID, "wb_step_noalloc takes a single box (patches = 1,1,1)");
  if (!U || !bx || !by || !bz || !U_out || !bx_out || !by_out || !bz_out)
    return noalloc_fail(WB_ERR_INVALID, "null state pointer");
  wb_desc one = *d;
  one.batch_patches = 0;
  one.keep_stages = 0;
  Layout L = layout(&one);
  if (L.total > kNoallocBytes) {
    char buf[200];
    std::snprintf(buf, sizeof(buf),
                  "box %dx%dx%d needs %zu bytes of scratch; the static limit is %zu bytes "
                  "(24 MiB: cubes up to 26^3 zones)",
                  d->n[0], d->n[1], d->n[2], L.total, kNoallocBytes);
    return noalloc_fail(WB_ERR_INVALID, buf);
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256)
    return noalloc_fail(WB_ERR_CUDA, "no current CUDA device");
  void* base = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
      void* p = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&p, wb_noalloc_scratch);
      if (e != cudaSuccess || !p)
        return noalloc_fail(WB_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      g_noalloc_addr[dev] = p;
    }
    base = g_noalloc_addr[dev];
  }
  // a grid object carved from the static array (no device allocation)
  wb_grid g;
  g.d = one;
  g.geo = make_geo(&one);
  for (int a = 0; a < 3; ++a) {
    g.map.N[a] = one.n[a];
    g.map.np[a] = 1;
    g.map.bc[a] = one.bc[a];
  }
  g.map.npatch = 1;
  g.npatch = 1;
  g.S = 1;
  g.phys = wb_phys_of(&one);
  g.stream = reinterpret_cast<cudaStream_t>(stream);
  g.mem = reinterpret_cast<char*>(base);
  g.bytes = kNoallocBytes;
  const size_t V = (size_t)g.geo.V;
  double* st = reinterpret_cast<double*>(g.mem);
  for (int c = 0; c < 8; ++c) g.q[c] = st + (size_t)c * V;
  for (int c = 0; c < 3; ++c) g.b[c] = st + (size_t)(8 + c) * V;
  double* w = reinterpret_cast<double*>(g.mem + L.state);
  carve_work(&g, w, V, false);
  g.staging = reinterpret_cast<double*>(g.mem + L.state + L.work);
  g.scal = reinterpret_cast<WbScalars*>(g.mem + L.state + L.work + L.staging);
  g.red = reinterpret_cast<unsigned long long*>(g.scal + 1);
  g.loaded = true;
  g.prof = false;
  g.ev_used = 0;
  cudaStream_t s = g.stream;
  // the array keeps the previous call's contents: the scalars (time, dt,
  // signal-rate accumulator, counters) must start at zero
  cudaError_t e = cudaMemsetAsync(g.scal, 0, L.scalars, s);
  if (e != cudaSuccess) return noalloc_fail(WB_ERR_CUDA, std::string("memset: ") + cudaGetErrorString(e));
  const double* faces[3] = {bx, by, bz};
  const long long nc = (long long)one.n[0] * one.n[1] * one.n[2];
  for (int comp = 0; comp < 8; ++comp) {
    const double* src = comp < 5 ? U + comp * nc : faces[comp - 5];
    double* dst = comp < 5 ? g.q[comp] : g.b[comp - 5];
    wb_launch_scatter(src, dst, comp, g.geo, g.map, s);
  }
  wb_launch_halo(g.q, g.b, g.geo, g.map, s);
  wb_launch_ccb(g.q, g.b, g.geo, 1, s);
  wb_launch_halo(g.q, g.b, g.geo, g.map, s);
  wb_launch_dt_init(g.q, g.geo, 1, g.phys, g.scal, s);
  wb_launch_dt_step(g.scal, one.cfl, 0.0, 0, s);
  enqueue_pass(&g, 0, 1);
  wb_launch_halo(g.q, g.b, g.geo, g.map, s);
  double* outs[3] = {bx_out, by_out, bz_out};
  for (int comp = 0; comp < 8; ++comp) {
    const double* src = comp < 5 ? g.q[comp] : g.b[comp - 5];
    double* dst = comp < 5 ? U_out + comp * nc : outs[comp - 5];
    wb_launch_gather(src, dst, comp, g.geo, g.map, s);
  }
  if (dt_out) {
    e = cudaMemcpyAsync(dt_out, &g.scal->dt, sizeof(double), cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return noalloc_fail(WB_ERR_CUDA, std::string("dt copy: ") + cudaGetErrorString(e));
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return noalloc_fail(WB_ERR_CUDA, std::string("launch: ") + cudaGetErrorString(e));
  return WB_OK;
}

}  // extern "C"

WB_CHECK_ACCESSOR(wb_check_take_capi)

#ifdef WB_CHECKED
namespace {
// Positive control of the checked build: forms the index of a zone one past
// the padded storage, which wb_at must flag; nothing is read or written at it.
__global__ void k_check_probe(WbGeo g, long long* sink) {
  const long long o = wb_at(g, g.pd[0] - WB_NG, 0, 0);
  if (o == -1 && sink) *sink = o;  // never true: keeps the index computation
}
}  // namespace
#endif

extern "C" {

int wb_check_flags(unsigned* flags) {
  if (!flags) return WB_ERR_INVALID;
  cudaDeviceSynchronize();
  *flags = wb_check_take_sweep() | wb_check_take_stages() | wb_check_take_capi() | wb_check_take_batch();
#ifdef WB_CHECKED
  return WB_OK;
#else
  return WB_ERR_INVALID;
#endif
}

int wb_check_selftest(int* detected) {
  if (!detected) return WB_ERR_INVALID;
  *detected = 0;
#ifdef WB_CHECKED
  WbGeo g{};
  for (int a = 0; a < 3; ++a) {
    g.n[a] = 4;
    g.pd[a] = 4 + 2 * WB_NG;
  }
  g.sy = g.pd[0];
  g.sz = (long long)g.pd[0] * g.pd[1];
  g.V = g.sz * g.pd[2];
  wb_check_take_capi();
  k_check_probe<<<1, 32>>>(g, nullptr);
  if (cudaDeviceSynchronize() != cudaSuccess) return WB_ERR_CUDA;
  *detected = wb_check_take_capi() != 0;
  return WB_OK;
#else
  return WB_ERR_INVALID;
#endif
}

}  // extern "C"
