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
// The default entropy-fix widths vanish on the linearly degenerate waves
// (Alfven and entropy); a specialisation with those eps_k = 0 known at compile
// time drops their Q-branch arithmetic.
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

// threads per block and resident blocks per SM the sweep is compiled for
// (registers per thread follow from their product; the face records take
// 2 x 38 doubles per thread of shared memory)
#ifndef WB_SWEEP_BLOCK
#define WB_SWEEP_BLOCK 64
#endif
// equal runs per warp once a launch has at least this many units per
// resident warp (measured: 128^3 sweeps 7 % faster than the one-segment-per-
// thread form at 54 units a warp, 64^3 2 % at 14)
#ifndef WB_BAL_MIN
#define WB_BAL_MIN 4
#endif
#ifndef WB_SWEEP_MIN_BLOCKS
#define WB_SWEEP_MIN_BLOCKS 4
#endif
constexpr int kBlock = WB_SWEEP_BLOCK;
using SRec = wbu::RecT<kBlock>;

using wbu::kEpsZeroLD;

template <int D, int EZ, bool PROT>
__global__ void __launch_bounds__(kBlock, WB_SWEEP_MIN_BLOCKS) k_sweep(SweepArgs A) {
  constexpr int U = (D == 0) ? 1 : 0;  // fastest transverse axis of the thread map
  constexpr int W = (D == 2) ? 1 : 2;
  __shared__ double srec[2][wbu::R_WORDS][kBlock];
  const double dt = *A.dt;
  if (!wb_pos(dt)) return;
  const int nu_ = A.box.hi[U] - A.box.lo[U] + 1;
  const int nw_ = A.box.hi[W] - A.box.lo[W] + 1;
  const long long npen = (long long)nu_ * nw_;
  const int len = A.box.hi[D] - A.box.lo[D] + 1;
  long long slot = blockIdx.y;
  const SRec rec[2] = {{&srec[0][0][threadIdx.x]}, {&srec[1][0][threadIdx.x]}};
  // Balanced: the work is the list of units (slot, group of 32 adjacent
  // pencils, face), slot- then group-major, over every slot of the pass; warp
  // w takes units [w U / C, (w+1) U / C) of the C warps of the launch (one
  // grid row) and marches one segment per group it touches, its 32 lanes on
  // the 32 pencils of the group (adjacent pencils: coalesced rows).
  // Otherwise one segment per thread: item = segment x pencils + pencil, one
  // grid row per slot.
  const long long ngroups = (npen + 31) / 32;
  const long long units = ngroups * len * (A.balanced ? A.nslots : 1);
  const long long C = (long long)gridDim.x * (kBlock / 32);
  const long long wid = ((long long)blockIdx.x * kBlock + threadIdx.x) / 32;
  const int lane = threadIdx.x % 32;
  long long u = wid * units / C;
  const long long u1 = (wid + 1) * units / C;
  const long long item = blockIdx.x * (long long)kBlock + threadIdx.x;
  bool once = !A.balanced;
  int nhll = 0;
  for (;;) {
    long long pen;
    int fa, fb;
    bool ok;
    if (A.balanced) {
      if (u >= u1) break;
      const long long sg = u / len;          // slot x ngroups + group
      slot = sg / ngroups;
      const long long grp = sg - slot * ngroups;
      const int off = (int)(u - sg * len);
      const int take = (int)((len - off) < (u1 - u) ? (len - off) : (u1 - u));
      pen = grp * 32 + lane;
      fa = A.box.lo[D] + off;
      fb = fa + take - 1;
      ok = pen < npen;
      u += take;
    } else {
      if (!once) break;
      once = false;
      const int seg = (int)(item / npen);
      pen = item - seg * npen;
      fa = A.box.lo[D] + seg * A.seg_len;
      fb = fa + A.seg_len - 1;
      if (fb > A.box.hi[D]) fb = A.box.hi[D];
      ok = item < npen * A.nseg && fa <= fb;
    }
    if (ok)
      nhll += wbu::sweep_segment<D, true, EZ, PROT>(A.geo, A.q, A.bn, A.F, slot * A.slot_in, slot * A.slot_out,
                                                    A.box.lo[U] + (int)(pen % nu_), A.box.lo[W] + (int)(pen / nu_),
                                                    fa, fb, dt, A.phys, rec);
  }
  if (nhll) atomicAdd((unsigned long long*)&A.scal->hll_faces, (unsigned long long)nhll);
}

template <int D, int EZ, bool PROT>
int blocks_per_sm() {
  static int cached = -1;
  if (cached < 0) {
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_sweep<D, EZ, PROT>, kBlock, 0) != cudaSuccess ||
        nb < 1)
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

template <int D, int EZ, bool PROT>
static void launch_sweep(SweepArgs a, int nslots, cudaStream_t s) {
  constexpr int U = (D == 0) ? 1 : 0;
  constexpr int W = (D == 2) ? 1 : 2;
  long long npen = (long long)(a.box.hi[U] - a.box.lo[U] + 1) * (a.box.hi[W] - a.box.lo[W] + 1);
  int len = a.box.hi[D] - a.box.lo[D] + 1;
  int resident = blocks_per_sm<D, EZ, PROT>() * sm_count() * kBlock;
  // big launches: equal runs of units per resident warp over every slot of
  // the pass, so every warp finishes with the others (no partial last wave)
  const long long units = (npen + 31) / 32 * (long long)len * nslots;
  const long long warps = resident / 32;
  if (a.nseg == 0 && units >= WB_BAL_MIN * warps) {
    a.balanced = 1;
    a.nslots = nslots;
    k_sweep<D, EZ, PROT><<<dim3((unsigned)(resident / kBlock), 1), kBlock, 0, s>>>(a);
    return;
  }
  a.balanced = 0;
  int nseg = a.nseg > 0 ? a.nseg : choose_segments(npen * nslots, len, resident);
  a.nseg = nseg;
  a.seg_len = (len + nseg - 1) / nseg;
  dim3 grid((unsigned)((npen * nseg + kBlock - 1) / kBlock), (unsigned)nslots);
  k_sweep<D, EZ, PROT><<<grid, kBlock, 0, s>>>(a);
}

template <int EZ, bool PROT>
static void launch_sweep_dir(int dir, const SweepArgs& a, int nslots, cudaStream_t s) {
  if (dir == 0) launch_sweep<0, EZ, PROT>(a, nslots, s);
  else if (dir == 1) launch_sweep<1, EZ, PROT>(a, nslots, s);
  else launch_sweep<2, EZ, PROT>(a, nslots, s);
}

// Kernel variants: eps_k = 0 on the linearly degenerate waves (the default)
// or general eps; protection floors off (the default) or on.
void wb_launch_sweep(int dir, const SweepArgs& a, int nslots, cudaStream_t s) {
  const bool ez = (a.phys.eps_zero & kEpsZeroLD) == kEpsZeroLD;
  if (a.phys.prot) {
    if (ez) launch_sweep_dir<kEpsZeroLD, true>(dir, a, nslots, s);
    else launch_sweep_dir<0, true>(dir, a, nslots, s);
  } else {
    if (ez) launch_sweep_dir<kEpsZeroLD, false>(dir, a, nslots, s);
    else launch_sweep_dir<0, false>(dir, a, nslots, s);
  }
}

// Self-test of the FP64 reciprocal helpers against the library division and
// reciprocal square root on n inputs spread over [1e-300, 1e300].
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
    double x = exp((u - 0.5) * 1381.55);
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

WB_CHECK_ACCESSOR(wb_check_take_sweep)
