// Host-side declarations of the kernel launchers (internal to the library).
#pragma once
#include <cuda_runtime.h>

#include "wb_device.cuh"
#include "wb_units.cuh"

struct wb_desc;
// Physics constants of a descriptor (gamma, CFL, eps_k, limiter, floors).
WbPhys wb_phys_of(const struct wb_desc* d);

struct SweepArgs {
  const double* q[8];      // input zone fields (slot 0)
  const double* bn;        // normal face field (slot 0)
  double* F[8];            // output flux fields (slot 0); F[F_BX + dir] unused
  long long slot_in, slot_out;
  WbGeo geo;
  WbBox box;               // faces along the sweep axis, zones across it
  const double* dt;
  WbPhys phys;
  WbScalars* scal;
  int nseg;                // segments per pencil (0: chosen at launch)
  int seg_len;             // faces per segment (set at launch)
  int balanced;            // 1: equal runs of (slot, 32-pencil group, face) units per warp
  int nslots;              // slots of the pass (balanced launches take them all in one row)
};

// Pointers of one pipeline pass over a batch of patches: the view holds the
// slot-0 pointers; slot s of the state is at +s*slot_q, of the workspace at
// +s*slot_w.
struct StageArgs {
  WbView v;
  long long slot_q, slot_w;
  WbPhys phys;
  int nslots;
  // the final update's view of the domain boundary: slot s holds patch
  // p0 + s of a grid with np[] patches per axis; bit a of ohi_bc is set when
  // axis a is outflow (its high boundary face is a copy of the last owned one)
  long long p0;
  int np[3];
  int ohi_bc;
};

// Global description needed by the halo fill and by load/read scatter.
struct GridMap {
  int N[3];        // global zones
  int np[3];       // patches per axis
  int bc[3];
  long long npatch;
};

void wb_launch_sweep(int dir, const SweepArgs& a, int nslots, cudaStream_t s);

void wb_launch_eref(const StageArgs& a, const WbBox& box, cudaStream_t s);
void wb_launch_edges(const StageArgs& a, bool corrector, const WbBox box[3], cudaStream_t s);
void wb_launch_ct(const StageArgs& a, bool final_step, const WbBox box[3], cudaStream_t s);
void wb_launch_transverse(const StageArgs& a, const WbBox box[3], cudaStream_t s);
void wb_launch_eref_half(const StageArgs& a, const WbBox& box, cudaStream_t s);
void wb_launch_final(const StageArgs& a, cudaStream_t s);

void wb_launch_halo(double* const q[8], double* const b[3], const WbGeo& geo, const GridMap& m,
                    cudaStream_t s);

// Arrays whose ghost points a periodic wrap fills (null entries skipped by
// the caller that builds the list).
struct WrapList {
  double* a[24];
  int n;
};
// Periodic images on every axis: one patch (the box's own interior) or all
// patches of a grid resident in one pass (slot = patch, neighbour patches).
void wb_launch_wrap(const WrapList& L, const WbGeo& geo, const GridMap& m, int depth, cudaStream_t s);
void wb_launch_dt_init(double* const q[8], const WbGeo& geo, long long npatch, const WbPhys& ph,
                       WbScalars* scal, cudaStream_t s);
void wb_launch_dt_step(WbScalars* scal, double cfl, double t_end, int lag, cudaStream_t s);
void wb_launch_ccb(double* const q[8], double* const b[3], const WbGeo& geo, long long npatch,
                   cudaStream_t s);
void wb_launch_prim_to_cons(double* const q[8], const WbGeo& geo, long long npatch,
                            const WbPhys& ph, cudaStream_t s);
// global <-> patch copies; comp: 0..4 zone field, 5..7 face field of axis comp-5
void wb_launch_scatter(const double* src, double* dst_field, int comp, const WbGeo& geo,
                       const GridMap& m, cudaStream_t s);
void wb_launch_gather(const double* src_field, double* dst, int comp, const WbGeo& geo,
                      const GridMap& m, cudaStream_t s);
// Conserved totals: nblocks partial pairs in part (16 doubles each), the 8
// totals x vol in out (device memory).
void wb_launch_totals(double* const q[8], double* const b[3], const WbGeo& geo, long long npatch, double vol,
                      double* part, int nblocks, double* out, cudaStream_t s);
void wb_launch_divb(double* const b[3], const WbGeo& geo, long long npatch,
                    unsigned long long* out_bits, cudaStream_t s);
void wb_launch_copy_box(const double* src, long long slot, const WbGeo& geo, const WbBox& box,
                        double* dst, cudaStream_t s);
void wb_launch_fp64_probe(double* out, int blocks, int iters, cudaStream_t s);
void wb_launch_math_selftest(int n, unsigned long long* worst, cudaStream_t s);
void wb_launch_bits_selftest(int n, unsigned long long* counts, cudaStream_t s);

// check words of the translation units (checked build; 0 otherwise)
unsigned wb_check_take_sweep();
unsigned wb_check_take_stages();
unsigned wb_check_take_capi();
unsigned wb_check_take_batch();
