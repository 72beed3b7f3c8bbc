// Host-side declarations of the kernel launchers (internal to the library).
#pragma once
#include <cuda_runtime.h>

#include "wb_device.cuh"

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
};

// Pointers of one pipeline pass over a batch of patches.
struct StageArgs {
  // state of the batch (slot 0 = first patch of the batch), stride slot_q
  double* q[8];
  double* b[3];
  long long slot_q;
  // workspace (stride slot_w)
  double* Fp[3][8];
  double* Fc[3][8];
  double* Eref[3];
  double* Eedge[3];
  double* bh[3];
  double* qh[3][8];
  double* Erefh[3];
  double* Eedgeh[3];
  long long slot_w;
  WbGeo geo;
  WbPhys phys;
  WbScalars* scal;
  int nslots;
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
void wb_launch_edge(const StageArgs& a, int axis, bool corrector, const WbBox& box,
                    cudaStream_t s);
void wb_launch_ct(const StageArgs& a, bool final_step, const WbBox box[3], cudaStream_t s);
void wb_launch_transverse(const StageArgs& a, int dir, const WbBox& box, cudaStream_t s);
void wb_launch_eref_half(const StageArgs& a, const WbBox& box, cudaStream_t s);
void wb_launch_final(const StageArgs& a, cudaStream_t s);

void wb_launch_halo(double* const q[8], double* const b[3], const WbGeo& geo, const GridMap& m,
                    cudaStream_t s);
void wb_launch_dt_init(double* const q[8], const WbGeo& geo, long long npatch, const WbPhys& ph,
                       WbScalars* scal, cudaStream_t s);
void wb_launch_dt_step(WbScalars* scal, double cfl, double t_end, cudaStream_t s);
void wb_launch_ccb(double* const q[8], double* const b[3], const WbGeo& geo, long long npatch,
                   cudaStream_t s);
void wb_launch_prim_to_cons(double* const q[8], const WbGeo& geo, long long npatch,
                            const WbPhys& ph, cudaStream_t s);
// global <-> patch copies; comp: 0..4 zone field, 5..7 face field of axis comp-5
void wb_launch_scatter(const double* src, double* dst_field, int comp, const WbGeo& geo,
                       const GridMap& m, cudaStream_t s);
void wb_launch_gather(const double* src_field, double* dst, int comp, const WbGeo& geo,
                      const GridMap& m, cudaStream_t s);
void wb_launch_divb(double* const b[3], const WbGeo& geo, long long npatch,
                    unsigned long long* out_bits, cudaStream_t s);
void wb_launch_copy_box(const double* src, long long slot, const WbGeo& geo, const WbBox& box,
                        double* dst, cudaStream_t s);
void wb_launch_fp64_probe(double* out, int blocks, int iters, cudaStream_t s);
void wb_launch_math_selftest(int n, unsigned long long* worst, cudaStream_t s);
