/*
 * wombat.h -- C ABI of the GB300-native (sm_103a) FP64 implementation of the
 * WOMBAT per-patch ideal-MHD step (Mendygral et al. 2017, arXiv:1701.07452):
 * the MHDTVD modified flux (Appendix A) inside the 3D CTU+CT 6-solve
 * integrator (Sec. "MHD in Three Dimensions", Steps 1-11), with 5 boundary
 * zones per patch filled once per step (Sec. "MHD in Two Dimensions") and a
 * global CFL time step (Sec. "MPI-RMA Engine": the non-blocking dt reduction).
 *
 * Conventions shared by every call
 *  - All floating point data are IEEE binary64.  Host arrays are row-major
 *    with x fastest:
 *      U  [5][nz][ny][nx]   conserved (rho, Mx, My, Mz, E)        (Sec. 3, q)
 *      W  [5][nz][ny][nx]   primitive (rho, vx, vy, vz, P)
 *      bx [nz][ny][nx+1], by [nz][ny+1][nx], bz [nz+1][ny][nx]
 *                           face-centred field; face index f is the low face
 *                           of zone f, the last face is the high boundary face
 *      B  [3][nz][ny][nx]   zone-centred field = face averages (Step 11)
 *  - Units absorb 4 pi (Sec. 3): P* = P + |B|^2/2.
 *  - Every call returns an int status (WB_OK = 0 or one of WB_ERR_*); details
 *    of the last failure on a handle are in wb_last_error().  No C++
 *    exception crosses this boundary.
 *  - Memory ownership: the caller allocates the device workspace (size from
 *    wb_grid_bytes) and keeps it alive until wb_grid_destroy; the library
 *    never allocates device memory for a grid and never frees caller memory.
 *  - Streams: all device work is enqueued on the stream given at create time
 *    (a cudaStream_t passed as void*, NULL = legacy default stream).  Calls
 *    that return host-visible values (dt, totals, t_out, counters) synchronise
 *    that stream; wb_advance without t_out does not.
 *  - A handle is not thread-safe; distinct handles are independent.
 */
#ifndef WOMBAT_H
#define WOMBAT_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define WB_OK 0
#define WB_ERR_INVALID 1     /* bad argument or descriptor */
#define WB_ERR_NOMEM 2       /* workspace smaller than wb_grid_bytes() */
#define WB_ERR_CUDA 3        /* a CUDA runtime call failed */
#define WB_ERR_UNPHYSICAL 4  /* rho <= 0, P <= 0 or non-finite state met */
#define WB_ERR_TIMEOUT 5     /* a bounded device wait ran out */

#define WB_BC_PERIODIC 0
#define WB_BC_OUTFLOW 1      /* zero-gradient copy of the nearest zone; on the high side the
                                boundary face is a copy of the last owned face, and the
                                last zone's field averages that copy (Step 11), so a read
                                followed by a load gives the same state */

/* Grid of equal patches (Sec. "Domain Decomposition": a Patch is a
 * self-contained sub-grid with its own 5 boundary zones).
 *  n[d]        global interior zones per axis.  n[2] = 1 with one patch
 *              along z and periodic z is the 2D problem (Sec. "MHD in Two
 *              Dimensions"): it is stored as one z plane (z stride 0), so z
 *              differences vanish exactly and the z sweep is one face per
 *              column; the zones equal those of the 11-plane 3D storage
 *              (outflow z) bit for bit.
 *  patches[d]  patches per axis; n[d] must be a multiple of patches[d]
 *  length[d]   box size; dx_d = length[d] / n[d]
 *  gamma       adiabatic index, 1 < gamma <= 2 (Sec. 3)
 *  cfl         Courant number of the time step
 *  bc[d]       WB_BC_PERIODIC or WB_BC_OUTFLOW
 *  eps[7]      entropy-fix parameters of Q_k (App. A), 0 <= eps < 0.5, waves
 *              ordered (v-cf, v-ca, v-cs, v, v+cs, v+ca, v+cf)
 *  sweby_beta  SWEBY limiter parameter, 1 <= beta <= 2 (1 = minmod)
 *  rho_floor, p_floor  floors applied to the updated state (App. A)
 *  batch_patches  patches processed together per pipeline pass (0 = all)
 *  prot_rho, prot_p  protection floors of App. A (>= 0; both 0 = off).  With
 *              a floor set, a face takes the HLL flux (App. A, Eqs. for the
 *              HLL u-bar, b+ and b-) when a zone state next to it, or an
 *              intermediate state of its linearised Riemann problem
 *              w_L + sum_{j<=k} alpha_j r_j, has rho < prot_rho or
 *              P < prot_p.  Independently of the floors, a face whose Roe
 *              state has no real sound speed always takes the HLL flux.
 *  dt_lag      0: each step's dt comes from its start state; 1: from the
 *              previous step's start state (the paper delays the dt
 *              reduction by one step to overlap it with work, Sec. on the
 *              MPI-RMA engine); the first two steps use the loaded state.
 *  keep_stages 0 (default): the corrector fluxes, the half-step reference
 *              EMF and the corrector corner EMFs reuse the arrays of their
 *              predictor counterparts, whose last reader has run by then
 *              (54 doubles of workspace per padded zone and patch of a pass);
 *              1: every intermediate of the step keeps its own array (81),
 *              so that wb_debug_stage can also return the predictor fluxes.
 *              Batches and pools ignore it (they always reuse). */
typedef struct wb_desc {
  int n[3];
  int patches[3];
  double length[3];
  double gamma;
  double cfl;
  int bc[3];
  double eps[7];
  double sweby_beta;
  double rho_floor;
  double p_floor;
  int batch_patches;
  double prot_rho;
  double prot_p;
  int dt_lag;
  int keep_stages;
} wb_desc;

typedef struct wb_counters_t {
  long long steps;          /* steps taken since load */
  long long floor_hits;     /* zones where a floor was applied */
  long long unphysical;     /* updated zones found non-finite or with rho <= 0 */
  double t;                 /* simulated time since load */
  double last_dt;           /* dt of the last step */
  long long hll_faces;      /* interior faces (the low faces of interior
                               zones, per predictor and per corrector sweep)
                               whose flux came from the HLL fallback */
} wb_counters_t;

typedef struct wb_grid wb_grid;

/* Fill *d with the defaults used by this library: gamma 5/3, cfl 0.8,
 * periodic, eps = (0.1, 0, 0.1, 0, 0.1, 0, 0.1), sweby 1, floors 1e-20. */
void wb_desc_default(wb_desc* d, int nx, int ny, int nz);

/* Device workspace bytes a grid with descriptor d needs (state, one step's
 * intermediates for batch_patches patches, staging, reductions). */
int wb_grid_bytes(const wb_desc* d, size_t* bytes);

/* Create a grid on the current CUDA device inside caller-owned device memory
 * dev_mem of at least wb_grid_bytes() bytes (256-byte aligned).  stream is a
 * cudaStream_t (borrowed).  The state is undefined until a load call. */
int wb_grid_create(const wb_desc* d, void* dev_mem, size_t bytes, void* stream,
                   wb_grid** out);
int wb_grid_destroy(wb_grid* g);

/* Load conserved U and faces bx, by, bz (layouts above).  on_device != 0:
 * the pointers are device memory, else host memory.  A host array in
 * page-locked memory the GPU can address (cudaHostAlloc, cudaHostRegister)
 * is read in place by the scatter kernel over the CPU-GPU link; any other
 * host array goes through a staging copy.  The call synchronises the stream.
 * The zone field is set to the face averages; the high boundary face of
 * each axis is taken from the ghost fill (periodic: face 0). */
int wb_load_state(wb_grid* g, const double* U, const double* bx, const double* by,
                  const double* bz, int on_device);
/* Same with primitive W = (rho, v, P); E from Eq. totenergy on the device. */
int wb_load_primitive(wb_grid* g, const double* W, const double* bx, const double* by,
                      const double* bz, int on_device);

/* CFL time step of the current state: dt = cfl / max over zones of
 * sum_d (|v_d| + c_f,d) / dx_d, c_f,d the fast speed along d (Sec. 3). */
int wb_compute_dt(wb_grid* g, double* dt);

/* Advance nsteps CTU+CT steps, each with the CFL dt of its start state,
 * clipped so that the time since load does not pass t_end (t_end <= 0: no
 * limit; steps past t_end do nothing).  The step that reaches t_end lands
 * on it exactly, and a step within 1e-10 of a CFL step of t_end is
 * stretched to it.  With t_end > 0 the call reads the device time back
 * every 64 steps (host synchronisation) and stops launching once t_end is
 * reached.  If t_out != NULL the stream is synchronised, *t_out receives
 * the time since load and an unphysical state met during these steps
 * returns WB_ERR_UNPHYSICAL. */
int wb_advance(wb_grid* g, int nsteps, double t_end, double* t_out);

/* Read back the state (any pointer may be NULL); on_device as for load
 * (page-locked host arrays are written in place by the gather kernel).
 * With host arrays the call synchronises the stream. */
int wb_read_state(wb_grid* g, double* U, double* bx, double* by, double* bz, double* B,
                  int on_device);

/* Conserved totals times zone volume: rho, Mx, My, Mz, E over zones and
 * bx, by, bz over owned faces (the low face of each zone).  Compensated
 * (Neumaier) sums in a fixed-order reduction on the device: the same state
 * gives the same totals bit for bit.  Synchronises the stream. */
int wb_conserved_totals(wb_grid* g, double tot[8]);
/* max over zones of |div b| with the face differences of Step 11. */
int wb_divb_max(wb_grid* g, double* divb);
int wb_counters(wb_grid* g, wb_counters_t* c);
const char* wb_last_error(const wb_grid* g);

/* Stage dump of the last step (debugging and parity tests): which = 0..2
 * predictor fluxes F, G, H (only for a grid created with keep_stages = 1;
 * WB_ERR_INVALID otherwise, the corrector has overwritten them); 3..5
 * corrector fluxes; 6..8 b^{n+1/2}; 9..11 q^{n+1/2}_x,y,z -- same layouts as
 * the oracle's dump (single patch only).  Copies to host memory out (cap
 * doubles); *written = doubles written. */
int wb_debug_stage(wb_grid* g, int which, double* out, long long cap, long long* written);

/* Kernel timing of the MHDTVD sweep launches (Steps 1, 6, 7): enable != 0
 * starts recording CUDA events around every sweep launch on the grid's stream
 * (at most 8192 launches; later ones are not recorded); enable == 0 stops.
 * wb_profile_read synchronises the stream and returns the summed duration in
 * milliseconds and the number of recorded launches since the last enable. */
int wb_profile_sweeps(wb_grid* g, int enable);
int wb_profile_read(wb_grid* g, double* sweep_ms, long long* launches);

/* One CTU+CT step of a single small box that allocates no device memory.
 * The paper has no counterpart.  Some callers cannot call cudaMalloc: a
 * plug-in inside a host application that owns every device allocation, an
 * embedding that is handed device buffers and nothing else, or a real-time
 * loop in which cudaMalloc's implicit device synchronisation is not allowed.
 * They cannot give wb_grid_create a workspace, so this entry point keeps one
 * step's intermediates in a static device array of 24 MiB inside this
 * library (held by every GPU that loads the library until process exit).  A
 * box needs about 520 (nx+10)(ny+10)(nz+10) + 8 (nx+1)(ny+1)(nz+1) bytes of
 * it (state, one step's intermediates with keep_stages = 0, reductions): a
 * cube of 26^3 interior zones fits, 27^3 does not; a box that does not fit
 * returns WB_ERR_INVALID with a message in wb_noalloc_last_error().
 *  d        descriptor of one box: patches must be (1,1,1); batch_patches is
 *           ignored
 *  U, bx, by, bz          device input state (layouts above)
 *  U_out, bx_out, by_out, bz_out   device outputs after one step with the
 *           CFL dt of the input (same layouts; may alias nothing else)
 *  dt_out   device double receiving the dt used (may be NULL)
 *  stream   cudaStream_t on which the work is enqueued; the call does not
 *           synchronise and does not report unphysical states (they show as
 *           non-finite outputs).
 * The first call on a device looks up the array's device address with
 * cudaGetSymbolAddress (a host-side set-up done once per device); make that
 * first call before any stream capture.  Every call on a device shares the
 * one array and finds the previous call's contents in it (the call clears
 * what must start at zero): calls whose GPU work overlaps (other streams,
 * other threads) race and corrupt each other's results, so serialise them on
 * one stream.  wb_noalloc_last_error returns the message of the calling
 * thread's last failed call (valid until that thread's next call). */
int wb_step_noalloc(const wb_desc* d, const double* U, const double* bx, const double* by,
                    const double* bz, double* U_out, double* bx_out, double* by_out,
                    double* bz_out, double* dt_out, void* stream);
const char* wb_noalloc_last_error(void);

/* ---- batching: many independent boxes in one persistent kernel ----
 * A batch holds nbox independent single-patch boxes (sizes may differ; every
 * box must share gamma, cfl, eps, sweby and floors).  One wb_batch_advance
 * launches one persistent kernel that advances every box with steps left by
 * up to nsteps CTU+CT steps, each box with its own CFL dt: thread blocks take
 * chunks of work items (pencil segments, zones, faces, edges) of all boxes
 * from a device work counter, and a bounded grid-wide barrier separates the
 * stages of a step.  The state of all boxes stays resident; the step's
 * intermediates are shared by workspace groups of boxes whose combined
 * workspace fits work_budget bytes (0 = 64 GiB).  Only boxes with steps
 * granted by wb_batch_set_steps are grouped (all resident boxes while none
 * has any), so a launch does no stage work for the others; a change of that
 * set regroups the batch before the next launch (and re-captures its
 * graph).  Boxes are periodic or outflow on their own; patches must be
 * (1,1,1).
 * wb_batch_bytes / wb_batch_create: caller-owned device memory as for grids.
 * wb_batch_load: as wb_load_state / wb_load_primitive for one box.
 * wb_batch_set_steps: steps left for one box (box = -1: all boxes); a box with
 * no steps left is skipped by wb_batch_advance.
 * wb_batch_advance: one persistent launch of nsteps steps; use_graph != 0
 * replays it from a captured CUDA graph (captured on first use per nsteps).
 * Synchronises the stream; returns WB_ERR_TIMEOUT if a barrier wait ran out.
 * wb_batch_autotune: times trial_steps real steps per candidate segment
 * length and blocks per SM in each form (below), keeps the fastest (cached
 * per box-size mix).
 * wb_batch_config: set them explicitly (0 = keep); barrier_budget_cycles is
 * the per-barrier wait limit in SM clock cycles (default 20 s worth).
 * wb_batch_stage_timer: on != 0 zeroes and starts the per-stage timer (one
 * block stamps the GPU global timer at the barrier closing every stage), 0
 * stops it; either drops a captured graph.  wb_batch_stage_times copies up to
 * n accumulated stage times in milliseconds, in the order: dt, predictor
 * sweeps (Step 1), reference EMF (2), images of both, corner EMFs (3), their
 * images, half CT (4), its images, transverse states (5, 7), their images,
 * corrector sweeps (6, 7), their images, half-step EMF (8), its images,
 * corner EMFs (9), their images, final CT (11), update (10), ghost fill;
 * *count = the number of stages (19).  The image stages copy periodic
 * images of intermediates for boxes periodic on every axis, whose other
 * stages then cover the interior only.  It synchronises the stream.
 * wb_batch_set_form: how wb_batch_advance runs the stages.
 * WB_BATCH_PERSISTENT (the default): the one persistent cooperative launch
 * above.  WB_BATCH_STAGED: one ordinary launch per stage of each step over
 * all boxes of a workspace group (the same work lists and results bit for
 * bit), each stage class compiled into its own kernel so that the zone
 * stages run with their own occupancy; no grid barrier, so no
 * WB_ERR_TIMEOUT.  With the stage timer on, the staged form times every
 * stage but dt.  Drops a captured graph.  wb_batch_autotune tries both forms
 * and keeps the faster; wb_batch_get_form reports the current one. */
#define WB_BATCH_PERSISTENT 0
#define WB_BATCH_STAGED 1
typedef struct wb_batch wb_batch;
int wb_batch_bytes(int nbox, const wb_desc* descs, size_t work_budget, size_t* bytes);
int wb_batch_create(int nbox, const wb_desc* descs, size_t work_budget, void* dev_mem,
                    size_t bytes, void* stream, wb_batch** out);
int wb_batch_destroy(wb_batch* b);
int wb_batch_load(wb_batch* b, int box, const double* U, const double* bx, const double* by,
                  const double* bz, int on_device, int primitive);
int wb_batch_set_steps(wb_batch* b, int box, int nsteps);
int wb_batch_advance(wb_batch* b, int nsteps, int use_graph);
int wb_batch_read(wb_batch* b, int box, double* U, double* bx, double* by, double* bz, double* B,
                  int on_device);
int wb_batch_counters(wb_batch* b, int box, wb_counters_t* c);
int wb_batch_autotune(wb_batch* b, int trial_steps, double* best_ms);
int wb_batch_config(wb_batch* b, int seg_len, int blocks_per_sm, long long barrier_budget_cycles);
int wb_batch_get_config(wb_batch* b, int* seg_len, int* blocks_per_sm, int* groups);
int wb_batch_stage_timer(wb_batch* b, int on);
int wb_batch_stage_times(wb_batch* b, double* ms, int n, int* count);
int wb_batch_set_form(wb_batch* b, int form);
int wb_batch_get_form(wb_batch* b, int* form);
const char* wb_batch_last_error(const wb_batch* b);

/* ---- serving: a batch as a pool boxes join and leave between launches ----
 * wb_pool_create makes an empty batch with a state region of state_bytes
 * (the HBM budget for resident runs), a shared workspace of work_bytes, up to
 * max_boxes boxes and box edges up to max_n; physics (gamma, cfl, eps, sweby,
 * floors) come from *physics and every admitted box must match them.
 * wb_pool_admit places one box (state allocated first-fit in the region) and
 * returns its slot in *box, or WB_ERR_NOMEM when the state region, the
 * workspace or the slots cannot hold it; wb_pool_release frees a slot.  The
 * wb_batch_* calls (load, set_steps, advance, read, counters) work on slots;
 * workspace groups are rebuilt before the next advance after any change.
 * wb_batch_steps_left copies the steps left of every slot (max_boxes ints).
 * wb_pool_free_bytes reports the largest free block and the total free state
 * bytes. */
int wb_pool_bytes(size_t state_bytes, size_t work_bytes, int max_boxes, int max_n, size_t* bytes);
int wb_pool_create(const wb_desc* physics, size_t state_bytes, size_t work_bytes, int max_boxes,
                   int max_n, void* dev_mem, size_t bytes, void* stream, wb_batch** out);
int wb_pool_admit(wb_batch* b, const wb_desc* d, int* box);
int wb_pool_release(wb_batch* b, int box);
int wb_pool_free_bytes(wb_batch* b, size_t* largest, size_t* total);
int wb_batch_steps_left(wb_batch* b, int* out);

/* Self-test of the library's FP64 reciprocal and reciprocal-square-root
 * helpers (PTX approximations refined by a third-order correction) against
 * the CUDA library division and rsqrt on n inputs spread over [1e-300, 1e300]:
 * worst[0] = max |rcp(x) x - 1|, worst[1] = max |rsqrt_ours / rsqrt_cuda - 1|.
 * Uses the grid's reduction words; synchronises the grid's stream. */
int wb_selftest_math(wb_grid* g, int n, double worst[2]);

/* Self-test of the integer-pipe helpers the kernels use in place of FP64
 * compares and sign operations (tests and edits on the IEEE bit patterns;
 * each FP64 compare would take an FP64-pipe issue slot): counts[h] = the
 * number of n inputs on which helper h disagrees with its FP64 definition,
 * for h = 0 zero test (x == 0), 1 exact doubling (x + x), 2 order (a < b),
 * 3 signal-rate max key, 4 x > 0 and finite, 5 x < 0, 6 positive normal,
 * 7 |a| < |b|, 8 minmod, 9 halving (x / 2 for |x| >= 2^-1021), 10 |x| and
 * 11 -x (not NaN), 12 a <= b for a, b >= 0, 13 x below a finite floor >= 0,
 * 14 finiteness.  The inputs: every pair of 16 special values (signed
 * zeros, subnormals, the ends of the normal range, infinities, NaN), then
 * random bit patterns with independent, adjacent, opposite or equal
 * partners.  Uses the grid's reduction words; synchronises the grid's
 * stream.  All counts are 0 for a correct build. */
#define WB_BITS_TESTS 15
int wb_selftest_bits(wb_grid* g, int n, long long counts[WB_BITS_TESTS]);

/* Checked build (the library compiled with -DWB_CHECKED; a substitute for a
 * device memory checker): every zone index a kernel forms, and the stencil
 * neighbours of each stage, are tested against the padded storage of a
 * patch; a bad index sets a check word and the access is redirected inside
 * the array.  wb_check_flags synchronises the device, returns the check words
 * of every translation unit OR-ed in *flags (0 = no bad index since the last
 * call) and clears them; wb_check_selftest forms one out-of-range index in a
 * probe kernel that accesses no memory and reports in *detected whether it
 * was flagged.  In an unchecked build both return WB_ERR_INVALID with 0. */
int wb_check_flags(unsigned* flags);
int wb_check_selftest(int* detected);

/* FP64 pipe probe: runs a dependent-free DFMA loop on every SM of the
 * current device and returns the achieved FP64 FLOP/s (FMA = 2 flops). */
int wb_measure_fp64_peak(void* stream, double* flops);

#ifdef __cplusplus
}
#endif
#endif
