/*
 * TEST INFRASTRUCTURE ONLY -- plain, slow FP64 CPU oracle of the WOMBAT
 * per-patch ideal-MHD step (Mendygral et al. 2017, arXiv:1701.07452).
 *
 * Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may
 * load this library.  It shares no code with the CUDA path.
 *
 * Scheme: MHDTVD modified flux (Appendix A, Eqs. for u-bar, f, beta, alpha,
 * gamma, g, g-tilde, Q) inside the 3D CTU+CT 6-solve integrator
 * (Sec. "MHD in Three Dimensions", Steps 1-11), 5 ghost zones, one ghost
 * fill per step.  State: zone-centred (rho, M, E, B) and face-centred b.
 *
 * Host arrays (all row-major, x fastest):
 *   U  [5][nz][ny][nx]  (rho, Mx, My, Mz, E)
 *   bx [nz][ny][nx+1], by [nz][ny+1][nx], bz [nz+1][ny][nx]
 *   B  [3][nz][ny][nx]  zone-centred field (read only)
 * Return codes: 0 ok, 1 invalid argument, 4 unphysical state met.
 * HLL flux (App. A): faces whose Roe state has no real sound speed take the
 * HLL flux; with protection floors set (> 0), so do faces where a zone state
 * or an intermediate state of the linearised Riemann problem has
 * rho < prot_rho or P < prot_p.
 */
#ifndef MHD_ORACLE_H
#define MHD_ORACLE_H
#ifdef __cplusplus
extern "C" {
#endif

typedef struct or_grid or_grid;

/* bc[d]: 0 periodic, 1 outflow (zero-gradient). eps[7]: entropy-fix
 * parameters of Q_k for waves k=1..7 ordered (v-cf, v-ca, v-cs, v, v+cs,
 * v+ca, v+cf). sweby: limiter parameter (1 = minmod). */
or_grid* or_create(int nx, int ny, int nz, double lx, double ly, double lz,
                   double gamma, double cfl, const int bc[3], const double eps[7],
                   double sweby, double rho_floor, double p_floor);
void or_destroy(or_grid* g);
int or_load(or_grid* g, const double* U, const double* bx, const double* by,
            const double* bz);
/* Primitive load: W[5][nz][ny][nx] = (rho, vx, vy, vz, P); the zone field
 * is the face average and E follows Eq. totenergy. */
int or_load_primitive(or_grid* g, const double* W, const double* bx, const double* by,
                      const double* bz);
int or_read(const or_grid* g, double* U, double* bx, double* by, double* bz,
            double* B);
/* CFL time step from the current state: C_cfl / max over interior zones of
 * sum_d (|v_d| + c_f,d) / dx_d (the paper gives no formula; reading R3). */
double or_compute_dt(const or_grid* g);
/* One CTU+CT step with the given dt. Returns 0 or 4 (unphysical). */
int or_step(or_grid* g, double dt);
/* Conserved totals x cell volume: rho, Mx, My, Mz, E, bx, by, bz. */
int or_totals(const or_grid* g, double tot[8]);
double or_divb_max(const or_grid* g);
/* floor hits, unphysical zones, and the interior faces (per predictor and
 * corrector sweep) that took the HLL flux, accumulated over all steps */
int or_counters(const or_grid* g, long long out[3]);
/* Protection floors (>= 0; 0 and 0, the default, turn protection off). */
int or_set_protection(or_grid* g, double prot_rho, double prot_p);
/* Test ablation of the div B source term of Steps 5 and 7: S is multiplied by
 * s (1 = the scheme; 0 drops the term, -1 flips its sign). */
int or_set_source_scale(or_grid* g, double s);
int or_set_threads(int n);

/* Stage dump: copy an intermediate of the last step, on interior cells
 * (faces [0, n] along the array's own normal), into out.  which:
 *   0..2  predictor flux F/G/H (8 comps each, layout [8][..])
 *   3..5  corrector fluxes (starred F, G, H)
 *   6..8  b^{n+1/2} x/y/z faces
 *   9..11 q^{n+1/2}_x/y/z (8 comps, interior cells)
 * Returns number of doubles written. */
long long or_stage(const or_grid* g, int which, double* out, long long cap);

/* ---- single-interface eigen-system (pins) ----
 * qL, qR: conserved 8-vectors in the sweep frame (rho, Mn, Mt1, Mt2, E,
 * Bn, Bt1, Bt2) with zone-centred B; b: face normal field.
 * Outputs (7-variable system ordered rho, Mn, Mt1, Mt2, Bt1, Bt2, E):
 * lam[7] eigenvalues, alpha[7] = L.dq, R[7*7] right eigenvectors as
 * columns (R[m*7+k] = component m of R_k), L[7*7] left eigenvectors as
 * rows (L[k*7+m]). Returns 0, or 4 if the Roe state is unphysical. */
int or_face_eigen(const double qL[8], const double qR[8], double b, double gamma,
                  double lam[7], double alpha[7], double R[49], double L[49]);

/* One MHDTVD flux pencil (pins): ncell cells (sweep frame 8-vectors,
 * row-major [ncell][8]) and ncell+1 face fields bface (face f between cells
 * f-1 and f).  Fluxes at faces [2, ncell-2] are written to out[(ncell+1)][7]
 * (other faces untouched).  Returns the number of those faces that took the
 * HLL flux, or -1 for invalid arguments. */
int or_flux_pencil(int ncell, const double* cells, const double* bface,
                   double dtdx, double dx_over_2dt, double gamma, const double eps[7],
                   double sweby, double prot_rho, double prot_p, double* out);

/* Independent 1D MHDTVD (RJ95-type) step on a line of n cells, periodic
 * (outflow = 0) or zero-gradient (outflow = 1) ends: q[n][8] conserved
 * sweep-frame vectors (B_n constant = b), updated in place by
 * q -= dt/dx (u_{i+1/2} - u_{i-1/2}) for all components.  Returns the number
 * of HLL faces, or -1 for invalid arguments. */
int or_step_1d(int n, double* q, double b, double dt, double dx, double gamma,
               const double eps[7], double sweby, double prot_rho, double prot_p, int outflow);

/* Operation counting (only in the build with -DORACLE_COUNT_FLOPS): per
 * section of the step (flop_count.h), the FP64 operations counted and the
 * units evaluated since the last or_flop_reset.  Returns the number of
 * sections written, or -1 in the ordinary build. */
int or_flop_report(long long* flops, long long* units, int cap);
void or_flop_reset(void);

#ifdef __cplusplus
}
#endif
#endif
