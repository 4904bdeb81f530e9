/*
 * jz.h -- C ABI of the GB300 stage-residual / Runge-Kutta library for the
 * JAZzY-style compressible LES solver (arXiv 2003.08746).
 *
 * The library advances the five conserved variables Q = [rho, rho u, rho v,
 * rho w, e] of the filtered Navier-Stokes equations (paper Sec. "Large Eddy
 * Simulation Formulation", eqs. les, vec-les, con-prop, rhs) on one
 * structured curvilinear (i, j, k) grid on one GPU, with the explicit
 * 5-stage Runge-Kutta scheme of Algorithm 2.
 *
 * Conventions common to every entry point
 *  - Every function returns an int status: JZ_OK (0) or a negative JZ_ERR_*
 *    code.  No function aborts the process.  jz_last_error() gives a
 *    thread-local message for the last failure on the calling thread.
 *  - Arrays passed in or out are FP64, structure-of-arrays, C order
 *    [var][nk][nj][ni] with i fastest, no ghost points.  N = ni * nj * nk.
 *  - Array pointers may be host or device pointers (CUDA unified
 *    addressing decides).  The caller owns them; the library never keeps
 *    them after the call returns.  Host transfers finish before the call
 *    returns; device transfers are ordered on the solver's stream.
 *  - Handles (jz_grid, jz_solver) are owned by the library and freed by
 *    the matching destroy call.  A grid must outlive the solvers built on it.
 *  - All device work of a solver is issued on the stream given to
 *    jz_create (NULL = legacy default stream).
 *  - Non-dimensionalisation: rho_inf = a_inf = T_inf = 1, p_inf = 1/gamma,
 *    lengths in jet diameters; mu_ref = mach_ref / Re.
 */
#ifndef JZ_H
#define JZ_H

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define JZ_OK             0
#define JZ_ERR_ARG       -1   /* invalid argument (sizes, pointers, flags)   */
#define JZ_ERR_CUDA      -2   /* a CUDA runtime call failed                  */
#define JZ_ERR_OOM       -3   /* device memory allocation failed             */
#define JZ_ERR_NONFINITE -4   /* NaN/Inf or non-positive rho or p in state   */
#define JZ_ERR_STATE     -5   /* call out of order (e.g. no metrics/state)   */

/* ---- grid topologies --------------------------------------------------- */
/* Triply periodic box: every node is advanced by the stencil; ghost points
 * are periodic images (coordinates shifted by the period vectors). */
#define JZ_TOPO_PERIODIC 1
/* Cylindrical jet grid (paper Sec. LES Formulation, boundary conditions):
 * i axial (i = 0 entrance, i = ni-1 exit), j radial (j = 0 on the jet axis,
 * j = nj-1 far field), k azimuthal with nk unique periodic points (nk even).
 * Nodes 1 <= i <= ni-2, 1 <= j <= nj-2 are advanced by the stencil; the
 * others are set by the boundary conditions after every stage. */
#define JZ_TOPO_JET      2

/* ---- precision forms --------------------------------------------------- */
#define JZ_PREC_FP64      0   /* every operation in FP64                      */
#define JZ_PREC_FP32FLUX  1   /* fluxes, dissipation, SGS in FP32; state,
                                 stage combination and totals in FP64        */
#define JZ_PREC_FP64PAIR  2   /* FP64 state, stage combination and totals;
                                 fluxes, dissipation, SGS in double-float
                                 arithmetic (pairs of FP32, ~48 bits) on the
                                 FP32 pipes: the FP64 form's results within
                                 its 1e-12 parity bar at FP32-pipe rates.
                                 488 bytes per padded node: 32 more than
                                 JZ_PREC_FP64 (pair copies of the metrics
                                 and state, 152; no stored face fluxes, -120).
                                 jz_adjoint_step on such a solver advances
                                 the states, regenerates the intermediates and
                                 runs the transposed passes in pair arithmetic
                                 (the running adjoint and the boundary-
                                 condition adjoints in FP64).                 */

#define JZ_N_MODES 8          /* azimuthal forcing modes m = 0..7            */
#define JZ_N_FREQ  4          /* forcing frequencies (Strouhal numbers)      */

typedef struct jz_grid jz_grid;
typedef struct jz_solver jz_solver;

/* Physical and numerical parameters (plain values).  Defaults used by the
 * workloads: gamma 1.4, Pr 0.72, Pr_sgs 0.9 (paper eqs. q_mod, kappa_sgs),
 * S1_K 110.4 K (eq. sutherland), T_ref_K 288.15, C_s 0.18, kappa2 1/4,
 * kappa4 1/64, sigma 2/3, cfl 0.5. */
typedef struct jz_params {
    double gamma, Pr, Pr_sgs;
    double Re;          /* Reynolds number built on U_ref = mach_ref * a_inf  */
    double mach_ref;
    double T_ref_K;     /* dimensional ambient temperature (Sutherland)      */
    double S1_K;        /* Sutherland constant in kelvin                      */
    double C_s;         /* Smagorinsky constant (0: no eddy viscosity)        */
    double kappa2, kappa4, sigma;   /* Turkel-Vatsa dissipation constants     */
    double cfl;         /* time step = cfl / max((l_xi + l_eta + l_zeta)/V)   */
    double dt_fixed;    /* > 0: use this fixed time step instead              */
    /* jet entrance (JZ_TOPO_JET only) */
    double jet_mach;    /* U_j / a_inf                                        */
    double theta_mom;   /* momentum thickness of the tanh profile (D)         */
    double forcing_amp[JZ_N_MODES * JZ_N_FREQ];   /* A[m][f], m-major          */
    double forcing_phi[JZ_N_MODES * JZ_N_FREQ];   /* azimuthal phase phi[m][f] */
    double forcing_psi[JZ_N_MODES * JZ_N_FREQ];   /* temporal phase psi[m][f]  */
    double strouhal[JZ_N_FREQ];
    int precision;      /* JZ_PREC_FP64, JZ_PREC_FP32FLUX or JZ_PREC_FP64PAIR */
} jz_params;

/* Per-call statistics returned by jz_rk_step. */
typedef struct jz_step_stats {
    double t;           /* time after the last step                           */
    double dt;          /* time step of the last step                         */
    double res_l2;      /* RMS over advanced nodes of RHS_rho at stage 1 of the last step */
    double totals[5];   /* sum over all nodes of Q_m V (conservation totals)  */
    double min_rho, min_p;
    long long steps;    /* steps taken since jz_set_state                      */
} jz_step_stats;

/* Message of the last failure on this thread ("" if none).  Never NULL. */
const char* jz_last_error(void);

/* Library ABI version (increments when a signature changes). */
int jz_version(void);

/* Create a grid from node coordinates (paper Algorithm 2: Read(Mesh)).
 *  xyz     [3][nk][nj][ni] Cartesian node coordinates, host or device
 *          (device coordinates are padded directly, host ones through a
 *          temporary device copy of the same size).
 *  period  [3][3] shift vectors of the i, j, k periods (JZ_TOPO_PERIODIC),
 *          host memory; may be NULL for JZ_TOPO_JET (ignored there).
 *  Sizes: JZ_TOPO_PERIODIC needs ni, nj, nk >= 1; JZ_TOPO_JET needs ni >= 4,
 *  nj >= 4 and an even nk >= 4.  Ghost coordinates are built here (two
 *  layers, paper Sec. "Parallel Implementation Aspects"): periodic images;
 *  on the jet the azimuthal wrap, the across-axis mirror (i, m, k + nk/2)
 *  and linear extrapolation beyond the far field and the entrance/exit.
 *  Returns JZ_ERR_ARG on bad sizes/pointers, JZ_ERR_OOM, JZ_ERR_CUDA. */
int jz_create_grid(int ni, int nj, int nk, const double* xyz, const double* period,
                   int topology, jz_grid** out);

/* Free the grid.  JZ_ERR_STATE (and nothing freed) while solvers created on it
 * are alive: destroy them first. */
int jz_destroy_grid(jz_grid* g);

/* Compute the metrics of the curvilinear transformation (Algorithm 2:
 * Calc(Jacob., Metric)): the area vectors S^xi = (xi_x, xi_y, xi_z)/J,
 * S^eta, S^zeta in the symmetric conservative (Thomas-Lombard) form built
 * from the centred index difference, and V = 1/J.  Runs on the default
 * stream and synchronises.  Returns JZ_ERR_ARG if V <= 0 on a node the
 * stencil advances (left-handed or degenerate grid). */
int jz_compute_metrics(jz_grid* g);

/* Copy the metrics to out [10][N] (host or device): S^xi_{x,y,z},
 * S^eta_{x,y,z}, S^zeta_{x,y,z}, V.  JZ_ERR_STATE before jz_compute_metrics
 * and on a compact grid. */
int jz_get_metrics(const jz_grid* g, double* out);

/* Compact a grid for the FP32-flux form (no counterpart in the paper; it
 * lets one GPU hold the paper's largest mesh, 1700 x 1700 x 361 points).
 * The metrics are converted to FP32 once and kept by the grid (S^xi, S^eta,
 * S^zeta, V, 1/V, V^(1/3): 48 bytes per padded node), the far-field normals and the
 * entrance-plane coordinates stay in FP64 surface arrays, and the FP64
 * coordinates and metrics (144 bytes per padded node) are freed.
 * Afterwards: FP32-flux solvers use the grid's FP32 metrics instead of their
 * own copy; the CFL rate of the first step after jz_set_state and the
 * conservation totals use the FP32 metrics widened to FP64 (relative
 * differences ~1e-7 from a full grid); FP64 solvers, jz_get_metrics and
 * jz_residual_noalloc refuse the grid (JZ_ERR_STATE).  Idempotent.
 * Errors: JZ_ERR_STATE (metrics not computed; a solver still uses the grid),
 * JZ_ERR_OOM, JZ_ERR_CUDA.  Synchronous (legacy default stream). */
int jz_grid_compact(jz_grid* g);

/* Create a solver on a grid with computed metrics (Algorithm 2: Read(Input)).
 *  stream  a cudaStream_t (may be NULL).  Allocates the state and the
 *  scratch arrays of the chosen precision form on the device. */
int jz_create(jz_grid* g, const jz_params* p, void* stream, jz_solver** out);
int jz_destroy(jz_solver* s);

/* Set the state Q (Algorithm 2: Calc(I.C.) / restart) and time t.  q is
 * [5][N], host or device.  The state is taken as given (no boundary
 * condition is applied); ghost points are filled.  Page-locked host memory
 * is read by the packing kernel directly over the host link; other host
 * memory goes through a device staging copy.  Host input: returns when the
 * copy is done; device input: queued on the solver's stream. */
int jz_set_state(jz_solver* s, const double* q, double t);

/* Copy the current state to q [5][N], host or device (page-locked host
 * memory is written by the unpacking kernel directly).  Host output:
 * returns when the data is there; device output: queued on the stream. */
int jz_get_state(jz_solver* s, double* q);

/* One evaluation of RHS(q) of eq. vec-les (dQ/dt = -RHS) on every node the
 * stencil advances; rhs [5][N] is 0 on the other nodes.  Does not touch the
 * solver's state.  q and rhs host or device. */
int jz_residual(jz_solver* s, const double* q, double* rhs);

/* Advance nsteps time steps (Algorithm 2 main loop): for each of the 5
 * stages, Q^(l) = Q^n - alpha_l dt RHS(Q^(l-1)), alpha = (1/4, 1/6, 3/8,
 * 1/2, 1), then the boundary conditions and the ghost points.  dt is the
 * CFL step of Q^n (or dt_fixed), kept on the device.  If out is non-NULL
 * the statistics are computed and copied to it (one stream
 * synchronisation); with out == NULL nothing waits for the GPU.
 * JZ_ERR_NONFINITE if out is requested and the state holds NaN/Inf or a
 * non-positive density or pressure. */
int jz_rk_step(jz_solver* s, int nsteps, jz_step_stats* out);

/* Gradient of an observer functional with respect to the entrance-forcing
 * amplitudes by the discrete adjoint of the time stepping (FP64 form, jet
 * grid).  Starting from the solver's current state Q^0 at time t0, with the
 * forcing amplitudes forcing_amps [8 modes][4 frequencies] (host; phases and
 * Strouhal numbers from jz_params) and a time step frozen at the CFL step of
 * Q^0 (or dt_fixed),
 *   J = sum_{n=1..nsteps} dt sum_{i,k} w_ik (p~_ik(Q^n) - p_inf)^2,
 * p~ the pressure on the cylinder r = r_obs (linear in r between the
 * bracketing grid lines), w_ik = r_obs dtheta dx_i (trapezoid in x).
 * The forward sweep stores Q^n every ckpt_every steps; the reverse sweep
 * recomputes each checkpoint segment and each step's five stage states and
 * runs the transposed stage, boundary-condition and ghost-fill kernels.
 * Writes J (*J_out, host) and dJ/dA (grad_out [32], host).  The solver's
 * state and parameters are unchanged on return; device memory for the
 * checkpoints and adjoint arrays is allocated for the call.
 * Errors: JZ_ERR_ARG (FP32-flux solver, periodic grid, r_obs outside the
 * grid, bad counts), JZ_ERR_STATE (no state), JZ_ERR_OOM, JZ_ERR_CUDA. */
int jz_adjoint_step(jz_solver* s, const double* forcing_amps, int nsteps, int ckpt_every, double r_obs,
                    double* J_out, double* grad_out);

/* ---- kernel timing ---------------------------------------------------- *
 * Kernel kinds of the stage (index of the arrays below). */
#define JZ_PROF_NODAL    0   /* FP64 nodal pass: primitives, spectral radii, inviscid fluxes */
#define JZ_PROF_VISCOUS  1   /* FP64 viscous pass: gradients, SGS, viscous fluxes, sensor   */
#define JZ_PROF_FACES    2   /* dissipation face fluxes (pair form: with the RHS and update) */
#define JZ_PROF_UPDATE   3   /* RHS assembly and stage update                              */
#define JZ_PROF_BC       4   /* boundary-condition kernels                                 */
#define JZ_PROF_GHOST    5   /* ghost-point fill                                           */
#define JZ_PROF_REDUCE   6   /* CFL, time, statistics reductions                           */
#define JZ_PROF_FUSED32  7   /* fused FP32-flux stage kernel                               */
#define JZ_PROF_ADJOINT  8   /* adjoint stage kernels                                      */
#define JZ_PROF_STATS    9   /* flow-statistics sampling                                   */
#define JZ_NPROF         10

/* Turn per-kernel timing on or off.  While on, the solver records a CUDA
 * event on its stream after every kernel it launches (intervals between
 * consecutive events are the kernels' device durations). */
int jz_profile(jz_solver* s, int enable);

/* Synchronise the solver's stream and return, per kernel kind, the summed
 * device time in milliseconds (ms[JZ_NPROF], may be NULL) since the last
 * read, and the number of kernel launches (launches[JZ_NPROF], may be NULL;
 * counted whether or not timing is on).  Both are reset. */
int jz_profile_read(jz_solver* s, double* ms, long long* launches);

/* Short name of a kernel kind ("" if out of range). */
const char* jz_profile_name(int kind);

/* ---- flow statistics ------------------------------------------------------ *
 * The paper validates the jet against measurements through time statistics
 * of the axial velocity (Sec. "Validation": mean axial velocity along the
 * centreline and radial profiles at x/D = 2.5 and 5, axial-velocity rms,
 * potential-core length).  The library accumulates them on the GPU:
 *
 *   u = (rho u_x) / rho at every real node, sampled from Q^n;
 *   per node: time mean  m = (1/S) sum_s u_s  and  rms = sqrt((1/S) sum_s (u_s - m)^2)
 *   (population definitions, accumulated with Welford's update);
 *   read-out: both averaged over the azimuth k, giving [nj][ni] arrays.
 *
 * jz_stats_begin allocates 2 x N accumulators plus 2 x ni x nj outputs
 * (device, owned by the solver), zeroes them, and makes jz_rk_step add a
 * sample after every `every`-th step (steps counted since jz_set_state or
 * the snapshot; every = 0: samples only through jz_stats_sample).  Calling
 * it again restarts the statistics.  jz_stats_sample adds Q^n now.
 * jz_stats_read writes mean and rms ([nj][ni], i fastest; host or device
 * pointers, either may be NULL) and the sample count (may be NULL); it
 * synchronises the stream when a pointer is on the host.  jz_stats_end
 * frees the accumulators (also freed by jz_destroy).
 * Errors: JZ_ERR_ARG (NULL solver, every < 0, nj or nk above 65535),
 * JZ_ERR_STATE (no state set; read/sample before begin; read with no
 * sample), JZ_ERR_OOM, JZ_ERR_CUDA. */
int jz_stats_begin(jz_solver* s, int every);
int jz_stats_sample(jz_solver* s);
int jz_stats_read(jz_solver* s, double* mean, double* rms, long long* nsamples);
int jz_stats_end(jz_solver* s);

/* Host-only helpers for the statistics' stations (no GPU involved):
 * jz_station_profile: the column profile of field [nj][ni] (i fastest) at
 * axial position x0, linearly interpolated in x between the two i lines
 * that bracket it (x [ni] strictly increasing; x0 = x[i] returns column i
 * exactly); out [nj].  JZ_ERR_ARG if x0 lies outside [x[0], x[ni-1]].
 * jz_potential_core: the first axial position where the centreline mean
 * axis [ni] drops below frac * u_jet (the paper uses 95% of U_j),
 * interpolated linearly between the bracketing i lines; NaN if it never
 * drops.  Both return JZ_ERR_ARG on NULL pointers or ni < 2. */
int jz_station_profile(const double* field, const double* x, int ni, int nj, double x0, double* out);
int jz_potential_core(const double* axis, const double* x, int ni, double u_jet, double frac, double* x_core);

/* ---- arithmetic self-check -------------------------------------------------- *
 * The FP64 form computes reciprocals (1/rho, the Sutherland and pressure-sensor
 * denominators), square roots (sound speed, strain-rate magnitude) and the
 * powers x^(1/3), x^(2/3) of the anisotropic spectral-radius scaling with the
 * library's own routines: a hardware seed (reciprocal) or an FP32 seed (inverse
 * square and cube root) refined by one third-order Householder step.
 * jz_check_math runs them on 2^20 arguments spread over [1e-30, 1e30] (and 0) on
 * the current device and returns the largest relative error against IEEE
 * division (1.0/x), the CUDA math library's cbrt (x^(1/3) and cbrt(x*x)) and
 * IEEE sqrt.  No counterpart in the paper.
 * Synchronous (legacy default stream).  Errors: JZ_ERR_ARG (NULL), JZ_ERR_CUDA. */
int jz_check_math(double* rcp_max_rel, double* cbrt_max_rel, double* sqrt_max_rel);

/* ---- self-check of the pair arithmetic ----------------------------------- *
 * The paper has no counterpart: JZ_PREC_FP64PAIR computes in double-float
 * (pairs of FP32).  This call evaluates its operations on 2^20 operand sets
 * (magnitudes 2^-40 .. 2^41, both signs) against FP64 and returns the largest
 * errors in max_rel9[9]: sum (relative to |x| + |y|), product, fused
 * multiply-add (relative to |x y| + |z|), reciprocal, square root, cube-root
 * pair, the FP64 -> pair -> FP64 round trip, and the square root and
 * cube-root pair of arguments below 1e-30 (their FP32 fallbacks).
 * Synchronous; legacy default stream; allocates 72 bytes.
 * Errors: JZ_ERR_ARG (NULL), JZ_ERR_OOM, JZ_ERR_CUDA. */
int jz_check_pair(double* max_rel9);

/* ---- self-check of the bounded wait ------------------------------------ *
 * The paper has no counterpart: the FP32-flux stage kernel waits for its TMA
 * copies on mbarriers with a bounded number of polls, and if a wait runs out
 * it stops requesting copies, sets an error flag that jz_rk_step reports as
 * JZ_ERR_CUDA, and finishes (the context stays usable).  This call runs the
 * same bounded wait on an mbarrier that nothing ever arrives at: *timed_out
 * is 1 when the wait ran out and returned, and *milliseconds how long it
 * took (from clock64 at the device's nominal clock).  Synchronous; uses the
 * legacy default stream; allocates 16 bytes of device memory.
 * Errors: JZ_ERR_ARG (NULL), JZ_ERR_OOM, JZ_ERR_CUDA. */
int jz_check_wait(int* timed_out, double* milliseconds);

/* ---- snapshots (checkpoint / restart) ------------------------------------ *
 * The paper restarts long runs from stored solution files (Algorithm 2
 * starts from an initial condition or a restart file; Sec. "Parallel I/O"
 * writes them per rank through CGNS/HDF5).  Here one GPU holds the whole
 * grid, so a snapshot is one raw binary file written from the host:
 *
 *   header, 256 bytes, little-endian:
 *     char     magic[8]  = "JZSNAP01"
 *     int32    version = 1, header_bytes = 256
 *     int32    ni, nj, nk, topology, precision, flags (bit 0: rate valid)
 *     int64    steps                 steps taken since jz_set_state
 *     float64  t, dt, rate, res_sum  time, last time step, CFL rate of Q^n
 *                                    (valid if flags bit 0), last residual sum
 *     uint64   params_hash           FNV-1a 64 of the jz_params fields
 *     uint64   data_hash             FNV-1a 64 over the data's 64-bit words
 *     zero padding to 256 bytes
 *   data: Q^n as [5][nk][nj][ni] float64, i fastest (the jz_get_state layout).
 *
 * jz_save_snapshot writes the solver's Q^n, time, step count and the CFL
 * rate the next step would use (FP32-flux form), so that continuing from
 * jz_load_snapshot reproduces an uninterrupted run bit for bit.
 * jz_load_snapshot requires the same grid shape and topology and the same
 * parameters (params_hash); the rate is restored only into an FP32-flux
 * solver from an FP32-flux snapshot, otherwise the next step reduces it
 * afresh (the FP64 form always reduces it in its first stage).  The file is created
 * or truncated by save; `path` is a NUL-terminated file name.
 * Both calls synchronise the solver's stream and allocate a device staging
 * buffer [5][N] (kept by the solver) and 2 x 64 MiB of pinned host memory
 * (freed on return).
 * Errors: JZ_ERR_ARG (NULL arguments, unreadable/unwritable file, bad magic
 * or version, shape/topology/parameter mismatch, short file, data hash
 * mismatch), JZ_ERR_STATE (save without a state), JZ_ERR_OOM, JZ_ERR_CUDA. */
#define JZ_SNAPSHOT_HEADER_BYTES 256
int jz_save_snapshot(jz_solver* s, const char* path);
int jz_load_snapshot(jz_solver* s, const char* path);

/* ---- allocation-free residual ------------------------------------------- *
 * The paper has no counterpart to this entry point; it is a service for
 * callers that cannot have the library allocate device memory: code whose
 * device memory belongs to another allocator under a fixed budget, and
 * latency-critical loops that cannot absorb cudaMalloc/cudaFree (cudaFree
 * synchronises the whole device).
 *
 * Same result as jz_residual (FP64 form) for the state q on grid g, with
 * parameters p (p->precision must be JZ_PREC_FP64).  q [5][N] and rhs [5][N]
 * are caller-owned DEVICE pointers; the work is queued on `stream` (a
 * cudaStream_t, NULL = legacy default stream) and the call returns without
 * waiting for it.  No device memory is allocated: the scratch is a fixed
 * array of JZ_NOALLOC_SCRATCH_BYTES (64 MiB) inside the library, charged on
 * every device where the library's module holding it is loaded and kept
 * until the process exits -- with CUDA's lazy module loading (the default
 * since CUDA 12.2) from the first call on that device, with eager loading
 * from context creation, whether or not this entry point is used.  q, rhs
 * and the grid must live on the current device.  A grid needs
 * 256 + 47 * 8 * (padded nodes) bytes, padded nodes = round4(ni+4) *
 * (nj+4) * (nk+4) (about 178,000 padded nodes, e.g. 48 x 48 x 48 real
 * nodes); larger grids are rejected with JZ_ERR_ARG and a message giving
 * the limit.  The first call on a device looks up the scratch address (make
 * it before any stream capture).  All calls on a device share the scratch:
 * calls whose kernels overlap on the GPU race; keep them on one stream.
 * Errors: JZ_ERR_ARG (NULL/host pointers, pointers or grid on another
 * device, bad parameters, grid too large), JZ_ERR_STATE (metrics not
 * computed, compact grid), JZ_ERR_CUDA (including a CUDA error that earlier
 * work left pending, which is reported and not cleared). */
#define JZ_NOALLOC_SCRATCH_BYTES (64u * 1024u * 1024u)
int jz_residual_noalloc(const jz_grid* g, const jz_params* p, const double* q, double* rhs, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* JZ_H */
