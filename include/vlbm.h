/* vlbm.h: C interface of the B300 (sm_103a) vectorial lattice Boltzmann step library.
 *
 * The library advances the vectorial lattice Boltzmann method (VLBM) of Hosseini & Karlin,
 * "Vectorial lattice Boltzmann solver for compressible inviscid flows with generic equation of
 * state", for the compressible Euler equations dW/dt + div Q(W) = 0 (Sec. II, Eqs. 9-10) with
 * W = (rho, rho u, rho E) (Eq. 2) on a uniform D = 1 or D = 2 grid, D1Q2 / D2Q4 lattices
 * (Sec. III A, Eq. 18).  One time step is, per cell (Secs. III A, III D, III E):
 *   W = sum_i f_i; P(rho, e) and c_s^2 from the EOS (Eqs. 11-17); s_max -> link speed c and dt
 *   (Eqs. 36-37, the last step shortened onto t_end); reprojection of f from the old to the new
 *   link speed (Eqs. 38-40); shock sensor beta(x) (Eqs. 28-35); relaxation
 *   f_i <- 2 beta f_i^eq(W) + (1 - 2 beta) f_i with f_i^eq = W/(2D) + c_i.Q(W)/(2c^2) (Eqs. 20, 22);
 *   exact transport f_i(x) <- f_i(x - dt c_i) (Eq. 21).
 *
 * Conventions for every call:
 *   - Field arrays are float64, laid out [component][y][x] with x fastest (1D: ny = 1), and may be
 *     device pointers or host pointers (unified addressing decides; host memory should be pinned
 *     for asynchronous copies).  The caller owns them.  The handle owns the populations, the
 *     device scalars, the time-step history and all scratch.
 *   - Work is issued on the CUDA stream given to vlbm_create, in stream order.  Only
 *     vlbm_step (at its end), vlbm_get_time, vlbm_get_dt_history, vlbm_get_W/vlbm_get_beta with a
 *     host destination, vlbm_save_state and the timing calls synchronise with the host.
 *   - Errors are return codes; no call aborts the process.  A state with rho <= 0, c_s^2 <= 0
 *     (Eq. 14 violated) or non-finite values detected on the device is reported as
 *     VLBM_E_NONPHYSICAL by the next synchronising call; the handle then stays in that state.
 *   - A handle is not thread-safe; use one handle per stream.
 */
#ifndef VLBM_H
#define VLBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct vlbm_s* vlbm_t;

typedef enum {
  VLBM_OK = 0,
  VLBM_E_INVAL = 1,       /* invalid argument (sizes, parameters, null pointers)          */
  VLBM_E_NOMEM = 2,       /* device or host allocation failed                             */
  VLBM_E_CUDA = 3,        /* a CUDA runtime call failed                                   */
  VLBM_E_NONPHYSICAL = 4, /* rho <= 0, c_s^2 <= 0 or non-finite state (Eq. 14)            */
  VLBM_E_TIMEOUT = 5,     /* a bounded wait ran out                                       */
  VLBM_E_STATE = 6,       /* call out of order (e.g. vlbm_step before vlbm_init)          */
  VLBM_E_CHECKSUM = 7,    /* saved state failed its integrity check                       */
  VLBM_E_UNSUPPORTED = 8  /* combination not built (reported, never silently substituted) */
} vlbm_status;

/* Boundary rule per domain side (periodic pairs both sides of an axis).  Zero-gradient is the
 * edge-replicated ghost cell of Secs. IV B and IV E: every stencil access and every streamed
 * population beyond the edge reads the edge cell.  Pinned inflow (x-lo side only, paired with a
 * zero-gradient x-hi side) is the inflow boundary of Sec. IV H: the ghost cells beyond the side
 * hold a fixed state W_in (vlbm_set_inflow), whose velocity and flux every stencil reads there and
 * whose equilibrium populations (Eq. 20, at the link speed of the step) stream into the domain. */
typedef enum { VLBM_BC_PERIODIC = 0, VLBM_BC_ZEROGRAD = 1, VLBM_BC_INFLOW = 2 } vlbm_bc;

typedef struct {
  int32_t dim;        /* 1 or 2                                                             */
  int64_t nx, ny;     /* cells per axis (ny ignored and taken as 1 when dim = 1)            */
  double x0, x1;      /* domain extent along x; dx = (x1 - x0) / nx; cells are square in 2D */
  double y0, y1;      /* extent along y (informational; dy is taken equal to dx)            */
  int32_t bc[4];      /* x-lo, x-hi, y-lo, y-hi (vlbm_bc)                                   */
} vlbm_grid;

/* Equations of state of Sec. II C: ideal gas P = (gamma-1) rho e (Eq. 15); polytropic van der
 * Waals P = R rho T / (1 - b rho) - a rho^2, e = cv T - a rho (Eqs. 16-17); and, as one of the
 * generic closures P(rho, e) of Eq. (11), the van der Waals thermal relation with a temperature-
 * dependent heat capacity c_v(T) = cv + cv1 T + cv2 T^2 (cv > 0, cv1, cv2 >= 0): e = cv T +
 * cv1 T^2/2 + cv2 T^3/3 - a rho, which satisfies the consistency condition Eq. (12) for any such
 * c_v.  Its temperature T(rho, e) is found by Newton's method in FP64 on every path (FP32 storage
 * too), stopping once a step changes T by at most 1e-15 T; a state where 50 steps do not get
 * there is reported as non-physical. */
typedef enum { VLBM_EOS_IDEAL = 0, VLBM_EOS_VDW = 1, VLBM_EOS_VDW_CVT = 2 } vlbm_eos_kind;

typedef struct {
  int32_t kind;                  /* vlbm_eos_kind                                  */
  double gamma;                  /* ideal gas                                      */
  double a, b, R, cv;            /* van der Waals (gamma ignored)                  */
  double cv1, cv2;               /* VLBM_EOS_VDW_CVT: c_v(T) = cv + cv1 T + cv2 T^2 */
} vlbm_eos;

typedef enum { VLBM_FP64 = 0, VLBM_FP32_STORE = 1 } vlbm_precision;
typedef enum { VLBM_BETA_SENSOR = 0, VLBM_BETA_CONST = 1 } vlbm_beta_mode;
typedef enum { VLBM_ALGO_AUTO = 0, VLBM_ALGO_TWO_PASS = 1, VLBM_ALGO_LOOKAHEAD = 2 } vlbm_algorithm;
/* How a 2D step kernel covers the grid: VLBM_TILING_STRIP walks a CTA down a column strip with
 * ring buffers (each quantity computed once per row), VLBM_TILING_TILE computes each 32 x 16 tile
 * with its own halo.  AUTO takes strips in 2D, except tiles for FP32 storage with an ideal gas on
 * grids of fewer than 2^19 cells (measured faster there).  Both give the same results up to
 * rounding order; 1D always uses tiles.  VLBM_ALGO_AUTO takes the look-ahead form for FP32 storage and the two-pass form
 * for FP64. */
typedef enum { VLBM_TILING_AUTO = 0, VLBM_TILING_TILE = 1, VLBM_TILING_STRIP = 2 } vlbm_tiling;

typedef struct {
  double cfl;             /* target Courant number in (0, 1) (Eq. 37)                           */
  int32_t beta_mode;      /* vlbm_beta_mode: shock sensor (Sec. III D) or constant beta         */
  double beta_const;      /* constant beta in (0, 1] (Eq. 24) for VLBM_BETA_CONST                */
  double beta_min;        /* sensor floor, 0 < beta_min <= beta_max <= 1 (Eqs. 34-35)            */
  double beta_max;        /* sensor ceiling                                                     */
  double c_sensor;        /* sensitivity C_sensor >= 0 (Eqs. 34-35)                              */
  double ducros_eps;      /* regulariser epsilon > 0 of the Ducros ratio (Eq. 33), in the units of */
                          /* |grad u|^2 (physical central differences); 1e-6 keeps theta smooth   */
  int32_t retarget_every; /* retarget the link speed every k >= 1 steps (Sec. III E)            */
  int32_t precision;      /* vlbm_precision: FP64 populations, or FP32 storage of deviations    */
  int32_t algorithm;      /* vlbm_algorithm: how the two global maxima of a step are obtained   */
  int32_t tiling;         /* vlbm_tiling: how the 2D step kernel covers the grid                */
} vlbm_params;

/* Creates a solver for the grid, EOS and parameters, bound to `cuda_stream` (a cudaStream_t, or
 * NULL for the legacy default stream).  Allocates the two population buffers (per cell 2D
 * directions x a 4-wide vector of the D+2 components, 8 bytes per value for VLBM_FP64, 4 for
 * VLBM_FP32_STORE; in FP64 with column strips also W, u and Q of the current state, 14 values per
 * cell, kept from the maxima pass for the step kernel) and scratch on the current
 * device.  Returns VLBM_E_INVAL for nx, ny < 1, more than (2^31 - 1) / (8 D) cells (134,217,727
 * in 2D, e.g. up to 11585^2), a periodic side without
 * its periodic partner, or parameters outside the ranges above; VLBM_E_NOMEM if allocation
 * fails.  *out receives the handle (NULL on failure). */
vlbm_status vlbm_create(const vlbm_grid* grid, const vlbm_eos* eos, const vlbm_params* params, void* cuda_stream,
                        vlbm_t* out);

/* Releases every resource of the handle after its stream has drained.  NULL is accepted. */
vlbm_status vlbm_destroy(vlbm_t h);

/* State W_in (host array of D+2 conserved values) held by the ghost cells of a pinned-inflow x-lo
 * side (Sec. IV H: the exact upstream state of the stationary shock).  Required before vlbm_init
 * on such a grid (else vlbm_init returns VLBM_E_STATE); may be changed between calls.  Returns
 * VLBM_E_STATE on a grid without a pinned-inflow side and VLBM_E_INVAL for rho <= 0 or a
 * non-finite or non-physical internal energy.  Synchronises. */
vlbm_status vlbm_set_inflow(vlbm_t h, const double* W_in);

/* Initial populations f_i = f_i^eq(W0; c0) with c0 = s_max(W0) / CFL (Eqs. 20, 36-37), time 0,
 * step counter 0, history cleared.  W0: (D+2) * ny * nx values.  A replayed schedule (see
 * vlbm_set_dt_schedule) supplies c0 instead.  A non-physical W0 is reported by the next
 * synchronising call. */
vlbm_status vlbm_init(vlbm_t h, const double* W0);

/* Advances up to n_steps time steps.  With t_end > 0 the run stops once t reaches t_end, the
 * last step being shortened to land on it exactly (Sec. III E); t_end <= 0 disables the end time.
 * All link-speed and time-step decisions are taken on the device (no host synchronisation per
 * step); the call synchronises once at its end and writes the number of steps taken to
 * *steps_done (may be NULL). */
vlbm_status vlbm_step(vlbm_t h, int64_t n_steps, double t_end, int64_t* steps_done);

/* W = sum_i f_i of the current state (Sec. III A), (D+2) * ny * nx float64 values. */
vlbm_status vlbm_get_W(vlbm_t h, double* W);

/* n_runs independent runs on this handle's grid, gas and parameters, one after another: run k is
 * vlbm_init(W0s[k]), vlbm_step(n_steps, t_end) and vlbm_get_W(Ws[k]), with the same results.
 * W0s[k], Ws[k]: (D+2) * ny * nx float64 values each, host or device memory (caller-owned; pinned
 * host memory lets the copies overlap the steps).  Host inputs and outputs move through two
 * device staging buffers per direction (4 (D+2) ny nx doubles, allocated on the first call and
 * kept by the handle) on two copy streams of their own, so that run k+1's upload and run k-1's
 * readback overlap run k's steps.  An output array must not overlap the input array of a later
 * run.  steps_done (may be NULL) receives n_runs step counts.  On return no copy is in flight
 * and the handle holds the last run's state (vlbm_step continues it).  Errors: VLBM_E_INVAL for
 * n_runs, n_steps < 0, a null array or element, or a non-finite t_end (nothing runs);
 * VLBM_E_STATE as vlbm_init; a failing run (VLBM_E_NONPHYSICAL, ...) ends the batch with its
 * status: later runs do not start and their outputs are not written.  Synchronises. */
vlbm_status vlbm_run_batch(vlbm_t h, int64_t n_runs, const double* const* W0s, int64_t n_steps, double t_end,
                           double* const* Ws, int64_t* steps_done);

/* beta(x) that the next step would use on the current state (Secs. III D; constant in
 * VLBM_BETA_CONST mode), ny * nx float64 values. */
vlbm_status vlbm_get_beta(vlbm_t h, double* beta);

/* Current populations f_i (the state whose zeroth moment vlbm_get_W returns), 2D * (D+2) * ny *
 * nx float64 values laid out [i][k][y][x], i in the lattice order {x-, x+, y-, y+} (1D: {x-, x+}).
 * FP32-storage handles return the stored FP32 deviation plus the FP64 reference share. */
vlbm_status vlbm_get_populations(vlbm_t h, double* f);

/* Time t, completed steps n and current link speed c (synchronises). Any pointer may be NULL. */
vlbm_status vlbm_get_time(vlbm_t h, double* t, int64_t* n, double* c);

/* Copies the per-step (dt, c) history of the run since vlbm_init into host arrays of capacity
 * `cap` (either may be NULL) and writes the number of recorded steps to *n (synchronises). */
vlbm_status vlbm_get_dt_history(vlbm_t h, double* dt_host, double* c_host, int64_t cap, int64_t* n);

/* Replays a fixed link-speed sequence instead of the CFL rule: c_host[0] is the initial link
 * speed used by vlbm_init, c_host[j] (j >= 1) the link speed of step j-1; dt = dx / c.  n = 0
 * returns to the adaptive rule.  Steps beyond the sequence fail with VLBM_E_INVAL.  Used to repeat
 * a recorded run exactly (finite differences, adjoint). */
vlbm_status vlbm_set_dt_schedule(vlbm_t h, const double* c_host, int64_t n);

/* Domain totals sum_x W_k(x) of the current state, k = 0..D+1 (mass, momentum, total energy per
 * unit cell volume), summed in FP64 with Neumaier compensation in a fixed order, written to the
 * host array totals[D+2] (synchronises).  On periodic domains the step conserves them up to
 * rounding (Sec. III A: the collision conserves W and streaming moves populations without loss);
 * zero-gradient sides let the boundary fluxes change them. */
vlbm_status vlbm_get_totals(vlbm_t h, double* totals);

/* Checkpoint / resume of a run.  vlbm_save_state writes the complete state (populations in
 * their storage precision, device scalars: time, step counter, link speed, FP32 reference share,
 * and the (dt, c) history) into the host buffer `host` of `cap` bytes and the size to *used;
 * host == NULL only queries the size.  The buffer ends with a 64-bit checksum.  It synchronises
 * and fails with VLBM_E_INVAL when cap is too small.  vlbm_load_state restores such a buffer
 * (n_bytes long) into a handle created with the same grid, lattice and precision (else
 * VLBM_E_INVAL; a damaged buffer gives VLBM_E_CHECKSUM); stepping then continues exactly as the
 * saving handle would have.  A replay schedule (vlbm_set_dt_schedule) belongs to the handle and
 * is not part of the state. */
vlbm_status vlbm_save_state(vlbm_t h, void* host, size_t cap, size_t* used);
vlbm_status vlbm_load_state(vlbm_t h, const void* host, size_t n_bytes);

/* Launches the dominant step kernel `reps` times on the handle's stream (without advancing the
 * state: each launch recomputes the same next state into the spare buffer) bracketed by CUDA
 * events, and writes the mean duration of one launch in milliseconds (synchronises).  The state
 * must have been initialised. */
vlbm_status vlbm_time_step_kernel(vlbm_t h, int32_t reps, double* ms_per_launch);

/* Live kernel timing.  With `on` != 0, every launch of the dominant step kernel by vlbm_step is
 * bracketed by a pair of CUDA events on the handle's stream: the graph chunks vlbm_step launches
 * are then captured with an event-record node before and after each step-kernel launch (the same
 * kernels, the same launches), and steps issued outside a chunk get an event pair each.  The
 * events of a chunk are read when vlbm_step synchronises at its end; a call that launches more
 * than one chunk synchronises once before each further chunk to read them.  vlbm_get_profile
 * returns the summed device time of the bracketed launches (ms) and their count, and resets both
 * (synchronises).  Turning profiling on or off also resets them. */
vlbm_status vlbm_set_profiling(vlbm_t h, int32_t on);
vlbm_status vlbm_get_profile(vlbm_t h, double* ms_total, int64_t* launches);

/* Gradient of an objective of the final state with respect to the initial field and the EOS
 * parameters (reverse mode of the whole run).  FP32-storage handles keep the checkpoints and the
 * recomputed states in FP32 storage and evaluate the adjoint in FP64 at those states.
 *
 * Runs vlbm_init(W0) and n_steps steps (adaptive link speed, or the replayed schedule), storing
 * the populations every checkpoint_every steps and recording the link-speed sequence; then walks
 * the run backwards segment by segment, recomputing each segment's states from its checkpoint
 * with the recorded link speeds and applying the adjoint of every step: streaming (Eq. 21),
 * relaxation and equilibrium (Eqs. 20, 22), the shock sensor with its global flux maxima
 * (Eqs. 28-35), reprojection (Eqs. 38-40), and flux and EOS Jacobians (Eqs. 10-17), and finally
 * the adjoint of the initial equilibrium.  The link speeds are held fixed (not differentiated);
 * the derivative of each maximum M_k goes to its first maximal element in (alpha, y, x) order;
 * d|x|/dx = 0 at 0, d sqrt = 0 at 0, and clip() has derivative 0 at and beyond its bounds.
 *
 *   W0:      (D+2) ny nx initial field (host or device).
 *   dJ_dWT:  (D+2) ny nx values dJ/dW(T) of the objective at the final state (host or device).
 *   dJ_dW0:  output, (D+2) ny nx values dJ/dW0 (host or device).
 *   dJ_deos: host[5] output dJ/d(gamma, a, b, R, cv) (the ideal gas uses gamma, van der Waals
 *            a, b, R, cv), or NULL.
 * Not available on a grid with a pinned-inflow side or with VLBM_EOS_VDW_CVT (VLBM_E_UNSUPPORTED).
 * Afterwards the handle holds the final state of the run (as after vlbm_step), and vlbm_step
 * continues it.  Device memory: (ceil(n_steps / checkpoint_every) + min(checkpoint_every,
 * n_steps) + 2) population states plus 43 FP64 fields per cell, plus the tape (see
 * vlbm_set_adjoint_tape): the last segments of the run, as many as the tape limit allows, are
 * stepped by the forward pass into slots of their own, so the reverse pass applies their adjoint
 * steps without recomputing them.  A slot holds each state of its segment and, on FP64 column
 * strips in sensor mode, the 8 sensor planes of each state (lean slot: the adjoint evaluates W, u,
 * Q itself) or all 22 kept planes (full slot); the memory left after the lean slots makes the last
 * ones full.  The gradient is the same either way up to rounding (6e-15 relative measured on FP64
 * strips, where taped and recomputed segments take W, u, Q and the sensor quantities from
 * different kernels).  The handle keeps the workspace and the tape for later calls.
 * Synchronises. */
vlbm_status vlbm_adjoint(vlbm_t h, const double* W0, int64_t n_steps, int32_t checkpoint_every, const double* dJ_dWT,
                         double* dJ_dW0, double* dJ_deos);

/* Device time (ms) of the reverse pass (segment recomputation and adjoint steps) of the last
 * vlbm_adjoint call, and of its segment recomputations alone (*recompute_ms, may be NULL). */
vlbm_status vlbm_adjoint_timing(vlbm_t h, double* reverse_ms, double* recompute_ms);

/* Limit of the adjoint tape, in bytes: max_bytes < 0 (the default) lets each vlbm_adjoint call
 * use up to 3/4 of the device memory free at that moment; 0 disables the tape (every segment is
 * recomputed from its checkpoint) and releases its memory; a positive value caps it (a held tape
 * above the cap is released).  Synchronises when it releases memory. */
vlbm_status vlbm_set_adjoint_tape(vlbm_t h, int64_t max_bytes);

/* Of the last vlbm_adjoint call: device time (ms) of its forward pass, the steps whose states
 * came from the tape rather than a recomputation, and the tape bytes used (each may be NULL). */
vlbm_status vlbm_adjoint_info(vlbm_t h, double* forward_ms, int64_t* taped_steps, int64_t* tape_bytes);

/* Number of kernel launches one time step issues (for launch accounting). */
vlbm_status vlbm_launches_per_step(vlbm_t h, int32_t* launches);

/* beta(x) of caller-owned FP64 populations without any device allocation.
 *
 * The paper has no counterpart: this entry point serves callers that cannot call cudaMalloc,
 * such as an application whose device memory all belongs to its own pool allocator, code that
 * must not allocate while a CUDA graph is being captured, or a loop with a fixed memory budget.
 * It computes what vlbm_get_beta returns for a handle holding the same state (Eqs. 28-35 with
 * the maxima of Eq. 30), but keeps all scratch (a scalar block, 1/M_k and per-CTA partial maxima)
 * in one file-scope static device array of about 330 KiB inside the library, which every GPU that
 * loads the library holds until the process exits.
 *
 *   grid, eos, params: as for vlbm_create (only the sensor fields of params are used).
 *   f:        device pointer, FP64 populations in the library's storage layout [i][y][x][4] (2D x 4 x
 *             ny nx values; component k of direction i at ((i ny + y) nx + x) 4 + k, slot 3 unused
 *             in 1D), caller-owned;
 *             in_place != 0: f holds the state itself (e.g. from vlbm_get_populations);
 *             in_place == 0: f holds post-collision populations to be pulled across the links.
 *   beta:     device pointer, ny nx FP64 values, caller-owned output.
 *   cuda_stream: stream for the work (NULL: legacy default stream); the call returns without
 *             waiting, beta is valid once the stream reaches this point.
 *
 * A grid with a pinned-inflow side returns VLBM_E_UNSUPPORTED (there is no handle holding W_in).
 * Limits and behaviour: at most 2,097,152 cells (nx ny, each axis checked first); larger grids
 * return VLBM_E_INVAL.  The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) and sets the kernels' shared-memory attribute, under a lock, so host
 * threads may make their first calls concurrently; make that first call before any stream
 * capture.  The call
 * allocates nothing (no cudaMalloc, cudaFree or allocating library routine).  Every call on a
 * device shares the one array and leaves its contents behind; the call clears the scalar block
 * at its start, and every other entry it reads it writes first.  Calls that overlap on the GPU
 * (different streams without ordering) race on the array: order them, e.g. one stream.  A
 * non-physical state is not reported (use a handle for that); beta is then meaningless. */
vlbm_status vlbm_beta_noalloc(const vlbm_grid* grid, const vlbm_eos* eos, const vlbm_params* params, const double* f,
                              int32_t in_place, double* beta, void* cuda_stream);

/* Measured FP64 throughput of the current GPU, the denominator of the FP64 step's ALU roofline
 * (the method has no counterpart; a measurement aid).  Runs `reps` timed launches of a kernel in
 * which every thread advances eight independent chains of dependent FP64 fused multiply-adds, on
 * a grid that fills every SM, and writes the best rate in TFLOP/s (an FMA counted as 2 flops) to
 * *tflops.  Synchronises; allocates no device memory. */
vlbm_status vlbm_measure_fp64_peak(int32_t reps, double* tflops);

/* Human-readable name of a status code (static storage). */
const char* vlbm_status_string(vlbm_status s);

/* Library version string (static storage). */
const char* vlbm_version(void);

#ifdef __cplusplus
}
#endif

#endif /* VLBM_H */
