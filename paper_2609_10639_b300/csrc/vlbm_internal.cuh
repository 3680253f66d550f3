// Internal declarations shared by the kernels and the C-ABI layer of the VLBM step library.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "vlbm.h"

namespace vlbm {

// Device-resident scalars of one solver.  Written only by the one-thread link-speed kernel
// (and the init kernels); read by every step kernel.  No host synchronisation per step.
struct Scalars {
  double c_prev;      // link speed of the stored populations
  double c_new;       // link speed of the step in flight (Eq. 37)
  double r;           // c_prev / c_new of the step in flight (reprojection, Eqs. 38-40)
  double inv_c;       // 1 / c_new
  double dt;          // time step of the step in flight
  double t;           // time once the step in flight has completed
  double t_end;       // end time of the current vlbm_step call (<= 0: none)
  double inv_M[4];    // 1 / max_{x,alpha} |Q_alpha,k| of the step in flight (0 where the max is 0)
  double smax;        // s_max of the step in flight (Eq. 36)
  double wref[4];     // FP32 storage: W_ref_k / Q, the share subtracted from every population
  float r_f, inv_c_f; // FP32 copies of r and 1/c_new (FP32-storage step)
  float inv_M_f[4];   // FP32 copy of 1/M_k
  float wq_f[4];      // FP32 storage: Q * W_ref_k / Q = W_ref_k as float
  long long n;        // steps completed once the step in flight has completed
  long long hist_cap; // capacity of the (dt, c) history arrays
  long long sched_len;// length of the replayed link-speed schedule (0: CFL rule)
  int active;         // the step in flight runs (0 once t_end has been reached)
  int done;           // t_end reached
  int err;            // error bits (1: non-physical state; 2: bad schedule)
  int nparts[2];      // per-CTA partial maxima written into partial slot s (see below)
};

// Global maxima of a step (s_max, Eq. 36; M_k, Eq. 30) are reduced in two levels without
// atomics: every CTA of the producing kernel writes its 5 partial maxima (s_max, M_0..M_3) to
// part[slot][cta][5] and CTA 0 records the count in Scalars::nparts[slot]; the one-CTA link-speed
// kernel folds them.  Slot of a step = (steps completed when the producer runs) & 1.
constexpr int kNV = 5;

enum { ERR_NONPHYSICAL = 1, ERR_SCHEDULE = 2 };

// Coefficients of the step in the arithmetic type of a path (FP64, or FP32 for FP32 storage),
// precomputed on the host so that no per-cell conversion runs on the FP64 pipe.
template <class M>
struct Coef {
  M gamma, gm1, ggm1;           // gamma, gamma - 1, gamma (gamma - 1)          (Eq. 15)
  M a, b, R, inv_cv, a_inv_cv;  // van der Waals a, b, R, 1/cv, a/cv         (Eqs. 16-17)
  M c_sensor, beta_max, dbeta;  // C_sensor, beta_max, beta_max - beta_min   (Eqs. 34-35)
  M c_chi2, c_chi1;             // chi = c_chi2 S T (2D) or c_chi1 S (1D), S and T the unnormalised
                                // filter sums of sqrt(sum_k s_hat_k^2) and theta: C / 512, C / (4 sqrt 3)
  M beta_const;                 // constant-beta mode
  M eps_lat;                    // Ducros regulariser (Eqs. 32-33) in units of unscaled central
                                // differences, eps (2 dx)^2: theta = D^2 / (D^2 + V^2 + eps_lat)
                                // with D, V the dilatation and vorticity times 2 dx
  M win[4];                     // state W_in of the pinned-inflow ghost cells (x-lo side)
  M cv0, cv1, cv2, cv1h, cv2t;  // non-polytropic van der Waals: c_v(T) = cv0 + cv1 T + cv2 T^2,
                                // cv1 / 2 and cv2 / 3 (the integral E(T))
};

// Constant per-solver parameters, passed to kernels by value.
struct KParams {
  int dim, nc, q;
  int nx, ny;
  long long plane;  // nx * ny
  int bc[4];        // x-lo, x-hi, y-lo, y-hi: 0 periodic, 1 zero-gradient, 2 pinned inflow (x-lo only)
  double dx, inv2dx;
  int eos_kind;
  double gamma, a, b, R, cv, inv_cv;  // eos_kind: 0 ideal, 1 van der Waals, 2 van der Waals with c_v(T)
  double cfl;
  int beta_mode;
  double beta_const, beta_min, beta_max, c_sensor, ducros_eps;
  int retarget_every;
  int max_parts;    // capacity of one partial-maxima slot (CTAs of the largest producer)
  int strip;        // 2D step kernel: column-strip form (1) or tiles (0)
  Coef<double> cd;
  Coef<float> cf;
};

// Problem set-up shared by vlbm_create and vlbm_beta_noalloc (defined in vlbm_capi.cu).
// valid_problem checks the grid's dimension, extent and boundary pairing, the EOS parameters and
// the sensor fields of the parameters (not the sizes: each entry point has its own limit);
// make_kparams fills the per-solver parameters and the precomputed coefficients of both
// arithmetic types.
bool valid_problem(const vlbm_grid* grid, const vlbm_eos* eos, const vlbm_params* params);
void make_kparams(const vlbm_grid* grid, const vlbm_eos* eos, const vlbm_params* params, KParams& p);

// Host-side launch helpers (defined in vlbm_kernels.cu).
struct Launch {
  const KParams* p;
  Scalars* sc;
  double* part;      // [2][max_parts][kNV]
  cudaStream_t stream;
  double* hist_dt;
  double* hist_c;
  const double* sched;
  double* fields = nullptr;  // FP64 two-pass strips: W, u, Q of the current state, 14 planes
                             // [W0..3, u0, u1, Qx0..3, Qy0..3][y][x], written by the maxima pass
                             // and read by the step kernel (nullptr: not kept)
  double* sens = nullptr;    // FP64 two-pass strips, adjoint recomputation only: the step kernel
                             // also writes s_hat_0..3, s, theta, dil, vort of every cell (8 planes)
  float* pkeep = nullptr;    // FP32 storage, look-ahead strips, non-ideal gas: pressure of the state
                             // a step kernel starts from, [2][y][x] by step parity, written by the
                             // pass that computed it for the same W (look-ahead stage, or init)
};

// precision: 0 = FP64, 1 = FP32 storage.  lookahead: fused single-kernel step.
// in_run: the reduction is a step of a run and is skipped once the run is done or failed;
// otherwise (beta readback, state restore) it always runs.
cudaError_t launch_reduce(const Launch& L, int precision, const void* fin, int pulled, bool in_run);
cudaError_t launch_dt(const Launch& L);
cudaError_t launch_step(const Launch& L, int precision, bool lookahead, const void* fin, void* fout, int pulled);
cudaError_t launch_beta(const Launch& L, int precision, const void* fin, int pulled, double* beta_out);
// maxima: also the maxima of the stored initial populations (the look-ahead form's first step)
cudaError_t launch_init(const Launch& L, int precision, const double* W0, void* fout, double* partial, int nblk_sum,
                        bool maxima);
cudaError_t launch_get_W(const Launch& L, int precision, const void* fin, int pulled, double* W);
cudaError_t launch_get_f(const Launch& L, int precision, const void* fin, int pulled, double* f);
cudaError_t launch_begin(const Launch& L, double t_end);
// Compensated domain totals sum_x W_k into out[0..nc) (W: nc planes of scratch, partial: per-block
// sums of sum_blocks() blocks).
cudaError_t launch_totals(const Launch& L, int precision, const void* fin, int pulled, double* W, double* partial,
                          int nblk_sum, double* out);
cudaError_t prepare_kernels();
// Column-strip form of the 2D step kernel (vlbm_roll.cu).
cudaError_t launch_roll(const Launch& L, int precision, bool lookahead, const void* fin, void* fout, int pulled);
cudaError_t prepare_roll_kernels();
// Pressure of the current state into slot (n & 1) of L.pkeep (after a state restore).
cudaError_t launch_fill_pressure(const Launch& L, const void* fin, int pulled);
long long roll_ctas(const KParams& p);
int sum_blocks(const KParams& p);
int max_partials(const KParams& p);

}  // namespace vlbm
