// Internal interface of the adjoint kernels (vlbm_adjoint.cu) for the C-ABI layer.
#pragma once

#include "vlbm_internal.cuh"

namespace vlbm {

// Device-resident scalars of one backward step and the accumulated EOS-parameter gradient.
struct AdjScalars {
  double M[4], invM[4];  // M_k = max |Q_alpha,k| of the step and 1/M_k (0 where M_k = 0)
  long long amax[4];     // linear index ((alpha NC + k) ny + y) nx + x of the first maximal element
  int amax_cell[4];      // its cell y nx + x and direction alpha
  int amax_alpha[4];
  double lamM[4];        // dJ/dM_k of the step
  double eos[5];         // dJ/d(gamma, a, b, R, cv), accumulated over the steps
  double eos_comp[5];    // compensation terms of that sum
  double r, inv_c;       // c_{n-1}/c_n and 1/c_n of the step
  double wref[4];        // FP32-storage states: the FP64 share W_ref/Q added to every stored value
};

struct AdjLaunch {
  const KParams* p;
  AdjScalars* as;
  cudaStream_t stream;
  const double* sched;  // [c0, c_0, ..., c_{N-1}]: link speed of the initial state and of each step
  double* F;            // adj_num_fields() planes of FP64 workspace
  double* pv;           // per-CTA argmax values [CTAs][4]
  long long* pi;        // per-CTA argmax indices [CTAs][4]
  double* part;         // per-CTA partial sums [adj_part_entries][8]
  double* gpart;        // first fold stage: group sums [adj_group_entries][8], or argmax values [..][4]
  long long* gidx;      // first fold stage: argmax indices [adj_group_entries][4]
};

int adj_num_fields();
int adj_part_entries(const KParams& p);
int adj_group_entries(const KParams& p);
// lambda^n from lambda^{n+1} for forward step n whose state f^n is `fin` (pulled or in place),
// stored in FP64 (precision 0) or as FP32 deviations (precision 1).  `kept`: 22 planes in the
// layout of the workspace's first planes (W, u, Q, s_hat, s, theta, dil, vort) of f^n, the
// first 14 stored by the maxima pass of the forward recomputation and, with kept_sensor, the
// other 8 by its step kernel; nullptr to recompute them all.  `sensor` (with kept == nullptr): the
// 8 sensor planes of f^n (s_hat, s, theta, dil, vort) written by the forward step kernel, so that
// only W, u, Q are evaluated here; nullptr to evaluate them too.
cudaError_t adj_step(const AdjLaunch& A, int precision, const void* fin, int pulled, const double* lam_in, double* lam_out,
                     long long n, double* kept, bool kept_sensor, const double* sensor = nullptr);
// lambda^N from dJ/dW(T); resets the EOS-gradient accumulator
cudaError_t adj_terminal(const AdjLaunch& A, const double* dJ_dW, double* lam);
// dJ/dW0 from lambda^0 through f^0 = f^eq(W0; c0); finishes the EOS-gradient sum
cudaError_t adj_init(const AdjLaunch& A, const double* W0, const double* lam0, double c0, double* dJ_dW0);
// step scalars for recomputing a segment from step n0 with a replayed link-speed sequence
cudaError_t adj_replay_scalars(cudaStream_t s, Scalars* sc, long long n0, const double* sched, long long sched_len);

}  // namespace vlbm
