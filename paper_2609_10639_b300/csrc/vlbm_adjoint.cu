// Adjoint (reverse mode) of the VLBM time step for a recorded link-speed sequence, evaluated in
// FP64 at the states of an FP64 or an FP32-storage run.
//
// Forward step n maps the pre-collision populations f^n to f^{n+1}:
//   W = sum_i f_i;  f' = R(r) f (reprojection, Eqs. 38-40, r = c_n-1 / c_n);  Q(W), u(W) (Eq. 10);
//   M_k = max_{x,alpha} |Q_alpha,k| (Eq. 30);  beta = sensor(Q, u, M) (Eqs. 28-35);
//   f*_i = 2 beta f_i^eq(W, Q; c_n) + (1 - 2 beta) f'_i (Eqs. 20, 22);  f^{n+1}_i(x) = f*_i(x - sigma_i).
// With the link speeds held fixed (they are recorded in the forward pass and not differentiated),
// the adjoint maps lambda^{n+1} = dJ/df^{n+1} to lambda^n = dJ/df^n and accumulates dJ/d(EOS
// parameters).  Non-smooth points follow the conventions of the dual-number oracle: the
// derivative of M_k goes to the first maximal element in (alpha, y, x) order, d|x| = 0 at 0,
// d sqrt = 0 at 0, and clip() has derivative 0 at and beyond its bounds.
//
// Each backward step runs cell-parallel kernels that exchange per-cell intermediates through a
// workspace of FP64 fields (the forward quantities of step n are recomputed from f^n first):
//   k_adj_fields   W, u, Q, per-CTA M_k candidates     k_adj_argmax_fold  M_k, argmax, 1/M_k
//                  (k_adj_argmax_kept: the candidates only, when the forward recomputation kept
//                  W, u, Q of the state; its step kernel then also kept the sensor quantities,
//                  and k_adj_sensor does not run)
//   k_adj_sensor   s_hat, s, theta, dil, vort
//   k_adj_local    beta; adjoints of relaxation, equilibrium and reprojection; d/d(s_bar, theta_bar)
//   k_adj_filter   transposed box filters; d/d(s_hat) -> d/dj; dM partial sums (+fold)
//   k_adj_flux     transposed differences; M fix-up at the argmax; flux/EOS Jacobian transposes;
//                  lambda^n += dJ/dW; EOS-parameter partial sums (+fold)
#include "vlbm.h"
#include "vlbm_device.cuh"
#include "vlbm_internal.cuh"
#include "vlbm_adjoint.cuh"

#include <cstddef>

namespace vlbm {

namespace {
constexpr int kNTA = 256;
// The per-CTA partials of a cell-parallel kernel are folded in two fixed-order stages: one warp
// per group of kGroup partials, then one CTA of kNTF threads over the groups.  A single CTA over
// all partials was bound by its one SM's FP64 pipe (2 FP64 results per clock per SM).
constexpr int kGroup = 32;
constexpr int kNTF = 128;

// workspace field indices (each a plane of FP64 values)
enum {
  F_W = 0,          // 4
  F_U = 4,          // 2
  F_Q = 6,          // 8: Q[alpha][k] at F_Q + 4 alpha + k
  F_SH = 14,        // 4: s_hat_k
  F_S = 18,         // activity s
  F_TH = 19,        // theta
  F_DIL = 20,
  F_VORT = 21,
  F_BETA = 22,      // (unused slot)
  F_LSB = 23,       // d/d s_bar
  F_LTB = 24,       // d/d theta_bar
  F_LWEQ = 25,      // 4: dJ/dW through the equilibrium
  F_LQEQ = 29,      // 8: dJ/dQ through the equilibrium
  F_LJ = 37,        // 4: dJ/dj_k
  F_LDIL = 41,
  F_LVORT = 42,
};
}  // namespace

int adj_num_fields() { return 43; }

// Distinct cells at positions j-1, j, j+1 along an axis (after the boundary rule), and the
// transposed weights of the operators built from them.
struct Cand {
  int c[3];
  int n;
};
__device__ __forceinline__ Cand candidates(int j, int n, int lo, int hi) {
  Cand r;
  r.n = 0;
  const int v[3] = {nb_index(j - 1, n, lo, hi), j, nb_index(j + 1, n, lo, hi)};
#pragma unroll
  for (int t = 0; t < 3; ++t) {
    bool dup = false;
    for (int q = 0; q < r.n; ++q) dup |= r.c[q] == v[t];
    if (!dup) r.c[r.n++] = v[t];
  }
  return r;
}
// weight with which the (1/4, 1/2, 1/4) filter centred at y reads cell x
__device__ __forceinline__ double filt_w(int y, int x, int n, int lo, int hi) {
  return (nb_index(y - 1, n, lo, hi) == x ? 0.25 : 0.0) + (y == x ? 0.5 : 0.0) + (nb_index(y + 1, n, lo, hi) == x ? 0.25 : 0.0);
}
// coefficient of cell x in the central difference v(y+1) - v(y-1) centred at y
__device__ __forceinline__ double diff_w(int y, int x, int n, int lo, int hi) {
  return (nb_index(y + 1, n, lo, hi) == x ? 1.0 : 0.0) - (nb_index(y - 1, n, lo, hi) == x ? 1.0 : 0.0);
}

// Reprojection (Eqs. 38-40) of one component's populations; the map is symmetric, so the same
// function applies its transpose.
template <int D>
__device__ __forceinline__ void reproject_k(const double (&f)[2 * D], double r, double (&o)[2 * D]) {
  if constexpr (D == 1) {
    const double w = 0.5 * (f[0] + f[1]), g = 0.5 * r * (f[1] - f[0]);
    o[0] = w - g;
    o[1] = w + g;
  } else {
    const double sx = f[0] + f[1], sy = f[2] + f[3];
    const double w = 0.25 * (sx + sy), kk = 0.25 * r * r * (sx - sy);
    const double gx = 0.5 * r * (f[1] - f[0]), gy = 0.5 * r * (f[3] - f[2]);
    o[0] = w - gx + kk;
    o[1] = w + gx + kk;
    o[2] = w - gy - kk;
    o[3] = w + gy - kk;
  }
}

// Transposed Jacobians of Q(W) and u(W) (Eq. 10 with the closure of Sec. II C) applied to
// (lamQ, lamu), added to lamW; returns the adjoint of P (for the EOS-parameter gradients) and the
// partial derivatives of P with respect to the EOS parameters at fixed W in dP_dprm[5]
// (gamma, a, b, R, cv).
template <int D>
__device__ __forceinline__ double flux_vjp(const KParams& p, const double (&W)[D + 2], const double (&lamQ)[D][D + 2],
                                           const double (&lamu)[D], double (&lamW)[D + 2], double (&dP_dprm)[5]) {
  constexpr int NC = D + 2;
  const double rho = W[0], ir = rcp_(rho), E = W[NC - 1];
  double u[D], usq = 0.0;
#pragma unroll
  for (int a = 0; a < D; ++a) {
    u[a] = W[1 + a] * ir;
    usq += u[a] * u[a];
  }
  const double e = E * ir - 0.5 * usq;
  double P, P_rho, P_e;
#pragma unroll
  for (int j = 0; j < 5; ++j) dP_dprm[j] = 0.0;
  if (p.eos_kind == 0) {
    const double gm1 = p.gamma - 1.0;
    P = gm1 * rho * e;
    P_rho = gm1 * e;
    P_e = gm1 * rho;
    dP_dprm[0] = rho * e;
  } else {
    const double T = (e + p.a * rho) / p.cv;
    const double omb = 1.0 - p.b * rho;
    const double dPdT = p.R * rho / omb;
    P = dPdT * T - p.a * rho * rho;
    P_rho = p.R * T / (omb * omb) - 2.0 * p.a * rho + dPdT * p.a / p.cv;
    P_e = dPdT / p.cv;
    dP_dprm[1] = dPdT * rho / p.cv - rho * rho;          // a (through T as well)
    dP_dprm[2] = p.R * rho * T * rho / (omb * omb);      // b
    dP_dprm[3] = rho * T / omb;                          // R
    dP_dprm[4] = -dPdT * T / p.cv;                       // cv
  }
  double lamP = 0.0;
  const double H = E + P;
#pragma unroll
  for (int a = 0; a < D; ++a) {
    lamW[1 + a] += lamQ[a][0];  // Q_a,0 = m_a
#pragma unroll
    for (int b = 0; b < D; ++b) {  // Q_a,1+b = m_b u_a + delta_ab P
      const double l = lamQ[a][1 + b];
      lamW[0] += -l * u[b] * u[a];
      lamW[1 + b] += l * u[a];
      lamW[1 + a] += l * u[b];
      if (a == b) lamP += l;
    }
    const double l = lamQ[a][NC - 1];  // Q_a,NC-1 = (E + P) u_a
    lamW[0] += -l * H * u[a] * ir;
    lamW[1 + a] += l * H * ir;
    lamW[NC - 1] += l * u[a];
    lamP += l * u[a];
    lamW[0] += -u[a] * lamu[a] * ir;  // u_a = m_a / rho
    lamW[1 + a] += lamu[a] * ir;
  }
  // dP/dW at fixed EOS parameters: P(rho, e(W))
  const double de_drho = (usq - E * ir) * ir, de_dE = ir;
  lamW[0] += lamP * (P_rho + P_e * de_drho);
#pragma unroll
  for (int c = 0; c < D; ++c) lamW[1 + c] += lamP * P_e * (-u[c] * ir);
  lamW[NC - 1] += lamP * P_e * de_dE;
  return lamP;
}

// Populations of a stored state in FP64 (FP32 storage: deviation plus the reference share).
template <int D, class S>
__device__ __forceinline__ void load_state(const S* __restrict__ fin, const KParams& p, int cx, int cy, int pulled,
                                           const double* wref, double (&fr)[2 * D][D + 2]) {
  typename Store<S>::M t[2 * D][D + 2];
  load_cell<D, S>(fin, p, cx, cy, pulled, false, t);
#pragma unroll
  for (int i = 0; i < 2 * D; ++i)
#pragma unroll
    for (int k = 0; k < D + 2; ++k) fr[i][k] = (double)t[i][k] + (Store<S>::kOffset ? wref[k] : 0.0);
}

// ------------------------------------------------------------------------------------------
// kernels (one thread per cell, 256-thread CTAs)
// ------------------------------------------------------------------------------------------
// Per-CTA (value, linear index) maxima of |Q_alpha,k| for each k; ties to the lowest index
// ((alpha NC + k) ny + y) nx + x.
// The values are non-negative doubles (or +0.0 for "none yet"), compared through their 64-bit
// patterns on the integer pipe (same order).
__device__ __forceinline__ bool better(double v, long long i, double bv, long long bi) {
  const unsigned long long a = (unsigned long long)__double_as_longlong(v), b = (unsigned long long)__double_as_longlong(bv);
  return a > b || (a == b && i < bi);
}

constexpr long long kNoIndex = 0x7fffffffffffffffll;  // loses every comparison of better()

// Warp-wide argmax of (value, index) pairs under better(), a strict total order on the pairs, so
// the unique best pair results whatever the order of the comparisons.
__device__ __forceinline__ void argmax_warp(double& v, long long& i) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const double ov = __shfl_xor_sync(0xffffffffu, v, off);
    const long long oi = __shfl_xor_sync(0xffffffffu, i, off);
    if (better(ov, oi, v, i)) {
      v = ov;
      i = oi;
    }
  }
}

// CTA-wide argmax of the per-thread candidates (v[k], i[k]), k < nc: within each warp by
// shuffles, then over the warps' results by warp 0, whose lane 0 ends with the CTA's best pairs.
template <int NT>
__device__ __forceinline__ void argmax_cta(double (&v)[4], long long (&i)[4], int nc) {
  __shared__ double wv[NT / 32][4];
  __shared__ long long wi[NT / 32][4];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    if (k >= nc) break;
    argmax_warp(v[k], i[k]);
    if (lane == 0) {
      wv[warp][k] = v[k];
      wi[warp][k] = i[k];
    }
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      if (k >= nc) break;
      v[k] = lane < NT / 32 ? wv[lane][k] : 0.0;
      i[k] = lane < NT / 32 ? wi[lane][k] : kNoIndex;
      argmax_warp(v[k], i[k]);
    }
  }
}

// W, u, Q of the forward state of the step, and the CTA's candidates for M_k (Eq. 30).
template <int D, class S>
__global__ void __launch_bounds__(kNTA) k_adj_fields(const S* __restrict__ fin, const KParams p, int pulled,
                                                      const AdjScalars* __restrict__ as, double* __restrict__ F,
                                                      double* __restrict__ pv, long long* __restrict__ pi) {
  constexpr int NC = D + 2;
  double sv[4];
  long long si[4];
  const int cell = blockIdx.x * kNTA + threadIdx.x;
  const long long P = p.plane;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    sv[k] = 0.0;
    si[k] = kNoIndex;
  }
  if (cell < p.plane) {
    const int cx = cell % p.nx, cy = cell / p.nx;
    double fr[2 * D][NC], W[NC], u[D], Qf[D][NC], cs;
    load_state<D, S>(fin, p, cx, cy, pulled, as->wref, fr);
    moments<D, double, false>(fr, nullptr, W);
    prim_flux<D, double, false>(p, W, u, Qf, cs);
#pragma unroll
    for (int k = 0; k < NC; ++k) F[(F_W + k) * P + cell] = W[k];
#pragma unroll
    for (int a = 0; a < D; ++a) {
      F[(F_U + a) * P + cell] = u[a];
#pragma unroll
      for (int k = 0; k < NC; ++k) F[(F_Q + 4 * a + k) * P + cell] = Qf[a][k];
    }
#pragma unroll
    for (int k = 0; k < NC; ++k) {
      // |Q| compared as 64-bit patterns (same order for non-negative doubles; integer pipe);
      // increasing alpha is increasing index, so a strict > keeps the first
      unsigned long long best = 0;
      int ba = -1;
#pragma unroll
      for (int a = 0; a < D; ++a) {
        const unsigned long long v = (unsigned long long)__double_as_longlong(Qf[a][k]) & 0x7fffffffffffffffull;
        if (ba < 0 || v > best) {
          best = v;
          ba = a;
        }
      }
      sv[k] = __longlong_as_double((long long)best);
      si[k] = (long long)(ba * NC + k) * P + cell;
    }
  }
  argmax_cta<kNTA>(sv, si, NC);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < NC; ++k) {
      pv[blockIdx.x * 4 + k] = sv[k];
      pi[blockIdx.x * 4 + k] = si[k];
    }
  }
}

// The CTA's candidates for M_k from Q kept by the forward recomputation (same layout as the
// workspace's first planes).
template <int D>
__global__ void __launch_bounds__(kNTA) k_adj_argmax_kept(const double* __restrict__ WQ, const KParams p,
                                                           double* __restrict__ pv, long long* __restrict__ pi) {
  constexpr int NC = D + 2;
  double sv[4];
  long long si[4];
  const int cell = blockIdx.x * kNTA + threadIdx.x;
  const long long P = p.plane;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    sv[k] = 0.0;
    si[k] = kNoIndex;
  }
  if (cell < p.plane) {
#pragma unroll
    for (int k = 0; k < NC; ++k) {
      unsigned long long best = 0;
      int ba = -1;
#pragma unroll
      for (int a = 0; a < D; ++a) {
        const unsigned long long v =
            (unsigned long long)__double_as_longlong(WQ[(F_Q + 4 * a + k) * P + cell]) & 0x7fffffffffffffffull;
        if (ba < 0 || v > best) {
          best = v;
          ba = a;
        }
      }
      sv[k] = __longlong_as_double((long long)best);
      si[k] = (long long)(ba * NC + k) * P + cell;
    }
  }
  argmax_cta<kNTA>(sv, si, NC);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < NC; ++k) {
      pv[blockIdx.x * 4 + k] = sv[k];
      pi[blockIdx.x * 4 + k] = si[k];
    }
  }
}

// Fold of the per-CTA candidates (one CTA): M_k, 1/M_k and the argmax of each k.
// First stage: the best candidate of each group of kGroup per-CTA candidates (one warp each).
__global__ void __launch_bounds__(kGroup) k_adj_argmax_groups(const double* __restrict__ pv,
                                                              const long long* __restrict__ pi, int nparts, int nc,
                                                              double* __restrict__ gv, long long* __restrict__ gi) {
  const int c = blockIdx.x * kGroup + threadIdx.x;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    if (k >= nc) break;
    double v = c < nparts ? pv[c * 4 + k] : 0.0;
    long long i = c < nparts ? pi[c * 4 + k] : kNoIndex;
    argmax_warp(v, i);
    if (threadIdx.x == 0) {
      gv[blockIdx.x * 4 + k] = v;
      gi[blockIdx.x * 4 + k] = i;
    }
  }
}

// Second stage over the groups' candidates.  Also sets the step's r = c_n / c_{n+1} and
// 1/c_{n+1} from the recorded link speeds (read by k_adj_local, which runs after this fold).
__global__ void __launch_bounds__(kNTF) k_adj_argmax_fold(const double* __restrict__ pv, const long long* __restrict__ pi,
                                                           int nparts, int nc, long long plane, AdjScalars* as,
                                                           const double* __restrict__ sched, long long n) {
  double sv[4];
  long long si[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    sv[k] = 0.0;
    si[k] = kNoIndex;
  }
  for (int c = threadIdx.x; c < nparts; c += kNTF)
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      if (k >= nc) break;
      const double v = pv[c * 4 + k];
      const long long i = pi[c * 4 + k];
      if (better(v, i, sv[k], si[k])) {
        sv[k] = v;
        si[k] = i;
      }
    }
  argmax_cta<kNTF>(sv, si, nc);
  if (threadIdx.x == 0) {
    const double c_old = sched[n], c_new = sched[n + 1];
    as->r = c_old / c_new;
    as->inv_c = 1.0 / c_new;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      if (k >= nc) break;
      const double bv = sv[k];
      as->M[k] = bv;
      as->invM[k] = bv > 0.0 ? 1.0 / bv : 0.0;
      const long long idx = si[k];
      as->amax[k] = idx;
      as->amax_cell[k] = (int)(idx % plane);
      as->amax_alpha[k] = (int)((idx / plane) / nc);
    }
  }
}

template <int D>
__global__ void __launch_bounds__(kNTA) k_adj_sensor(const KParams p, const AdjScalars* __restrict__ as,
                                                      double* F, const double* WQ) {
  constexpr int NC = D + 2;
  const int cell = blockIdx.x * kNTA + threadIdx.x;
  if (cell >= p.plane) return;
  const int x = cell % p.nx, y = cell / p.nx;
  const long long P = p.plane;
  const int xp = nb_index(x + 1, p.nx, p.bc[0], p.bc[1]) + y * p.nx, xm = nb_index(x - 1, p.nx, p.bc[0], p.bc[1]) + y * p.nx;
  int yp = 0, ym = 0;
  if constexpr (D == 2) {
    yp = x + nb_index(y + 1, p.ny, p.bc[2], p.bc[3]) * p.nx;
    ym = x + nb_index(y - 1, p.ny, p.bc[2], p.bc[3]) * p.nx;
  }
  double acc = 0.0;
#pragma unroll
  for (int k = 0; k < NC; ++k) {
    double jk = WQ[(F_Q + k) * P + xp] - WQ[(F_Q + k) * P + xm];
    if constexpr (D == 2) jk += WQ[(F_Q + 4 + k) * P + yp] - WQ[(F_Q + 4 + k) * P + ym];
    const double sh = 0.5 * jk * as->invM[k];
    F[(F_SH + k) * P + cell] = sh;
    acc += sh * sh;
  }
  F[F_S * P + cell] = sqrt(acc * (1.0 / NC));
  if constexpr (D == 2) {
    const double* ux = WQ + F_U * P;
    const double* uy = WQ + (F_U + 1) * P;
    const double dil = ((ux[xp] - ux[xm]) + (uy[yp] - uy[ym])) * p.inv2dx;
    const double vort = ((uy[xp] - uy[xm]) - (ux[yp] - ux[ym])) * p.inv2dx;
    F[F_DIL * P + cell] = dil;
    F[F_VORT * P + cell] = vort;
    F[F_TH * P + cell] = dil * dil / (dil * dil + vort * vort + p.ducros_eps);
  }
}

// beta at a cell from the stored s, theta (box filter x then y, Sensor A / B), and the raw
// argument C s_bar theta_bar with the filtered values.
template <int D>
__device__ __forceinline__ double sensor_at(const KParams& p, const double* __restrict__ F, int x, int y, double& chi_raw,
                                            double& sbar, double& tbar) {
  const long long P = p.plane;
  const double* s = F + F_S * P;
  const double* th = F + F_TH * P;
  if (D == 2 && x >= 1 && x < p.nx - 1 && y >= 1 && y < p.ny - 1) {  // interior: plain neighbours
    const int c = y * p.nx + x;
    double rs[3], rt[3];  // unnormalised (1, 2, 1) sums: the 1/16 is exact
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const int c0 = c + (j - 1) * p.nx;
      rs[j] = fma(2.0, s[c0], s[c0 - 1]) + s[c0 + 1];
      rt[j] = fma(2.0, th[c0], th[c0 - 1]) + th[c0 + 1];
    }
    sbar = 0.0625 * (fma(2.0, rs[1], rs[0]) + rs[2]);
    tbar = 0.0625 * (fma(2.0, rt[1], rt[0]) + rt[2]);
    chi_raw = p.c_sensor * sbar * tbar;
    const double chi = chi_raw <= 0.0 ? 0.0 : (chi_raw >= 1.0 ? 1.0 : chi_raw);
    return p.beta_max - (p.beta_max - p.beta_min) * chi;
  }
  const int xm = nb_index(x - 1, p.nx, p.bc[0], p.bc[1]), xp = nb_index(x + 1, p.nx, p.bc[0], p.bc[1]);
  if constexpr (D == 1) {
    sbar = 0.25 * s[xm] + 0.5 * s[x] + 0.25 * s[xp];
    tbar = 1.0;
  } else {
    const int ys[3] = {nb_index(y - 1, p.ny, p.bc[2], p.bc[3]), y, nb_index(y + 1, p.ny, p.bc[2], p.bc[3])};
    double rs[3], rt[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const int row = ys[j] * p.nx;
      rs[j] = 0.25 * s[row + xm] + 0.5 * s[row + x] + 0.25 * s[row + xp];
      rt[j] = 0.25 * th[row + xm] + 0.5 * th[row + x] + 0.25 * th[row + xp];
    }
    sbar = 0.25 * rs[0] + 0.5 * rs[1] + 0.25 * rs[2];
    tbar = 0.25 * rt[0] + 0.5 * rt[1] + 0.25 * rt[2];
  }
  chi_raw = p.c_sensor * sbar * tbar;
  const double chi = chi_raw <= 0.0 ? 0.0 : (chi_raw >= 1.0 ? 1.0 : chi_raw);
  return p.beta_max - (p.beta_max - p.beta_min) * chi;
}

template <int D, class S>
__global__ void __launch_bounds__(kNTA) k_adj_local(const S* __restrict__ fin, const double* __restrict__ lam_in,
                                                     double* __restrict__ lam_out, const KParams p, int pulled,
                                                     const AdjScalars* __restrict__ as, double* __restrict__ F,
                                                     const double* __restrict__ WQ) {
  constexpr int NC = D + 2, Q = 2 * D;
  const int cell = blockIdx.x * kNTA + threadIdx.x;
  if (cell >= p.plane) return;
  const int x = cell % p.nx, y = cell / p.nx;
  const long long P = p.plane;
  const int plane = (int)p.plane;
  const double r = as->r, inv_c = as->inv_c;
  // beta of the forward step
  double chi_raw = 0.0, sbar = 0.0, tbar = 1.0, beta;
  if (p.beta_mode == 0) beta = sensor_at<D>(p, WQ, x, y, chi_raw, sbar, tbar);
  else beta = p.beta_const;
  // adjoint of the streaming: lam*_i(x) = sum over y with nb(y - sigma_i) = x of lam_i(y)
  double ls[Q][NC];
  const bool inner = x >= 1 && x < p.nx - 1 && (D == 1 || (y >= 1 && y < p.ny - 1));
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    if (inner) {  // interior: lam*_i(x) = lam_i(x + sigma_i)
      double v[4];
      const int src = cell + ((i & 1) ? 1 : -1) * (i < 2 ? 1 : p.nx);
      ld4g(lam_in + (i * plane + src) * 4, v);
#pragma unroll
      for (int k = 0; k < NC; ++k) ls[i][k] = v[k];
      continue;
    }
    const int sgn = (i & 1) ? 1 : -1;
    const bool ax = i < 2;
    const int n = ax ? p.nx : p.ny;
    const int lo = ax ? p.bc[0] : p.bc[2], hi = ax ? p.bc[1] : p.bc[3];
    const int j = ax ? x : y;
    const int yA = nb_index(j + sgn, n, lo, hi);
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    if (nb_index(yA - sgn, n, lo, hi) == j) {
      double v[4];
      ld4g(lam_in + (i * plane + (ax ? y * p.nx + yA : yA * p.nx + x)) * 4, v);
#pragma unroll
      for (int k = 0; k < 4; ++k) acc[k] += v[k];
    }
    if (yA != j && nb_index(j - sgn, n, lo, hi) == j) {
      double v[4];
      ld4g(lam_in + (i * plane + cell) * 4, v);
#pragma unroll
      for (int k = 0; k < 4; ++k) acc[k] += v[k];
    }
#pragma unroll
    for (int k = 0; k < NC; ++k) ls[i][k] = acc[k];
  }
  // forward populations, reprojection, equilibrium
  double fr[Q][NC];
  load_state<D, S>(fin, p, x, y, pulled, as->wref, fr);
  double W[NC], Qc[D][NC];
#pragma unroll
  for (int k = 0; k < NC; ++k) W[k] = WQ[(F_W + k) * P + cell];
#pragma unroll
  for (int a = 0; a < D; ++a)
#pragma unroll
    for (int k = 0; k < NC; ++k) Qc[a][k] = WQ[(F_Q + 4 * a + k) * P + cell];
  // f*_i = 2 beta f^eq_i + (1 - 2 beta) (R f)_i with R the (symmetric) reprojection:
  //   dJ/df = (1 - 2 beta) R lam*,  dJ/dbeta = 2 sum_i lam*_i f^eq_i - 2 sum_i (R lam*)_i f_i,
  // and sum_i lam*_i f^eq_i = W/(2D) sum_i lam*_i + 1/(2c) sum_a Q_a (lam*_a+ - lam*_a-).
  double lam_beta = 0.0;
  const double omb = 1.0 - 2.0 * beta;
  const double hr = 0.5 * r, qr2 = 0.25 * r * r, hic = 0.5 * inv_c, bic = beta * inv_c, bd = beta / D;
  double out[Q][NC];
#pragma unroll
  for (int k = 0; k < NC; ++k) {
    // g = R lam* from the pair sums and differences (which the equilibrium terms reuse)
    double g[Q], d[D], sum, qd;
    if constexpr (D == 1) {
      d[0] = ls[1][k] - ls[0][k];
      sum = ls[0][k] + ls[1][k];
      const double w = 0.5 * sum, gx = hr * d[0];
      g[0] = w - gx;
      g[1] = w + gx;
      qd = Qc[0][k] * d[0];
    } else {
      const double sx = ls[0][k] + ls[1][k], sy = ls[2][k] + ls[3][k];
      d[0] = ls[1][k] - ls[0][k];
      d[1] = ls[3][k] - ls[2][k];
      sum = sx + sy;
      const double w = 0.25 * sum, kk = qr2 * (sx - sy), gx = hr * d[0], gy = hr * d[1];
      const double wx = w + kk, wy = w - kk;
      g[0] = wx - gx;
      g[1] = wx + gx;
      g[2] = wy - gy;
      g[3] = wy + gy;
      qd = fma(Qc[0][k], d[0], Qc[1][k] * d[1]);
    }
    double gf = 0.0;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      out[i][k] = omb * g[i];
      gf = fma(g[i], fr[i][k], gf);
    }
#pragma unroll
    for (int a = 0; a < D; ++a) F[(F_LQEQ + 4 * a + k) * P + cell] = bic * d[a];
    lam_beta += 2.0 * ((W[k] * (1.0 / (2 * D))) * sum + hic * qd - gf);
    F[(F_LWEQ + k) * P + cell] = bd * sum;  // 2 beta / (2D) sum_i lam*_i
  }
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    double v[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
    for (int k = 0; k < NC; ++k) v[k] = out[i][k];
    st4g(lam_out + (i * plane + cell) * 4, v);
  }
  // beta = beta_max - (beta_max - beta_min) clip(C s_bar theta_bar)
  double lsb = 0.0, ltb = 0.0;
  if (p.beta_mode == 0 && chi_raw > 0.0 && chi_raw < 1.0) {
    const double lchi = -(p.beta_max - p.beta_min) * lam_beta;
    lsb = p.c_sensor * tbar * lchi;
    ltb = p.c_sensor * sbar * lchi;
  }
  F[F_LSB * P + cell] = lsb;
  F[F_LTB * P + cell] = ltb;
}

// Transposed box filters; adjoint of s = sqrt(mean s_hat^2), s_hat = j / M, theta(dil, vort);
// per-CTA partial sums of dJ/dM_k.
template <int D>
__global__ void __launch_bounds__(kNTA) k_adj_filter(const KParams p, const AdjScalars* __restrict__ as,
                                                      double* __restrict__ F, double* __restrict__ part,
                                                      const double* __restrict__ WQ) {
  constexpr int NC = D + 2;
  __shared__ double red[kNTA][4];
  const int cell = blockIdx.x * kNTA + threadIdx.x;
  double lM[4] = {0.0, 0.0, 0.0, 0.0};
  if (cell < p.plane) {
    const int x = cell % p.nx, y = cell / p.nx;
    const long long P = p.plane;
    double ls = 0.0, lt = 0.0;
    const bool inner = x >= 1 && x < p.nx - 1 && (D == 1 || (y >= 1 && y < p.ny - 1));
    if (inner) {  // the (1/4, 1/2, 1/4) filters are symmetric: their transposes are the filters
      const double* l1 = F + F_LSB * P;
      if constexpr (D == 1) {
        ls = 0.25 * (l1[cell - 1] + 2.0 * l1[cell] + l1[cell + 1]);
      } else {
        const double* l2 = F + F_LTB * P;
        const int nx = p.nx;
        double rs[3], rt[3];
#pragma unroll
        for (int j = 0; j < 3; ++j) {
          const int c0 = cell + (j - 1) * nx;
          rs[j] = (l1[c0 - 1] + 2.0 * l1[c0]) + l1[c0 + 1];
          rt[j] = (l2[c0 - 1] + 2.0 * l2[c0]) + l2[c0 + 1];
        }
        ls = 0.0625 * ((rs[0] + 2.0 * rs[1]) + rs[2]);
        lt = 0.0625 * ((rt[0] + 2.0 * rt[1]) + rt[2]);
      }
    } else {  // boundary cells: the distinct cells of the stencil after the boundary rule
      const Cand cx = candidates(x, p.nx, p.bc[0], p.bc[1]);
      Cand cy;
      if constexpr (D == 2) cy = candidates(y, p.ny, p.bc[2], p.bc[3]);
      else {
        cy.n = 1;
        cy.c[0] = 0;
      }
      for (int a = 0; a < cx.n; ++a) {
        const double wx = filt_w(cx.c[a], x, p.nx, p.bc[0], p.bc[1]);
        for (int b = 0; b < cy.n; ++b) {
          const double wy = D == 2 ? filt_w(cy.c[b], y, p.ny, p.bc[2], p.bc[3]) : 1.0;
          const int src = cy.c[b] * p.nx + cx.c[a];
          ls += wx * wy * F[F_LSB * P + src];
          if constexpr (D == 2) lt += wx * wy * F[F_LTB * P + src];
        }
      }
    }
    const double s = WQ[F_S * P + cell];
    const double ls_s = s > 0.0 ? ls * rcp_(NC * s) : 0.0;  // d s / d s_hat_k = s_hat_k / (NC s)
#pragma unroll
    for (int k = 0; k < NC; ++k) {
      const double sh = WQ[(F_SH + k) * P + cell];
      const double lsh = ls_s * sh;
      F[(F_LJ + k) * P + cell] = lsh * 0.5 * as->invM[k];  // s_hat = (1/2)(dQ sums) / M
      lM[k] = -lsh * sh * as->invM[k];
    }
    if constexpr (D == 2) {
      const double dil = WQ[F_DIL * P + cell], vort = WQ[F_VORT * P + cell];
      const double den = dil * dil + vort * vort + p.ducros_eps;
      const double l2 = 2.0 * lt * rcp_(den * den);
      F[F_LDIL * P + cell] = l2 * dil * (vort * vort + p.ducros_eps);
      F[F_LVORT * P + cell] = -l2 * vort * dil * dil;
    }
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) red[threadIdx.x][k] = lM[k];
  __syncthreads();
  for (int s = kNTA / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s)
#pragma unroll
      for (int k = 0; k < 4; ++k) red[threadIdx.x][k] += red[threadIdx.x + s][k];
    __syncthreads();
  }
  if ((int)threadIdx.x < 4) part[blockIdx.x * 8 + threadIdx.x] = red[0][threadIdx.x];
}

// Fixed-order (deterministic) fold of per-CTA partial sums: out[j] = sum_c part[c * 8 + j], j < nv.
// First stage: the sum of each group of kGroup per-CTA partials (one warp each, a fixed shuffle
// tree).
__global__ void __launch_bounds__(kGroup) k_adj_fold_groups(const double* __restrict__ part, int nparts, int nv,
                                                            double* __restrict__ gpart) {
  const int c = blockIdx.x * kGroup + threadIdx.x;
#pragma unroll
  for (int j = 0; j < 5; ++j) {
    if (j >= nv) break;
    double v = c < nparts ? part[c * 8 + j] : 0.0;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    if (threadIdx.x == 0) gpart[blockIdx.x * 8 + j] = v;
  }
}

__global__ void __launch_bounds__(kNTF) k_adj_fold(const double* __restrict__ part, int nparts, int nv, double* out,
                                                    double* comp, int accumulate) {
  // fixed order: thread t sums partials t, t + kNTF, ... in turn; then a fixed shuffle tree per
  // warp and one over the warps (deterministic)
  __shared__ double red[kNTF / 32][5];
  double v[5] = {0, 0, 0, 0, 0};
  for (int c = threadIdx.x; c < nparts; c += kNTF)
#pragma unroll
    for (int j = 0; j < 5; ++j)
      if (j < nv) v[j] += part[c * 8 + j];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int j = 0; j < 5; ++j) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v[j] += __shfl_xor_sync(0xffffffffu, v[j], off);
    if (lane == 0) red[warp][j] = v[j];
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int j = 0; j < 5; ++j) {
      v[j] = lane < kNTF / 32 ? red[lane][j] : 0.0;
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) v[j] += __shfl_xor_sync(0xffffffffu, v[j], off);
    }
  }
  if (threadIdx.x == 0)
#pragma unroll
    for (int j = 0; j < 5; ++j) {
      if (j >= nv) break;
      const double x = v[j];
      if (!accumulate) {
        out[j] = x;
      } else {  // Neumaier-compensated running sum
        const double s = out[j], t = s + x;
        comp[j] += fabs(s) >= fabs(x) ? (s - t) + x : (x - t) + s;
        out[j] = t;
      }
    }
}

template <int D>
__global__ void __launch_bounds__(kNTA) k_adj_flux(double* __restrict__ lam_out, const KParams p,
                                                    const AdjScalars* __restrict__ as, const double* __restrict__ F,
                                                    double* __restrict__ part,
                                                    const double* __restrict__ WQ) {
  constexpr int NC = D + 2, Q = 2 * D;
  __shared__ double red[kNTA][5];
  const int cell = blockIdx.x * kNTA + threadIdx.x;
  double le[5] = {0, 0, 0, 0, 0};
  if (cell < p.plane) {
    const int x = cell % p.nx, y = cell / p.nx;
    const long long P = p.plane;
    const int plane = (int)p.plane;
    double lQ[D][NC], lu[D];
#pragma unroll
    for (int a = 0; a < D; ++a) {
      lu[a] = 0.0;
#pragma unroll
      for (int k = 0; k < NC; ++k) lQ[a][k] = F[(F_LQEQ + 4 * a + k) * P + cell];
    }
    // transposed central differences along each axis (sensor jumps, dilatation, vorticity):
    // v(x) enters the differences centred at x - 1 (+1) and x + 1 (-1)
    const bool inner = x >= 1 && x < p.nx - 1 && (D == 1 || (y >= 1 && y < p.ny - 1));
    if (inner) {
#pragma unroll
      for (int a = 0; a < D; ++a) {
        const int dn = a == 0 ? 1 : p.nx;
        const int cm = cell - dn, cp = cell + dn;
#pragma unroll
        for (int k = 0; k < NC; ++k) lQ[a][k] += F[(F_LJ + k) * P + cm] - F[(F_LJ + k) * P + cp];
        if constexpr (D == 2) {
          const double ld = F[F_LDIL * P + cm] - F[F_LDIL * P + cp], lv = F[F_LVORT * P + cm] - F[F_LVORT * P + cp];
          lu[a] += p.inv2dx * ld;
          if (a == 0) lu[1] += p.inv2dx * lv;
          else lu[0] -= p.inv2dx * lv;
        }
      }
    } else {
#pragma unroll
    for (int a = 0; a < D; ++a) {
      const bool ax = a == 0;
      const int n = ax ? p.nx : p.ny, lo = ax ? p.bc[0] : p.bc[2], hi = ax ? p.bc[1] : p.bc[3];
      const int j = ax ? x : y;
      const Cand c = candidates(j, n, lo, hi);
      for (int q = 0; q < c.n; ++q) {
        const double w = diff_w(c.c[q], j, n, lo, hi);
        if (w == 0.0) continue;
        const int src = ax ? y * p.nx + c.c[q] : c.c[q] * p.nx + x;
#pragma unroll
        for (int k = 0; k < NC; ++k) lQ[a][k] += w * F[(F_LJ + k) * P + src];  // F_LJ: d/d(raw jump)
        if constexpr (D == 2) {
          const double ld = F[F_LDIL * P + src], lv = F[F_LVORT * P + src];
          lu[a] += w * p.inv2dx * ld;                    // dil: d u_a / d a
          if (ax) lu[1] += w * p.inv2dx * lv;            // vort: + d u_y / dx
          else lu[0] -= w * p.inv2dx * lv;               //       - d u_x / dy
        }
      }
    }
    }  // generic (boundary) branch
    // derivative of M_k goes to its argmax element
#pragma unroll
    for (int k = 0; k < NC; ++k) {
      if (as->amax_cell[k] == cell) {
        const int a = as->amax_alpha[k];
        const double q = WQ[(F_Q + 4 * a + k) * P + cell];
        lQ[a][k] += (q > 0.0 ? 1.0 : (q < 0.0 ? -1.0 : 0.0)) * as->lamM[k];
      }
    }
    double W[NC], lW[NC], dprm[5];
#pragma unroll
    for (int k = 0; k < NC; ++k) {
      W[k] = WQ[(F_W + k) * P + cell];
      lW[k] = F[(F_LWEQ + k) * P + cell];
    }
    const double lP = flux_vjp<D>(p, W, lQ, lu, lW, dprm);
#pragma unroll
    for (int j = 0; j < 5; ++j) le[j] = lP * dprm[j];
    // lambda^n_i += dJ/dW (W = sum_i f_i)
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      double v[4];
      ld4g(lam_out + (i * plane + cell) * 4, v);
#pragma unroll
      for (int k = 0; k < NC; ++k) v[k] += lW[k];
      st4g(lam_out + (i * plane + cell) * 4, v);
    }
  }
#pragma unroll
  for (int j = 0; j < 5; ++j) red[threadIdx.x][j] = le[j];
  __syncthreads();
  for (int s = kNTA / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s)
#pragma unroll
      for (int j = 0; j < 5; ++j) red[threadIdx.x][j] += red[threadIdx.x + s][j];
    __syncthreads();
  }
  if ((int)threadIdx.x < 5) part[blockIdx.x * 8 + threadIdx.x] = red[0][threadIdx.x];
}

// lambda^N_{i,k} = dJ/dW_k(T) for every direction i (W(T) = sum_i f^N_i).
template <int D>
__global__ void __launch_bounds__(kNTA) k_adj_terminal(const double* __restrict__ dJ_dW, double* __restrict__ lam,
                                                        const KParams p) {
  constexpr int NC = D + 2;
  const int cell = blockIdx.x * kNTA + threadIdx.x;
  if (cell >= p.plane) return;
  double v[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
  for (int k = 0; k < NC; ++k) v[k] = dJ_dW[k * p.plane + cell];
#pragma unroll
  for (int i = 0; i < 2 * D; ++i) st4g(lam + (i * (int)p.plane + cell) * 4, v);
}

// Initialisation f^0 = f^eq(W0; c0) (Eq. 20): dJ/dW0 and the EOS-parameter partial sums.
template <int D>
__global__ void __launch_bounds__(kNTA) k_adj_init(const double* __restrict__ W0, const double* __restrict__ lam0,
                                                    const KParams p, double c0, double* __restrict__ dJ_dW0,
                                                    double* __restrict__ part) {
  constexpr int NC = D + 2;
  __shared__ double red[kNTA][5];
  const int cell = blockIdx.x * kNTA + threadIdx.x;
  double le[5] = {0, 0, 0, 0, 0};
  if (cell < p.plane) {
    double W[NC], lW[NC], lQ[D][NC], lu[D], dprm[5], l[2 * D][4];
#pragma unroll
    for (int i = 0; i < 2 * D; ++i) ld4g(lam0 + (i * (int)p.plane + cell) * 4, l[i]);
#pragma unroll
    for (int k = 0; k < NC; ++k) {
      W[k] = W0[k * p.plane + cell];
      double s = 0.0;
#pragma unroll
      for (int i = 0; i < 2 * D; ++i) s += l[i][k];
      lW[k] = s / (2.0 * D);
    }
#pragma unroll
    for (int a = 0; a < D; ++a) {
      lu[a] = 0.0;
#pragma unroll
      for (int k = 0; k < NC; ++k) lQ[a][k] = (l[2 * a + 1][k] - l[2 * a][k]) / (2.0 * c0);
    }
    const double lP = flux_vjp<D>(p, W, lQ, lu, lW, dprm);
#pragma unroll
    for (int j = 0; j < 5; ++j) le[j] = lP * dprm[j];
#pragma unroll
    for (int k = 0; k < NC; ++k) dJ_dW0[k * p.plane + cell] = lW[k];
  }
#pragma unroll
  for (int j = 0; j < 5; ++j) red[threadIdx.x][j] = le[j];
  __syncthreads();
  for (int s = kNTA / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s)
#pragma unroll
      for (int j = 0; j < 5; ++j) red[threadIdx.x][j] += red[threadIdx.x + s][j];
    __syncthreads();
  }
  if ((int)threadIdx.x < 5) part[blockIdx.x * 8 + threadIdx.x] = red[0][threadIdx.x];
}

__global__ void k_adj_begin(AdjScalars* as) {
  for (int j = 0; j < 5; ++j) {
    as->eos[j] = 0.0;
    as->eos_comp[j] = 0.0;
  }
}

__global__ void k_adj_finish(AdjScalars* as) {
  for (int j = 0; j < 5; ++j) as->eos[j] += as->eos_comp[j];
}

// Scalars of the forward recomputation of a segment: start at step n0 with link speed c_{n0-1}.
__global__ void k_adj_replay_scalars(Scalars* sc, long long n0, const double* sched, long long sched_len) {
  sc->n = n0;
  sc->c_prev = sched[n0];
  sc->t = 0.0;
  sc->t_end = 0.0;
  sc->done = 0;
  sc->err = 0;
  sc->sched_len = sched_len;
}

// ------------------------------------------------------------------------------------------
// host launchers
// ------------------------------------------------------------------------------------------
namespace {
unsigned cells_blocks(const KParams& p) { return (unsigned)((p.plane + kNTA - 1) / kNTA); }
// device address of a member of the (device-resident) adjoint scalar block
double* adj_field(AdjScalars* as, size_t off) { return reinterpret_cast<double*>(reinterpret_cast<char*>(as) + off); }
}  // namespace

int adj_part_entries(const KParams& p) { return (int)cells_blocks(p) + 1; }
int adj_group_entries(const KParams& p) { return (int)((cells_blocks(p) + kGroup - 1) / kGroup) + 1; }

template <int D, class S>
static cudaError_t adj_step_t(const AdjLaunch& A, const S* fin, int pulled, const double* lam_in, double* lam_out,
                              long long n, double* kept, bool kept_sensor, const double* sensor) {
  const KParams& p = *A.p;
  const unsigned nb = cells_blocks(p);
  double* WQ = kept ? kept : A.F;  // planes F_W .. F_VORT of this step
  if (!kept && sensor) {
    const cudaError_t e = cudaMemcpyAsync(A.F + (size_t)F_SH * p.plane, sensor, (size_t)8 * p.plane * sizeof(double),
                                          cudaMemcpyDeviceToDevice, A.stream);
    if (e != cudaSuccess) return e;
  }
  if (kept) k_adj_argmax_kept<D><<<nb, kNTA, 0, A.stream>>>(kept, p, A.pv, A.pi);
  else k_adj_fields<D, S><<<nb, kNTA, 0, A.stream>>>(fin, p, pulled, A.as, A.F, A.pv, A.pi);
  const unsigned ng = (nb + kGroup - 1) / kGroup;
  k_adj_argmax_groups<<<ng, kGroup, 0, A.stream>>>(A.pv, A.pi, nb, p.nc, A.gpart, A.gidx);
  k_adj_argmax_fold<<<1, kNTF, 0, A.stream>>>(A.gpart, A.gidx, ng, p.nc, p.plane, A.as, A.sched, n);
  if (!(kept && kept_sensor) && !(!kept && sensor)) k_adj_sensor<D><<<nb, kNTA, 0, A.stream>>>(p, A.as, WQ, WQ);
  k_adj_local<D, S><<<nb, kNTA, 0, A.stream>>>(fin, lam_in, lam_out, p, pulled, A.as, A.F, WQ);
  k_adj_filter<D><<<nb, kNTA, 0, A.stream>>>(p, A.as, A.F, A.part, WQ);
  k_adj_fold_groups<<<ng, kGroup, 0, A.stream>>>(A.part, nb, p.nc, A.gpart);
  k_adj_fold<<<1, kNTF, 0, A.stream>>>(A.gpart, ng, p.nc, adj_field(A.as, offsetof(AdjScalars, lamM)), nullptr, 0);
  k_adj_flux<D><<<nb, kNTA, 0, A.stream>>>(lam_out, p, A.as, A.F, A.part, WQ);
  k_adj_fold_groups<<<ng, kGroup, 0, A.stream>>>(A.part, nb, 5, A.gpart);
  k_adj_fold<<<1, kNTF, 0, A.stream>>>(A.gpart, ng, 5, adj_field(A.as, offsetof(AdjScalars, eos)),
                                       adj_field(A.as, offsetof(AdjScalars, eos_comp)), 1);
  return cudaGetLastError();
}

cudaError_t adj_step(const AdjLaunch& A, int precision, const void* fin, int pulled, const double* lam_in, double* lam_out,
                     long long n, double* kept, bool kept_sensor, const double* sensor) {
  if (A.p->dim == 1) kept = nullptr, sensor = nullptr;  // kept fields exist for 2D strips only
  if (precision == 0)
    return A.p->dim == 1 ? adj_step_t<1, double>(A, (const double*)fin, pulled, lam_in, lam_out, n, kept, kept_sensor, sensor)
                         : adj_step_t<2, double>(A, (const double*)fin, pulled, lam_in, lam_out, n, kept, kept_sensor, sensor);
  return A.p->dim == 1 ? adj_step_t<1, float>(A, (const float*)fin, pulled, lam_in, lam_out, n, kept, kept_sensor, sensor)
                       : adj_step_t<2, float>(A, (const float*)fin, pulled, lam_in, lam_out, n, kept, kept_sensor, sensor);
}

cudaError_t adj_terminal(const AdjLaunch& A, const double* dJ_dW, double* lam) {
  const KParams& p = *A.p;
  if (p.dim == 1) k_adj_terminal<1><<<cells_blocks(p), kNTA, 0, A.stream>>>(dJ_dW, lam, p);
  else k_adj_terminal<2><<<cells_blocks(p), kNTA, 0, A.stream>>>(dJ_dW, lam, p);
  k_adj_begin<<<1, 1, 0, A.stream>>>(A.as);
  return cudaGetLastError();
}

cudaError_t adj_init(const AdjLaunch& A, const double* W0, const double* lam0, double c0, double* dJ_dW0) {
  const KParams& p = *A.p;
  const unsigned nb = cells_blocks(p);
  if (p.dim == 1) k_adj_init<1><<<nb, kNTA, 0, A.stream>>>(W0, lam0, p, c0, dJ_dW0, A.part);
  else k_adj_init<2><<<nb, kNTA, 0, A.stream>>>(W0, lam0, p, c0, dJ_dW0, A.part);
  const unsigned ng = (nb + kGroup - 1) / kGroup;
  k_adj_fold_groups<<<ng, kGroup, 0, A.stream>>>(A.part, nb, 5, A.gpart);
  k_adj_fold<<<1, kNTF, 0, A.stream>>>(A.gpart, ng, 5, adj_field(A.as, offsetof(AdjScalars, eos)),
                                       adj_field(A.as, offsetof(AdjScalars, eos_comp)), 1);
  k_adj_finish<<<1, 1, 0, A.stream>>>(A.as);
  return cudaGetLastError();
}

cudaError_t adj_replay_scalars(cudaStream_t s, Scalars* sc, long long n0, const double* sched, long long sched_len) {
  k_adj_replay_scalars<<<1, 1, 0, s>>>(sc, n0, sched, sched_len);
  return cudaGetLastError();
}

}  // namespace vlbm
