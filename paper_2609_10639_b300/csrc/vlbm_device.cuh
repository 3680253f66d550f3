// Device helpers shared by the step kernels and the adjoint kernels of the VLBM library:
// boundary index rules, vector access to the population layout [i][y][x][4], arithmetic helpers,
// thermodynamics (Sec. II C), primitives and flux (Eqs. 1-2, 10), population loads and stores,
// and the two-level reduction of the global maxima (Eqs. 30, 36).
#pragma once

#include <cmath>
#include <type_traits>

#include "vlbm_internal.cuh"

namespace vlbm {

// ------------------------------------------------------------------------------------------
// index rules
// ------------------------------------------------------------------------------------------
// Cell index read at position j along an axis of n cells: wrap (periodic) or clamp to the edge
// (zero-gradient).  Positions beyond a pinned-inflow side (lo == 2) hold the ghost state, which
// the callers supply themselves; the clamp only keeps any index inside the buffer.
__device__ __forceinline__ int nb_index(int j, int n, int lo, int hi) {
  if (j < 0) {
    if (lo == 0) {
      do { j += n; } while (j < 0);
      return j;
    }
    return 0;
  }
  if (j >= n) {
    if (hi == 0) {
      do { j -= n; } while (j >= n);
      return j;
    }
    return n - 1;
  }
  return j;
}

// Position at which a stencil quantity "at" position j is evaluated: the edge cell beyond a
// zero-gradient side (the ghost replicates the edge cell), j itself otherwise (periodic sides are
// unwrapped, the region holds the wrapped values there; beyond a pinned-inflow side the region
// holds the ghost cells' own values).
__device__ __forceinline__ int centre_pos(int j, int n, int lo, int hi) {
  if (j < 0 && lo == 1) return 0;
  if (j >= n && hi == 1) return n - 1;
  return j;
}

// Lattice unit vectors sigma_i in the order {x-, x+, y-, y+} (Eq. 18).
__device__ __forceinline__ int sig_x(int i) { return i == 0 ? -1 : (i == 1 ? 1 : 0); }
__device__ __forceinline__ int sig_y(int i) { return i == 2 ? -1 : (i == 3 ? 1 : 0); }

// 4-wide vector access (one lattice direction of one cell: its components k = 0..3, slot 3 unused
// in 1D).  FP32: one 128-bit access; FP64: two.
__device__ __forceinline__ void ld4g(const float* p, float (&v)[4]) {
  const float4 t = __ldg(reinterpret_cast<const float4*>(p));
  v[0] = t.x, v[1] = t.y, v[2] = t.z, v[3] = t.w;
}
__device__ __forceinline__ void ld4g(const double* p, double (&v)[4]) {
  const double2 a = __ldg(reinterpret_cast<const double2*>(p)), b = __ldg(reinterpret_cast<const double2*>(p) + 1);
  v[0] = a.x, v[1] = a.y, v[2] = b.x, v[3] = b.y;
}
__device__ __forceinline__ void st4g(float* p, const float (&v)[4]) {
  *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
__device__ __forceinline__ void st4g(double* p, const double (&v)[4]) {
  reinterpret_cast<double2*>(p)[0] = make_double2(v[0], v[1]);
  reinterpret_cast<double2*>(p)[1] = make_double2(v[2], v[3]);
}
__device__ __forceinline__ void ld4s(const float* p, float (&v)[4]) {
  const float4 t = *reinterpret_cast<const float4*>(p);
  v[0] = t.x, v[1] = t.y, v[2] = t.z, v[3] = t.w;
}
__device__ __forceinline__ void ld4s(const double* p, double (&v)[4]) {
  const double2 a = reinterpret_cast<const double2*>(p)[0], b = reinterpret_cast<const double2*>(p)[1];
  v[0] = a.x, v[1] = a.y, v[2] = b.x, v[3] = b.y;
}
__device__ __forceinline__ void st4s(float* p, const float (&v)[4]) { st4g(p, v); }
__device__ __forceinline__ void st4s(double* p, const double (&v)[4]) { st4g(p, v); }

// Reciprocal, quotient and square root.  FP64 reciprocal: two Newton-Raphson steps for 1/a
// (e = 1 - a y, y <- y + y e; the relative error squares at each step) from the PTX
// rcp.approx.ftz.f64 seed (relative error ~1e-6 measured on a B300), i.e. ~1e-24 before
// rounding: in a 4M-sample sweep over [6e-6, 2e5] it equalled 1.0/a in every case.  Four FP64
// FMAs, against the longer correctly rounded division sequence.  Zero, infinite and subnormal
// arguments are not meaningful here (rho and 1 - b rho are checked positive and finite); they
// give a non-finite or zero result.  FP32-storage path: the hardware approximations (<= 2 ulp),
// well inside that path's error budget.
__device__ __forceinline__ double rcp_(double a) {
  double y;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(a));
  double e = fma(-a, y, 1.0);
  y = fma(y, e, y);
  e = fma(-a, y, 1.0);
  return fma(y, e, y);
}
__device__ __forceinline__ float rcp_(float x) { return __fdividef(1.0f, x); }
__device__ __forceinline__ double div_(double a, double b) { return a * rcp_(b); }
__device__ __forceinline__ float div_(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double sqrt_(double x) { return sqrt(x); }
__device__ __forceinline__ float sqrt_(float x) { return x > 0.0f ? x * rsqrtf(x) : 0.0f; }

template <class M>
__device__ __forceinline__ const Coef<M>& coef(const KParams& p);
template <>
__device__ __forceinline__ const Coef<double>& coef<double>(const KParams& p) { return p.cd; }
template <>
__device__ __forceinline__ const Coef<float>& coef<float>(const KParams& p) { return p.cf; }

// Step scalars in the arithmetic type of a path (the FP32 copies are written by k_dt).
template <class M>
struct StepScalars;
template <>
struct StepScalars<double> {
  static __device__ __forceinline__ double r(const Scalars* s) { return s->r; }
  static __device__ __forceinline__ double inv_c(const Scalars* s) { return s->inv_c; }
  static __device__ __forceinline__ const double* inv_M(const Scalars* s) { return s->inv_M; }
  static __device__ __forceinline__ double wq(const Scalars* s, int k) { return 0.0; }
};
template <>
struct StepScalars<float> {
  static __device__ __forceinline__ float r(const Scalars* s) { return s->r_f; }
  static __device__ __forceinline__ float inv_c(const Scalars* s) { return s->inv_c_f; }
  static __device__ __forceinline__ const float* inv_M(const Scalars* s) { return s->inv_M_f; }
  static __device__ __forceinline__ float wq(const Scalars* s, int k) { return s->wq_f[k]; }
};

// ------------------------------------------------------------------------------------------
// thermodynamics (Sec. II C)
// ------------------------------------------------------------------------------------------
template <class E>
__device__ __forceinline__ void eos_eval(const KParams& p, const Coef<E>& c, E rho, E inv_rho, E e, E& P, E& cs2) {
  if (p.eos_kind == 0) {  // ideal gas, Eq. (15)
    P = c.gm1 * rho * e;
    cs2 = c.ggm1 * e;
  } else {  // van der Waals, Eqs. (16)-(17); c_s^2 by Eq. (13)
    E T, a_inv_cv = c.a_inv_cv, inv_cv = c.inv_cv;
    if (p.eos_kind == 2) {
      // c_v(T) = cv + cv1 T + cv2 T^2, e = E(T) - a rho with E(T) = cv T + cv1 T^2/2 + cv2 T^3/3:
      // Newton's method on E(T) = e + a rho from T0 = (e + a rho)/cv (E is increasing and convex, so
      // the iterates fall monotonically onto the root); stops when a step changes T by at most
      // 1e-15 T, else after 50 steps T is NaN and the state is reported non-physical
      const E target = e + c.a * rho;
      T = target * c.inv_cv;
      bool conv = false;
#pragma unroll 1
      for (int it = 0; it < 50; ++it) {
        const E ET = T * fma(T, fma(T, c.cv2t, c.cv1h), c.cv0);
        const E cvT = fma(T, fma(T, c.cv2, c.cv1), c.cv0);
        const E step = div_(ET - target, cvT);
        T -= step;
        if (fabs(step) <= (E)1e-15 * fabs(T)) {
          conv = true;
          break;
        }
      }
      if (!conv) T = (E)NAN;
      inv_cv = rcp_(fma(T, fma(T, c.cv2, c.cv1), c.cv0));  // 1 / c_v(T)
      a_inv_cv = c.a * inv_cv;
    } else {
      T = (e + c.a * rho) * c.inv_cv;
    }
    const E inv_omb = rcp_((E)1 - c.b * rho);
    const E RT_omb = c.R * T * inv_omb;
    P = rho * RT_omb - c.a * rho * rho;
    const E dPdT = c.R * rho * inv_omb;                                     // (dP/dT)_rho
    const E P_rho = RT_omb * inv_omb - (E)2 * c.a * rho + dPdT * a_inv_cv;  // (dP/drho)_e
    const E P_e = dPdT * inv_cv;                                            // (dP/de)_rho
    cs2 = P_rho + P * inv_rho * inv_rho * P_e;
  }
}

// Primitives and flux of one state (Eqs. 1-2, 10); with NEED_CS also c_s and the physical-state
// check (returns false for rho <= 0, c_s^2 <= 0 or non-finite values).  In the FP32 path the van
// der Waals energy-to-temperature inversion and pressure run in FP64.
template <int D, class M, bool NEED_CS>
__device__ __forceinline__ bool prim_flux(const KParams& p, const M (&W)[D + 2], M (&u)[D], M (&Qf)[D][D + 2], M& cs,
                                          M* P_out = nullptr) {
  constexpr int NC = D + 2;
  const M rho = W[0];
  M P, cs2;
  if (std::is_same<M, float>::value && p.eos_kind != 0) {
    const double rd = (double)rho, ird = 1.0 / rd;
    double usq = 0.0;
#pragma unroll
    for (int a = 0; a < D; ++a) {
      const double ua = (double)W[1 + a] * ird;
      u[a] = (M)ua;
      usq += ua * ua;
    }
    const double e = (double)W[NC - 1] * ird - 0.5 * usq;
    double Pd, cd;
    eos_eval<double>(p, p.cd, rd, ird, e, Pd, cd);
    P = (M)Pd;
    cs2 = (M)cd;
  } else {
    const M inv_rho = rcp_(rho);
    M usq = 0;
#pragma unroll
    for (int a = 0; a < D; ++a) {
      u[a] = W[1 + a] * inv_rho;
      usq += u[a] * u[a];
    }
    const M e = W[NC - 1] * inv_rho - (M)0.5 * usq;
    eos_eval<M>(p, coef<M>(p), rho, inv_rho, e, P, cs2);
  }
  bool ok = true;
  if (NEED_CS) {
    ok = (rho > (M)0) && (cs2 > (M)0) && isfinite(cs2) && isfinite(P);
    cs = sqrt_(cs2 > (M)0 ? cs2 : (M)0);
  }
  if (P_out) *P_out = P;
#pragma unroll
  for (int a = 0; a < D; ++a) {
    Qf[a][0] = W[1 + a];
#pragma unroll
    for (int b = 0; b < D; ++b) Qf[a][1 + b] = W[1 + b] * u[a] + (a == b ? P : (M)0);
    Qf[a][NC - 1] = (W[NC - 1] + P) * u[a];
  }
  return ok;
}

// FP32 storage with a non-ideal gas: velocity and flux of W with the pressure P already known
// (kept from the pass that computed it for the same W), the same operations as prim_flux's
// non-ideal FP32 branch without the FP64 EOS evaluation, so the result is bit-identical.
template <int D>
__device__ __forceinline__ void flux_given_P(const float (&W)[D + 2], float P, float (&u)[D], float (&Qf)[D][D + 2]) {
  constexpr int NC = D + 2;
  const double ird = 1.0 / (double)W[0];
#pragma unroll
  for (int a = 0; a < D; ++a) u[a] = (float)((double)W[1 + a] * ird);
#pragma unroll
  for (int a = 0; a < D; ++a) {
    Qf[a][0] = W[1 + a];
#pragma unroll
    for (int b = 0; b < D; ++b) Qf[a][1 + b] = W[1 + b] * u[a] + (a == b ? P : 0.0f);
    Qf[a][NC - 1] = (W[NC - 1] + P) * u[a];
  }
}

// ------------------------------------------------------------------------------------------
// storage: FP64 holds f_i; FP32 holds d_i = f_i - W_ref/Q (W_ref a per-run FP64 constant)
// ------------------------------------------------------------------------------------------
template <class S>
struct Store;
template <>
struct Store<double> {
  using M = double;
  static constexpr bool kOffset = false;
};
template <>
struct Store<float> {
  using M = float;
  static constexpr bool kOffset = true;
};

// ------------------------------------------------------------------------------------------
// pinned inflow (x-lo side, VLBM_BC_INFLOW; Sec. IV H): every ghost cell x < 0 holds the state
// W_in; its populations are the equilibrium of W_in (Eq. 20) at the link speed of the stored
// populations, 1/c = ginv (a relaxed ghost stays that equilibrium, reprojected to the new speed).
// ------------------------------------------------------------------------------------------
template <int D, class M>
__device__ __forceinline__ void ghost_state(const KParams& p, M (&W)[D + 2], M (&u)[D], M (&Qf)[D][D + 2]) {
  const Coef<M>& co = coef<M>(p);
#pragma unroll
  for (int k = 0; k < D + 2; ++k) W[k] = co.win[k];
  M cs;
  prim_flux<D, M, false>(p, W, u, Qf, cs);
}

// Population i of a ghost cell, in the storage representation (FP32 storage: minus W_ref/Q; wq
// holds Q W_ref/Q per component).
template <int D, class M, bool OFFSET>
__device__ __forceinline__ void ghost_population(const KParams& p, const M* wq, M ginv, int i, M (&v)[D + 2]) {
  M W[D + 2], u[D], Qf[D][D + 2];
  ghost_state<D, M>(p, W, u, Qf);
  constexpr M inv_q = (M)1 / (M)(2 * D);
#pragma unroll
  for (int k = 0; k < D + 2; ++k) {
    M ciQ = (M)sig_x(i) * Qf[0][k];
    if constexpr (D == 2) ciQ += (M)sig_y(i) * Qf[1][k];
    v[k] = (OFFSET ? W[k] - wq[k] : W[k]) * inv_q + (M)0.5 * ginv * ciQ;
  }
}

// The values of a pinned-inflow ghost cell, the same for every ghost and every thread of a launch:
// populations (storage representation), W, u, Q.  Filled once per CTA (fill_ghost_tab, one thread,
// then a barrier) into shared memory, so that the ghost paths of the kernels are plain loads.
template <int D, class M>
struct GhostTab {
  M f[2 * D][D + 2];
  M W[D + 2], u[D], Q[D][D + 2];
};

template <int D, class M, bool OFFSET>
__device__ __noinline__ void fill_ghost_tab(const KParams& p, const M* wq, M ginv, GhostTab<D, M>& g) {
#pragma unroll 1
  for (int i = 0; i < 2 * D; ++i) ghost_population<D, M, OFFSET>(p, wq, ginv, i, g.f[i]);
  ghost_state<D, M>(p, g.W, g.u, g.Q);
}

// Loads the populations of cell (cx, cy), pulled across the links (or in place), into fr[i][k].
// Layout [i][y][x][4]: one vector access per direction.  `interior`: the caller guarantees that
// (cx, cy) and its four neighbours lie inside the domain (no boundary rule needed).  gpop: the
// ghost populations [i][k] of a pinned-inflow side (GhostTab::f), nullptr without one; a pull from
// beyond that side takes them.  Offsets are 32-bit (vlbm_create bounds 2D * 4 * nx * ny below 2^31).
template <int D, class S>
__device__ __forceinline__ void load_cell(const S* __restrict__ fin, const KParams& p, int cx, int cy, int pulled,
                                          bool interior, typename Store<S>::M (&fr)[2 * D][D + 2],
                                          const typename Store<S>::M* gpop = nullptr) {
  using M = typename Store<S>::M;
  constexpr int NC = D + 2, Q = 2 * D;
  const int plane = (int)p.plane;
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    int sx = cx, sy = cy;
    if (pulled) {
      if (interior) {
        sx = cx - sig_x(i);
        sy = cy - sig_y(i);
      } else {
        if (gpop && cx - sig_x(i) < 0) {
#pragma unroll
          for (int k = 0; k < NC; ++k) fr[i][k] = gpop[i * NC + k];
          continue;
        }
        sx = nb_index(cx - sig_x(i), p.nx, p.bc[0], p.bc[1]);
        if (D == 2) sy = nb_index(cy - sig_y(i), p.ny, p.bc[2], p.bc[3]);
      }
    }
    S v[4];
    ld4g(fin + (i * plane + sy * p.nx + sx) * 4, v);
#pragma unroll
    for (int k = 0; k < NC; ++k) fr[i][k] = (M)v[k];
  }
}

// Stores one cell's populations f[i][k] (layout [i][y][x][4]).
template <int D, class S, class M>
__device__ __forceinline__ void store_cell(S* __restrict__ fout, const KParams& p, int cell, const M (&f)[2 * D][D + 2]) {
  const int plane = (int)p.plane;
#pragma unroll
  for (int i = 0; i < 2 * D; ++i) {
    S v[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) v[k] = k < D + 2 ? (S)f[i][k] : (S)0;
    st4g(fout + (i * plane + cell) * 4, v);
  }
}

// Zeroth moment of one cell: W_k = sum_i f_i (direction pairs first); in FP32 storage the sum of
// deviations plus Q W_ref/Q (wq).
template <int D, class M, bool OFFSET>
__device__ __forceinline__ void moments(const M (&fr)[2 * D][D + 2], const M* wq, M (&W)[D + 2]) {
#pragma unroll
  for (int k = 0; k < D + 2; ++k) {
    M acc = fr[0][k] + fr[1][k];
    if constexpr (D == 2) acc += fr[2][k] + fr[3][k];
    if constexpr (OFFSET) acc += wq[k];
    W[k] = acc;
  }
}

// Fused reprojection (c_old -> c_new, Eqs. 38-40) and relaxation (Eqs. 20, 22) of one cell:
//   f*_{a,+-} = W/Q  +-  [ beta Q_a / c + (1 - 2 beta) r (f_{a+} - f_{a-}) / 2 ]
//               (+ for x, - for y)  (1 - 2 beta) r^2 ((f_x+ + f_x-) - (f_y+ + f_y-)) / 4   (D2Q4 K-term),
// r = c_old / c_new.  In 2D the W/4 and K-terms of a direction pair combine into
//   (1/4 + k) S_x + (1/4 - k) S_y  (x pair),   (1/4 - k) S_x + (1/4 + k) S_y  (y pair),
// with S_a = f_{a+} + f_{a-} and k = (1 - 2 beta) r^2 / 4.  In FP32 storage the same update acts
// on the deviations (W/Q -> dW/Q).
template <int D, class M>
__device__ __forceinline__ void relax_cell(M (&f)[2 * D][D + 2], const M (&Qc)[D][D + 2], M beta, M r, M inv_c) {
  constexpr int NC = D + 2;
  const M om = (M)1 - (M)2 * beta;
  const M bq = beta * inv_c;
  const M omr = om * r * (M)0.5;
  if constexpr (D == 1) {
#pragma unroll
    for (int k = 0; k < NC; ++k) {
      const M w = (f[0][k] + f[1][k]) * (M)0.5;
      const M gx = bq * Qc[0][k] + omr * (f[1][k] - f[0][k]);
      f[0][k] = w - gx;
      f[1][k] = w + gx;
    }
  } else {
    const M omk = om * r * r * (M)0.25;
    const M cp = (M)0.25 + omk, cm = (M)0.25 - omk;
#pragma unroll
    for (int k = 0; k < NC; ++k) {
      const M sx = f[0][k] + f[1][k], sy = f[2][k] + f[3][k];
      const M gx = bq * Qc[0][k] + omr * (f[1][k] - f[0][k]);
      const M gy = bq * Qc[1][k] + omr * (f[3][k] - f[2][k]);
      const M wx = cp * sx + cm * sy, wy = cm * sx + cp * sy;
      f[0][k] = wx - gx;
      f[1][k] = wx + gx;
      f[2][k] = wy - gy;
      f[3][k] = wy + gy;
    }
  }
}

// FP32 storage, D2Q4: the same two updates on component pairs (k = 0,1 and k = 2,3) with the
// packed two-lane FP32 instructions of sm_100 and later (each lane rounds like the scalar
// operation), halving the FP32 instruction count of the hottest arithmetic.  The moments keep the
// scalar summation order ((f_x- + f_x+) + (f_y- + f_y+)) + W_ref/Q, so they are bit-identical.
__device__ __forceinline__ float2 pk(float a, float b) { return make_float2(a, b); }

template <>
__device__ __forceinline__ void moments<2, float, true>(const float (&fr)[4][4], const float* wq, float (&W)[4]) {
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int k = 2 * h;
    const float2 a = __fadd2_rn(pk(fr[0][k], fr[0][k + 1]), pk(fr[1][k], fr[1][k + 1]));
    const float2 b = __fadd2_rn(pk(fr[2][k], fr[2][k + 1]), pk(fr[3][k], fr[3][k + 1]));
    const float2 w = __fadd2_rn(__fadd2_rn(a, b), pk(wq[k], wq[k + 1]));
    W[k] = w.x;
    W[k + 1] = w.y;
  }
}

template <>
__device__ __forceinline__ void relax_cell<2, float>(float (&f)[4][4], const float (&Qc)[2][4], float beta, float r,
                                                     float inv_c) {
  const float om = 1.0f - 2.0f * beta;
  const float bq = beta * inv_c;
  const float omr = om * r * 0.5f;
  const float omk = om * r * r * 0.25f;
  const float2 cp = pk(0.25f + omk, 0.25f + omk), cm = pk(0.25f - omk, 0.25f - omk);
  const float2 bq2 = pk(bq, bq), omr2 = pk(omr, omr), m1 = pk(-1.0f, -1.0f);
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int k = 2 * h;
    const float2 f0 = pk(f[0][k], f[0][k + 1]), f1 = pk(f[1][k], f[1][k + 1]);
    const float2 f2 = pk(f[2][k], f[2][k + 1]), f3 = pk(f[3][k], f[3][k + 1]);
    const float2 sx = __fadd2_rn(f0, f1), sy = __fadd2_rn(f2, f3);
    const float2 dx = __ffma2_rn(m1, f0, f1), dy = __ffma2_rn(m1, f2, f3);  // f+ - f-
    const float2 gx = __ffma2_rn(bq2, pk(Qc[0][k], Qc[0][k + 1]), __fmul2_rn(omr2, dx));
    const float2 gy = __ffma2_rn(bq2, pk(Qc[1][k], Qc[1][k + 1]), __fmul2_rn(omr2, dy));
    const float2 wx = __ffma2_rn(cp, sx, __fmul2_rn(cm, sy));
    const float2 wy = __ffma2_rn(cm, sx, __fmul2_rn(cp, sy));
    const float2 o0 = __ffma2_rn(m1, gx, wx), o1 = __fadd2_rn(wx, gx);
    const float2 o2 = __ffma2_rn(m1, gy, wy), o3 = __fadd2_rn(wy, gy);
    f[0][k] = o0.x, f[0][k + 1] = o0.y;
    f[1][k] = o1.x, f[1][k + 1] = o1.y;
    f[2][k] = o2.x, f[2][k + 1] = o2.y;
    f[3][k] = o3.x, f[3][k + 1] = o3.y;
  }
}

// Separable (1/4, 1/2, 1/4) box filter (Sec. III D) without its normalisation: a + 2b + c.  Two
// passes give 16 x the filtered value; the powers of two are exact, so scaling at the end
// reproduces the normalised filter bit for bit.
__device__ __forceinline__ double box3(double a, double b, double c) { return fma(2.0, b, a) + c; }
__device__ __forceinline__ float box3(float a, float b, float c) { return fmaf(2.0f, b, a) + c; }

// Sensor A/B map (Eqs. 34-35) from chi before clipping (C s_bar theta_bar).
template <class M>
__device__ __forceinline__ M beta_of(const Coef<M>& co, M chi) {
  chi = chi <= (M)0 ? (M)0 : (chi >= (M)1 ? (M)1 : chi);
  return co.beta_max - co.dbeta * chi;
}

// ------------------------------------------------------------------------------------------
// Maxima: per-cell values reduced within a CTA and stored as the CTA's partial (no atomics).
// FP64: non-negative doubles compared as their 64-bit patterns (same order, integer pipe);
// FP32: float max.  The one-CTA link-speed kernel folds the partials.
// ------------------------------------------------------------------------------------------
template <class M>
struct Red;
template <>
struct Red<double> {
  using T = unsigned long long;
  static __device__ __forceinline__ T make(double x) {  // |x| as an ordered bit pattern
    return (T)__double_as_longlong(x) & 0x7fffffffffffffffull;
  }
  static __device__ __forceinline__ T mx(T a, T b) { return a > b ? a : b; }
  static __device__ __forceinline__ double value(T v) { return __longlong_as_double((long long)v); }
};
template <>
struct Red<float> {
  using T = float;
  static __device__ __forceinline__ T make(float x) { return fabsf(x); }
  static __device__ __forceinline__ T mx(T a, T b) { return fmaxf(a, b); }
  static __device__ __forceinline__ double value(T v) { return (double)v; }
};

// Per-cell contributions to (s_max, M_0..M_{NC-1}) (Eqs. 30, 36).
template <int D, class M>
__device__ __forceinline__ void cell_maxima(const M (&u)[D], M cs, const M (&Qf)[D][D + 2], typename Red<M>::T (&v)[kNV]) {
  using R = Red<M>;
#pragma unroll
  for (int a = 0; a < D; ++a) {
    v[0] = R::mx(v[0], R::make(fabs(u[a]) + cs));
#pragma unroll
    for (int k = 0; k < D + 2; ++k) v[1 + k] = R::mx(v[1 + k], R::make(Qf[a][k]));
  }
}

template <class M, int NT>
__device__ __forceinline__ void block_max_store(typename Red<M>::T (&v)[kNV], double* __restrict__ part_slot, int cta,
                                                int ncta, int* nparts_slot) {
  using R = Red<M>;
  using T = typename R::T;
  __shared__ T red_s[NT / 32][kNV];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int j = 0; j < kNV; ++j) {
    T x = v[j];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) x = R::mx(x, __shfl_xor_sync(0xffffffffu, x, off));
    if (lane == 0) red_s[warp][j] = x;
  }
  __syncthreads();
  if (threadIdx.x < kNV) {
    T x = red_s[0][threadIdx.x];
#pragma unroll 4
    for (int w = 1; w < NT / 32; ++w) x = R::mx(x, red_s[w][threadIdx.x]);
    part_slot[(long long)cta * kNV + threadIdx.x] = R::value(x);
  }
  if (cta == 0 && threadIdx.x == 0) *nparts_slot = ncta;
}

// Fold the partials of one slot with one CTA of NT threads into out[j] (valid in thread 0).  The
// partials are non-negative doubles and are compared as 64-bit patterns on the integer pipe (a
// single SM's FP64 pipe would make this fold cost tens of microseconds).
template <int NT>
__device__ __forceinline__ void fold_partials(const double* __restrict__ part_slot, int nparts, double (&out)[kNV]) {
  using T = unsigned long long;
  __shared__ T red_s[NT / 32][kNV];
  const T* bits = reinterpret_cast<const T*>(part_slot);
  T v[kNV];
#pragma unroll
  for (int j = 0; j < kNV; ++j) v[j] = 0ull;
  for (int c = threadIdx.x; c < nparts; c += NT)
#pragma unroll
    for (int j = 0; j < kNV; ++j) {
      const T x = __ldg(bits + (long long)c * kNV + j);
      v[j] = x > v[j] ? x : v[j];
    }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int j = 0; j < kNV; ++j) {
    T x = v[j];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      const T y = __shfl_xor_sync(0xffffffffu, x, off);
      x = y > x ? y : x;
    }
    if (lane == 0) red_s[warp][j] = x;
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int j = 0; j < kNV; ++j) {
      T x = lane < NT / 32 ? red_s[lane][j] : 0ull;
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        const T y = __shfl_xor_sync(0xffffffffu, x, off);
        x = y > x ? y : x;
      }
      out[j] = __longlong_as_double((long long)x);
    }
  }
}


}  // namespace vlbm
