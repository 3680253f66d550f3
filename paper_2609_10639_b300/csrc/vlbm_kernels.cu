// CUDA kernels of the VLBM step (sm_103a).
//
// Populations live in HBM as one plane per lattice direction i in {x-, x+, y-, y+}, each cell
// holding its (D+2) conserved components contiguously in a 4-wide vector: [i][y][x][4] (one 128-bit
// access per direction and cell in FP32 storage, two in FP64), double-buffered.  A buffer holds post-collision
// populations; a step pulls them across the lattice links on read (exact transport, Eq. 21), so
// each population is read once and written once per step.  The first step after vlbm_init reads
// the equilibrium populations in place ("unpulled").
//
// Step kernels: the 2D default is the column-strip kernel k_roll (vlbm_roll.cu).  This file holds
// the tile kernel k_tile (1D, beta readback, and 2D on request): one CTA owns a TX x TY tile and
// stages, in shared memory, the primitive velocity and the flux Q_alpha(W) of a halo region
// around it (radius 2, or 3 for the look-ahead form); the shock sensor (Eqs. 28-35) and its
// separable box filter read that region; the reprojection (Eqs. 38-40) and relaxation (Eqs. 20,
// 22) are fused into one register update.
// Boundary rules are applied to every stencil access: a region position outside a zero-gradient
// side takes the values of the edge cell (edge-replicated ghost) and every derived stencil
// quantity there is evaluated at the edge cell; periodic sides are simply unwrapped.
//
// The two domain-wide maxima a step needs (s_max, Eq. 36; M_k, Eq. 30) are reduced with warp
// shuffles and a per-CTA combine into per-CTA partials, folded by the one-CTA link-speed kernel
// (no atomics, deterministic).  Two forms:
//   two-pass:   k_reduce (reads the state once more; in FP64 with strips it also keeps W, u, Q
//               for the step kernel) -> k_dt -> step kernel;
//   look-ahead: k_dt -> step kernel, which also forms W^{n+1} of its cells from the relaxed
//               populations (k_tile: a one-cell ring around its tile) and reduces them for the
//               next step, so a step moves each population through HBM exactly twice.
// k_dt is a one-CTA kernel that folds the partial maxima and turns them into c, dt, r and 1/M_k
// on the device.
#include "vlbm.h"
#include "vlbm_device.cuh"
#include "vlbm_internal.cuh"

#include <atomic>
#include <cfloat>
#include <cstddef>
#include <cmath>
#include <mutex>
#include <type_traits>

namespace vlbm {

// ------------------------------------------------------------------------------------------
// k_reduce: s_max and M_k of the current state (two-pass form; also feeds vlbm_get_beta)
// ------------------------------------------------------------------------------------------
// With `fields` (FP64, 2D) the pass also stores W, u and Q of every cell, so that the step
// kernel reads them instead of recomputing moments, primitives and flux.  With `pk` it stores the
// pressure of every cell into pk[n & 1] (the kept pressure the next FP32 look-ahead step reads;
// used after a state restore).
template <int D, class S, int NT>
__global__ void __launch_bounds__(NT) k_reduce(const S* __restrict__ fin, Scalars* __restrict__ sc, const KParams p,
                                                const int pulled, double* __restrict__ part, const int in_run,
                                                double* __restrict__ fields, float* __restrict__ pk) {
  using M = typename Store<S>::M;
  using R = Red<M>;
  constexpr int NC = D + 2;
  if (in_run && (sc->done || sc->err)) return;  // a finished or failed run skips its remaining steps
  const int slot = (int)(sc->n & 1);
  M wq[NC];
#pragma unroll
  for (int k = 0; k < NC; ++k) wq[k] = StepScalars<M>::wq(sc, k);
  // pinned inflow: the ghost values, with the stored populations' link speed c_prev
  __shared__ GhostTab<D, M> gtab;
  const bool inflow = p.bc[0] == 2;
  if (inflow) {
    if (threadIdx.x == 0) fill_ghost_tab<D, M, Store<S>::kOffset>(p, wq, (M)(1.0 / sc->c_prev), gtab);
    __syncthreads();
  }
  typename R::T v[kNV];
#pragma unroll
  for (int j = 0; j < kNV; ++j) v[j] = typename R::T(0);
  bool bad = false;
  for (long long cell = (long long)blockIdx.x * NT + threadIdx.x; cell < p.plane; cell += (long long)gridDim.x * NT) {
    const int cx = (int)(cell % p.nx), cy = (int)(cell / p.nx);
    M fr[2 * D][NC], W[NC], u[D], Qf[D][NC], cs;
    load_cell<D, S>(fin, p, cx, cy, pulled, false, fr, inflow ? &gtab.f[0][0] : nullptr);
    moments<D, M, Store<S>::kOffset>(fr, wq, W);
    M Pc;
    bad |= !prim_flux<D, M, true>(p, W, u, Qf, cs, &Pc);
    if (pk) pk[(long long)slot * p.plane + cell] = (float)Pc;
    cell_maxima<D, M>(u, cs, Qf, v);
    if constexpr (D == 2 && std::is_same<M, double>::value) {
      if (fields) {
#pragma unroll
        for (int k = 0; k < 4; ++k) fields[k * p.plane + cell] = W[k];
        fields[4 * p.plane + cell] = u[0];
        fields[5 * p.plane + cell] = u[1];
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
          for (int k = 0; k < 4; ++k) fields[(6 + 4 * a + k) * p.plane + cell] = Qf[a][k];
      }
    }
  }
  if (bad) atomicOr(&sc->err, ERR_NONPHYSICAL);
  block_max_store<M, NT>(v, part + (long long)slot * p.max_parts * kNV, blockIdx.x, gridDim.x, &sc->nparts[slot]);
}

// ------------------------------------------------------------------------------------------
// k_dt: link speed and time step of the next step (Eqs. 36-37), final-step shortening, and the
// reciprocals the step kernels use.  One CTA folds the partial maxima; thread 0 decides.
// ------------------------------------------------------------------------------------------
constexpr int kNTD = 1024;  // threads of the one-CTA scalar kernels

__global__ void __launch_bounds__(kNTD) k_dt(Scalars* sc, const KParams p, const double* __restrict__ part,
                                              double* hist_dt, double* hist_c, const double* sched) {
  // Every scalar the decision reads is loaded before the fold, as independent loads, so that
  // their latencies overlap instead of forming a chain behind the fold (the kernel is
  // latency-bound; nothing else writes these fields while it runs).
  const long long n = sc->n;
  const int slot = (int)(n & 1);
  const int nparts = sc->nparts[slot];
  const double t = sc->t, t_end = sc->t_end, c_prev = sc->c_prev;
  const int done0 = sc->done, err0 = sc->err;
  const long long sched_len = sc->sched_len, hist_cap = sc->hist_cap;
  const double c_sched = (sched_len > 0 && n + 1 < sched_len) ? sched[n + 1] : 0.0;
  double mx[kNV];
  fold_partials<kNTD>(part + (long long)slot * p.max_parts * kNV, nparts, mx);
  if (threadIdx.x != 0) return;
  const bool done = done0 || (t_end > 0.0 && t >= t_end);
  if (done && !done0) sc->done = 1;
  if (done || err0) {
    sc->active = 0;
    return;
  }
  const double smax = mx[0];
  double c;
  if (sched_len > 0) {
    if (n + 1 >= sched_len) {
      sc->err = err0 | ERR_SCHEDULE;
      sc->active = 0;
      return;
    }
    c = c_sched;
  } else {
    const bool retarget = p.retarget_every <= 1 || (n % p.retarget_every) == 0;
    c = retarget ? smax / p.cfl : c_prev;
  }
  double dt = p.dx / c;
  bool last = false;
  if (sched_len == 0 && t_end > 0.0 && t + dt >= t_end) {  // land on t_end
    dt = t_end - t;
    c = p.dx / dt;
    last = true;
  }
  if (!(c > 0.0) || !isfinite(c) || !(dt > 0.0)) {
    sc->err = err0 | ERR_NONPHYSICAL;
    sc->active = 0;
    return;
  }
  const double r = c_prev / c, inv_c = 1.0 / c;
  sc->smax = smax;
  sc->r = r;
  sc->c_new = c;
  sc->inv_c = inv_c;
  sc->dt = dt;
  sc->r_f = (float)r;
  sc->inv_c_f = (float)inv_c;
  for (int k = 0; k < p.nc; ++k) {
    const double im = mx[1 + k] > 0.0 ? 1.0 / mx[1 + k] : 0.0;
    sc->inv_M[k] = im;
    sc->inv_M_f[k] = (float)im;
  }
  if (n < hist_cap) {
    hist_dt[n] = dt;
    hist_c[n] = c;
  }
  sc->t = last ? t_end : t + dt;
  sc->c_prev = c;
  sc->n = n + 1;
  sc->active = 1;
  if (last) sc->done = 1;
}

// ------------------------------------------------------------------------------------------
// k_tile: the step (or, with BETA_OUT, only beta(x) of the current state)
// ------------------------------------------------------------------------------------------
template <int D, class S, bool LOOK, int TX, int TY>
struct TileGeom {
  static constexpr int NC = D + 2, Q = 2 * D;
  static constexpr int H = LOOK ? 3 : 2;                          // u/Q region radius
  static constexpr int HY = D == 2 ? H : 0;
  static constexpr int RX = TX + 2 * H, RY = TY + 2 * HY;         // u/Q region
  static constexpr int SX = TX + 2 * (H - 1), SY = TY + 2 * (D == 2 ? H - 1 : 0);  // s, theta region
  static constexpr int RB = LOOK ? 1 : 0, RBY = D == 2 ? RB : 0;  // relaxed ring
  static constexpr int BX = TX + 2 * RB, BY = TY + 2 * RBY;       // relaxed region
  static constexpr int NT = TX * TY;
  using M = typename Store<S>::M;
  static constexpr size_t smem_elems = (size_t)D * 4 * RY * RX + (size_t)Q * 4 * BY * BX + (size_t)D * RY * RX +
                                       (size_t)SY * SX * (D == 2 ? 2 : 1);
  static constexpr size_t smem_bytes = smem_elems * sizeof(M);
};

// beta at region-local centre (sx, sy) of the s/theta arrays: box filter x then y (Sec. III D),
// Sensor A (1D, Eq. 34) or Sensor B (2D, Eq. 35).
template <int D, class M, int SX>
__device__ __forceinline__ M sensor_beta(const KParams& p, const Coef<M>& c, const M* s_s, const M* s_t, int sx, int sy) {
  if (p.beta_mode == 1) return c.beta_const;
  if constexpr (D == 1) {
    // 1D: theta = 1, one filter pass
    return beta_of<M>(c, c.c_chi1 * box3(s_s[sx - 1], s_s[sx], s_s[sx + 1]));
  } else {
    M rs[3], rt[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const M* rows = s_s + (sy - 1 + j) * SX;
      const M* rowt = s_t + (sy - 1 + j) * SX;
      rs[j] = box3(rows[sx - 1], rows[sx], rows[sx + 1]);
      rt[j] = box3(rowt[sx - 1], rowt[sx], rowt[sx + 1]);
    }
    return beta_of<M>(c, c.c_chi2 * box3(rs[0], rs[1], rs[2]) * box3(rt[0], rt[1], rt[2]));
  }
}

// Two resident CTAs per SM requested: without it the compiler caps the FP32 form at 40 registers
// with spills and the kernel runs 12% slower at 4096^2 (0.62 vs 0.55 ms on a B300).
template <int D, class S, bool LOOK, bool BETA_OUT, int TX, int TY>
__global__ void __launch_bounds__(TX * TY, 2) k_tile(const S* __restrict__ fin, S* __restrict__ fout, Scalars* __restrict__ sc,
                                                    const KParams p, const int pulled,
                                                    const typename Store<S>::M* __restrict__ invM_src,
                                                    double* __restrict__ beta_out, double* __restrict__ part) {
  using G = TileGeom<D, S, LOOK, TX, TY>;
  using M = typename G::M;
  constexpr int NC = G::NC, Q = G::Q, H = G::H, HY = G::HY, RX = G::RX, RY = G::RY, SX = G::SX, SY = G::SY;
  constexpr int RB = G::RB, RBY = G::RBY, BX = G::BX, BY = G::BY, NT = G::NT;
  constexpr bool OFF = Store<S>::kOffset;
  if (!BETA_OUT && !sc->active) return;

  extern __shared__ __align__(16) unsigned char smem_raw[];
  M* s_Q = reinterpret_cast<M*>(smem_raw);  // [D][RY][RX][4]  flux Q_alpha of the region
  M* s_f = s_Q + D * RY * RX * 4;           // [Q][BY][BX][4]  populations of the relaxed region
  M* s_u = s_f + Q * BY * BX * 4;           // [D][RY][RX]     velocity of the region
  M* s_s = s_u + D * RY * RX;               // [SY][SX]        activity s
  M* s_t = s_s + SY * SX;                   // [SY][SX]        Ducros ratio (2D)

  const Coef<M>& co = coef<M>(p);
  const int x0 = blockIdx.x * TX, y0 = (D == 2) ? blockIdx.y * TY : 0;
  M wq[NC];
#pragma unroll
  for (int k = 0; k < NC; ++k) wq[k] = StepScalars<M>::wq(sc, k);
  // Interior tile: every region position and its pull sources lie inside the domain, so no
  // boundary rule is evaluated (uniform per CTA).
  const bool interior = x0 - H - 1 >= 0 && x0 + TX + H + 1 <= p.nx &&
                        (D == 1 || (y0 - HY - 1 >= 0 && y0 + TY + HY + 1 <= p.ny));
  // pinned inflow: the ghost values, at the link speed of the stored populations (readback:
  // c_prev; in a step, after the link-speed kernel: c_new r)
  __shared__ GhostTab<D, M> gtab;
  const bool inflow = p.bc[0] == 2;
  if (inflow) {
    if (threadIdx.x == 0)
      fill_ghost_tab<D, M, OFF>(p, wq, BETA_OUT ? (M)(1.0 / sc->c_prev) : StepScalars<M>::inv_c(sc) / StepScalars<M>::r(sc),
                                gtab);
    __syncthreads();
  }

  // ---- phase A: populations, primitives and flux over the region (row-major, coalesced) ----
  for (int idx = threadIdx.x; idx < RX * RY; idx += NT) {
    const int rx = idx % RX, ry = idx / RX;
    const int px = x0 - H + rx, py = y0 - HY + ry;
    const int cx = interior ? px : nb_index(px, p.nx, p.bc[0], p.bc[1]);
    const int cy = (D == 2) ? (interior ? py : nb_index(py, p.ny, p.bc[2], p.bc[3])) : 0;
    M fr[Q][NC], W[NC], u[D], Qf[D][NC], cs;
    if (!interior && inflow && px < 0) {  // ghost cell of the pinned-inflow side
#pragma unroll
      for (int k = 0; k < NC; ++k) {
#pragma unroll
        for (int i = 0; i < Q; ++i) fr[i][k] = gtab.f[i][k];
        W[k] = gtab.W[k];
#pragma unroll
        for (int a = 0; a < D; ++a) Qf[a][k] = gtab.Q[a][k];
      }
#pragma unroll
      for (int a = 0; a < D; ++a) u[a] = gtab.u[a];
    } else {
      load_cell<D, S>(fin, p, cx, cy, pulled, interior, fr, inflow ? &gtab.f[0][0] : nullptr);
      moments<D, M, OFF>(fr, wq, W);
      prim_flux<D, M, false>(p, W, u, Qf, cs);
    }
#pragma unroll
    for (int a = 0; a < D; ++a) {
      s_u[a * RY * RX + idx] = u[a];
      M v[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) v[k] = k < NC ? Qf[a][k] : (M)0;
      st4s(s_Q + (a * RY * RX + idx) * 4, v);
    }
    const int bx = rx - (H - RB), by = ry - (HY - RBY);
    if (!BETA_OUT && bx >= 0 && bx < BX && by >= 0 && by < BY) {
#pragma unroll
      for (int i = 0; i < Q; ++i) {
        M v[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) v[k] = k < NC ? fr[i][k] : (M)0;
        st4s(s_f + (i * BY * BX + by * BX + bx) * 4, v);
      }
    }
  }
  __syncthreads();

  // ---- phase B: activity s (Eqs. 28-31) and Ducros ratio theta (Eqs. 32-33) ----
  if (p.beta_mode == 0) {
    M invMh[NC];  // M_k^-1 / 2: s_hat_k = (jump over two cells) / 2 / M_k (Eqs. 29-30)
#pragma unroll
    for (int k = 0; k < NC; ++k) invMh[k] = (M)0.5 * invM_src[k];
    for (int j = threadIdx.x; j < SX * SY; j += NT) {
      const int sx = j % SX, sy = j / SX;
      const int px = x0 - (H - 1) + sx;
      const int py = y0 - (D == 2 ? H - 1 : 0) + sy;
      const int rx = (interior ? px : centre_pos(px, p.nx, p.bc[0], p.bc[1])) - (x0 - H);
      const int ry = (D == 2) ? (interior ? py : centre_pos(py, p.ny, p.bc[2], p.bc[3])) - (y0 - HY) : 0;
      const int c = ry * RX + rx;
      M qxp[4], qxm[4], qyp[4], qym[4];
      ld4s(s_Q + (c + 1) * 4, qxp);
      ld4s(s_Q + (c - 1) * 4, qxm);
      if constexpr (D == 2) {
        ld4s(s_Q + (RY * RX + c + RX) * 4, qyp);
        ld4s(s_Q + (RY * RX + c - RX) * 4, qym);
      }
      M acc = 0;
#pragma unroll
      for (int k = 0; k < NC; ++k) {
        M jk = qxp[k] - qxm[k];
        if constexpr (D == 2) jk += qyp[k] - qym[k];
        const M sh = jk * invMh[k];
        acc += sh * sh;
      }
      // sqrt(acc) = sqrt(NC) s (Eq. 31): 2 s in 2D, sqrt(3) s in 1D; the constant is folded into
      // the sensor map
      s_s[j] = sqrt_(acc);
      if constexpr (D == 2) {
        const M* ux = s_u;
        const M* uy = s_u + RY * RX;
        const M dl = (ux[c + 1] - ux[c - 1]) + (uy[c + RX] - uy[c - RX]);
        const M vt = (uy[c + 1] - uy[c - 1]) - (ux[c + RX] - ux[c - RX]);
        s_t[j] = div_(dl * dl, dl * dl + vt * vt + co.eps_lat);
      }
    }
    __syncthreads();
  }

  // ---- phase C/D: beta, fused reprojection + relaxation, single write ----
  const M r = StepScalars<M>::r(sc), inv_c = StepScalars<M>::inv_c(sc);
  for (int idx = threadIdx.x; idx < BX * BY; idx += NT) {
    const int bx = idx % BX, by = idx / BX;
    const int px = x0 - RB + bx, py = y0 - RBY + by;
    const bool in_tile = bx >= RB && bx < RB + TX && by >= RBY && by < RBY + TY;
    const bool in_dom = px >= 0 && px < p.nx && py >= 0 && py < p.ny;
    // ring positions beyond a zero-gradient side are never read (their pulls land on the edge)
    if (!in_tile && (centre_pos(px, p.nx, p.bc[0], p.bc[1]) != px ||
                     (D == 2 && centre_pos(py, p.ny, p.bc[2], p.bc[3]) != py)))
      continue;
    const int ccx = centre_pos(px, p.nx, p.bc[0], p.bc[1]) - (x0 - (H - 1));
    const int ccy = (D == 2) ? centre_pos(py, p.ny, p.bc[2], p.bc[3]) - (y0 - (H - 1)) : 0;
    const M beta = sensor_beta<D, M, SX>(p, co, s_s, s_t, ccx, ccy);
    if constexpr (BETA_OUT) {
      if (in_dom) beta_out[(long long)py * p.nx + px] = (double)beta;
      continue;
    } else {
      M f[Q][NC], Qc[D][NC];
      const int ri = (by + (HY - RBY)) * RX + (bx + (H - RB));
#pragma unroll
      for (int i = 0; i < Q; ++i) {
        M v[4];
        ld4s(s_f + (i * BY * BX + idx) * 4, v);
#pragma unroll
        for (int k = 0; k < NC; ++k) f[i][k] = v[k];
      }
#pragma unroll
      for (int a = 0; a < D; ++a) {
        M v[4];
        ld4s(s_Q + (a * RY * RX + ri) * 4, v);
#pragma unroll
        for (int k = 0; k < NC; ++k) Qc[a][k] = v[k];
      }
      relax_cell<D, M>(f, Qc, beta, r, inv_c);
      if (in_tile && in_dom) store_cell<D, S, M>(fout, p, py * p.nx + px, f);
      if constexpr (LOOK) {
#pragma unroll
        for (int i = 0; i < Q; ++i) {
          M v[4];
#pragma unroll
          for (int k = 0; k < 4; ++k) v[k] = k < NC ? f[i][k] : (M)0;
          st4s(s_f + (i * BY * BX + idx) * 4, v);
        }
      }
    }
  }

  // ---- look-ahead: W^{n+1}(x) = sum_i f*_i(x - sigma_i) of the tile, reduced for the next step ----
  if constexpr (LOOK && !BETA_OUT) {
    __syncthreads();
    using R = Red<M>;
    typename R::T v[kNV];
#pragma unroll
    for (int j = 0; j < kNV; ++j) v[j] = typename R::T(0);
    bool bad = false;
    const int tx = threadIdx.x % TX, ty = threadIdx.x / TX;
    const int gx = x0 + tx, gy = y0 + ty;
    if (gx < p.nx && gy < p.ny) {
      M fr[Q][NC], W[NC];
#pragma unroll
      for (int i = 0; i < Q; ++i) {
        const int qx = centre_pos(gx - sig_x(i), p.nx, p.bc[0], p.bc[1]) - (x0 - RB);
        const int qy = (D == 2) ? centre_pos(gy - sig_y(i), p.ny, p.bc[2], p.bc[3]) - (y0 - RBY) : 0;
        M v[4];
        ld4s(s_f + (i * BY * BX + qy * BX + qx) * 4, v);
#pragma unroll
        for (int k = 0; k < NC; ++k) fr[i][k] = v[k];
      }
      // same summation order as every other moment evaluation (the maxima are those k_reduce
      // would compute from the stored state)
      moments<D, M, OFF>(fr, wq, W);
      M u[D], Qf[D][NC], cs;
      bad = !prim_flux<D, M, true>(p, W, u, Qf, cs);
      cell_maxima<D, M>(u, cs, Qf, v);
    }
    if (bad) atomicOr(&sc->err, ERR_NONPHYSICAL);
    const int slot = (int)(sc->n & 1);
    block_max_store<M, NT>(v, part + (long long)slot * p.max_parts * kNV, blockIdx.y * gridDim.x + blockIdx.x,
                           gridDim.x * gridDim.y, &sc->nparts[slot]);
  }
}

// ------------------------------------------------------------------------------------------
// initialisation, readback
// ------------------------------------------------------------------------------------------
__global__ void k_init_begin(Scalars* sc) {
  for (int k = 0; k < 4; ++k) sc->wq_f[k] = 0.0f;
  sc->n = 0;
  sc->t = 0.0;
  sc->active = 0;
  sc->done = 0;
  sc->err = 0;
  sc->nparts[0] = sc->nparts[1] = 0;
  for (int k = 0; k < 4; ++k) sc->wref[k] = 0.0;
}

// s_max of W0 into partial slot 1 (Eq. 36), with the physical-state check.
template <int D, int NT>
__global__ void __launch_bounds__(NT) k_reduce_W0(const double* __restrict__ W0, Scalars* __restrict__ sc, const KParams p,
                                                   double* __restrict__ part) {
  constexpr int NC = D + 2;
  using R = Red<double>;
  R::T v[kNV];
#pragma unroll
  for (int j = 0; j < kNV; ++j) v[j] = 0ull;
  bool bad = false;
  for (long long cell = (long long)blockIdx.x * NT + threadIdx.x; cell < p.plane; cell += (long long)gridDim.x * NT) {
    double W[NC], u[D], Qf[D][NC], cs;
#pragma unroll
    for (int k = 0; k < NC; ++k) W[k] = W0[k * p.plane + cell];
    bad |= !prim_flux<D, double, true>(p, W, u, Qf, cs);
    cell_maxima<D, double>(u, cs, Qf, v);
  }
  if (bad) atomicOr(&sc->err, ERR_NONPHYSICAL);
  block_max_store<double, NT>(v, part + (long long)1 * p.max_parts * kNV, blockIdx.x, gridDim.x, &sc->nparts[1]);
}

// Per-block compensated (Neumaier) sums of W0_k (FP32-storage reference), fixed order.
template <int NT>
__global__ void __launch_bounds__(NT) k_sum_partial(const double* __restrict__ W0, const KParams p, double* __restrict__ partial) {
  __shared__ double ss[NT], sc_[NT];
  for (int k = 0; k < p.nc; ++k) {
    double s = 0.0, c = 0.0;
    for (long long cell = (long long)blockIdx.x * NT + threadIdx.x; cell < p.plane; cell += (long long)gridDim.x * NT) {
      const double x = W0[k * p.plane + cell];
      const double t = s + x;
      c += fabs(s) >= fabs(x) ? (s - t) + x : (x - t) + s;
      s = t;
    }
    ss[threadIdx.x] = s;
    sc_[threadIdx.x] = c;
    __syncthreads();
    if (threadIdx.x < 32) {
      // fixed order: lane l folds the threads [l NT/32, (l+1) NT/32), then the lanes in order
      constexpr int PER = NT / 32;
      double S = 0.0, Cc = 0.0;
      for (int j = threadIdx.x * PER; j < (threadIdx.x + 1) * PER; ++j) {
        const double x = ss[j];
        const double t = S + x;
        Cc += fabs(S) >= fabs(x) ? (S - t) + x : (x - t) + S;
        S = t;
        Cc += sc_[j];
      }
      double T = 0.0, Ct = 0.0;
      for (int l = 0; l < 32; ++l) {
        const double x = __shfl_sync(0xffffffffu, S, l), cx = __shfl_sync(0xffffffffu, Cc, l);
        const double t = T + x;
        Ct += fabs(T) >= fabs(x) ? (T - t) + x : (x - t) + T;
        T = t;
        Ct += cx;
      }
      if (threadIdx.x == 0) partial[blockIdx.x * 4 + k] = T + Ct;
    }
    __syncthreads();
  }
}

// Compensated (Neumaier) sum of the per-block partials of component k by one warp, in a fixed
// order: lane l folds the contiguous blocks [l n/32, (l+1) n/32), then lane 0 folds the 32 lane
// sums in lane order and adds their compensations.  Returns the total in lane 0.
__device__ double warp_sum_partials(const double* __restrict__ partial, int nblk, int k) {
  const int lane = threadIdx.x & 31;
  const int b0 = (int)((long long)nblk * lane / 32), b1 = (int)((long long)nblk * (lane + 1) / 32);
  double S = 0.0, Cc = 0.0;
  for (int b = b0; b < b1; ++b) {
    const double x = partial[b * 4 + k];
    const double t = S + x;
    Cc += fabs(S) >= fabs(x) ? (S - t) + x : (x - t) + S;
    S = t;
  }
  double T = 0.0, Ct = 0.0;
  for (int l = 0; l < 32; ++l) {
    const double x = __shfl_sync(0xffffffffu, S, l), cx = __shfl_sync(0xffffffffu, Cc, l);
    const double t = T + x;
    Ct += fabs(T) >= fabs(x) ? (T - t) + x : (x - t) + T;
    T = t;
    Ct += cx;
  }
  return T + Ct;
}

// One warp.
__global__ void k_sum_final(const double* __restrict__ partial, int nblk, const KParams p, Scalars* sc) {
  for (int k = 0; k < p.nc; ++k) {
    const double total = warp_sum_partials(partial, nblk, k);
    if (threadIdx.x == 0) {
      sc->wref[k] = total / (double)p.plane / (double)p.q;
      sc->wq_f[k] = (float)(p.q * sc->wref[k]);
    }
  }
}

// Domain totals sum_x W_k of the current state: the per-block partials of k_sum_partial folded
// with the same compensation (the discrete conservation law of the step, Sec. III A).  One warp.
__global__ void k_sum_out(const double* __restrict__ partial, int nblk, const KParams p, double* __restrict__ out) {
  for (int k = 0; k < p.nc; ++k) {
    const double total = warp_sum_partials(partial, nblk, k);
    if (threadIdx.x == 0) out[k] = total;
  }
}

// Initial link speed c0 = s_max(W0)/CFL (or the replayed c0).  One CTA.
__global__ void __launch_bounds__(kNTD) k_init_c0(Scalars* sc, const KParams p, const double* __restrict__ part,
                                                   const double* sched) {
  double mx[kNV];
  fold_partials<kNTD>(part + (long long)1 * p.max_parts * kNV, sc->nparts[1], mx);
  if (threadIdx.x != 0) return;
  const double c0 = sc->sched_len > 0 ? sched[0] : mx[0] / p.cfl;
  if (!(c0 > 0.0) || !isfinite(c0)) sc->err |= ERR_NONPHYSICAL;
  sc->c_prev = c0;
  sc->c_new = c0;
  sc->r = 1.0;
}

// f_i = f_i^eq(W0; c0) (Eq. 20), stored in place (unpulled); maxima of W^0 = sum_i f_i into
// partial slot 0.
// MAXIMA: also the maxima of the stored populations into partial slot 0, which the first step of
// the look-ahead form reads (the two-pass form's first step takes them itself).
template <int D, class S, int NT, bool MAXIMA>
__global__ void __launch_bounds__(NT) k_init_eq(const double* __restrict__ W0, S* __restrict__ fout, Scalars* __restrict__ sc,
                                                 const KParams p, double* __restrict__ part, float* __restrict__ pk) {
  using M = typename Store<S>::M;
  using R = Red<M>;
  constexpr int NC = D + 2, Q = 2 * D;
  typename R::T v[kNV];
#pragma unroll
  for (int j = 0; j < kNV; ++j) v[j] = typename R::T(0);
  M wq[NC];
#pragma unroll
  for (int k = 0; k < NC; ++k) wq[k] = Store<S>::kOffset ? (M)(Q * sc->wref[k]) : (M)0;
  bool bad = false;
  const double h2c = 0.5 / sc->c_prev;  // 1 / (2 c0): c_i.Q / (2 c^2) with |c_i| = c
  static_assert(sizeof(S) == 4 || sizeof(S) == 8, "storage type");
  for (long long cell = (long long)blockIdx.x * NT + threadIdx.x; cell < p.plane; cell += (long long)gridDim.x * NT) {
    double W[NC], u[D], Qf[D][NC], cs;
#pragma unroll
    for (int k = 0; k < NC; ++k) W[k] = W0[k * p.plane + cell];
    prim_flux<D, double, false>(p, W, u, Qf, cs);
    M fr[Q][NC];
#pragma unroll
    for (int k = 0; k < NC; ++k)
#pragma unroll
      for (int i = 0; i < Q; ++i) {
        const int a = i >> 1;
        const double sgn = (i & 1) ? 1.0 : -1.0;
        const double fe = W[k] * (1.0 / (2.0 * D)) + sgn * (Qf[a][k] * h2c);
        const S st = Store<S>::kOffset ? (S)(fe - sc->wref[k]) : (S)fe;
        fr[i][k] = (M)st;
      }
    store_cell<D, S, M>(fout, p, (int)cell, fr);
    if constexpr (MAXIMA) {
      M Ws[NC], us[D], Qs[D][NC], css;
      moments<D, M, Store<S>::kOffset>(fr, wq, Ws);
      M Pc;
      bad |= !prim_flux<D, M, true>(p, Ws, us, Qs, css, &Pc);
      if (pk) pk[cell] = (float)Pc;  // kept pressure of the state n = 0 (slot 0)
      cell_maxima<D, M>(us, css, Qs, v);
    }
  }
  if constexpr (MAXIMA) {
    if (bad) atomicOr(&sc->err, ERR_NONPHYSICAL);
    block_max_store<M, NT>(v, part, blockIdx.x, gridDim.x, &sc->nparts[0]);
  }
}

// W = sum_i f_i (FP32 storage: FP64 sum of the reference share and the deviations).
template <int D, class S, int NT>
__global__ void __launch_bounds__(NT) k_get_W(const S* __restrict__ fin, const Scalars* __restrict__ sc, const KParams p,
                                               const int pulled, double* __restrict__ W) {
  constexpr int NC = D + 2, Q = 2 * D;
  const long long cell = (long long)blockIdx.x * NT + threadIdx.x;
  if (cell >= p.plane) return;
  const int cx = (int)(cell % p.nx), cy = (int)(cell / p.nx);
  double acc[NC];
#pragma unroll
  for (int k = 0; k < NC; ++k) acc[k] = 0.0;
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    int sx = cx, sy = cy;
    if (pulled) {
      if (p.bc[0] == 2 && cx - sig_x(i) < 0) {  // from a pinned-inflow ghost cell, at c_prev
        double g[NC];
        ghost_population<D, double, false>(p, nullptr, 1.0 / sc->c_prev, i, g);
#pragma unroll
        for (int k = 0; k < NC; ++k) acc[k] += g[k];
        continue;
      }
      sx = nb_index(cx - sig_x(i), p.nx, p.bc[0], p.bc[1]);
      if (D == 2) sy = nb_index(cy - sig_y(i), p.ny, p.bc[2], p.bc[3]);
    }
    S v[4];
    ld4g(fin + (i * (int)p.plane + sy * p.nx + sx) * 4, v);
#pragma unroll
    for (int k = 0; k < NC; ++k) acc[k] += Store<S>::kOffset ? ((double)v[k] + sc->wref[k]) : (double)v[k];
  }
#pragma unroll
  for (int k = 0; k < NC; ++k) W[k * p.plane + cell] = acc[k];
}

// Populations in the interface layout [i][k][y][x] (FP32 storage: reference share added in FP64).
template <int D, class S, int NT>
__global__ void __launch_bounds__(NT) k_get_f(const S* __restrict__ fin, const Scalars* __restrict__ sc, const KParams p,
                                               const int pulled, double* __restrict__ f) {
  constexpr int NC = D + 2, Q = 2 * D;
  const long long cell = (long long)blockIdx.x * NT + threadIdx.x;
  if (cell >= p.plane) return;
  const int cx = (int)(cell % p.nx), cy = (int)(cell / p.nx);
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    int sx = cx, sy = cy;
    if (pulled) {
      if (p.bc[0] == 2 && cx - sig_x(i) < 0) {  // from a pinned-inflow ghost cell, at c_prev
        double g[NC];
        ghost_population<D, double, false>(p, nullptr, 1.0 / sc->c_prev, i, g);
#pragma unroll
        for (int k = 0; k < NC; ++k) f[(long long)(i * NC + k) * p.plane + cell] = g[k];
        continue;
      }
      sx = nb_index(cx - sig_x(i), p.nx, p.bc[0], p.bc[1]);
      if (D == 2) sy = nb_index(cy - sig_y(i), p.ny, p.bc[2], p.bc[3]);
    }
    S v[4];
    ld4g(fin + (i * (int)p.plane + sy * p.nx + sx) * 4, v);
#pragma unroll
    for (int k = 0; k < NC; ++k)
      f[(long long)(i * NC + k) * p.plane + cell] = Store<S>::kOffset ? (double)v[k] + sc->wref[k] : (double)v[k];
  }
}

// beta-only preparation: 1/M_k of the current state (partial slot n & 1) into separate scratch.
__global__ void __launch_bounds__(kNTD) k_beta_prep(Scalars* sc, const KParams p, const double* __restrict__ part,
                                                     double* invM_beta) {
  const int slot = (int)(sc->n & 1);
  double mx[kNV];
  fold_partials<kNTD>(part + (long long)slot * p.max_parts * kNV, sc->nparts[slot], mx);
  if (threadIdx.x == 0)
    for (int k = 0; k < p.nc; ++k) {
      invM_beta[k] = mx[1 + k] > 0.0 ? 1.0 / mx[1 + k] : 0.0;
      reinterpret_cast<float*>(invM_beta + 4)[k] = (float)invM_beta[k];
    }
}

__global__ void k_begin(Scalars* sc, double t_end) {
  sc->t_end = t_end;
  sc->done = (t_end > 0.0 && sc->t >= t_end) ? 1 : 0;
}

// ------------------------------------------------------------------------------------------
// host launchers
// ------------------------------------------------------------------------------------------
namespace {
constexpr int kNT1 = 256;        // threads of the cell-parallel kernels
constexpr int kGridStride = 592; // CTAs of the grid-stride producers (4 per SM on 148 SMs)

template <int D>
struct TileCfg;
template <>
struct TileCfg<2> {  // 2D tiles of 32 x 16 cells
  static constexpr int TX = 32, TY = 16;
};
template <>
struct TileCfg<1> {  // 1D tiles of 64 cells: a 1000-cell problem spreads over 16 SMs (its FP64 work
                     // took 4 SMs 12 us per step with 256-cell tiles)
  static constexpr int TX = 64, TY = 1;
};

template <int D, class S, bool LOOK, bool BOUT>
cudaError_t launch_tile_t(const Launch& L, const void* fin, void* fout, int pulled, const void* invM, double* beta_out) {
  constexpr int TX = TileCfg<D>::TX, TY = TileCfg<D>::TY;
  using G = TileGeom<D, S, LOOK, TX, TY>;
  const KParams& p = *L.p;
  dim3 grid((p.nx + TX - 1) / TX, D == 2 ? (p.ny + TY - 1) / TY : 1);
  k_tile<D, S, LOOK, BOUT, TX, TY><<<grid, TX * TY, G::smem_bytes, L.stream>>>((const S*)fin, (S*)fout, L.sc, p, pulled,
                                                                              (const typename Store<S>::M*)invM, beta_out,
                                                                              L.part);
  return cudaGetLastError();
}

template <int D, class S, bool LOOK, bool BOUT>
cudaError_t prepare_tile_t() {
  constexpr int TX = TileCfg<D>::TX, TY = TileCfg<D>::TY;
  using G = TileGeom<D, S, LOOK, TX, TY>;
  return cudaFuncSetAttribute(k_tile<D, S, LOOK, BOUT, TX, TY>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)G::smem_bytes);
}

template <class S, bool LOOK, bool BOUT>
cudaError_t launch_tile_d(const Launch& L, const void* fin, void* fout, int pulled, const void* invM, double* beta_out) {
  return L.p->dim == 1 ? launch_tile_t<1, S, LOOK, BOUT>(L, fin, fout, pulled, invM, beta_out)
                       : launch_tile_t<2, S, LOOK, BOUT>(L, fin, fout, pulled, invM, beta_out);
}

unsigned blocks1(const KParams& p) { return (unsigned)((p.plane + kNT1 - 1) / kNT1); }
unsigned blocks_gs(const KParams& p) {
  const long long b = (p.plane + kNT1 - 1) / kNT1;
  return (unsigned)(b < kGridStride ? b : kGridStride);
}

template <int D, class S>
void launch_reduce_t(const Launch& L, const void* fin, int pulled, int in_run, float* pk = nullptr) {
  if constexpr (D == 1) {  // CTAs of 64 cells, as the 1D tiles: the small 1D problems spread over more SMs
    const long long b = (L.p->plane + 63) / 64;
    k_reduce<D, S, 64><<<(unsigned)(b < kGridStride ? b : kGridStride), 64, 0, L.stream>>>(
        (const S*)fin, L.sc, *L.p, pulled, L.part, in_run, nullptr, pk);
  } else {
    k_reduce<D, S, kNT1><<<blocks_gs(*L.p), kNT1, 0, L.stream>>>((const S*)fin, L.sc, *L.p, pulled, L.part, in_run,
                                                                   in_run ? L.fields : nullptr, pk);
  }
}
}  // namespace

// Opt-in shared memory sizes of every step-kernel instantiation (current device); called once
// per solver before any launch or graph capture.
cudaError_t prepare_kernels() {
  cudaError_t e = cudaSuccess;
#define VLBM_PREP(D, S, LK, B) \
  if (e == cudaSuccess) e = prepare_tile_t<D, S, LK, B>();
  VLBM_PREP(1, double, false, false) VLBM_PREP(1, double, true, false) VLBM_PREP(1, double, false, true)
  VLBM_PREP(1, float, false, false) VLBM_PREP(1, float, true, false) VLBM_PREP(1, float, false, true)
  VLBM_PREP(2, double, false, false) VLBM_PREP(2, double, true, false) VLBM_PREP(2, double, false, true)
  VLBM_PREP(2, float, false, false) VLBM_PREP(2, float, true, false) VLBM_PREP(2, float, false, true)
#undef VLBM_PREP
  if (e == cudaSuccess) e = prepare_roll_kernels();
  return e;
}

int sum_blocks(const KParams& p) {
  long long b = (p.plane + kNT1 - 1) / kNT1;
  return (int)(b < 1184 ? b : 1184);
}

// Largest number of CTAs any partial-maxima producer launches for this grid.
int max_partials(const KParams& p) {
  long long tiles = p.dim == 2 ? (long long)((p.nx + TileCfg<2>::TX - 1) / TileCfg<2>::TX) * ((p.ny + TileCfg<2>::TY - 1) / TileCfg<2>::TY)
                               : (long long)((p.nx + TileCfg<1>::TX - 1) / TileCfg<1>::TX);
  long long gs = blocks_gs(p);
  long long m = tiles > gs ? tiles : gs;
  const long long rc = roll_ctas(p);
  return (int)(rc > m ? rc : m);
}

cudaError_t launch_reduce(const Launch& L, int precision, const void* fin, int pulled, bool in_run) {
  const int r = in_run ? 1 : 0;
  if (L.p->dim == 1) {
    if (precision == 0) launch_reduce_t<1, double>(L, fin, pulled, r);
    else launch_reduce_t<1, float>(L, fin, pulled, r);
  } else {
    if (precision == 0) launch_reduce_t<2, double>(L, fin, pulled, r);
    else launch_reduce_t<2, float>(L, fin, pulled, r);
  }
  return cudaGetLastError();
}

cudaError_t launch_fill_pressure(const Launch& L, const void* fin, int pulled) {
  if (!L.pkeep || L.p->dim != 2) return cudaSuccess;
  launch_reduce_t<2, float>(L, fin, pulled, 0, L.pkeep);
  return cudaGetLastError();
}

cudaError_t launch_dt(const Launch& L) {
  k_dt<<<1, kNTD, 0, L.stream>>>(L.sc, *L.p, L.part, L.hist_dt, L.hist_c, L.sched);
  return cudaGetLastError();
}

cudaError_t launch_step(const Launch& L, int precision, bool lookahead, const void* fin, void* fout, int pulled) {
  if (L.p->dim == 2 && L.p->strip) return launch_roll(L, precision, lookahead, fin, fout, pulled);
  const char* base = reinterpret_cast<const char*>(L.sc);
  if (precision == 0) {
    const void* invM = base + offsetof(Scalars, inv_M);
    return lookahead ? launch_tile_d<double, true, false>(L, fin, fout, pulled, invM, nullptr)
                     : launch_tile_d<double, false, false>(L, fin, fout, pulled, invM, nullptr);
  }
  const void* invM = base + offsetof(Scalars, inv_M_f);
  return lookahead ? launch_tile_d<float, true, false>(L, fin, fout, pulled, invM, nullptr)
                   : launch_tile_d<float, false, false>(L, fin, fout, pulled, invM, nullptr);
}

cudaError_t launch_beta(const Launch& L, int precision, const void* fin, int pulled, double* beta_out) {
  const KParams& p = *L.p;
  // maxima of the current state into partial slot n & 1 (the same values any producer of that
  // slot writes for this state), then 1/M_k into the beta scratch
  cudaError_t e = launch_reduce(L, precision, fin, pulled, false);
  if (e != cudaSuccess) return e;
  double* invM_beta = beta_out + p.plane;  // caller provides plane + 8 doubles (1/M_k in FP64, FP32)
  k_beta_prep<<<1, kNTD, 0, L.stream>>>(L.sc, p, L.part, invM_beta);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (precision == 0) return launch_tile_d<double, false, true>(L, fin, nullptr, pulled, invM_beta, beta_out);
  return launch_tile_d<float, false, true>(L, fin, nullptr, pulled, invM_beta + 4, beta_out);
}

cudaError_t launch_init(const Launch& L, int precision, const double* W0, void* fout, double* partial, int nblk_sum,
                        bool maxima) {
  const KParams& p = *L.p;
  k_init_begin<<<1, 1, 0, L.stream>>>(L.sc);
  if (p.dim == 1) k_reduce_W0<1, kNT1><<<blocks_gs(p), kNT1, 0, L.stream>>>(W0, L.sc, p, L.part);
  else k_reduce_W0<2, kNT1><<<blocks_gs(p), kNT1, 0, L.stream>>>(W0, L.sc, p, L.part);
  if (precision == 1) {
    k_sum_partial<kNT1><<<nblk_sum, kNT1, 0, L.stream>>>(W0, p, partial);
    k_sum_final<<<1, 32, 0, L.stream>>>(partial, nblk_sum, p, L.sc);
  }
  k_init_c0<<<1, kNTD, 0, L.stream>>>(L.sc, p, L.part, L.sched);
  const unsigned g = blocks_gs(p);
#define VLBM_INIT_EQ(D, S, PK)                                                                          \
  (maxima ? k_init_eq<D, S, kNT1, true><<<g, kNT1, 0, L.stream>>>(W0, (S*)fout, L.sc, p, L.part, PK)    \
          : k_init_eq<D, S, kNT1, false><<<g, kNT1, 0, L.stream>>>(W0, (S*)fout, L.sc, p, L.part, PK))
  if (p.dim == 1) {
    if (precision == 0) VLBM_INIT_EQ(1, double, nullptr);
    else VLBM_INIT_EQ(1, float, nullptr);
  } else {
    if (precision == 0) VLBM_INIT_EQ(2, double, nullptr);
    else VLBM_INIT_EQ(2, float, L.pkeep);
  }
#undef VLBM_INIT_EQ
  return cudaGetLastError();
}

cudaError_t launch_get_W(const Launch& L, int precision, const void* fin, int pulled, double* W) {
  const KParams& p = *L.p;
  if (p.dim == 1) {
    if (precision == 0) k_get_W<1, double, kNT1><<<blocks1(p), kNT1, 0, L.stream>>>((const double*)fin, L.sc, p, pulled, W);
    else k_get_W<1, float, kNT1><<<blocks1(p), kNT1, 0, L.stream>>>((const float*)fin, L.sc, p, pulled, W);
  } else {
    if (precision == 0) k_get_W<2, double, kNT1><<<blocks1(p), kNT1, 0, L.stream>>>((const double*)fin, L.sc, p, pulled, W);
    else k_get_W<2, float, kNT1><<<blocks1(p), kNT1, 0, L.stream>>>((const float*)fin, L.sc, p, pulled, W);
  }
  return cudaGetLastError();
}

cudaError_t launch_get_f(const Launch& L, int precision, const void* fin, int pulled, double* f) {
  const KParams& p = *L.p;
  if (p.dim == 1) {
    if (precision == 0) k_get_f<1, double, kNT1><<<blocks1(p), kNT1, 0, L.stream>>>((const double*)fin, L.sc, p, pulled, f);
    else k_get_f<1, float, kNT1><<<blocks1(p), kNT1, 0, L.stream>>>((const float*)fin, L.sc, p, pulled, f);
  } else {
    if (precision == 0) k_get_f<2, double, kNT1><<<blocks1(p), kNT1, 0, L.stream>>>((const double*)fin, L.sc, p, pulled, f);
    else k_get_f<2, float, kNT1><<<blocks1(p), kNT1, 0, L.stream>>>((const float*)fin, L.sc, p, pulled, f);
  }
  return cudaGetLastError();
}

cudaError_t launch_totals(const Launch& L, int precision, const void* fin, int pulled, double* W, double* partial,
                          int nblk_sum, double* out) {
  const KParams& p = *L.p;
  cudaError_t e = launch_get_W(L, precision, fin, pulled, W);
  if (e != cudaSuccess) return e;
  k_sum_partial<kNT1><<<nblk_sum, kNT1, 0, L.stream>>>(W, p, partial);
  k_sum_out<<<1, 32, 0, L.stream>>>(partial, nblk_sum, p, out);
  return cudaGetLastError();
}

// begin-of-call marker (end time and done flag), used by the C-ABI layer
cudaError_t launch_begin(const Launch& L, double t_end) {
  k_begin<<<1, 1, 0, L.stream>>>(L.sc, t_end);
  return cudaGetLastError();
}

}  // namespace vlbm

// ==========================================================================================
// Allocation-free beta(x) of caller-owned populations.
//
// For callers that cannot call cudaMalloc: an application whose device memory belongs entirely
// to its own pool allocator, code that must not allocate while a CUDA graph is being captured,
// or a loop with a fixed memory budget.  The scratch of the beta computation (the device scalar
// block, 1/M_k and the per-CTA partial maxima) lives in one file-scope static device array
// instead of memory owned by a vlbm handle.  The kernels are the ones vlbm_get_beta runs; the
// maxima kernel is launched with one CTA per 256 cells so that its partials fit the array.
// ==========================================================================================
namespace vlbm {
namespace {
constexpr int kNoallocCtaCells = 256;
constexpr int kNoallocMaxCtas = 8192;
constexpr long long kNoallocMaxCells = (long long)kNoallocCtaCells * kNoallocMaxCtas;  // 2,097,152
constexpr int kNoallocScalarsBytes = 1024;                                             // >= sizeof(Scalars)
constexpr int kNoallocInvMBytes = 256;                                                 // 4 FP64 + 4 FP32
constexpr size_t kNoallocBytes =
    kNoallocScalarsBytes + kNoallocInvMBytes + (size_t)kNoallocMaxCtas * kNV * sizeof(double);
static_assert(sizeof(Scalars) <= kNoallocScalarsBytes, "scalar block does not fit its slot");

// Shared by every call on a device; holds the last call's contents until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

constexpr int kNoallocMaxDevices = 64;
std::atomic<unsigned char*> g_noalloc_addr[kNoallocMaxDevices];  // device address, per device ordinal
std::mutex g_noalloc_mutex;                                        // serialises the first-call set-up
}  // namespace

}  // namespace vlbm

extern "C" vlbm_status vlbm_beta_noalloc(const vlbm_grid* grid, const vlbm_eos* eos, const vlbm_params* params,
                                         const double* f, int32_t in_place, double* beta, void* cuda_stream) {
  using namespace vlbm;
  if (!grid || !eos || !params || !f || !beta) return VLBM_E_INVAL;
  if (!valid_problem(grid, eos, params)) return VLBM_E_INVAL;
  if (grid->bc[0] == VLBM_BC_INFLOW) return VLBM_E_UNSUPPORTED;  // no pinned state to read from
  // beyond the fixed scratch: rejected (each axis first, so that nx * ny cannot overflow)
  const long long nx = grid->nx, ny = grid->dim == 1 ? 1 : grid->ny;
  if (nx > kNoallocMaxCells || ny > kNoallocMaxCells || nx * ny > kNoallocMaxCells) return VLBM_E_INVAL;

  // Set-up, once per device, with that device current: the device address of the static array
  // and the kernels' shared-memory attribute.  Guarded, so that host threads making their first
  // calls at the same time set it up once.
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNoallocMaxDevices) return VLBM_E_CUDA;
  unsigned char* base = g_noalloc_addr[dev].load(std::memory_order_acquire);
  if (!base) {
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    base = g_noalloc_addr[dev].load(std::memory_order_relaxed);
    if (!base) {
      void* ptr = nullptr;
      if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) return VLBM_E_CUDA;
      if (cudaFuncSetAttribute(k_tile<1, double, false, true, TileCfg<1>::TX, TileCfg<1>::TY>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)TileGeom<1, double, false, TileCfg<1>::TX, TileCfg<1>::TY>::smem_bytes) != cudaSuccess ||
          cudaFuncSetAttribute(k_tile<2, double, false, true, TileCfg<2>::TX, TileCfg<2>::TY>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)TileGeom<2, double, false, TileCfg<2>::TX, TileCfg<2>::TY>::smem_bytes) != cudaSuccess)
        return VLBM_E_CUDA;
      base = static_cast<unsigned char*>(ptr);
      g_noalloc_addr[dev].store(base, std::memory_order_release);
    }
  }
  Scalars* sc = reinterpret_cast<Scalars*>(base);
  double* invM = reinterpret_cast<double*>(base + kNoallocScalarsBytes);
  double* part = reinterpret_cast<double*>(base + kNoallocScalarsBytes + kNoallocInvMBytes);

  KParams p{};
  make_kparams(grid, eos, params, p);  // the same parameters and coefficients as vlbm_create
  const int ncta = (int)((p.plane + kNoallocCtaCells - 1) / kNoallocCtaCells);
  p.max_parts = ncta;

  cudaStream_t s = (cudaStream_t)cuda_stream;
  const int pulled = in_place ? 0 : 1;
  // The scalar block must start at zero (no error bit, step 0); the partials and 1/M_k are
  // fully written by this call before they are read.
  if (cudaMemsetAsync(sc, 0, sizeof(Scalars), s) != cudaSuccess) return VLBM_E_CUDA;
  if (p.dim == 1) k_reduce<1, double, kNoallocCtaCells><<<ncta, kNoallocCtaCells, 0, s>>>(f, sc, p, pulled, part, 0, nullptr, nullptr);
  else k_reduce<2, double, kNoallocCtaCells><<<ncta, kNoallocCtaCells, 0, s>>>(f, sc, p, pulled, part, 0, nullptr, nullptr);
  k_beta_prep<<<1, kNTD, 0, s>>>(sc, p, part, invM);
  if (p.dim == 1) {
    constexpr int TX = TileCfg<1>::TX, TY = TileCfg<1>::TY;
    k_tile<1, double, false, true, TX, TY><<<dim3((p.nx + TX - 1) / TX, 1), TX * TY,
                                             TileGeom<1, double, false, TX, TY>::smem_bytes, s>>>(f, nullptr, sc, p, pulled,
                                                                                                 invM, beta, part);
  } else {
    constexpr int TX = TileCfg<2>::TX, TY = TileCfg<2>::TY;
    k_tile<2, double, false, true, TX, TY><<<dim3((p.nx + TX - 1) / TX, (p.ny + TY - 1) / TY), TX * TY,
                                             TileGeom<2, double, false, TX, TY>::smem_bytes, s>>>(f, nullptr, sc, p, pulled,
                                                                                                 invM, beta, part);
  }
  return cudaGetLastError() == cudaSuccess ? VLBM_OK : VLBM_E_CUDA;
}


// ==========================================================================================
// FP64 throughput of this GPU (the denominator of the FP64 path's ALU roofline): every thread
// runs eight independent chains of dependent FP64 fused multiply-adds, the grid fills every SM.
// ==========================================================================================
namespace vlbm {
namespace {
__device__ double g_fma_sink;

constexpr int kFmaThreads = 256, kFmaChains = 8;

__global__ void __launch_bounds__(kFmaThreads) k_dfma_rate(double m, double c, int iters, int write) {
  double a[kFmaChains];
#pragma unroll
  for (int j = 0; j < kFmaChains; ++j) a[j] = 1.0 + 1e-3 * (threadIdx.x + j);
  for (int it = 0; it < iters; ++it)
#pragma unroll
    for (int j = 0; j < kFmaChains; ++j) a[j] = fma(a[j], m, c);
  double sum = 0.0;
#pragma unroll
  for (int j = 0; j < kFmaChains; ++j) sum += a[j];
  if (write) g_fma_sink = sum;  // never taken at run time; keeps the chains live
}
}  // namespace
}  // namespace vlbm

extern "C" vlbm_status vlbm_measure_fp64_peak(int32_t reps, double* tflops) {
  using namespace vlbm;
  if (reps < 1 || !tflops) return VLBM_E_INVAL;
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_dfma_rate, kFmaThreads, 0) != cudaSuccess || per_sm < 1)
    return VLBM_E_CUDA;
  const int grid = sms * per_sm, iters = 8192;
  cudaStream_t s = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  vlbm_status st = VLBM_OK;
  if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
      cudaEventCreate(&e1) != cudaSuccess)
    st = VLBM_E_CUDA;
  double best = 0.0;
  k_dfma_rate<<<grid, kFmaThreads, 0, s>>>(0.9999999, 1e-7, iters, 0);  // warm-up
  for (int r = 0; r < reps && st == VLBM_OK; ++r) {
    float ms = 0.f;
    if (cudaEventRecord(e0, s) != cudaSuccess) st = VLBM_E_CUDA;
    k_dfma_rate<<<grid, kFmaThreads, 0, s>>>(0.9999999, 1e-7, iters, 0);
    if (st == VLBM_OK && (cudaGetLastError() != cudaSuccess || cudaEventRecord(e1, s) != cudaSuccess ||
                          cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
      st = VLBM_E_CUDA;
    const double flops = 2.0 * (double)grid * kFmaThreads * kFmaChains * iters;
    if (st == VLBM_OK && ms > 0.f) best = flops / (ms * 1e-3) / 1e12 > best ? flops / (ms * 1e-3) / 1e12 : best;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (s) cudaStreamDestroy(s);
  *tflops = best;
  return st;
}
