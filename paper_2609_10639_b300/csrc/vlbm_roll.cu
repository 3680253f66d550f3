// Column-marching form of the 2D step kernel (sm_103a).
//
// The grid is cut into column strips of TXO output columns; the strip-rows of all strips, taken
// strip by strip, are split evenly over a persistent grid of CTAs (as many as fit on the GPU at
// once, so every SM gets the same work), and each CTA walks down its share (one or two strip
// segments) RR rows at a time.  Every quantity of the step is computed once per row and kept in
// shared-memory ring buffers for as long as the stencils below need it, so the only
// recomputation is the x-halo of the strip (H columns on each side) and H rows at each end of a
// segment, instead of a halo all around a small tile.  Per iteration (block start F):
//
//   S1  rows [F, F+RR):        pulled populations (Eq. 21), W, u, flux Q_alpha (Eqs. 10, 15-17),
//                              or in the FP64 two-pass form W, u, Q kept by the maxima pass
//                              -> ring of Q and u (2 RR rows); the populations stay in registers
//   S2  rows [F-RR+1, F+1):    flux-divergence activity s (Eqs. 28-31) and Ducros ratio theta
//                              (Eqs. 32-33) -> ring of (s, theta) (RR + 2 rows)
//   S3  rows [F-RR, F):        box filters and beta (Eqs. 34-35), fused reprojection (Eqs. 38-40)
//                              and relaxation (Eqs. 20, 22) on the populations S1 loaded one
//                              iteration earlier (same thread), single write to HBM
//   S4  rows [F-RR-1, F-1):    (look-ahead) W^{n+1} = sum_i f*_i(x - sigma_i) from the rings of
//                              relaxed populations (RR + 2 rows, RR + 1 for f*_{y-}), and the
//                              maxima of the next step (Eqs. 30, 36) accumulated in registers
//                              over the whole strip
//
// Boundary rules as in the tile kernel: positions and rows outside a zero-gradient side hold the
// edge cell's populations (S1 maps them), and every stencil read of s, theta (S3) and of the
// relaxed populations (S4) is taken at the edge cell there; periodic sides are unwrapped.
#include <type_traits>

#include "vlbm.h"
#include "vlbm_device.cuh"
#include "vlbm_internal.cuh"

namespace vlbm {

namespace {

template <class S, bool LOOK, int XW, int RR>
struct RollGeom {
  using M = typename Store<S>::M;
  static constexpr int H = LOOK ? 3 : 2;  // halo of u and Q around the output columns
  static constexpr int TXO = XW - 2 * H;  // output columns of a strip
  static constexpr int NT = XW * RR;
  static constexpr int RQ = 2 * RR;       // rows of the u/Q ring: [F-RR, F+RR)
  static constexpr int RS = RR + 2;       // rows of the (s, theta) ring: [F-RR-1, F+1)
  // Relaxed-population rings, one per direction, each as deep as the rows S4 still reads after
  // S3 wrote rows [F-RR, F): x pairs and f*_{y-} (read at the row itself, or the row below it
  // only where that is the edge row) [F-RR-1, F); f*_{y+} (read from the row above) [F-RR-2, F).
  // The y- ring is one row short of the others (less shared memory per resident CTA).
  __host__ __device__ static constexpr int RF(int i) { return i == 2 ? RR + 1 : RR + 2; }
  __host__ __device__ static constexpr int OF(int i) { return i <= 2 ? i * (RR + 2) : 2 * (RR + 2) + RR + 1; }
  // FP64 two-pass form: the x pass of the box filter runs once per row in a stage of its own (S2x)
  // into a ring of x-filtered (s, theta) rows, instead of three times per cell in S3 (8 FP64
  // operations per cell fewer on the FP64 pipe that bounds that kernel); the raw (s, theta) ring
  // then only holds the RR rows S2 has just written.
  static constexpr bool XF = sizeof(M) == 8 && !LOOK;
  static constexpr int RSR = XF ? RR : RS;  // rows of the raw (s, theta) ring
  static constexpr size_t nQ = (size_t)RQ * 2 * XW * 4;
  static constexpr size_t nU = (size_t)RQ * XW * 2;
  static constexpr size_t nS = (size_t)RSR * XW * 2;
  static constexpr size_t nF = LOOK ? (size_t)(OF(3) + RF(3)) * XW * 4 : 0;
  static constexpr size_t nX = XF ? (size_t)RS * XW * 2 : 0;  // x-filtered (s, theta) ring
  static constexpr size_t smem_bytes = (nQ + nU + nS + nF + nX) * sizeof(M);
  static_assert(RR >= 2, "stage S2 of a block reads u/Q one row beyond it");
};

// Asks the TMA unit to bring `bytes` (a multiple of 16, from a 16-byte aligned address inside the
// buffer) into L2; nothing waits for it and no register receives data.
__device__ __forceinline__ void prefetch_l2(const void* src, unsigned bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}

// Ring slot of row r (rows never lie more than 8 R below the strip's first row `base`).
template <int R>
__device__ __forceinline__ int ring(int r, int base) {
  return (int)((unsigned)(r - base + 8 * R) % (unsigned)R);
}

// FP32 storage: about 1024 resident threads per SM (64 registers) to hide memory latency (0.46 vs
// 0.73 ms per two-pass step kernel at 4096^2 with half of them); FP64 is bound by its FP64 pipe
// and runs two CTAs of up to 128 registers per SM, so that one CTA's stage S1 (loads only, with
// W, u, Q kept by the maxima pass) overlaps the other's arithmetic.  INFLOW: the grid has a
// pinned-inflow x-lo side (a separate instantiation: the ghost paths cost the FP32 kernel register
// spills, 76 bytes, which the other grids need not pay).  KEEP (FP32 storage, look-ahead, non-ideal
// gas): stage S4 keeps the pressure it computes for the next state in pk[(n) & 1] and stage S1 reads
// it from pk[(n - 1) & 1] instead of evaluating the FP64 equation of state a second time for the
// same W (the FP64 EOS, with its Newton inversion for c_v(T), bounds that path); bit-identical.
template <class S, bool LOOK, int XW, int RR, bool INFLOW, bool KEEP>
__global__ void __launch_bounds__(XW * RR, sizeof(S) == 4 ? 1024 / (XW * RR) : 512 / (XW * RR)) k_roll(const S* __restrict__ fin, S* __restrict__ fout,
                                                  Scalars* __restrict__ sc, const KParams p, const int pulled,
                                                  const typename Store<S>::M* __restrict__ invM_src,
                                                  double* __restrict__ part, const double* __restrict__ fields,
                                                  double* __restrict__ sens, float* __restrict__ pk) {
  using G = RollGeom<S, LOOK, XW, RR>;
  using M = typename G::M;
  constexpr int H = G::H, TXO = G::TXO, RQ = G::RQ, RS = G::RS;
  constexpr bool OFF = Store<S>::kOffset;
  if (!sc->active) return;

  extern __shared__ __align__(16) unsigned char smem_raw[];
  M* sQ = reinterpret_cast<M*>(smem_raw);  // [RQ][2][XW][4]
  M* sU = sQ + G::nQ;                      // [RQ][XW][2]
  M* sS = sU + G::nU;                      // [RS][XW][2]
  M* sF = sS + G::nS;                      // direction i: [RF(i)][XW][4] from row OF(i) (look-ahead)
  M* sX = sF + G::nF;                      // [RS][XW][2] x-filtered (s, theta) (FP64 two-pass)

  const Coef<M>& co = coef<M>(p);
  const int tx = threadIdx.x % XW, ty = threadIdx.x / XW;
  // zero-gradient sides in x (each side alone: a pinned-inflow x-lo side pairs with a
  // zero-gradient x-hi side) and in y (both sides alike, checked at vlbm_create)
  const bool zxl = p.bc[0] == 1, zxh = p.bc[1] == 1, zy = p.bc[2] == 1;
  constexpr bool gx = INFLOW;  // pinned-inflow x-lo side: ghost cells x < 0 hold W_in
  // centre_pos of a row.  Both sides of the y axis share their rule, so a zero-gradient axis
  // clamps and a periodic one keeps the unwrapped index; the FP32 kernel takes that branch-free
  // form (0.495 against 0.527 ms per look-ahead step kernel at 4096^2), the FP64 kernel the
  // general one (4.90 against 4.95 ms).
  auto yc = [&](int r) -> int {
    if constexpr (sizeof(S) == 4) return zy ? min(max(r, 0), p.ny - 1) : r;
    else return centre_pos(r, p.ny, p.bc[2], p.bc[3]);
  };

  M wq[4], invMh[4];  // invMh: M_k^-1 / 2 (s_hat_k = jump over two cells / 2 / M_k, Eqs. 29-30)
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    wq[k] = StepScalars<M>::wq(sc, k);
    invMh[k] = (M)0.5 * invM_src[k];
  }
  const M r_c = StepScalars<M>::r(sc), inv_c = StepScalars<M>::inv_c(sc);
  const int slot_n = (int)(sc->n & 1);
  static_assert(!KEEP || (sizeof(S) == 4 && LOOK), "kept pressure: FP32 storage, look-ahead form only");
  const float* pk_in = KEEP ? pk + (long long)(slot_n ^ 1) * p.plane : nullptr;  // written by the previous step
  float* pk_out = KEEP ? pk + (long long)slot_n * p.plane : nullptr;
  // pinned inflow: the ghost values at the link speed of the stored populations, c_new r (read
  // after the barrier at the start of the first segment)
  __shared__ GhostTab<2, M> gtab;
  if constexpr (INFLOW) {
    if (threadIdx.x == 0) fill_ghost_tab<2, M, OFF>(p, wq, inv_c / r_c, gtab);
  }

  using R = Red<M>;
  typename R::T vmax[kNV];
#pragma unroll
  for (int j = 0; j < kNV; ++j) vmax[j] = typename R::T(0);
  bool bad = false;

  M fcar[4][4];  // populations this thread loaded in S1 of the previous iteration
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int k = 0; k < 4; ++k) fcar[i][k] = (M)0;

  // this CTA's share of the strip-rows, strip-major
  const int nstrips = (p.nx + TXO - 1) / TXO;
  const long long total = (long long)nstrips * p.ny;
  long long a = total * blockIdx.x / gridDim.x;
  const long long b_end = total * (blockIdx.x + 1) / gridDim.x;
  for (; a < b_end;) {
  const int strip = (int)(a / p.ny);
  const int y0 = (int)(a - (long long)strip * p.ny);
  const int yend = (int)min((long long)p.ny, (long long)y0 + (b_end - a));
  a += yend - y0;
  const int x0 = strip * TXO;
  const int xs = x0 - H;  // column of strip position 0
  const int px = xs + tx;
  const int xend = min(x0 + TXO, p.nx);
  const int base = y0 - H;
  // strip positions or their pull sources outside [0, nx): boundary rules needed in x
  const bool xedge = xs - 1 < 0 || xs + XW + 1 > p.nx;
  // strip index of the value read at column px + d (the edge cell beyond a zero-gradient side)
  auto xi = [&](int d) -> int {
    if constexpr (sizeof(S) == 4) {
      if (!xedge) return tx + d;
      int j = px + d;
      if (zxl) j = max(j, 0);
      if (zxh) j = min(j, p.nx - 1);
      return j - xs;
    } else {
      return xedge ? centre_pos(px + d, p.nx, p.bc[0], p.bc[1]) - xs : tx + d;
    }
  };
  // positions beyond a zero-gradient x side hold no values of their own (reads land on the edge)
  const bool x_void = (zxl && px < 0) || (zxh && px >= p.nx);
  // the column and row-range predicates of the stages, constant over the segment
  const bool c1 = px >= x0 - H && px < xend + H;
  const bool c2 = px >= x0 - H + 1 && px < xend + H - 1 && !x_void && p.beta_mode == 0;
  const bool c3 = px >= x0 - H + 2 && px < xend + H - 2 && !x_void;
  const bool cout = px >= x0 && px < xend;
  const int r1hi = yend + H, r2lo = y0 - H + 1, r2hi = yend + H - 1, r3lo = y0 - H + 2, r3hi = yend + H - 2;
  // S4 (look-ahead) of block Fb: W^{n+1} of rows [Fb-RR-1, Fb-1) from the rings of relaxed
  // populations and the next step's maxima.  It runs after a barrier at the end of its block, when
  // only the populations carried to the next block are live (run alongside the next block's S2,
  // which would save that barrier, it kept both blocks' populations live and spilled registers).
  auto s4 = [&](int Fb) {
    const int r = Fb - RR - 1 + ty;
    if (cout && r >= y0 && r < yend) {
      M fr[4][4], W[4];
      const int xm = xi(-1), xp = xi(1);
      const int sfy = ring<G::RF(0)>(r, base);
      const int sfm = ring<G::RF(3)>(yc(r - 1), base), sfp = ring<G::RF(2)>(yc(r + 1), base);
      ld4s(sF + ((G::OF(0) + sfy) * XW + xp) * 4, fr[0]);  // f*_{x-} from x+1
      ld4s(sF + ((G::OF(1) + sfy) * XW + xm) * 4, fr[1]);  // f*_{x+} from x-1
      ld4s(sF + ((G::OF(2) + sfp) * XW + tx) * 4, fr[2]);  // f*_{y-} from y+1
      ld4s(sF + ((G::OF(3) + sfm) * XW + tx) * 4, fr[3]);  // f*_{y+} from y-1
      moments<2, M, OFF>(fr, wq, W);
      M u[2], Qf[2][4], cs, Pc;
      bad |= !prim_flux<2, M, true>(p, W, u, Qf, cs, KEEP ? &Pc : nullptr);
      if constexpr (KEEP) pk_out[r * p.nx + px] = (float)Pc;
      cell_maxima<2, M>(u, cs, Qf, vmax);
    }
  };
  __syncthreads();  // the rings of a previous segment are no longer read

  // FP32 look-ahead form: two blocks per loop trip, so that the populations carried from S1 to the
  // next block's S3 change roles instead of being copied (0.480 against 0.494 ms per step kernel at
  // 4096^2); the FP64 forms would spill at their 128 registers.
#pragma unroll (sizeof(S) == 4 && LOOK ? 2 : 1)
  for (int F = base; F - RR - (LOOK ? 1 : 0) < yend; F += RR) {
    // FP32 storage: L2 prefetch of the populations S1 of the next iteration reads (rows
    // [F+RR, F+2RR)), per direction the contiguous run of its pull sources in the strip's
    // columns, one bulk prefetch per lane of the first warp.  An iteration takes microseconds, so
    // those loads then hit L2 (measured at 4096^2: 0.553 against 0.585 ms per look-ahead step
    // kernel).  The FP64 kernel is bound by its FP64 pipe and ran slower with it (5.40 against
    // 5.25 ms), also when the kept W, u, Q planes were prefetched as well.
    if constexpr (sizeof(S) == 4) {
      const int t = threadIdx.x;
      if (t < 4 * RR) {
        const int c0 = max(xs - 1, 0), c1 = min(xs + XW + 1, p.nx);
        const int i = t % 4, rr = F + RR + t / 4;
        const int sr = pulled ? rr - sig_y(i) : rr;
        if (rr < yend + H && sr >= 0 && sr < p.ny && c1 > c0)
          prefetch_l2(fin + ((long long)i * p.plane + (long long)sr * p.nx + c0) * 4, (unsigned)(c1 - c0) * 16u);
      }
    }

    // ---- S1: pulled populations, W, u, Q of rows [F, F+RR) ----
    M fnew[4][4];
    {
      const int r = F + ty;
      const bool act = c1 && r < r1hi;
      if (act) {
        const int cy = (r >= 0 && r < p.ny) ? r : nb_index(r, p.ny, p.bc[2], p.bc[3]);
        const int cx = xedge ? nb_index(px, p.nx, p.bc[0], p.bc[1]) : px;
        const bool inner = !xedge && cy >= 1 && cy < p.ny - 1;
        const bool ghost = gx && px < 0;  // a ghost cell of the pinned-inflow side
        M W[4], u[2], Qf[2][4], cs;
        bool have = false;
        if constexpr (INFLOW) {
          if (ghost) {
#pragma unroll
          for (int k = 0; k < 4; ++k) {
#pragma unroll
            for (int i = 0; i < 4; ++i) fnew[i][k] = gtab.f[i][k];
            W[k] = gtab.W[k];
            Qf[0][k] = gtab.Q[0][k];
            Qf[1][k] = gtab.Q[1][k];
          }
          u[0] = gtab.u[0];
          u[1] = gtab.u[1];
          have = true;
          } else {
            load_cell<2, S>(fin, p, cx, cy, pulled, inner, fnew, &gtab.f[0][0]);
          }
        } else {
          load_cell<2, S>(fin, p, cx, cy, pulled, inner, fnew);
        }
        if constexpr (!LOOK && std::is_same<M, double>::value) {
          if (fields && !ghost) {  // W, u, Q of this state, stored by the maxima pass
            const int c = cy * p.nx + cx;
            const long long P = p.plane;
#pragma unroll
            for (int k = 0; k < 4; ++k) W[k] = fields[k * P + c];
            u[0] = fields[4 * P + c];
            u[1] = fields[5 * P + c];
#pragma unroll
            for (int al = 0; al < 2; ++al)
#pragma unroll
              for (int k = 0; k < 4; ++k) Qf[al][k] = fields[(6 + 4 * al + k) * P + c];
            have = true;
          }
        }
        if (!have) {
          moments<2, M, OFF>(fnew, wq, W);
          if constexpr (KEEP) {
            flux_given_P<2>(W, pk_in[cy * p.nx + cx], u, Qf);
          } else {
            prim_flux<2, M, false>(p, W, u, Qf, cs);
          }
        }
        const int s = ring<RQ>(r, base);
#pragma unroll
        for (int al = 0; al < 2; ++al) st4s(sQ + ((s * 2 + al) * XW + tx) * 4, Qf[al]);
        if constexpr (sizeof(M) == 8) {
          reinterpret_cast<double2*>(sU)[s * XW + tx] = make_double2((double)u[0], (double)u[1]);
        } else {
          reinterpret_cast<float2*>(sU)[s * XW + tx] = make_float2((float)u[0], (float)u[1]);
        }
      }
    }
    __syncthreads();

    // ---- S2: s and theta of rows [F-RR+1, F+1) ----
    {
      const int r = F - RR + 1 + ty;
      const bool act = c2 && r >= r2lo && r < r2hi && !(zy && (r < 0 || r >= p.ny));
      if (act) {
        const int sm = ring<RQ>(r - 1, base), s0 = ring<RQ>(r, base), sp = ring<RQ>(r + 1, base);
        M qxp[4], qxm[4], qyp[4], qym[4];
        ld4s(sQ + ((s0 * 2 + 0) * XW + tx + 1) * 4, qxp);
        ld4s(sQ + ((s0 * 2 + 0) * XW + tx - 1) * 4, qxm);
        ld4s(sQ + ((sp * 2 + 1) * XW + tx) * 4, qyp);
        ld4s(sQ + ((sm * 2 + 1) * XW + tx) * 4, qym);
        M acc = 0, shk[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const M jk = (qxp[k] - qxm[k]) + (qyp[k] - qym[k]);
          const M sh = jk * invMh[k];
          shk[k] = sh;
          acc += sh * sh;
        }
        const M sval = sqrt_(acc);  // 2 s (Eq. 31); the 2 is folded into c_chi2
        M uxp, uxm, vxp, vxm, uyp, uym, vyp, vym;
        if constexpr (sizeof(M) == 8) {
          const double2* u2 = reinterpret_cast<const double2*>(sU);
          const double2 a = u2[s0 * XW + tx + 1], b = u2[s0 * XW + tx - 1], c = u2[sp * XW + tx], d = u2[sm * XW + tx];
          uxp = a.x, vxp = a.y, uxm = b.x, vxm = b.y, uyp = c.x, vyp = c.y, uym = d.x, vym = d.y;
        } else {
          const float2* u2 = reinterpret_cast<const float2*>(sU);
          const float2 a = u2[s0 * XW + tx + 1], b = u2[s0 * XW + tx - 1], c = u2[sp * XW + tx], d = u2[sm * XW + tx];
          uxp = a.x, vxp = a.y, uxm = b.x, vxm = b.y, uyp = c.x, vyp = c.y, uym = d.x, vym = d.y;
        }
        const M dl = (uxp - uxm) + (vyp - vym), vt = (vxp - vxm) - (uyp - uym);  // 2 dx (dil, vort)
        const M th = div_(dl * dl, dl * dl + vt * vt + co.eps_lat);
        if constexpr (sizeof(M) == 8) {
          // adjoint recomputation: the sensor quantities of the cells this CTA owns, in the
          // adjoint's units (s_hat_k, s, theta, dil, vort)
          if (sens && r >= y0 && r < yend && px >= x0 && px < xend) {
            const long long P = p.plane, c = (long long)r * p.nx + px;
#pragma unroll
            for (int k = 0; k < 4; ++k) sens[k * P + c] = shk[k];
            sens[4 * P + c] = 0.5 * sval;
            sens[5 * P + c] = th;
            sens[6 * P + c] = dl * p.inv2dx;
            sens[7 * P + c] = vt * p.inv2dx;
          }
        }
        const int ss = ring<G::RSR>(r, base);
        if constexpr (sizeof(M) == 8) {
          reinterpret_cast<double2*>(sS)[ss * XW + tx] = make_double2((double)sval, (double)th);
        } else {
          reinterpret_cast<float2*>(sS)[ss * XW + tx] = make_float2((float)sval, (float)th);
        }
      }
    }
    __syncthreads();

    // ---- S2x (FP64 two-pass): x pass of the box filter of rows [F-RR+1, F+1) ----
    if constexpr (G::XF) {
      const int r = F - RR + 1 + ty;
      const bool act = r >= y0 - H + 1 && r < yend + H - 1 && px >= x0 - H + 2 && px < xend + H - 2 &&
                       !(zy && (r < 0 || r >= p.ny)) && !x_void && p.beta_mode == 0;
      if (act) {
        const double2* s2 = reinterpret_cast<const double2*>(sS) + ring<G::RSR>(r, base) * XW;
        const double2 e0 = s2[xi(-1)], e1 = s2[tx], e2 = s2[xi(1)];
        reinterpret_cast<double2*>(sX)[ring<RS>(r, base) * XW + tx] =
            make_double2(box3(e0.x, e1.x, e2.x), box3(e0.y, e1.y, e2.y));
      }
      __syncthreads();
    }

    // ---- S3: beta, fused reprojection + relaxation of rows [F-RR, F), single write ----
    {
      const int r = F - RR + ty;
      const bool act = c3 && r >= r3lo && r < r3hi && !(zy && (r < 0 || r >= p.ny));
      if (act) {
        M beta = co.beta_const;
        if (p.beta_mode == 0 && G::XF) {
          M rs[3], rt[3];
#pragma unroll
          for (int j = 0; j < 3; ++j) {
            const double2 e = reinterpret_cast<const double2*>(sX)[ring<RS>(yc(r - 1 + j), base) * XW + tx];
            rs[j] = (M)e.x;
            rt[j] = (M)e.y;
          }
          beta = beta_of<M>(co, co.c_chi2 * box3(rs[0], rs[1], rs[2]) * box3(rt[0], rt[1], rt[2]));
        } else if (p.beta_mode == 0) {
          const int xm = xi(-1), xp = xi(1);
          M rs[3], rt[3];
#pragma unroll
          for (int j = 0; j < 3; ++j) {
            const int ss = ring<RS>(yc(r - 1 + j), base);
            M a0, a1, a2, b0, b1, b2;
            if constexpr (sizeof(M) == 8) {
              const double2* s2 = reinterpret_cast<const double2*>(sS) + ss * XW;
              const double2 e0 = s2[xm], e1 = s2[tx], e2 = s2[xp];
              a0 = e0.x, b0 = e0.y, a1 = e1.x, b1 = e1.y, a2 = e2.x, b2 = e2.y;
            } else {
              const float2* s2 = reinterpret_cast<const float2*>(sS) + ss * XW;
              const float2 e0 = s2[xm], e1 = s2[tx], e2 = s2[xp];
              a0 = e0.x, b0 = e0.y, a1 = e1.x, b1 = e1.y, a2 = e2.x, b2 = e2.y;
            }
            rs[j] = box3(a0, a1, a2);
            rt[j] = box3(b0, b1, b2);
          }
          beta = beta_of<M>(co, co.c_chi2 * box3(rs[0], rs[1], rs[2]) * box3(rt[0], rt[1], rt[2]));
        }
        M Qc[2][4];
        const int sq = ring<RQ>(r, base);
        ld4s(sQ + ((sq * 2 + 0) * XW + tx) * 4, Qc[0]);
        ld4s(sQ + ((sq * 2 + 1) * XW + tx) * 4, Qc[1]);
        relax_cell<2, M>(fcar, Qc, beta, r_c, inv_c);
        if (cout && r >= y0 && r < yend) store_cell<2, S, M>(fout, p, r * p.nx + px, fcar);
        if constexpr (LOOK) {
          const int s4 = ring<G::RF(0)>(r, base), s3 = ring<G::RF(2)>(r, base);
          st4s(sF + ((G::OF(0) + s4) * XW + tx) * 4, fcar[0]);
          st4s(sF + ((G::OF(1) + s4) * XW + tx) * 4, fcar[1]);
          st4s(sF + ((G::OF(2) + s3) * XW + tx) * 4, fcar[2]);
          st4s(sF + ((G::OF(3) + s4) * XW + tx) * 4, fcar[3]);
        }
      }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int k = 0; k < 4; ++k) fcar[i][k] = fnew[i][k];

    if constexpr (LOOK) {
      __syncthreads();
      s4(F);
    }
  }
  }  // segments

  if constexpr (LOOK) {
    if (bad) atomicOr(&sc->err, ERR_NONPHYSICAL);
    block_max_store<M, XW * RR>(vmax, part + (long long)slot_n * p.max_parts * kNV, blockIdx.x, gridDim.x,
                                &sc->nparts[slot_n]);
  }
}

// Strip shapes: XW columns per row (TXO = XW - 2H of them outputs), RR rows per iteration.
// FP32 storage: 160 x 2 threads (rings of 3-4 rows, 69 KB, three CTAs per SM); measured on a B300
// at 4096^2 the look-ahead step kernel takes 0.459 ms this way against 0.480 ms with 128 x 2 (four
// CTAs per SM), 0.479 with 96 x 2 (five) and 0.503-0.519 with 192, 224 or 256 x 2 (two); with
// 128 x 4 the two-pass step kernel took 0.46 against 0.42 ms with 128 x 2.  KEEP (a non-ideal gas,
// whose FP64 equation of state bounds the kernel) keeps 128 x 2 and four CTAs per SM: 7,417 against
// 7,155 MLUPS on the 2048^2 van der Waals interface.
// FP64: 128 x 2 threads, two CTAs per SM (4.90 ms per two-pass step kernel at 4096^2 against
// 5.26 ms with one CTA of 128 x 4, whose FP64 pipe idled while all its warps were in S1).
template <class S, bool LOOK, bool KEEP = false>
struct RollCfg {
  static constexpr int XW = sizeof(S) == 4 && !KEEP ? 160 : 128, RR = 2;
};

constexpr int kMaxDevices = 64;
int g_grid[kMaxDevices][16];  // persistent grid size per device and configuration (0: not set)

template <class S, bool LOOK, bool INFLOW, bool KEEP>
constexpr int cfg_index() {
  return (sizeof(S) == 8 ? 0 : 2) + (LOOK ? 1 : 0) + (INFLOW ? 4 : 0) + (KEEP ? 8 : 0);
}

template <class S, bool LOOK, bool INFLOW, bool KEEP = false>
cudaError_t launch_roll_t(const Launch& L_, const void* fin, void* fout, int pulled, const void* invM) {
  using C = RollCfg<S, LOOK, KEEP>;
  using G = RollGeom<S, LOOK, C::XW, C::RR>;
  const KParams& p = *L_.p;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const int grid = (dev >= 0 && dev < kMaxDevices) ? g_grid[dev][cfg_index<S, LOOK, INFLOW, KEEP>()] : 0;
  if (grid <= 0) return cudaErrorInitializationError;  // prepare_roll_kernels() not run on this device
  k_roll<S, LOOK, C::XW, C::RR, INFLOW, KEEP><<<grid, G::NT, G::smem_bytes, L_.stream>>>(
      (const S*)fin, (S*)fout, L_.sc, p, pulled, (const typename Store<S>::M*)invM, L_.part,
      (!LOOK && sizeof(S) == 8) ? L_.fields : nullptr, (!LOOK && sizeof(S) == 8) ? L_.sens : nullptr,
      KEEP ? L_.pkeep : nullptr);
  return cudaGetLastError();
}

// Opt-in shared memory, and the persistent grid: SMs x resident CTAs per SM.
template <class S, bool LOOK, bool INFLOW, bool KEEP>
cudaError_t prepare_roll_t(int dev, int sms) {
  using C = RollCfg<S, LOOK, KEEP>;
  using G = RollGeom<S, LOOK, C::XW, C::RR>;
  cudaError_t e = cudaFuncSetAttribute(k_roll<S, LOOK, C::XW, C::RR, INFLOW, KEEP>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)G::smem_bytes);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_roll<S, LOOK, C::XW, C::RR, INFLOW, KEEP>, G::NT,
                                                    G::smem_bytes);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  g_grid[dev][cfg_index<S, LOOK, INFLOW, KEEP>()] = sms * per_sm;
  return cudaSuccess;
}

template <class S, bool LOOK>
cudaError_t prepare_roll_pair(int dev, int sms) {
  cudaError_t e = prepare_roll_t<S, LOOK, false, false>(dev, sms);
  if (e == cudaSuccess) e = prepare_roll_t<S, LOOK, true, false>(dev, sms);
  if constexpr (sizeof(S) == 4 && LOOK) {
    if (e == cudaSuccess) e = prepare_roll_t<S, LOOK, false, true>(dev, sms);
    if (e == cudaSuccess) e = prepare_roll_t<S, LOOK, true, true>(dev, sms);
  }
  return e;
}

}  // namespace

cudaError_t prepare_roll_kernels() {
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  e = prepare_roll_pair<double, false>(dev, sms);
  if (e == cudaSuccess) e = prepare_roll_pair<double, true>(dev, sms);
  if (e == cudaSuccess) e = prepare_roll_pair<float, false>(dev, sms);
  if (e == cudaSuccess) e = prepare_roll_pair<float, true>(dev, sms);
  return e;
}

// Upper bound of the CTAs a strip launch uses (partial-maxima capacity): every SM full of CTAs.
long long roll_ctas(const KParams& p) {
  if (p.dim != 2) return 0;
  int dev = 0, sms = 0, thr = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&thr, cudaDevAttrMaxThreadsPerMultiProcessor, dev) != cudaSuccess) {
    cudaGetLastError();
    return 4096;
  }
  // the smallest CTA of any strip configuration
  constexpr int nt32 = RollGeom<float, false, RollCfg<float, false>::XW, RollCfg<float, false>::RR>::NT;
  constexpr int nt64 = RollGeom<double, false, RollCfg<double, false>::XW, RollCfg<double, false>::RR>::NT;
  constexpr int nt = nt32 < nt64 ? nt32 : nt64;
  return (long long)sms * ((thr + nt - 1) / nt);
}

cudaError_t launch_roll(const Launch& L, int precision, bool lookahead, const void* fin, void* fout, int pulled) {
  const char* base = reinterpret_cast<const char*>(L.sc);
  const bool inflow = L.p->bc[0] == 2;
  if (precision == 0) {
    const void* invM = base + offsetof(Scalars, inv_M);
    if (inflow)
      return lookahead ? launch_roll_t<double, true, true>(L, fin, fout, pulled, invM)
                       : launch_roll_t<double, false, true>(L, fin, fout, pulled, invM);
    return lookahead ? launch_roll_t<double, true, false>(L, fin, fout, pulled, invM)
                     : launch_roll_t<double, false, false>(L, fin, fout, pulled, invM);
  }
  const void* invM = base + offsetof(Scalars, inv_M_f);
  if (lookahead && L.pkeep && L.p->eos_kind != 0)  // non-ideal gas: pressure kept between the stages
    return inflow ? launch_roll_t<float, true, true, true>(L, fin, fout, pulled, invM)
                  : launch_roll_t<float, true, false, true>(L, fin, fout, pulled, invM);
  if (inflow)
    return lookahead ? launch_roll_t<float, true, true>(L, fin, fout, pulled, invM)
                     : launch_roll_t<float, false, true>(L, fin, fout, pulled, invM);
  return lookahead ? launch_roll_t<float, true, false>(L, fin, fout, pulled, invM)
                   : launch_roll_t<float, false, false>(L, fin, fout, pulled, invM);
}

}  // namespace vlbm
