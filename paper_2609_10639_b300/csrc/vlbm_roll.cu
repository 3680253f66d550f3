// Column-marching form of the 2D step kernel (sm_103a).
//
// One CTA owns a strip of TXO output columns and L output rows and walks down it RR rows at a
// time.  Every quantity of the step is computed once per row of the strip and kept in
// shared-memory ring buffers for as long as the stencils below need it, so the only
// recomputation is the x-halo of the strip (H columns on each side) and H rows at each end of
// the strip, instead of a halo all around a small tile.  Per iteration (block start F):
//
//   S1  rows [F, F+RR):        pulled populations (Eq. 21), W, u, flux Q_alpha (Eqs. 10, 15-17)
//                              -> ring of Q and u (2 RR rows); the populations stay in registers
//   S2  rows [F-RR+1, F+1):    flux-divergence activity s (Eqs. 28-31) and Ducros ratio theta
//                              (Eqs. 32-33) -> ring of (s, theta) (RR + 2 rows)
//   S3  rows [F-RR, F):        box filters and beta (Eqs. 34-35), fused reprojection (Eqs. 38-40)
//                              and relaxation (Eqs. 20, 22) on the populations S1 loaded one
//                              iteration earlier (same thread), single write to HBM
//   S4  rows [F-RR-1, F-1):    (look-ahead) W^{n+1} = sum_i f*_i(x - sigma_i) from the ring of
//                              relaxed populations (RR + 2 rows), and the maxima of the next
//                              step (Eqs. 30, 36) accumulated in registers over the whole strip
//
// Boundary rules as in the tile kernel: positions and rows outside a zero-gradient side hold the
// edge cell's populations (S1 maps them), and every stencil read of s, theta (S3) and of the
// relaxed populations (S4) is taken at the edge cell there; periodic sides are unwrapped.
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
  static constexpr int RF = RR + 2;       // rows of the relaxed-population ring: [F-RR-2, F)
  static constexpr size_t nQ = (size_t)RQ * 2 * XW * 4;
  static constexpr size_t nU = (size_t)RQ * XW * 2;
  static constexpr size_t nS = (size_t)RS * XW * 2;
  static constexpr size_t nF = LOOK ? (size_t)RF * 4 * XW * 4 : 0;
  static constexpr size_t smem_bytes = (nQ + nU + nS + nF) * sizeof(M);
};

// Ring slot of row r (rows never lie more than 8 R below the strip's first row `base`).
template <int R>
__device__ __forceinline__ int ring(int r, int base) {
  return (r - base + 8 * R) % R;
}

template <class S, bool LOOK, int XW, int RR, int L>
__global__ void __launch_bounds__(XW * RR) k_roll(const S* __restrict__ fin, S* __restrict__ fout,
                                                  Scalars* __restrict__ sc, const KParams p, const int pulled,
                                                  const typename Store<S>::M* __restrict__ invM_src,
                                                  double* __restrict__ part) {
  using G = RollGeom<S, LOOK, XW, RR>;
  using M = typename G::M;
  constexpr int H = G::H, TXO = G::TXO, RQ = G::RQ, RS = G::RS, RF = G::RF;
  constexpr bool OFF = Store<S>::kOffset;
  if (!sc->active) return;

  extern __shared__ __align__(16) unsigned char smem_raw[];
  M* sQ = reinterpret_cast<M*>(smem_raw);  // [RQ][2][XW][4]
  M* sU = sQ + G::nQ;                      // [RQ][XW][2]
  M* sS = sU + G::nU;                      // [RS][XW][2]
  M* sF = sS + G::nS;                      // [RF][4][XW][4]  (look-ahead)

  const Coef<M>& co = coef<M>(p);
  const int tx = threadIdx.x % XW, ty = threadIdx.x / XW;
  const int x0 = blockIdx.x * TXO, y0 = blockIdx.y * L;
  const int xs = x0 - H;  // column of strip position 0
  const int px = xs + tx;
  const int xend = min(x0 + TXO, p.nx), yend = min(y0 + L, p.ny);
  const int base = y0 - H;
  // strip positions or their pull sources outside [0, nx): boundary rules needed in x
  const bool xedge = xs - 1 < 0 || xs + XW + 1 > p.nx;
  const bool zx = p.bc[0] == 1, zy = p.bc[2] == 1;  // zero-gradient in x / y (both sides alike)
  const bool x_in = px >= 0 && px < p.nx;

  // strip index of the value read at column px + d (the edge cell beyond a zero-gradient side)
  auto xi = [&](int d) -> int { return xedge ? centre_pos(px + d, p.nx, p.bc[0], p.bc[1]) - xs : tx + d; };
  auto yc = [&](int r) -> int { return centre_pos(r, p.ny, p.bc[2], p.bc[3]); };

  M wq[4], invM[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    wq[k] = StepScalars<M>::wq(sc, k);
    invM[k] = invM_src[k];
  }
  const M r_c = StepScalars<M>::r(sc), inv_c = StepScalars<M>::inv_c(sc);
  const int slot_n = (int)(sc->n & 1);

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

  for (int F = base; F - RR - (LOOK ? 1 : 0) < yend; F += RR) {
    // ---- S1: pulled populations, W, u, Q of rows [F, F+RR) ----
    M fnew[4][4];
    {
      const int r = F + ty;
      const bool act = r < yend + H && px >= x0 - H && px < xend + H;
      if (act) {
        const int cy = nb_index(r, p.ny, p.bc[2], p.bc[3]);
        const int cx = xedge ? nb_index(px, p.nx, p.bc[0], p.bc[1]) : px;
        const bool inner = !xedge && cy >= 1 && cy < p.ny - 1;
        load_cell<2, S>(fin, p, cx, cy, pulled, inner, fnew);
        M W[4], u[2], Qf[2][4], cs;
        moments<2, M, OFF>(fnew, wq, W);
        prim_flux<2, M, false>(p, W, u, Qf, cs);
        const int s = ring<RQ>(r, base);
#pragma unroll
        for (int a = 0; a < 2; ++a) st4s(sQ + ((s * 2 + a) * XW + tx) * 4, Qf[a]);
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
      const bool act = r >= y0 - H + 1 && r < yend + H - 1 && px >= x0 - H + 1 && px < xend + H - 1 &&
                       !(zy && (r < 0 || r >= p.ny)) && !(zx && !x_in) && p.beta_mode == 0;
      if (act) {
        const int sm = ring<RQ>(r - 1, base), s0 = ring<RQ>(r, base), sp = ring<RQ>(r + 1, base);
        M qxp[4], qxm[4], qyp[4], qym[4];
        ld4s(sQ + ((s0 * 2 + 0) * XW + tx + 1) * 4, qxp);
        ld4s(sQ + ((s0 * 2 + 0) * XW + tx - 1) * 4, qxm);
        ld4s(sQ + ((sp * 2 + 1) * XW + tx) * 4, qyp);
        ld4s(sQ + ((sm * 2 + 1) * XW + tx) * 4, qym);
        M acc = 0;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const M jk = (qxp[k] - qxm[k]) + (qyp[k] - qym[k]);
          const M sh = (M)0.5 * jk * invM[k];
          acc += sh * sh;
        }
        const M sval = sqrt_(acc * (M)0.25);
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
        const M dil = ((uxp - uxm) + (vyp - vym)) * co.inv2dx;
        const M vort = ((vxp - vxm) - (uyp - uym)) * co.inv2dx;
        const M th = div_(dil * dil, dil * dil + vort * vort + co.eps);
        const int ss = ring<RS>(r, base);
        if constexpr (sizeof(M) == 8) {
          reinterpret_cast<double2*>(sS)[ss * XW + tx] = make_double2((double)sval, (double)th);
        } else {
          reinterpret_cast<float2*>(sS)[ss * XW + tx] = make_float2((float)sval, (float)th);
        }
      }
    }
    __syncthreads();

    // ---- S3: beta, fused reprojection + relaxation of rows [F-RR, F), single write ----
    {
      const int r = F - RR + ty;
      const bool act = r >= y0 - H + 2 && r < yend + H - 2 && px >= x0 - H + 2 && px < xend + H - 2 &&
                       !(zy && (r < 0 || r >= p.ny)) && !(zx && !x_in);
      if (act) {
        M beta = co.beta_const;
        if (p.beta_mode == 0) {
          const int xm = xi(-1), xp = xi(1);
          const M q = (M)0.25, h = (M)0.5;
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
            rs[j] = q * a0 + h * a1 + q * a2;
            rt[j] = q * b0 + h * b1 + q * b2;
          }
          const M sbar = q * rs[0] + h * rs[1] + q * rs[2];
          const M tbar = q * rt[0] + h * rt[1] + q * rt[2];
          M chi = co.c_sensor * sbar * tbar;
          chi = chi <= (M)0 ? (M)0 : (chi >= (M)1 ? (M)1 : chi);
          beta = co.beta_max - co.dbeta * chi;
        }
        M Qc[2][4];
        const int sq = ring<RQ>(r, base);
        ld4s(sQ + ((sq * 2 + 0) * XW + tx) * 4, Qc[0]);
        ld4s(sQ + ((sq * 2 + 1) * XW + tx) * 4, Qc[1]);
        relax_cell<2, M>(fcar, Qc, beta, r_c, inv_c);
        if (r >= y0 && r < yend && px >= x0 && px < xend) store_cell<2, S, M>(fout, p, r * p.nx + px, fcar);
        if constexpr (LOOK) {
          const int sf = ring<RF>(r, base);
#pragma unroll
          for (int i = 0; i < 4; ++i) st4s(sF + ((sf * 4 + i) * XW + tx) * 4, fcar[i]);
        }
      }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int k = 0; k < 4; ++k) fcar[i][k] = fnew[i][k];

    // ---- S4: W^{n+1} of rows [F-RR-1, F-1) and the next step's maxima ----
    if constexpr (LOOK) {
      __syncthreads();
      const int r = F - RR - 1 + ty;
      if (r >= y0 && r < yend && px >= x0 && px < xend) {
        M fr[4][4], W[4];
        const int xm = xi(-1), xp = xi(1);
        const int sfy = ring<RF>(r, base);
        const int sfm = ring<RF>(yc(r - 1), base), sfp = ring<RF>(yc(r + 1), base);
        ld4s(sF + ((sfy * 4 + 0) * XW + xp) * 4, fr[0]);  // f*_{x-} from x+1
        ld4s(sF + ((sfy * 4 + 1) * XW + xm) * 4, fr[1]);  // f*_{x+} from x-1
        ld4s(sF + ((sfp * 4 + 2) * XW + tx) * 4, fr[2]);  // f*_{y-} from y+1
        ld4s(sF + ((sfm * 4 + 3) * XW + tx) * 4, fr[3]);  // f*_{y+} from y-1
        moments<2, M, OFF>(fr, wq, W);
        M u[2], Qf[2][4], cs;
        bad |= !prim_flux<2, M, true>(p, W, u, Qf, cs);
        cell_maxima<2, M>(u, cs, Qf, vmax);
      }
    }
  }

  if constexpr (LOOK) {
    if (bad) atomicOr(&sc->err, ERR_NONPHYSICAL);
    block_max_store<M, XW * RR>(vmax, part + (long long)slot_n * p.max_parts * kNV, blockIdx.y * gridDim.x + blockIdx.x,
                                gridDim.x * gridDim.y, &sc->nparts[slot_n]);
  }
}

// Strip shapes: XW columns per row (TXO = XW - 2H of them outputs), RR rows per iteration, L
// output rows per CTA.
template <class S, bool LOOK>
struct RollCfg {
  static constexpr int XW = 128, RR = 4, L = 128;
};

template <class S, bool LOOK>
cudaError_t launch_roll_t(const Launch& L_, const void* fin, void* fout, int pulled, const void* invM) {
  using C = RollCfg<S, LOOK>;
  using G = RollGeom<S, LOOK, C::XW, C::RR>;
  const KParams& p = *L_.p;
  dim3 grid((p.nx + G::TXO - 1) / G::TXO, (p.ny + C::L - 1) / C::L);
  k_roll<S, LOOK, C::XW, C::RR, C::L><<<grid, G::NT, G::smem_bytes, L_.stream>>>(
      (const S*)fin, (S*)fout, L_.sc, p, pulled, (const typename Store<S>::M*)invM, L_.part);
  return cudaGetLastError();
}

template <class S, bool LOOK>
cudaError_t prepare_roll_t() {
  using C = RollCfg<S, LOOK>;
  using G = RollGeom<S, LOOK, C::XW, C::RR>;
  return cudaFuncSetAttribute(k_roll<S, LOOK, C::XW, C::RR, C::L>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)G::smem_bytes);
}

}  // namespace

cudaError_t prepare_roll_kernels() {
  cudaError_t e = prepare_roll_t<double, false>();
  if (e == cudaSuccess) e = prepare_roll_t<double, true>();
  if (e == cudaSuccess) e = prepare_roll_t<float, false>();
  if (e == cudaSuccess) e = prepare_roll_t<float, true>();
  return e;
}

long long roll_ctas(const KParams& p) {
  if (p.dim != 2) return 0;
  long long m = 0;
  auto upd = [&](int txo, int l) {
    const long long c = (long long)((p.nx + txo - 1) / txo) * ((p.ny + l - 1) / l);
    if (c > m) m = c;
  };
  upd(RollGeom<double, false, RollCfg<double, false>::XW, RollCfg<double, false>::RR>::TXO, RollCfg<double, false>::L);
  upd(RollGeom<double, true, RollCfg<double, true>::XW, RollCfg<double, true>::RR>::TXO, RollCfg<double, true>::L);
  upd(RollGeom<float, false, RollCfg<float, false>::XW, RollCfg<float, false>::RR>::TXO, RollCfg<float, false>::L);
  upd(RollGeom<float, true, RollCfg<float, true>::XW, RollCfg<float, true>::RR>::TXO, RollCfg<float, true>::L);
  return m;
}

cudaError_t launch_roll(const Launch& L, int precision, bool lookahead, const void* fin, void* fout, int pulled) {
  const char* base = reinterpret_cast<const char*>(L.sc);
  if (precision == 0) {
    const void* invM = base + offsetof(Scalars, inv_M);
    return lookahead ? launch_roll_t<double, true>(L, fin, fout, pulled, invM)
                     : launch_roll_t<double, false>(L, fin, fout, pulled, invM);
  }
  const void* invM = base + offsetof(Scalars, inv_M_f);
  return lookahead ? launch_roll_t<float, true>(L, fin, fout, pulled, invM)
                   : launch_roll_t<float, false>(L, fin, fout, pulled, invM);
}

}  // namespace vlbm
