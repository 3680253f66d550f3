// C interface of the VLBM step library (declared in include/vlbm.h).
//
// Each handle owns two population buffers, a device-resident scalar block, the (dt, c) history
// and scratch.  vlbm_step issues the step kernels in chunks captured once as CUDA graphs (one
// graph per buffer parity), launched on the caller's stream; the device decides the link speed
// and time step, so the host synchronises only once at the end of the call (or once per chunk
// when an end time is given and the number of steps is not known in advance).
#include "vlbm.h"
#include "vlbm_adjoint.cuh"
#include "vlbm_internal.cuh"

#include <cmath>
#include <cstddef>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

using vlbm::KParams;
using vlbm::Scalars;

struct vlbm_s {
  int device = 0;
  cudaStream_t stream = nullptr;      // caller's stream
  cudaStream_t cap_stream = nullptr;  // private stream used only to capture graphs
  KParams p{};
  int precision = 0;
  bool lookahead = false;
  size_t elem = 8;  // bytes per stored population value
  void* buf[2] = {nullptr, nullptr};
  Scalars* sc = nullptr;       // device
  Scalars* sc_host = nullptr;  // pinned mirror for readback
  double* hist_dt = nullptr;
  double* hist_c = nullptr;
  long long hist_cap = 0;
  double* sched = nullptr;
  long long sched_len = 0;
  double* partial = nullptr;  // compensated-sum partials (FP32 reference)
  int nblk_sum = 0;
  double* part = nullptr;     // per-CTA partial maxima, [2][max_parts][5]
  double* scratch = nullptr;  // (D+2) * plane doubles + plane + 8 (beta + 1/M)
  size_t scratch_elems = 0;
  double* fscratch = nullptr;  // populations readback (lazily allocated)
  double* fields = nullptr;    // FP64 strips: W, u, Q kept from the maxima pass (14 planes)
  float* pkeep = nullptr;      // FP32 storage, look-ahead strips, non-ideal gas: kept pressure [2][plane]
  bool initialised = false;
  bool inflow_set = false;     // pinned-inflow grids: vlbm_set_inflow has supplied W_in
  bool unpulled = true;        // the current buffer holds equilibrium populations in place
  bool last_step_pulled = true;
  long long n_host = 0;        // steps completed, as of the last synchronisation
  static constexpr int kChunk = 32;
  // Graph chunks of kChunk steps: graph[0], graph[1] start on buffer 0 / 1; graph[2] is the first
  // chunk after vlbm_init (its first step reads the equilibrium populations in place).  pgraph:
  // the same chunks with an event-record node before and after every step-kernel launch
  // (profiling), whose events are gev[which][2j], gev[which][2j + 1] for step j of the chunk.
  cudaGraphExec_t graph[3] = {nullptr, nullptr, nullptr};
  cudaGraphExec_t pgraph[3] = {nullptr, nullptr, nullptr};
  cudaEvent_t gev[3][2 * kChunk] = {};
  int gev_pending = -1;       // event set of the last profiled chunk launch, not yet read
  double prof_ms = 0.0;       // summed step-kernel time of the profiled chunks read so far
  long long prof_n = 0;       // their step-kernel launches
  cudaEvent_t ev0 = nullptr, ev1 = nullptr, ev2 = nullptr;
  // adjoint workspace (allocated on first use, grown when needed)
  struct Adj {
    double* ckpt = nullptr;   // checkpoint states
    size_t ckpt_states = 0;
    double* seg = nullptr;    // recomputed states of one segment
    size_t seg_states = 0;
    double* kept = nullptr;   // FP64 strips: W, u, Q and sensor quantities of each recomputed state
    size_t kept_cap = 0;
    double* lam[2] = {nullptr, nullptr};
    double* F = nullptr;      // workspace fields
    double* pv = nullptr;
    long long* pi = nullptr;
    double* part = nullptr;
    double* gpart = nullptr;  // first stage of the folds of the per-CTA partials
    long long* gidx = nullptr;
    double* sched = nullptr;  // [c0, c_0, ..., c_{N-1}]
    size_t sched_cap = 0;
    double* dJ = nullptr;     // device copy of dJ/dW(T)
    double* dW0 = nullptr;    // device copy of W0 / result
    vlbm::AdjScalars* as = nullptr;
    vlbm::AdjScalars* as_host = nullptr;
    Scalars* sc_backup = nullptr;
    double fwd_ms = 0.0, rev_ms = 0.0, recompute_ms = 0.0;
    // tape: the last segments' states (and, FP64 strips, their W, u, Q and sensor quantities)
    // kept by the forward pass, so that the reverse pass does not recompute those segments
    double* tape = nullptr;
    size_t tape_cap = 0;          // doubles
    long long tape_limit = -1;    // bytes; < 0: 3/4 of the free device memory; 0: no tape
    long long taped_steps = 0;    // of the last call
    size_t tape_used = 0;         // bytes of the last call
  } adj;
  // vlbm_run_batch: device staging of host inputs and outputs ([4][nc * plane]: in 0, in 1,
  // out 0, out 1; allocated on first use), one stream per copy direction, and the events that
  // order the copies against the handle's stream: in_ready[2], in_free[2], out_ready[2], out_free[2]
  double* bstage = nullptr;
  cudaStream_t h2d = nullptr, d2h = nullptr;
  cudaEvent_t bev[8] = {};
  bool profile = false;            // bracket step-kernel launches with events
  std::vector<cudaEvent_t> pev;    // event pool, used in pairs
  size_t pev_used = 0;
};

namespace {

vlbm::Launch launch_of(vlbm_t h, cudaStream_t s) {
  vlbm::Launch L;
  L.p = &h->p;
  L.sc = h->sc;
  L.part = h->part;
  L.stream = s;
  L.hist_dt = h->hist_dt;
  L.hist_c = h->hist_c;
  L.sched = h->sched;
  L.fields = h->fields;
  L.pkeep = h->pkeep;
  return L;
}

vlbm_status cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return VLBM_OK;
  if (e == cudaErrorMemoryAllocation) return VLBM_E_NOMEM;
  return VLBM_E_CUDA;
}

#define VLBM_TRY(expr)                      \
  do {                                      \
    cudaError_t _e = (expr);                \
    if (_e != cudaSuccess) return cuda_status(_e); \
  } while (0)

bool is_device_ptr(const void* ptr) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

void destroy_graphs(vlbm_t h) {
  for (int j = 0; j < 3; ++j) {
    if (h->graph[j]) {
      cudaGraphExecDestroy(h->graph[j]);
      h->graph[j] = nullptr;
    }
    if (h->pgraph[j]) {
      cudaGraphExecDestroy(h->pgraph[j]);
      h->pgraph[j] = nullptr;
    }
  }
}

// Next pair of profiling events (grows the pool).
cudaError_t profile_pair(vlbm_t h, cudaEvent_t* a, cudaEvent_t* b) {
  while (h->pev.size() < h->pev_used + 2) {
    cudaEvent_t e;
    cudaError_t r = cudaEventCreate(&e);
    if (r != cudaSuccess) return r;
    h->pev.push_back(e);
  }
  *a = h->pev[h->pev_used];
  *b = h->pev[h->pev_used + 1];
  h->pev_used += 2;
  return cudaSuccess;
}

// Issues one step (reading buffer `par`) on stream s.  With events ea, eb the step-kernel launch
// is bracketed by them (recorded as event-record nodes when s is being captured).
cudaError_t issue_step(vlbm_t h, cudaStream_t s, int par, int pulled, cudaEvent_t ea = nullptr,
                       cudaEvent_t eb = nullptr, bool capturing = false) {
  vlbm::Launch L = launch_of(h, s);
  const void* fin = h->buf[par];
  void* fout = h->buf[par ^ 1];
  cudaError_t e;
  if (!h->lookahead) {
    e = vlbm::launch_reduce(L, h->precision, fin, pulled, true);
    if (e != cudaSuccess) return e;
  }
  e = vlbm::launch_dt(L);
  if (e != cudaSuccess) return e;
  const unsigned flags = capturing ? cudaEventRecordExternal : cudaEventRecordDefault;
  if (ea) {
    e = cudaEventRecordWithFlags(ea, s, flags);
    if (e != cudaSuccess) return e;
  }
  e = vlbm::launch_step(L, h->precision, h->lookahead, fin, fout, pulled);
  if (e != cudaSuccess || !eb) return e;
  return cudaEventRecordWithFlags(eb, s, flags);
}

// One step issued on its own (outside a graph chunk), bracketed by a pool event pair when
// profiling.
cudaError_t issue_single(vlbm_t h, int par, int pulled) {
  cudaEvent_t ea = nullptr, eb = nullptr;
  if (h->profile) {
    cudaError_t e = profile_pair(h, &ea, &eb);
    if (e != cudaSuccess) return e;
  }
  return issue_step(h, h->stream, par, pulled, ea, eb, false);
}

// Captures graph chunk `which` (0, 1: kChunk pulled steps starting on buffer 0 / 1; 2: the first
// chunk after vlbm_init, starting on buffer 0 with the in-place step), with event-record nodes
// around the step kernels when `prof`.
cudaError_t build_graph(vlbm_t h, int which, bool prof) {
  if (prof)
    for (int j = 0; j < 2 * vlbm_s::kChunk; ++j)
      if (!h->gev[which][j]) {
        cudaError_t e = cudaEventCreate(&h->gev[which][j]);
        if (e != cudaSuccess) return e;
      }
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return e;
  cudaError_t le = cudaSuccess;
  for (int j = 0; j < vlbm_s::kChunk && le == cudaSuccess; ++j) {
    const int par = which == 2 ? (j & 1) : which ^ (j & 1);
    const int pulled = (which == 2 && j == 0) ? 0 : 1;
    cudaEvent_t ea = prof ? h->gev[which][2 * j] : nullptr, eb = prof ? h->gev[which][2 * j + 1] : nullptr;
    le = issue_step(h, h->cap_stream, par, pulled, ea, eb, true);
  }
  e = cudaStreamEndCapture(h->cap_stream, &g);
  if (le != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return le;
  }
  if (e != cudaSuccess) return e;
  e = cudaGraphInstantiate(prof ? &h->pgraph[which] : &h->graph[which], g, 0);
  cudaGraphDestroy(g);
  return e;
}

// Reads the step-kernel times of the last profiled chunk (the stream must have drained).
cudaError_t harvest_chunk_events(vlbm_t h) {
  if (h->gev_pending < 0) return cudaSuccess;
  const int w = h->gev_pending;
  h->gev_pending = -1;
  for (int j = 0; j < vlbm_s::kChunk; ++j) {
    float ms = 0.f;
    cudaError_t e = cudaEventElapsedTime(&ms, h->gev[w][2 * j], h->gev[w][2 * j + 1]);
    if (e != cudaSuccess) return e;
    h->prof_ms += ms;
  }
  h->prof_n += vlbm_s::kChunk;
  return cudaSuccess;
}

// Launches graph chunk `which` on the caller's stream (captured on first use).  When profiling,
// a chunk whose events have not been read yet is read first (one host synchronisation; a
// vlbm_step call of at most one chunk never needs it, its events are read at the call's end).
cudaError_t launch_chunk(vlbm_t h, int which) {
  if (h->profile) {
    if (h->gev_pending >= 0) {
      cudaError_t e = cudaStreamSynchronize(h->stream);
      if (e == cudaSuccess) e = harvest_chunk_events(h);
      if (e != cudaSuccess) return e;
    }
    if (!h->pgraph[which]) {
      cudaError_t e = build_graph(h, which, true);
      if (e != cudaSuccess) return e;
    }
    cudaError_t e = cudaGraphLaunch(h->pgraph[which], h->stream);
    if (e == cudaSuccess) h->gev_pending = which;
    return e;
  }
  if (!h->graph[which]) {
    cudaError_t e = build_graph(h, which, false);
    if (e != cudaSuccess) return e;
  }
  return cudaGraphLaunch(h->graph[which], h->stream);
}

// Grows the history arrays to hold at least `need` steps (keeps the recorded part).
vlbm_status ensure_history(vlbm_t h, long long need) {
  if (need <= h->hist_cap) return VLBM_OK;
  long long cap = h->hist_cap > 0 ? h->hist_cap : 4096;
  while (cap < need) cap *= 2;
  double *ndt = nullptr, *nc = nullptr;
  if (cudaMalloc(&ndt, cap * sizeof(double)) != cudaSuccess) return VLBM_E_NOMEM;
  if (cudaMalloc(&nc, cap * sizeof(double)) != cudaSuccess) {
    cudaFree(ndt);
    return VLBM_E_NOMEM;
  }
  if (h->hist_cap > 0) {
    VLBM_TRY(cudaMemcpyAsync(ndt, h->hist_dt, h->hist_cap * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
    VLBM_TRY(cudaMemcpyAsync(nc, h->hist_c, h->hist_cap * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
  }
  VLBM_TRY(cudaStreamSynchronize(h->stream));
  cudaFree(h->hist_dt);
  cudaFree(h->hist_c);
  h->hist_dt = ndt;
  h->hist_c = nc;
  h->hist_cap = cap;
  h->sc_host->hist_cap = cap;
  VLBM_TRY(cudaMemcpyAsync(&h->sc->hist_cap, &cap, sizeof(long long), cudaMemcpyHostToDevice, h->stream));
  VLBM_TRY(cudaStreamSynchronize(h->stream));
  destroy_graphs(h);  // the graphs captured the old history pointers
  return VLBM_OK;
}

// Copies the device scalars to the pinned mirror and waits.
vlbm_status sync_scalars(vlbm_t h) {
  VLBM_TRY(cudaMemcpyAsync(h->sc_host, h->sc, sizeof(Scalars), cudaMemcpyDeviceToHost, h->stream));
  VLBM_TRY(cudaStreamSynchronize(h->stream));
  h->n_host = h->sc_host->n;
  if (h->sc_host->err & vlbm::ERR_SCHEDULE) return VLBM_E_INVAL;
  if (h->sc_host->err) return VLBM_E_NONPHYSICAL;
  return VLBM_OK;
}

bool valid_params(const vlbm_params* q) {
  if (!(q->cfl > 0.0 && q->cfl < 1.0)) return false;
  if (q->retarget_every < 1) return false;
  if (q->precision != VLBM_FP64 && q->precision != VLBM_FP32_STORE) return false;
  if (q->algorithm < VLBM_ALGO_AUTO || q->algorithm > VLBM_ALGO_LOOKAHEAD) return false;
  if (q->tiling < VLBM_TILING_AUTO || q->tiling > VLBM_TILING_STRIP) return false;
  return true;
}

}  // namespace

namespace vlbm {

bool valid_problem(const vlbm_grid* grid, const vlbm_eos* eos, const vlbm_params* q) {
  if (grid->dim != 1 && grid->dim != 2) return false;
  const long long nx = grid->nx, ny = grid->dim == 1 ? 1 : grid->ny;
  if (nx < 1 || ny < 1) return false;
  if (!(grid->x1 > grid->x0)) return false;
  for (int j = 0; j < 4; ++j)
    if (grid->bc[j] != VLBM_BC_PERIODIC && grid->bc[j] != VLBM_BC_ZEROGRAD && !(j == 0 && grid->bc[j] == VLBM_BC_INFLOW))
      return false;
  // a pinned-inflow x-lo side pairs with a zero-gradient (outflow) x-hi side
  if (grid->bc[0] == VLBM_BC_INFLOW && grid->bc[1] != VLBM_BC_ZEROGRAD) return false;
  if ((grid->bc[0] == VLBM_BC_PERIODIC) != (grid->bc[1] == VLBM_BC_PERIODIC)) return false;
  if (grid->dim == 2 && (grid->bc[2] == VLBM_BC_PERIODIC) != (grid->bc[3] == VLBM_BC_PERIODIC)) return false;
  if (eos->kind == VLBM_EOS_IDEAL) {
    if (!(eos->gamma > 1.0)) return false;
  } else if (eos->kind == VLBM_EOS_VDW || eos->kind == VLBM_EOS_VDW_CVT) {
    if (!(eos->a >= 0.0 && eos->b >= 0.0 && eos->R > 0.0 && eos->cv > 0.0)) return false;
    if (eos->kind == VLBM_EOS_VDW_CVT && !(eos->cv1 >= 0.0 && eos->cv2 >= 0.0)) return false;
  } else {
    return false;
  }
  if (q->beta_mode != VLBM_BETA_SENSOR && q->beta_mode != VLBM_BETA_CONST) return false;
  if (q->beta_mode == VLBM_BETA_CONST && !(q->beta_const > 0.0 && q->beta_const <= 1.0)) return false;
  if (q->beta_mode == VLBM_BETA_SENSOR) {
    if (!(q->beta_min > 0.0 && q->beta_min <= q->beta_max && q->beta_max <= 1.0)) return false;
    if (!(q->c_sensor >= 0.0) || !(q->ducros_eps > 0.0)) return false;
  }
  return true;
}

void make_kparams(const vlbm_grid* grid, const vlbm_eos* eos, const vlbm_params* params, KParams& p) {
  const long long nx = grid->nx, ny = grid->dim == 1 ? 1 : grid->ny;
  p.dim = grid->dim;
  p.nc = grid->dim + 2;
  p.q = 2 * grid->dim;
  p.nx = (int)nx;
  p.ny = (int)ny;
  p.plane = nx * ny;
  for (int j = 0; j < 4; ++j) p.bc[j] = grid->bc[j];
  if (grid->dim == 1) p.bc[2] = p.bc[3] = VLBM_BC_ZEROGRAD;
  p.dx = (grid->x1 - grid->x0) / (double)nx;
  p.inv2dx = 1.0 / (2.0 * p.dx);
  p.eos_kind = eos->kind;
  p.gamma = eos->kind == VLBM_EOS_IDEAL ? eos->gamma : 1.0 + eos->R / eos->cv;
  p.a = eos->a;
  p.b = eos->b;
  p.R = eos->R;
  p.cv = eos->cv;
  p.inv_cv = eos->kind != VLBM_EOS_IDEAL ? 1.0 / eos->cv : 0.0;
  p.cfl = params->cfl;
  p.beta_mode = params->beta_mode;
  p.beta_const = params->beta_const;
  p.beta_min = params->beta_min;
  p.beta_max = params->beta_max;
  p.c_sensor = params->c_sensor;
  p.ducros_eps = params->ducros_eps;
  p.retarget_every = params->retarget_every;
  // Column strips in 2D (each quantity computed once per row).  Measured on a B300 (per step):
  // FP64 strips beat tiles on every grid tried (4096^2: 6.7 vs 8.9 ms; 800 x 300: 148 vs 200 us); in
  // FP32 storage strips win on large grids (1024^2: 51 vs 63 us) and tiles on small ones with an
  // ideal gas, where a strip segment is only a few rows long and its halo rows weigh (800 x 300:
  // 25 vs 33 us, 512^2: 22 vs 28 us); with a non-ideal gas the strips keep the pressure between the
  // stages and win (1200 x 450: 113 vs 153 us).
  const long long cells = (long long)grid->nx * (grid->dim == 1 ? 1 : grid->ny);
  const bool small_fp32_ideal = params->precision == VLBM_FP32_STORE && eos->kind == VLBM_EOS_IDEAL && cells < (1LL << 19);
  p.strip = (grid->dim == 2 && (params->tiling == VLBM_TILING_STRIP ||
                                (params->tiling == VLBM_TILING_AUTO && !small_fp32_ideal))) ? 1 : 0;
  Coef<double>& c = p.cd;
  c.gamma = p.gamma;
  c.gm1 = p.gamma - 1.0;
  c.ggm1 = p.gamma * (p.gamma - 1.0);
  c.a = p.a;
  c.b = p.b;
  c.R = p.R;
  c.inv_cv = p.inv_cv;
  c.a_inv_cv = p.a * p.inv_cv;
  c.c_sensor = p.c_sensor;
  c.beta_max = p.beta_max;
  c.dbeta = p.beta_max - p.beta_min;
  c.beta_const = p.beta_const;
  c.eps_lat = p.ducros_eps * (2.0 * p.dx) * (2.0 * p.dx);
  c.c_chi2 = p.c_sensor / 512.0;
  c.c_chi1 = p.c_sensor / (4.0 * std::sqrt(3.0));
  const bool cvt = eos->kind == VLBM_EOS_VDW_CVT;
  c.cv0 = eos->kind != VLBM_EOS_IDEAL ? eos->cv : 0.0;
  c.cv1 = cvt ? eos->cv1 : 0.0;
  c.cv2 = cvt ? eos->cv2 : 0.0;
  c.cv1h = c.cv1 / 2.0;
  c.cv2t = c.cv2 / 3.0;
  Coef<float>& f = p.cf;
  f.gamma = (float)c.gamma;
  f.gm1 = (float)c.gm1;
  f.ggm1 = (float)c.ggm1;
  f.a = (float)c.a;
  f.b = (float)c.b;
  f.R = (float)c.R;
  f.inv_cv = (float)c.inv_cv;
  f.a_inv_cv = (float)c.a_inv_cv;
  f.c_sensor = (float)c.c_sensor;
  f.beta_max = (float)c.beta_max;
  f.dbeta = (float)c.dbeta;
  f.beta_const = (float)c.beta_const;
  f.eps_lat = (float)c.eps_lat;
  f.c_chi2 = (float)c.c_chi2;
  f.c_chi1 = (float)c.c_chi1;
  f.cv0 = (float)c.cv0;
  f.cv1 = (float)c.cv1;
  f.cv2 = (float)c.cv2;
  f.cv1h = (float)c.cv1h;
  f.cv2t = (float)c.cv2t;
}

}  // namespace vlbm

extern "C" {

const char* vlbm_status_string(vlbm_status s) {
  switch (s) {
    case VLBM_OK: return "ok";
    case VLBM_E_INVAL: return "invalid argument";
    case VLBM_E_NOMEM: return "out of memory";
    case VLBM_E_CUDA: return "CUDA error";
    case VLBM_E_NONPHYSICAL: return "non-physical state (rho <= 0, c_s^2 <= 0 or non-finite)";
    case VLBM_E_TIMEOUT: return "timeout";
    case VLBM_E_STATE: return "call out of order";
    case VLBM_E_CHECKSUM: return "checksum mismatch";
    case VLBM_E_UNSUPPORTED: return "unsupported combination";
  }
  return "unknown status";
}

const char* vlbm_version(void) { return "vlbm-b300 0.1 (sm_103a)"; }

vlbm_status vlbm_create(const vlbm_grid* grid, const vlbm_eos* eos, const vlbm_params* params, void* cuda_stream,
                        vlbm_t* out) {
  if (out) *out = nullptr;
  if (!grid || !eos || !params || !out) return VLBM_E_INVAL;
  if (!vlbm::valid_problem(grid, eos, params) || !valid_params(params)) return VLBM_E_INVAL;
  const long long nx = grid->nx, ny = grid->dim == 1 ? 1 : grid->ny;
  // 32-bit population offsets: 2D * 4 * nx * ny values per buffer must stay below 2^31
  const long long nvals = 2LL * grid->dim * 4;
  if (nx > 2147483647LL || ny > 2147483647LL || nx * ny > 2147483647LL / nvals) return VLBM_E_INVAL;

  vlbm_s* h = new (std::nothrow) vlbm_s();
  if (!h) return VLBM_E_NOMEM;
  cudaGetDevice(&h->device);
  h->stream = (cudaStream_t)cuda_stream;
  KParams& p = h->p;
  vlbm::make_kparams(grid, eos, params, p);
  p.max_parts = vlbm::max_partials(p);
  h->precision = params->precision;
  h->elem = params->precision == VLBM_FP64 ? 8 : 4;
  // Look-ahead (one pass over HBM per step) for FP32 storage, which is bandwidth-bound: 0.59 vs
  // 0.64 ms per step with strips at 4096^2.  Two-pass for FP64, which is bound by the FP64 pipe:
  // the look-ahead's second reduction inside the step kernel costs more there than the separate
  // reduction pass (8.2 vs 8.0 ms).
  h->lookahead = params->algorithm == VLBM_ALGO_LOOKAHEAD ||
                 (params->algorithm == VLBM_ALGO_AUTO && params->precision == VLBM_FP32_STORE);

  vlbm_status st = VLBM_OK;
  const size_t fbytes = (size_t)p.q * 4 * p.plane * h->elem;  // layout [i][y][x][4]
  h->scratch_elems = (size_t)p.nc * p.plane + p.plane + 8;
  h->nblk_sum = vlbm::sum_blocks(p);
  if (cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreate(&h->ev0) != cudaSuccess || cudaEventCreate(&h->ev1) != cudaSuccess ||
      cudaEventCreate(&h->ev2) != cudaSuccess) {
    st = VLBM_E_CUDA;
  } else if (cudaMalloc(&h->buf[0], fbytes) != cudaSuccess || cudaMalloc(&h->buf[1], fbytes) != cudaSuccess ||
             cudaMalloc(&h->sc, sizeof(Scalars)) != cudaSuccess ||
             cudaMallocHost(&h->sc_host, sizeof(Scalars)) != cudaSuccess ||
             cudaMalloc(&h->scratch, h->scratch_elems * sizeof(double)) != cudaSuccess ||
             cudaMalloc(&h->partial, (size_t)h->nblk_sum * 4 * sizeof(double)) != cudaSuccess ||
             cudaMalloc(&h->part, (size_t)2 * p.max_parts * vlbm::kNV * sizeof(double)) != cudaSuccess) {
    st = VLBM_E_NOMEM;
  } else if (p.strip && h->precision == VLBM_FP64 &&
             cudaMalloc(&h->fields, (size_t)14 * p.plane * sizeof(double)) != cudaSuccess) {
    st = VLBM_E_NOMEM;
  } else if (p.strip && h->precision == VLBM_FP32_STORE && h->lookahead && p.eos_kind != VLBM_EOS_IDEAL &&
             cudaMalloc(&h->pkeep, (size_t)2 * p.plane * sizeof(float)) != cudaSuccess) {
    st = VLBM_E_NOMEM;
  } else if (vlbm::prepare_kernels() != cudaSuccess) {
    st = VLBM_E_CUDA;
  }
  if (st == VLBM_OK) {
    std::memset(h->sc_host, 0, sizeof(Scalars));
    if (cudaMemsetAsync(h->sc, 0, sizeof(Scalars), h->stream) != cudaSuccess ||
        cudaStreamSynchronize(h->stream) != cudaSuccess)
      st = VLBM_E_CUDA;
  }
  if (st == VLBM_OK) st = ensure_history(h, 4096);
  if (st != VLBM_OK) {
    cudaGetLastError();
    vlbm_destroy(h);
    return st;
  }
  *out = h;
  return VLBM_OK;
}

vlbm_status vlbm_destroy(vlbm_t h) {
  if (!h) return VLBM_OK;
  if (h->stream || h->cap_stream) cudaStreamSynchronize(h->stream);
  if (h->h2d) cudaStreamSynchronize(h->h2d);
  if (h->d2h) cudaStreamSynchronize(h->d2h);
  destroy_graphs(h);
  cudaFree(h->buf[0]);
  cudaFree(h->buf[1]);
  cudaFree(h->sc);
  if (h->sc_host) cudaFreeHost(h->sc_host);
  cudaFree(h->hist_dt);
  cudaFree(h->hist_c);
  cudaFree(h->sched);
  cudaFree(h->partial);
  cudaFree(h->part);
  cudaFree(h->scratch);
  cudaFree(h->fscratch);
  cudaFree(h->fields);
  cudaFree(h->pkeep);
  cudaFree(h->adj.ckpt);
  cudaFree(h->adj.seg);
  cudaFree(h->adj.kept);
  cudaFree(h->adj.lam[0]);
  cudaFree(h->adj.lam[1]);
  cudaFree(h->adj.F);
  cudaFree(h->adj.pv);
  cudaFree(h->adj.pi);
  cudaFree(h->adj.part);
  cudaFree(h->adj.gpart);
  cudaFree(h->adj.gidx);
  cudaFree(h->adj.sched);
  cudaFree(h->adj.dJ);
  cudaFree(h->adj.dW0);
  cudaFree(h->adj.tape);
  cudaFree(h->adj.as);
  cudaFree(h->adj.sc_backup);
  if (h->adj.as_host) cudaFreeHost(h->adj.as_host);
  for (cudaEvent_t e : h->pev) cudaEventDestroy(e);
  for (auto& set : h->gev)
    for (cudaEvent_t e : set)
      if (e) cudaEventDestroy(e);
  if (h->ev0) cudaEventDestroy(h->ev0);
  if (h->ev1) cudaEventDestroy(h->ev1);
  if (h->ev2) cudaEventDestroy(h->ev2);
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  for (cudaEvent_t e : h->bev)
    if (e) cudaEventDestroy(e);
  if (h->h2d) cudaStreamDestroy(h->h2d);
  if (h->d2h) cudaStreamDestroy(h->d2h);
  cudaFree(h->bstage);
  delete h;
  return VLBM_OK;
}

vlbm_status vlbm_set_dt_schedule(vlbm_t h, const double* c_host, int64_t n) {
  if (!h || n < 0 || (n > 0 && !c_host)) return VLBM_E_INVAL;
  for (int64_t j = 0; j < n; ++j)
    if (!(c_host[j] > 0.0) || !std::isfinite(c_host[j])) return VLBM_E_INVAL;
  VLBM_TRY(cudaStreamSynchronize(h->stream));
  cudaFree(h->sched);
  h->sched = nullptr;
  h->sched_len = 0;
  if (n > 0) {
    VLBM_TRY(cudaMalloc(&h->sched, n * sizeof(double)));
    VLBM_TRY(cudaMemcpy(h->sched, c_host, n * sizeof(double), cudaMemcpyHostToDevice));
  }
  h->sched_len = n;
  long long len = n;
  VLBM_TRY(cudaMemcpy(&h->sc->sched_len, &len, sizeof(long long), cudaMemcpyHostToDevice));
  destroy_graphs(h);  // the graphs captured the old schedule pointer
  return VLBM_OK;
}

vlbm_status vlbm_set_inflow(vlbm_t h, const double* W_in) {
  if (!h || !W_in) return VLBM_E_INVAL;
  if (h->p.bc[0] != VLBM_BC_INFLOW) return VLBM_E_STATE;
  const KParams& p = h->p;
  for (int k = 0; k < p.nc; ++k)
    if (!std::isfinite(W_in[k])) return VLBM_E_INVAL;
  const double rho = W_in[0];
  double usq = 0.0;
  for (int a = 0; a < p.dim; ++a) usq += (W_in[1 + a] / rho) * (W_in[1 + a] / rho);
  const double e = W_in[p.nc - 1] / rho - 0.5 * usq;
  if (!(rho > 0.0) || !std::isfinite(e)) return VLBM_E_INVAL;
  if (p.eos_kind == VLBM_EOS_IDEAL && !(e > 0.0)) return VLBM_E_INVAL;
  if (p.eos_kind != VLBM_EOS_IDEAL && !(1.0 - p.b * rho > 0.0)) return VLBM_E_INVAL;
  VLBM_TRY(cudaStreamSynchronize(h->stream));
  for (int k = 0; k < 4; ++k) {
    h->p.cd.win[k] = k < p.nc ? W_in[k] : 0.0;
    h->p.cf.win[k] = (float)h->p.cd.win[k];
  }
  h->inflow_set = true;
  destroy_graphs(h);  // the graphs captured the kernel parameters
  return VLBM_OK;
}

namespace {

// Equilibrium populations of W0 (device memory) on the handle's stream; resets time and counters.
vlbm_status init_from_device(vlbm_t h, const double* src) {
  vlbm::Launch L = launch_of(h, h->stream);
  VLBM_TRY(vlbm::launch_init(L, h->precision, src, h->buf[0], h->partial, h->nblk_sum, h->lookahead || h->pkeep));
  h->initialised = true;
  h->unpulled = true;
  h->last_step_pulled = false;
  h->n_host = 0;
  return VLBM_OK;
}

// W of the current state into device memory, on the handle's stream.
cudaError_t get_W_to_device(vlbm_t h, double* dst) {
  vlbm::Launch L = launch_of(h, h->stream);
  return vlbm::launch_get_W(L, h->precision, h->buf[(int)(h->n_host & 1)], h->unpulled ? 0 : 1, dst);
}

}  // namespace

vlbm_status vlbm_init(vlbm_t h, const double* W0) {
  if (!h || !W0) return VLBM_E_INVAL;
  if (h->p.bc[0] == VLBM_BC_INFLOW && !h->inflow_set) return VLBM_E_STATE;
  const size_t wbytes = (size_t)h->p.nc * h->p.plane * sizeof(double);
  const double* src = W0;
  if (!is_device_ptr(W0)) {
    VLBM_TRY(cudaMemcpyAsync(h->scratch, W0, wbytes, cudaMemcpyDefault, h->stream));
    src = h->scratch;
  }
  return init_from_device(h, src);
}

vlbm_status vlbm_step(vlbm_t h, int64_t n_steps, double t_end, int64_t* steps_done) {
  if (steps_done) *steps_done = 0;
  if (!h || n_steps < 0 || !std::isfinite(t_end)) return VLBM_E_INVAL;
  if (!h->initialised) return VLBM_E_STATE;
  if (n_steps == 0) return VLBM_OK;
  vlbm_status st = VLBM_OK;
  const long long n0 = h->n_host;
  vlbm::Launch L = launch_of(h, h->stream);
  VLBM_TRY(vlbm::launch_begin(L, t_end));
  long long issued = 0, n_expect = n0;
  const bool poll = t_end > 0.0;  // an end time may stop the run early: check once per chunk
  while (issued < n_steps) {
    // history room for the next chunk (grows by doubling; rebuilds the graphs when it moves)
    st = ensure_history(h, n_expect + vlbm_s::kChunk + 1);
    if (st != VLBM_OK) break;
    const int par = (int)(n_expect & 1);
    const bool first = h->unpulled;  // first step after vlbm_init reads the equilibrium in place
    if (n_steps - issued >= vlbm_s::kChunk) {
      VLBM_TRY(launch_chunk(h, first ? 2 : par));
      issued += vlbm_s::kChunk;
      n_expect += vlbm_s::kChunk;
      h->last_step_pulled = true;
    } else {
      VLBM_TRY(issue_single(h, par, first ? 0 : 1));
      ++issued;
      ++n_expect;
      h->last_step_pulled = !first;
    }
    h->unpulled = false;
    if (poll && issued < n_steps) {
      st = sync_scalars(h);
      if (st == VLBM_OK) st = cuda_status(harvest_chunk_events(h));
      if (st != VLBM_OK) break;
      if (h->sc_host->done) break;
      n_expect = h->n_host;
    }
  }
  vlbm_status st2 = sync_scalars(h);
  if (st2 == VLBM_OK) st2 = cuda_status(harvest_chunk_events(h));
  if (steps_done) *steps_done = h->n_host - n0;
  if (h->n_host == n0 + 1 && n0 == 0) h->last_step_pulled = false;
  if (st != VLBM_OK) return st;
  return st2;
}

vlbm_status vlbm_get_W(vlbm_t h, double* W) {
  if (!h || !W) return VLBM_E_INVAL;
  if (!h->initialised) return VLBM_E_STATE;
  const bool dev = is_device_ptr(W);
  VLBM_TRY(get_W_to_device(h, dev ? W : h->scratch));
  if (!dev) {
    VLBM_TRY(cudaMemcpyAsync(W, h->scratch, (size_t)h->p.nc * h->p.plane * sizeof(double), cudaMemcpyDefault, h->stream));
    VLBM_TRY(cudaStreamSynchronize(h->stream));
  }
  return VLBM_OK;
}

namespace {

vlbm_status batch_resources(vlbm_t h) {
  if (h->bstage) return VLBM_OK;
  if (cudaStreamCreateWithFlags(&h->h2d, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&h->d2h, cudaStreamNonBlocking) != cudaSuccess)
    return VLBM_E_CUDA;
  for (cudaEvent_t& e : h->bev)
    if (!e) VLBM_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  VLBM_TRY(cudaMalloc(&h->bstage, (size_t)4 * h->p.nc * h->p.plane * sizeof(double)));
  return VLBM_OK;
}

}  // namespace

vlbm_status vlbm_run_batch(vlbm_t h, int64_t n_runs, const double* const* W0s, int64_t n_steps, double t_end,
                           double* const* Ws, int64_t* steps_done) {
  if (!h || n_runs < 0 || n_steps < 0 || !std::isfinite(t_end)) return VLBM_E_INVAL;
  if (n_runs == 0) return VLBM_OK;
  if (!W0s || !Ws) return VLBM_E_INVAL;
  for (int64_t k = 0; k < n_runs; ++k) {
    if (!W0s[k] || !Ws[k]) return VLBM_E_INVAL;
    if (steps_done) steps_done[k] = 0;
  }
  if (h->p.bc[0] == VLBM_BC_INFLOW && !h->inflow_set) return VLBM_E_STATE;
  vlbm_status st = batch_resources(h);
  if (st != VLBM_OK) {
    cudaGetLastError();
    return st;
  }
  const size_t n = (size_t)h->p.nc * h->p.plane, wbytes = n * sizeof(double);
  double* const in[2] = {h->bstage, h->bstage + n};
  double* const out[2] = {h->bstage + 2 * n, h->bstage + 3 * n};
  cudaEvent_t* const in_ready = h->bev;
  cudaEvent_t* const in_free = h->bev + 2;
  cudaEvent_t* const out_ready = h->bev + 4;
  cudaEvent_t* const out_free = h->bev + 6;
  // Upload of run k into staging buffer k mod 2 on the upload stream, once the run two before
  // it has read that buffer (vlbm_init of run k - 2).
  auto upload = [&](int64_t k) -> cudaError_t {
    if (is_device_ptr(W0s[k])) return cudaSuccess;
    const int j = (int)(k & 1);
    cudaError_t e = cudaStreamWaitEvent(h->h2d, in_free[j], 0);
    if (e == cudaSuccess) e = cudaMemcpyAsync(in[j], W0s[k], wbytes, cudaMemcpyHostToDevice, h->h2d);
    if (e == cudaSuccess) e = cudaEventRecord(in_ready[j], h->h2d);
    return e;
  };
  cudaError_t e = upload(0);
  for (int64_t k = 0; k < n_runs && e == cudaSuccess && st == VLBM_OK; ++k) {
    const int j = (int)(k & 1);
    const bool dev_in = is_device_ptr(W0s[k]), dev_out = is_device_ptr(Ws[k]);
    if (!dev_in) e = cudaStreamWaitEvent(h->stream, in_ready[j], 0);
    if (e != cudaSuccess) break;
    st = init_from_device(h, dev_in ? W0s[k] : in[j]);
    if (st != VLBM_OK) break;
    e = cudaEventRecord(in_free[j], h->stream);
    // the next run's upload runs while this run steps
    if (e == cudaSuccess && k + 1 < n_runs) e = upload(k + 1);
    if (e != cudaSuccess) break;
    int64_t done = 0;
    st = vlbm_step(h, n_steps, t_end, &done);
    if (steps_done) steps_done[k] = done;
    if (st != VLBM_OK) break;
    // W into staging buffer k mod 2 once the readback of run k - 2 has left it; its readback
    // runs on the download stream while the next run steps
    if (dev_out) {
      e = get_W_to_device(h, Ws[k]);
    } else {
      e = cudaStreamWaitEvent(h->stream, out_free[j], 0);
      if (e == cudaSuccess) e = get_W_to_device(h, out[j]);
      if (e == cudaSuccess) e = cudaEventRecord(out_ready[j], h->stream);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(h->d2h, out_ready[j], 0);
      if (e == cudaSuccess) e = cudaMemcpyAsync(Ws[k], out[j], wbytes, cudaMemcpyDeviceToHost, h->d2h);
      if (e == cudaSuccess) e = cudaEventRecord(out_free[j], h->d2h);
    }
  }
  // no copy into or out of the caller's arrays is left in flight on return
  const cudaError_t e1 = cudaStreamSynchronize(h->h2d);
  const cudaError_t e2 = cudaStreamSynchronize(h->d2h);
  const cudaError_t e3 = cudaStreamSynchronize(h->stream);
  if (st != VLBM_OK) return st;
  if (e != cudaSuccess) return cuda_status(e);
  if (e1 != cudaSuccess) return cuda_status(e1);
  if (e2 != cudaSuccess) return cuda_status(e2);
  return cuda_status(e3);
}

vlbm_status vlbm_get_populations(vlbm_t h, double* f) {
  if (!h || !f) return VLBM_E_INVAL;
  if (!h->initialised) return VLBM_E_STATE;
  const size_t bytes = (size_t)h->p.q * h->p.nc * h->p.plane * sizeof(double);
  const bool dev = is_device_ptr(f);
  double* dst = f;
  if (!dev) {
    if (!h->fscratch) VLBM_TRY(cudaMalloc(&h->fscratch, bytes));
    dst = h->fscratch;
  }
  const int cur = (int)(h->n_host & 1);
  vlbm::Launch L = launch_of(h, h->stream);
  VLBM_TRY(vlbm::launch_get_f(L, h->precision, h->buf[cur], h->unpulled ? 0 : 1, dst));
  if (!dev) {
    VLBM_TRY(cudaMemcpyAsync(f, dst, bytes, cudaMemcpyDefault, h->stream));
    VLBM_TRY(cudaStreamSynchronize(h->stream));
  }
  return VLBM_OK;
}

vlbm_status vlbm_get_beta(vlbm_t h, double* beta) {
  if (!h || !beta) return VLBM_E_INVAL;
  if (!h->initialised) return VLBM_E_STATE;
  const int cur = (int)(h->n_host & 1);
  double* out = h->scratch + (size_t)h->p.nc * h->p.plane;  // plane + 4 doubles (beta, 1/M_k)
  vlbm::Launch L = launch_of(h, h->stream);
  VLBM_TRY(vlbm::launch_beta(L, h->precision, h->buf[cur], h->unpulled ? 0 : 1, out));
  VLBM_TRY(cudaMemcpyAsync(beta, out, (size_t)h->p.plane * sizeof(double), cudaMemcpyDefault, h->stream));
  VLBM_TRY(cudaStreamSynchronize(h->stream));
  VLBM_TRY(cudaMemcpy(h->sc_host, h->sc, sizeof(Scalars), cudaMemcpyDeviceToHost));
  return h->sc_host->err ? VLBM_E_NONPHYSICAL : VLBM_OK;
}

vlbm_status vlbm_get_time(vlbm_t h, double* t, int64_t* n, double* c) {
  if (!h) return VLBM_E_INVAL;
  vlbm_status st = sync_scalars(h);
  if (t) *t = h->sc_host->t;
  if (n) *n = h->sc_host->n;
  if (c) *c = h->sc_host->c_prev;
  return st;
}

vlbm_status vlbm_get_dt_history(vlbm_t h, double* dt_host, double* c_host, int64_t cap, int64_t* n) {
  if (!h || cap < 0) return VLBM_E_INVAL;
  vlbm_status st = sync_scalars(h);
  const long long m = h->n_host < cap ? h->n_host : cap;
  if (m > 0 && dt_host) VLBM_TRY(cudaMemcpy(dt_host, h->hist_dt, m * sizeof(double), cudaMemcpyDeviceToHost));
  if (m > 0 && c_host) VLBM_TRY(cudaMemcpy(c_host, h->hist_c, m * sizeof(double), cudaMemcpyDeviceToHost));
  if (n) *n = h->n_host;
  return st;
}

vlbm_status vlbm_get_totals(vlbm_t h, double* totals) {
  if (!h || !totals) return VLBM_E_INVAL;
  if (!h->initialised) return VLBM_E_STATE;
  const int cur = (int)(h->n_host & 1);
  double* out = h->scratch + (size_t)h->p.nc * h->p.plane;
  vlbm::Launch L = launch_of(h, h->stream);
  VLBM_TRY(vlbm::launch_totals(L, h->precision, h->buf[cur], h->unpulled ? 0 : 1, h->scratch, h->partial, h->nblk_sum,
                               out));
  double tmp[4];
  VLBM_TRY(cudaMemcpyAsync(tmp, out, (size_t)h->p.nc * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  VLBM_TRY(cudaStreamSynchronize(h->stream));
  std::memcpy(totals, tmp, (size_t)h->p.nc * sizeof(double));
  return VLBM_OK;
}

namespace {

// Serialised state: header, device scalar block, (dt, c) history, population buffer, checksum.
struct StateHeader {
  char magic[8];
  uint32_t version;
  int32_t dim, nx, ny, nc, q, precision, elem;
  int32_t unpulled, last_step_pulled;
  int64_t n;
  uint64_t scalars_bytes, hist_len, pop_bytes;
};
constexpr char kStateMagic[8] = {'V', 'L', 'B', 'M', 'S', 'T', 'A', 'T'};
constexpr uint32_t kStateVersion = 1;

// 64-bit FNV-1a applied to little-endian 8-byte words (then the trailing bytes).
uint64_t state_checksum(const unsigned char* p, size_t n) {
  uint64_t hsh = 1469598103934665603ull;
  const uint64_t prime = 1099511628211ull;
  size_t i = 0;
  for (; i + 8 <= n; i += 8) {
    uint64_t w;
    std::memcpy(&w, p + i, 8);
    hsh = (hsh ^ w) * prime;
  }
  for (; i < n; ++i) hsh = (hsh ^ p[i]) * prime;
  return hsh;
}

size_t state_bytes(vlbm_t h, long long n) {
  return sizeof(StateHeader) + sizeof(Scalars) + 2 * (size_t)n * sizeof(double) +
         (size_t)h->p.q * 4 * h->p.plane * h->elem + sizeof(uint64_t);
}

}  // namespace

vlbm_status vlbm_save_state(vlbm_t h, void* host, size_t cap, size_t* used) {
  if (used) *used = 0;
  if (!h) return VLBM_E_INVAL;
  if (!h->initialised) return VLBM_E_STATE;
  vlbm_status st = sync_scalars(h);
  if (st != VLBM_OK && st != VLBM_E_NONPHYSICAL) return st;
  const long long n = h->n_host;
  const size_t need = state_bytes(h, n);
  if (used) *used = need;
  if (!host) return VLBM_OK;  // size query
  if (cap < need) return VLBM_E_INVAL;
  unsigned char* out = static_cast<unsigned char*>(host);
  StateHeader hd;
  std::memset(&hd, 0, sizeof(hd));
  std::memcpy(hd.magic, kStateMagic, 8);
  hd.version = kStateVersion;
  hd.dim = h->p.dim;
  hd.nx = h->p.nx;
  hd.ny = h->p.ny;
  hd.nc = h->p.nc;
  hd.q = h->p.q;
  hd.precision = h->precision;
  hd.elem = (int32_t)h->elem;
  hd.unpulled = h->unpulled ? 1 : 0;
  hd.last_step_pulled = h->last_step_pulled ? 1 : 0;
  hd.n = n;
  hd.scalars_bytes = sizeof(Scalars);
  hd.hist_len = (uint64_t)n;
  hd.pop_bytes = (uint64_t)h->p.q * 4 * h->p.plane * h->elem;
  size_t off = 0;
  std::memcpy(out + off, &hd, sizeof(hd));
  off += sizeof(hd);
  std::memcpy(out + off, h->sc_host, sizeof(Scalars));
  off += sizeof(Scalars);
  if (n > 0) {
    VLBM_TRY(cudaMemcpy(out + off, h->hist_dt, n * sizeof(double), cudaMemcpyDeviceToHost));
    off += n * sizeof(double);
    VLBM_TRY(cudaMemcpy(out + off, h->hist_c, n * sizeof(double), cudaMemcpyDeviceToHost));
    off += n * sizeof(double);
  }
  VLBM_TRY(cudaMemcpy(out + off, h->buf[(int)(n & 1)], hd.pop_bytes, cudaMemcpyDeviceToHost));
  off += hd.pop_bytes;
  const uint64_t cs = state_checksum(out, off);
  std::memcpy(out + off, &cs, sizeof(cs));
  return st;
}

vlbm_status vlbm_load_state(vlbm_t h, const void* host, size_t n_bytes) {
  if (!h || !host || n_bytes < sizeof(StateHeader) + sizeof(uint64_t)) return VLBM_E_INVAL;
  const unsigned char* in = static_cast<const unsigned char*>(host);
  StateHeader hd;
  std::memcpy(&hd, in, sizeof(hd));
  if (std::memcmp(hd.magic, kStateMagic, 8) != 0 || hd.version != kStateVersion) return VLBM_E_INVAL;
  if (hd.n < 0 || n_bytes != state_bytes(h, hd.n)) return VLBM_E_INVAL;
  uint64_t cs;
  std::memcpy(&cs, in + n_bytes - sizeof(uint64_t), sizeof(cs));
  if (state_checksum(in, n_bytes - sizeof(uint64_t)) != cs) return VLBM_E_CHECKSUM;
  if (hd.dim != h->p.dim || hd.nx != h->p.nx || hd.ny != h->p.ny || hd.nc != h->p.nc || hd.q != h->p.q ||
      hd.precision != h->precision || hd.elem != (int32_t)h->elem || hd.scalars_bytes != sizeof(Scalars) ||
      hd.pop_bytes != (uint64_t)h->p.q * 4 * h->p.plane * h->elem)
    return VLBM_E_INVAL;
  const long long n = hd.n;
  VLBM_TRY(cudaStreamSynchronize(h->stream));
  vlbm_status st = ensure_history(h, n + vlbm_s::kChunk + 1);
  if (st != VLBM_OK) return st;
  size_t off = sizeof(hd);
  Scalars sc;
  std::memcpy(&sc, in + off, sizeof(Scalars));
  off += sizeof(Scalars);
  // handle-owned fields are not part of the state
  sc.hist_cap = h->hist_cap;
  sc.sched_len = h->sched_len;
  sc.done = 0;
  sc.active = 0;
  if (n > 0) {
    VLBM_TRY(cudaMemcpy(h->hist_dt, in + off, n * sizeof(double), cudaMemcpyHostToDevice));
    off += n * sizeof(double);
    VLBM_TRY(cudaMemcpy(h->hist_c, in + off, n * sizeof(double), cudaMemcpyHostToDevice));
    off += n * sizeof(double);
  }
  const int cur = (int)(n & 1);
  VLBM_TRY(cudaMemcpy(h->buf[cur], in + off, hd.pop_bytes, cudaMemcpyHostToDevice));
  VLBM_TRY(cudaMemcpy(h->sc, &sc, sizeof(Scalars), cudaMemcpyHostToDevice));
  h->initialised = true;
  h->unpulled = hd.unpulled != 0;
  h->last_step_pulled = hd.last_step_pulled != 0;
  h->n_host = n;
  // the maxima of the current state (partial slot n & 1), which the look-ahead step of the
  // saving handle had left in its own partials
  vlbm::Launch L = launch_of(h, h->stream);
  VLBM_TRY(vlbm::launch_reduce(L, h->precision, h->buf[cur], h->unpulled ? 0 : 1, false));
  // the kept pressure of the restored state (FP32 look-ahead with a non-ideal gas)
  VLBM_TRY(vlbm::launch_fill_pressure(L, h->buf[cur], h->unpulled ? 0 : 1));
  return sync_scalars(h);
}

vlbm_status vlbm_time_step_kernel(vlbm_t h, int32_t reps, double* ms_per_launch) {
  if (!h || reps < 1 || !ms_per_launch) return VLBM_E_INVAL;
  if (!h->initialised || h->n_host < 1) return VLBM_E_STATE;
  // Re-run the last step kernel (same input buffer, same device scalars): it rewrites the
  // current state with identical values, so the state does not change.
  const int cur = (int)(h->n_host & 1);
  vlbm::Launch L = launch_of(h, h->stream);
  const int pulled = h->last_step_pulled ? 1 : 0;
  VLBM_TRY(cudaEventRecord(h->ev0, h->stream));
  for (int j = 0; j < reps; ++j)
    VLBM_TRY(vlbm::launch_step(L, h->precision, h->lookahead, h->buf[cur ^ 1], h->buf[cur], pulled));
  VLBM_TRY(cudaEventRecord(h->ev1, h->stream));
  VLBM_TRY(cudaEventSynchronize(h->ev1));
  float ms = 0.f;
  VLBM_TRY(cudaEventElapsedTime(&ms, h->ev0, h->ev1));
  *ms_per_launch = (double)ms / reps;
  return VLBM_OK;
}

vlbm_status vlbm_set_profiling(vlbm_t h, int32_t on) {
  if (!h) return VLBM_E_INVAL;
  VLBM_TRY(cudaStreamSynchronize(h->stream));
  h->profile = on != 0;
  h->pev_used = 0;
  h->gev_pending = -1;
  h->prof_ms = 0.0;
  h->prof_n = 0;
  return VLBM_OK;
}

vlbm_status vlbm_get_profile(vlbm_t h, double* ms_total, int64_t* launches) {
  if (!h) return VLBM_E_INVAL;
  VLBM_TRY(cudaStreamSynchronize(h->stream));
  VLBM_TRY(harvest_chunk_events(h));
  double tot = h->prof_ms;
  for (size_t j = 0; j + 1 < h->pev_used; j += 2) {
    float ms = 0.f;
    VLBM_TRY(cudaEventElapsedTime(&ms, h->pev[j], h->pev[j + 1]));
    tot += ms;
  }
  if (ms_total) *ms_total = tot;
  if (launches) *launches = (int64_t)(h->pev_used / 2) + h->prof_n;
  h->pev_used = 0;
  h->prof_ms = 0.0;
  h->prof_n = 0;
  return VLBM_OK;
}

vlbm_status vlbm_adjoint(vlbm_t h, const double* W0, int64_t n_steps, int32_t checkpoint_every, const double* dJ_dWT,
                         double* dJ_dW0, double* dJ_deos) {
  if (!h || !W0 || !dJ_dWT || !dJ_dW0 || n_steps < 1 || checkpoint_every < 1) return VLBM_E_INVAL;
  if (h->p.bc[0] == VLBM_BC_INFLOW) return VLBM_E_UNSUPPORTED;  // the adjoint has no ghost cells
  if (h->p.eos_kind == VLBM_EOS_VDW_CVT) return VLBM_E_UNSUPPORTED;  // nor a Newton-inversion Jacobian
  auto& A = h->adj;
  const KParams& p = h->p;
  // population states are kept in the handle's storage precision (FP64, or FP32 deviations);
  // sizes below are in doubles (an FP32 state takes half of one FP64 state's doubles)
  const size_t state_vals = (size_t)p.q * 4 * p.plane;
  const size_t state = h->precision == VLBM_FP64 ? state_vals : (state_vals + 1) / 2;
  const size_t lam_state = state_vals;
  const size_t wsz = (size_t)p.nc * p.plane;
  const long long N = n_steps, K = checkpoint_every;
  const size_t nseg = (size_t)((N + K - 1) / K);
  const size_t segn = (size_t)(K < N ? K : N);
  // workspace (grown on demand)
  auto grow = [](double** ptr, size_t* cap, size_t need) -> bool {
    if (*cap >= need && *ptr) return true;
    cudaFree(*ptr);
    *ptr = nullptr;
    *cap = 0;
    if (cudaMalloc(ptr, need * sizeof(double)) != cudaSuccess) return false;
    *cap = need;
    return true;
  };
  if (!grow(&A.ckpt, &A.ckpt_states, nseg * state) || !grow(&A.seg, &A.seg_states, segn * state) ||
      !grow(&A.sched, &A.sched_cap, (size_t)N + 1))
    return VLBM_E_NOMEM;
  // FP64 strips: the recomputation keeps, for each state of a segment but the last, W, u, Q
  // (stored by its maxima pass) and in sensor mode s_hat, s, theta, dil, vort (stored by its step
  // kernel) in a slot of its own, which the adjoint of that step reads instead of recomputing
  // them; used when the slots fit in half of the free device memory
  bool use_kept = false;
  const size_t kept_per_state = (size_t)22 * p.plane;
  const bool kept_sensor = p.beta_mode == 0;
  if (h->fields && p.dim == 2 && segn > 1) {
    const size_t need = (segn - 1) * kept_per_state;
    size_t fr = 0, tot = 0;
    if (A.kept_cap >= need) {
      use_kept = true;
    } else if (cudaMemGetInfo(&fr, &tot) == cudaSuccess && need * sizeof(double) <= fr / 2) {
      use_kept = grow(&A.kept, &A.kept_cap, need);
    }
    cudaGetLastError();
  }
  if (!A.as) {
    if (cudaMalloc(&A.lam[0], lam_state * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&A.lam[1], lam_state * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&A.F, (size_t)vlbm::adj_num_fields() * p.plane * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&A.pv, (size_t)vlbm::adj_part_entries(p) * 4 * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&A.pi, (size_t)vlbm::adj_part_entries(p) * 4 * sizeof(long long)) != cudaSuccess ||
        cudaMalloc(&A.part, (size_t)vlbm::adj_part_entries(p) * 8 * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&A.gpart, (size_t)vlbm::adj_group_entries(p) * 8 * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&A.gidx, (size_t)vlbm::adj_group_entries(p) * 4 * sizeof(long long)) != cudaSuccess ||
        cudaMalloc(&A.dJ, wsz * sizeof(double)) != cudaSuccess || cudaMalloc(&A.dW0, wsz * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&A.sc_backup, sizeof(Scalars)) != cudaSuccess ||
        cudaMallocHost(&A.as_host, sizeof(vlbm::AdjScalars)) != cudaSuccess ||
        cudaMalloc(&A.as, sizeof(vlbm::AdjScalars)) != cudaSuccess)
      return VLBM_E_NOMEM;
  }
  // Tape: the last T segments are stepped by the forward pass into slots of their own, so the
  // reverse pass applies their adjoint steps without recomputing them.  A lean slot keeps every
  // state of the segment and, on FP64 strips in sensor mode, the 8 sensor planes of each state
  // (written by the step kernel), whose adjoint then evaluates W, u, Q itself; a full slot keeps
  // all 22 planes (W, u, Q from the maxima pass too).  T is as large as the tape limit allows in
  // lean slots (by default 3/4 of the free device memory: a B300's HBM holds about a thousand
  // steps of a 1024^2 run that way); the memory left over turns the last T_full of them into
  // full slots.  Avoiding a recomputation saves about a forward step per step, a full slot about
  // a fifth of one more.
  const bool tape_kept = h->fields && p.dim == 2;
  const size_t sens_per_state = kept_sensor ? (size_t)8 * p.plane : 0;
  const size_t lean_seg = segn * state + (tape_kept ? segn * sens_per_state : 0);      // doubles
  const size_t full_seg = segn * state + (tape_kept ? segn * kept_per_state : 0);
  size_t T = 0, T_full = 0;
  if (A.tape_limit != 0) {
    size_t budget = 0;
    if (A.tape_limit > 0) {
      budget = (size_t)A.tape_limit;
    } else {
      size_t fr = 0, tot = 0;
      if (cudaMemGetInfo(&fr, &tot) == cudaSuccess) budget = fr / 4 * 3 + A.tape_cap * sizeof(double);
      cudaGetLastError();
    }
    T = budget / (lean_seg * sizeof(double));
    if (T > nseg) T = nseg;
    if (full_seg > lean_seg) {
      T_full = (budget / sizeof(double) - T * lean_seg) / (full_seg - lean_seg);
      if (T_full > T) T_full = T;
    }
    if (T > 0 && !grow(&A.tape, &A.tape_cap, (T - T_full) * lean_seg + T_full * full_seg)) {
      cudaGetLastError();
      T = T_full = 0;
    }
  }
  const size_t first_taped = nseg - T, first_full = nseg - T_full;
  A.taped_steps = T > 0 ? N - (long long)first_taped * K : 0;
  A.tape_used = ((T - T_full) * lean_seg + T_full * full_seg) * sizeof(double);
  // a taped segment's slot: its states, then its kept planes (22 per state in a full slot, the
  // 8 sensor planes in a lean one); lean slots first, the full ones (the last segments) after
  struct TapeSlot {
    double* states;
    double* kept;     // full slot: 22 planes per state (nullptr otherwise)
    double* sensor;   // lean slot in sensor mode: 8 planes per state (nullptr otherwise)
  };
  auto tape_slot = [&](size_t sgi) -> TapeSlot {
    const bool full = sgi >= first_full;
    double* base = A.tape + (full ? (first_full - first_taped) * lean_seg + (sgi - first_full) * full_seg
                                  : (sgi - first_taped) * lean_seg);
    double* extra = base + segn * state;
    TapeSlot t{base, nullptr, nullptr};
    if (tape_kept && full) t.kept = extra;
    if (tape_kept && !full && kept_sensor) t.sensor = extra;
    return t;
  };
  VLBM_TRY(cudaMemcpyAsync(A.dW0, W0, wsz * sizeof(double), cudaMemcpyDefault, h->stream));
  VLBM_TRY(cudaMemcpyAsync(A.dJ, dJ_dWT, wsz * sizeof(double), cudaMemcpyDefault, h->stream));

  // One taped segment of the forward pass: from the handle's current state n0 (buffer n0 & 1),
  // `steps` steps in the two-pass form with live link-speed decisions, as vlbm_step takes them,
  // every state into the segment's slots and the last one into buffer (n0 + steps) & 1.
  auto tape_forward = [&](size_t sgi, long long steps) -> vlbm_status {
    const long long n0 = (long long)sgi * K;
    if (h->n_host != n0) return VLBM_E_STATE;
    vlbm_status ts = ensure_history(h, n0 + steps + 1);
    if (ts != VLBM_OK) return ts;
    const TapeSlot ts_ = tape_slot(sgi);
    double* tst = ts_.states;
    vlbm::Launch TL = launch_of(h, h->stream);
    VLBM_TRY(vlbm::launch_begin(TL, 0.0));
    VLBM_TRY(cudaMemcpyAsync(tst, h->buf[(int)(n0 & 1)], state * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
    for (long long j = 0; j < steps; ++j) {
      const long long n = n0 + j;
      const int pulled = n >= 1 ? 1 : 0;  // the run's first step reads the equilibrium in place
      double* fin = tst + (size_t)j * state;
      void* fout = j + 1 < steps ? static_cast<void*>(tst + (size_t)(j + 1) * state) : h->buf[(int)((n + 1) & 1)];
      if (ts_.kept) {
        TL.fields = ts_.kept + (size_t)j * kept_per_state;
        TL.sens = kept_sensor ? TL.fields + (size_t)14 * p.plane : nullptr;
      } else if (ts_.sensor) {  // W, u, Q in the handle's own planes; the sensor planes taped
        TL.sens = ts_.sensor + (size_t)j * sens_per_state;
      }
      VLBM_TRY(vlbm::launch_reduce(TL, h->precision, fin, pulled, true));
      VLBM_TRY(vlbm::launch_dt(TL));
      VLBM_TRY(vlbm::launch_step(TL, h->precision, false, fin, fout, pulled));
    }
    ts = sync_scalars(h);
    if (ts != VLBM_OK) return ts;
    if (h->n_host != n0 + steps) return VLBM_E_STATE;
    h->unpulled = false;
    h->last_step_pulled = true;
    return VLBM_OK;
  };

  // ---- forward pass: checkpoints every K steps, recorded link speeds ----
  VLBM_TRY(cudaEventRecord(h->ev0, h->stream));
  vlbm_status st = vlbm_init(h, A.dW0);
  if (st != VLBM_OK) return st;
  double c0 = 0.0;
  st = vlbm_get_time(h, nullptr, nullptr, &c0);
  if (st != VLBM_OK) return st;
  VLBM_TRY(cudaMemcpyAsync(reinterpret_cast<char*>(A.as) + offsetof(vlbm::AdjScalars, wref),
                           reinterpret_cast<const char*>(h->sc) + offsetof(Scalars, wref), 4 * sizeof(double),
                           cudaMemcpyDeviceToDevice, h->stream));
  for (size_t sgi = 0; sgi < nseg; ++sgi) {
    const long long steps = (long long)((N - (long long)sgi * K) < K ? (N - (long long)sgi * K) : K);
    if (sgi >= first_taped) {
      st = tape_forward(sgi, steps);
      if (st != VLBM_OK) return st;
      continue;
    }
    const int cur = (int)(h->n_host & 1);
    VLBM_TRY(cudaMemcpyAsync(A.ckpt + sgi * state, h->buf[cur], state * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
    int64_t done = 0;
    st = vlbm_step(h, steps, 0.0, &done);
    if (st != VLBM_OK) return st;
    if (done != steps) return VLBM_E_STATE;
  }
  VLBM_TRY(cudaMemcpyAsync(A.sched, &c0, sizeof(double), cudaMemcpyHostToDevice, h->stream));
  VLBM_TRY(cudaMemcpyAsync(A.sched + 1, h->hist_c, N * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
  VLBM_TRY(cudaMemcpyAsync(A.sc_backup, h->sc, sizeof(Scalars), cudaMemcpyDeviceToDevice, h->stream));
  VLBM_TRY(cudaEventRecord(h->ev1, h->stream));

  // ---- reverse pass ----
  vlbm::AdjLaunch L{&p, A.as, h->stream, A.sched, A.F, A.pv, A.pi, A.part, A.gpart, A.gidx};
  vlbm::Launch FL = launch_of(h, h->stream);
  FL.sched = A.sched;
  int li = (int)(N & 1);  // lambda^N lives in lam[li]
  VLBM_TRY(vlbm::adj_terminal(L, A.dJ, A.lam[li]));
  const size_t pev_base = h->pev_used;  // event pairs bracketing the recomputations
  for (long long sgi = (long long)nseg - 1; sgi >= 0; --sgi) {
    const long long n0 = sgi * K, n1 = (n0 + K < N) ? n0 + K : N;
    if ((size_t)sgi >= first_taped) {  // taped: every state (and its kept planes) at hand
      const TapeSlot t = tape_slot((size_t)sgi);
      for (long long n = n1 - 1; n >= n0; --n) {
        const int pulled = n >= 1 ? 1 : 0;
        const size_t j = (size_t)(n - n0);
        double* kept = t.kept ? t.kept + j * kept_per_state : nullptr;
        const double* sensor = t.sensor ? t.sensor + j * sens_per_state : nullptr;
        VLBM_TRY(vlbm::adj_step(L, h->precision, t.states + j * state, pulled, A.lam[li], A.lam[li ^ 1], n, kept,
                                kept_sensor, sensor));
        li ^= 1;
      }
      continue;
    }
    VLBM_TRY(cudaMemcpyAsync(A.seg, A.ckpt + (size_t)sgi * state, state * sizeof(double), cudaMemcpyDeviceToDevice,
                             h->stream));
    if (n1 - n0 > 1) {  // recompute the segment's states with the recorded link speeds (two-pass form)
      cudaEvent_t ra, rb;
      VLBM_TRY(profile_pair(h, &ra, &rb));
      VLBM_TRY(cudaEventRecord(ra, h->stream));
      VLBM_TRY(vlbm::adj_replay_scalars(h->stream, h->sc, n0, A.sched, N + 1));
      for (long long j = 0; j + 1 < n1 - n0; ++j) {
        const int pulled = (n0 + j >= 1) ? 1 : 0;
        double* fin = A.seg + (size_t)j * state;
        double* fout = A.seg + (size_t)(j + 1) * state;
        if (use_kept) {
          FL.fields = A.kept + (size_t)j * kept_per_state;
          FL.sens = kept_sensor ? FL.fields + (size_t)14 * p.plane : nullptr;
        }
        VLBM_TRY(vlbm::launch_reduce(FL, h->precision, fin, pulled, true));
        VLBM_TRY(vlbm::launch_dt(FL));
        VLBM_TRY(vlbm::launch_step(FL, h->precision, false, fin, fout, pulled));
      }
      VLBM_TRY(cudaEventRecord(rb, h->stream));
    }
    for (long long n = n1 - 1; n >= n0; --n) {
      const int pulled = n >= 1 ? 1 : 0;
      double* kept = (use_kept && n + 1 < n1) ? A.kept + (size_t)(n - n0) * kept_per_state : nullptr;
      VLBM_TRY(vlbm::adj_step(L, h->precision, A.seg + (size_t)(n - n0) * state, pulled, A.lam[li], A.lam[li ^ 1], n,
                              kept, kept_sensor));
      li ^= 1;
    }
  }
  VLBM_TRY(vlbm::adj_init(L, A.dW0, A.lam[li], c0, A.dW0));
  VLBM_TRY(cudaMemcpyAsync(h->sc, A.sc_backup, sizeof(Scalars), cudaMemcpyDeviceToDevice, h->stream));
  {
    // the recomputations overwrote the partial maxima (and the kept pressure) that a look-ahead
    // step reads for the state it starts from: take them again from the final state
    vlbm::Launch RL = launch_of(h, h->stream);
    const int cur = (int)(N & 1);
    VLBM_TRY(vlbm::launch_reduce(RL, h->precision, h->buf[cur], 1, false));
    VLBM_TRY(vlbm::launch_fill_pressure(RL, h->buf[cur], 1));
  }
  VLBM_TRY(cudaEventRecord(h->ev2, h->stream));
  VLBM_TRY(cudaMemcpyAsync(dJ_dW0, A.dW0, wsz * sizeof(double), cudaMemcpyDefault, h->stream));
  VLBM_TRY(cudaMemcpyAsync(A.as_host, A.as, sizeof(vlbm::AdjScalars), cudaMemcpyDeviceToHost, h->stream));
  VLBM_TRY(cudaStreamSynchronize(h->stream));
  float r_ms = 0.f, f_ms = 0.f;
  // forward pass = [ev0, ev1], reverse pass = [ev1, ev2]
  VLBM_TRY(cudaEventElapsedTime(&r_ms, h->ev1, h->ev2));
  VLBM_TRY(cudaEventElapsedTime(&f_ms, h->ev0, h->ev1));
  A.rev_ms = r_ms;
  A.fwd_ms = f_ms;
  A.recompute_ms = 0.0;
  for (size_t e = pev_base; e + 1 < h->pev_used; e += 2) {
    float m = 0.f;
    VLBM_TRY(cudaEventElapsedTime(&m, h->pev[e], h->pev[e + 1]));
    A.recompute_ms += m;
  }
  h->pev_used = pev_base;
  if (dJ_deos)
    for (int j = 0; j < 5; ++j) dJ_deos[j] = A.as_host->eos[j];
  st = sync_scalars(h);
  return st;
}

vlbm_status vlbm_set_adjoint_tape(vlbm_t h, int64_t max_bytes) {
  if (!h) return VLBM_E_INVAL;
  h->adj.tape_limit = max_bytes;
  if (max_bytes == 0 || (max_bytes > 0 && h->adj.tape_cap * sizeof(double) > (size_t)max_bytes)) {
    VLBM_TRY(cudaStreamSynchronize(h->stream));
    cudaFree(h->adj.tape);
    h->adj.tape = nullptr;
    h->adj.tape_cap = 0;
  }
  return VLBM_OK;
}

vlbm_status vlbm_adjoint_info(vlbm_t h, double* forward_ms, int64_t* taped_steps, int64_t* tape_bytes) {
  if (!h) return VLBM_E_INVAL;
  if (forward_ms) *forward_ms = h->adj.fwd_ms;
  if (taped_steps) *taped_steps = h->adj.taped_steps;
  if (tape_bytes) *tape_bytes = (int64_t)h->adj.tape_used;
  return VLBM_OK;
}

vlbm_status vlbm_adjoint_timing(vlbm_t h, double* reverse_ms, double* recompute_ms) {
  if (!h || !reverse_ms) return VLBM_E_INVAL;
  *reverse_ms = h->adj.rev_ms;
  if (recompute_ms) *recompute_ms = h->adj.recompute_ms;
  return VLBM_OK;
}

vlbm_status vlbm_launches_per_step(vlbm_t h, int32_t* launches) {
  if (!h || !launches) return VLBM_E_INVAL;
  *launches = h->lookahead ? 2 : 3;
  return VLBM_OK;
}

}  // extern "C"
