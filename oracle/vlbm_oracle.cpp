// ORACLE: test infrastructure only.
//
// Plain, slow, obviously-correct FP64 CPU implementation of the vectorial lattice Boltzmann
// (VLBM) time step of Hosseini & Karlin, "Vectorial lattice Boltzmann solver for compressible
// inviscid flows with generic equation of state" (Secs. II-III).  Only the test-suite, the
// package smoke check and the CPU-baseline leg of the benchmark may load it; the product path
// never does.  It shares no code, header, table or constant with the CUDA library.
//
// Every routine is templated on the scalar type T so that the same source runs in plain
// double and in first-order dual numbers (forward-mode derivative, used to check the adjoint).
// Compile with -O2 -ffp-contract=off: no fused multiply-add, the summation orders written here
// are the ones executed.
//
// Parity status: every function below is pinned by the CPU tests (closed forms, invariants,
// the paper's printed numbers, brute force).  The shock sensor beta(x,t) (Sec. III D) is pinned
// by closed forms on states where its chain is exact: a density ramp (activity, normalisation,
// beta map), slope kinks of the density and of the velocity (the (1/4, 1/2, 1/4) filter along
// each axis applied to s and to the Ducros ratio theta, theta itself, and the gate s_bar theta_bar),
// and the Ducros gate on shear; and by the paper's printed accuracy numbers.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <type_traits>
#include <vector>

#ifdef _OPENMP
#include <omp.h>
#endif

namespace orc {

// ------------------------------------------------------------------------------------------
// First-order dual numbers: v + d*eps, eps^2 = 0.  Non-smooth points follow fixed conventions:
// d|x| = 0 at x = 0, d sqrt(x) = 0 at x = 0, max() takes the derivative of the first maximal
// element in iteration order, clip() has derivative 0 at and beyond its bounds.
// ------------------------------------------------------------------------------------------
struct Dual {
  double v, d;
  Dual() : v(0), d(0) {}
  Dual(double x) : v(x), d(0) {}
  Dual(double x, double dx) : v(x), d(dx) {}
};
inline Dual operator+(Dual a, Dual b) { return Dual(a.v + b.v, a.d + b.d); }
inline Dual operator-(Dual a, Dual b) { return Dual(a.v - b.v, a.d - b.d); }
inline Dual operator-(Dual a) { return Dual(-a.v, -a.d); }
inline Dual operator*(Dual a, Dual b) { return Dual(a.v * b.v, a.d * b.v + a.v * b.d); }
inline Dual operator/(Dual a, Dual b) {
  double q = a.v / b.v;
  return Dual(q, (a.d - q * b.d) / b.v);
}
inline Dual& operator+=(Dual& a, Dual b) { a = a + b; return a; }
inline Dual sqrt(Dual a) {
  double s = std::sqrt(a.v);
  return Dual(s, s > 0 ? a.d / (2.0 * s) : 0.0);
}
inline Dual fabs(Dual a) {
  if (a.v > 0) return a;
  if (a.v < 0) return -a;
  return Dual(0.0, 0.0);
}
inline double val(double x) { return x; }
inline double val(const Dual& x) { return x.v; }
inline double der(double) { return 0.0; }
inline double der(const Dual& x) { return x.d; }
inline bool finite_(double x) { return std::isfinite(x); }
inline bool finite_(const Dual& x) { return std::isfinite(x.v) && std::isfinite(x.d); }
using std::fabs;
using std::sqrt;

template <class T>
inline T clip01(T x) {  // clip(., 0, 1) of Eqs. (34)-(35)
  if (val(x) <= 0.0) return T(0.0);
  if (val(x) >= 1.0) return T(1.0);
  return x;
}

// ------------------------------------------------------------------------------------------
// Equation of state (Sec. II C).
// ------------------------------------------------------------------------------------------
enum { EOS_IDEAL = 0, EOS_VDW = 1, EOS_VDW_CVT = 2 };

template <class T>
struct Eos {
  int kind;
  T gamma, a, b, R, cv;
  T cv1, cv2;  // EOS_VDW_CVT: c_v(T) = cv + cv1 T + cv2 T^2
};

// Caloric part of the non-polytropic van der Waals gas (EOS_VDW_CVT): the heat capacity
// c_v(T) = cv + cv1 T + cv2 T^2 integrates to E(T) = cv T + cv1 T^2/2 + cv2 T^3/3, and
// e = E(T) - a rho.  For the thermal relation of Eq. (16), (dP/dT)_rho = R rho / (1 - b rho), so
// the consistency condition Eq. (12) gives (de/drho)_T = [P - T (dP/dT)_rho] / rho^2 = -a whatever
// c_v(T) is: any positive c_v(T) is admissible.  The paper's Eq. (11) is this P(rho, e) with T(rho, e)
// from inverting E(T) = e + a rho, done here by Newton's method from T0 = (e + a rho)/cv; E is
// increasing and convex for cv > 0, cv1, cv2 >= 0, so E(T0) >= e + a rho and the iterates fall
// monotonically onto the root.  The iteration stops when a step changes T by at most 1e-15 T;
// after 50 steps without that, T is returned as NaN (a non-physical state).
template <class T>
T vdw_cvt_temperature(const Eos<T>& q, T rho, T e) {
  T target = e + q.a * rho;
  T temp = target / q.cv;
  for (int it = 0; it < 50; ++it) {
    T E = q.cv * temp + q.cv1 * temp * temp / 2.0 + q.cv2 * temp * temp * temp / 3.0;
    T cvT = q.cv + q.cv1 * temp + q.cv2 * temp * temp;
    T step = (E - target) / cvT;
    temp = temp - step;
    if (std::fabs(val(step)) <= 1e-15 * std::fabs(val(temp))) return temp;
  }
  return T(std::nan(""));
}

// Pressure P(rho, e) (Eq. 11) and frozen sound speed c_s^2 = P_rho + P P_e / rho^2 (Eq. 13).
// Ideal gas: Eq. (15).  Polytropic van der Waals: Eqs. (16)-(17), with the caloric relation
// e = cv T - a rho inverted for T; the partial derivatives at fixed e (P_rho) and fixed rho
// (P_e) are written out from Eq. (16) by the chain rule.
template <class T>
void eos_eval(const Eos<T>& q, T rho, T e, T* P, T* cs2) {
  if (q.kind == EOS_IDEAL) {
    *P = (q.gamma - 1.0) * rho * e;
    *cs2 = q.gamma * (q.gamma - 1.0) * e;
    return;
  }
  // T from the caloric relation: Eq. (17) solved for T, or the Newton inversion of E(T)
  T temp = q.kind == EOS_VDW_CVT ? vdw_cvt_temperature(q, rho, e) : (e + q.a * rho) / q.cv;
  T cvT = q.kind == EOS_VDW_CVT ? q.cv + q.cv1 * temp + q.cv2 * temp * temp : q.cv;  // c_v at T
  T omb = 1.0 - q.b * rho;
  T p = q.R * rho * temp / omb - q.a * rho * rho;                        // Eq. (16)
  T dP_dT_rho = q.R * rho / omb;                                         // (dP/dT)_rho
  T dP_drho_T = q.R * temp / (omb * omb) - 2.0 * q.a * rho;              // (dP/drho)_T
  T dT_drho_e = q.a / cvT;                                               // from e = E(T) - a rho
  T dT_de_rho = 1.0 / cvT;
  T P_rho = dP_drho_T + dP_dT_rho * dT_drho_e;  // (dP/drho)_e
  T P_e = dP_dT_rho * dT_de_rho;                // (dP/de)_rho
  *P = p;
  *cs2 = P_rho + p / (rho * rho) * P_e;  // Eq. (13)
}

// Fundamental derivative Gamma = 1 + (rho/c_s)(dc_s/drho)_s (Sec. II C and Eq. 46).  Along an
// isentrope T ds = de - (P/rho^2) drho = 0 (Sec. II C), so (d/drho)_s = d/drho|_e + (P/rho^2)
// d/de|_rho.  The derivative of c_s^2 along that direction is taken exactly with a dual number,
// and Gamma = 1 + rho/(2 c_s^2) (dc_s^2/drho)_s.
inline double fundamental_derivative(const Eos<double>& q, double rho, double e) {
  double P, cs2;
  eos_eval(q, rho, e, &P, &cs2);
  Eos<Dual> qd{q.kind, Dual(q.gamma), Dual(q.a), Dual(q.b), Dual(q.R), Dual(q.cv), Dual(q.cv1), Dual(q.cv2)};
  Dual Pd, cs2d;
  eos_eval(qd, Dual(rho, 1.0), Dual(e, P / (rho * rho)), &Pd, &cs2d);
  return 1.0 + rho / (2.0 * cs2) * cs2d.d;
}

// ------------------------------------------------------------------------------------------
// Lattice (Sec. III A, Eq. 18): DdQ2^d, Q = 2D velocities c_i = c sigma_i.  Order of i:
// D2Q4 {x-, x+, y-, y+}; D1Q2 {x-, x+}.
// ------------------------------------------------------------------------------------------
static const int SIGMA[4][2] = {{-1, 0}, {1, 0}, {0, -1}, {0, 1}};

// Flux Q_alpha(W) (Eq. 10): Q_alpha = (rho u_alpha, rho u u_alpha + P e_alpha, (rho E + P) u_alpha).
// W = (rho, rho u_1..rho u_D, rho E) (Eq. 2); E = e + |u|^2/2 (Eq. 1).  Output Qf[alpha*NC + k].
template <class T>
int primitives_and_flux(int D, const Eos<T>& eos, const T* W, T* u, T* P, T* cs2, T* Qf) {
  const int NC = D + 2;
  T rho = W[0];
  if (!(val(rho) > 0.0) || !finite_(rho)) return 1;
  T usq = 0.0;
  for (int a = 0; a < D; ++a) {
    u[a] = W[1 + a] / rho;
    usq = usq + u[a] * u[a];
  }
  T E = W[NC - 1] / rho;
  T e = E - 0.5 * usq;
  eos_eval(eos, rho, e, P, cs2);
  if (!(val(*cs2) > 0.0) || !finite_(*cs2) || !finite_(*P)) return 1;  // Eq. (14)
  if (Qf) {
    for (int a = 0; a < D; ++a) {
      T* q = Qf + a * NC;
      q[0] = W[1 + a];
      for (int b = 0; b < D; ++b) q[1 + b] = W[1 + b] * u[a] + (a == b ? *P : T(0.0));
      q[NC - 1] = (W[NC - 1] + *P) * u[a];
    }
  }
  return 0;
}

// Vector equilibrium f_i^eq = W/(2D) + c_i . Q(W) / (2 c^2) (Eq. 20), c_i = c sigma_i.
template <class T>
void feq(int D, double c, const T* W, const T* Qf, int i, T* out) {
  const int NC = D + 2;
  for (int k = 0; k < NC; ++k) {
    T ciQ = 0.0;
    for (int a = 0; a < D; ++a) ciQ = ciQ + (c * SIGMA[i][a]) * Qf[a * NC + k];
    out[k] = W[k] / (2.0 * D) + ciQ / (2.0 * c * c);
  }
}

// Reprojection at a new link speed (Sec. III E, Eqs. 38-40).  Moments J_alpha = sum_i c_i,alpha f_i
// and (D = 2) K = sum_i (c_ix^2 - c_iy^2) f_i are taken with the old link speed, then the
// populations are rebuilt from (W, J, K) with the new one.  For D = 1 the K term is absent and
// the share is W/2 (the single-direction D1Q2 form).  f is laid out f[i*NC + k] for one cell.
template <class T>
void reproject(int D, double c_old, double c_new, T* f) {
  const int NC = D + 2, Q = 2 * D;
  for (int k = 0; k < NC; ++k) {
    T W = 0.0, J[2] = {T(0.0), T(0.0)}, K = 0.0;
    for (int i = 0; i < Q; ++i) W = W + f[i * NC + k];
    for (int a = 0; a < D; ++a)
      for (int i = 0; i < Q; ++i) J[a] = J[a] + (c_old * SIGMA[i][a]) * f[i * NC + k];
    if (D == 2)
      for (int i = 0; i < Q; ++i) {
        double cx = c_old * SIGMA[i][0], cy = c_old * SIGMA[i][1];
        K = K + (cx * cx - cy * cy) * f[i * NC + k];
      }
    for (int i = 0; i < Q; ++i) {
      T ciJ = 0.0;
      for (int a = 0; a < D; ++a) ciJ = ciJ + (c_new * SIGMA[i][a]) * J[a];
      T fi = W / (double)Q + ciJ / (2.0 * c_new * c_new);
      if (D == 2) {
        double cx = c_new * SIGMA[i][0], cy = c_new * SIGMA[i][1];
        fi = fi + (cx * cx - cy * cy) / (4.0 * c_new * c_new * c_new * c_new) * K;
      }
      f[i * NC + k] = fi;
    }
  }
}

// ------------------------------------------------------------------------------------------
// Solver
// ------------------------------------------------------------------------------------------
enum { BC_PERIODIC = 0, BC_ZEROGRAD = 1, BC_INFLOW = 2 };
enum { BETA_SENSOR = 0, BETA_CONST = 1 };
enum { OK = 0, E_NONPHYSICAL = 4 };

struct Params {
  double cfl, beta_const, beta_min, beta_max, c_sensor, ducros_eps;
  int beta_mode, retarget_every;
};

// Index rule shared by streaming and every stencil (periodic: wrap; zero-gradient: clamp to
// the edge cell, i.e. an edge-replicated ghost, Secs. IV B and IV E).  A pinned-inflow side
// (Sec. IV H) is handled by the solver before this rule is reached (its ghost cells hold a fixed
// state); the clamp below is never used for it.
inline long nb(long j, long n, int bc_lo, int bc_hi) {
  if (j < 0) return bc_lo == BC_PERIODIC ? j + n : 0;
  if (j >= n) return bc_hi == BC_PERIODIC ? j - n : n - 1;
  return j;
}

template <class T>
struct Solver {
  int D, Q, NC;
  long nx, ny, N;
  double dx;
  int bc[4];  // x-lo, x-hi, y-lo, y-hi
  Eos<T> eos;
  Params prm;
  std::vector<T> f, fnext, W, u, P, cs2, Qf, s, th, tmp, beta;
  std::vector<T> s_raw, th_raw;  // s and theta before the filter (kept only on request)
  bool keep_raw = false;
  // Pinned inflow on the x-lo side (Sec. IV H): every ghost cell x < 0 holds the fixed state
  // W_in, whose velocity and flux are uin, qin; its post-collision populations are the
  // equilibrium of W_in at the step's link speed.  s and theta of the ghost column x = -1 feed
  // the box filter of the first column.
  bool inflow = false;
  T win[4], uin[2], qin[8];
  std::vector<T> s_gh, th_gh;
  double c_prev = 0, t = 0;
  long n = 0;
  std::vector<double> hist_dt, hist_c, sched;
  int nthreads = 1;

  long cell(long x, long y) const { return y * nx + x; }
  long fidx(int i, int k, long c) const { return ((long)(i * NC + k)) * N + c; }
  long xn(long x, int d) const { return nb(x + d, nx, bc[0], bc[1]); }
  long yn(long y, int d) const { return nb(y + d, ny, bc[2], bc[3]); }
  bool ghost(long x) const { return inflow && x < 0; }
  // Flux component Q_{a,k} and velocity u_a at position (x, y) after the boundary rules.
  T Qat(int a, int k, long x, long y) const {
    if (ghost(x)) return qin[a * NC + k];
    return Qf[(size_t)(a * NC + k) * N + cell(xn(x, 0), yn(y, 0))];
  }
  T uat(int a, long x, long y) const {
    if (ghost(x)) return uin[a];
    return u[(size_t)a * N + cell(xn(x, 0), yn(y, 0))];
  }

  int set_inflow(const T* w) {
    T P_, cs2_;
    for (int k = 0; k < NC; ++k) win[k] = w[k];
    if (primitives_and_flux(D, eos, win, uin, &P_, &cs2_, qin)) return E_NONPHYSICAL;
    inflow = bc[0] == BC_INFLOW;
    return OK;
  }

  // Local activity s at (x, y) (Eqs. 28-31): central differences, j_k = dx (div Q)_k,
  // s_hat_k = j_k / M_k (taken as 0 where M_k = 0), s = sqrt(sum_k s_hat_k^2 / NC).
  T activity(long x, long y, const T* M) const {
    T acc = 0.0;
    for (int k = 0; k < NC; ++k) {
      T divq = 0.0;
      for (int a = 0; a < D; ++a) {
        T qp = a == 0 ? Qat(a, k, x + 1, y) : Qat(a, k, x, y + 1);
        T qm = a == 0 ? Qat(a, k, x - 1, y) : Qat(a, k, x, y - 1);
        divq = divq + (qp - qm) / (2.0 * dx);
      }
      T j = dx * divq;
      T sh = val(M[k]) != 0.0 ? j / M[k] : T(0.0);
      acc = acc + sh * sh;
    }
    return sqrt(acc / (double)NC);
  }

  // Ducros ratio at (x, y): dilatation and vorticity by central differences (Eq. 32), Eq. (33).
  T ducros(long x, long y) const {
    T dux_dx = (uat(0, x + 1, y) - uat(0, x - 1, y)) / (2.0 * dx);
    T duy_dy = (uat(1, x, y + 1) - uat(1, x, y - 1)) / (2.0 * dx);
    T duy_dx = (uat(1, x + 1, y) - uat(1, x - 1, y)) / (2.0 * dx);
    T dux_dy = (uat(0, x, y + 1) - uat(0, x, y - 1)) / (2.0 * dx);
    T dil = dux_dx + duy_dy;
    T vort = duy_dx - dux_dy;
    return dil * dil / (dil * dil + vort * vort + prm.ducros_eps);
  }

  void alloc() {
    Q = 2 * D;
    NC = D + 2;
    N = nx * ny;
    f.assign((size_t)Q * NC * N, T(0.0));
    fnext.assign((size_t)Q * NC * N, T(0.0));
    W.assign((size_t)NC * N, T(0.0));
    u.assign((size_t)D * N, T(0.0));
    P.assign(N, T(0.0));
    cs2.assign(N, T(0.0));
    Qf.assign((size_t)D * NC * N, T(0.0));
    s.assign(N, T(0.0));
    th.assign(N, T(0.0));
    tmp.assign(N, T(0.0));
    beta.assign(N, T(1.0));
  }

  // Steps 1-2 of the cycle: W = sum_i f_i (sum in i order, Sec. III A), then primitives,
  // EOS and flux at every cell.  Returns nonzero on a non-physical state (rho <= 0, c_s^2 <= 0).
  int moments_and_flux() {
    int bad = 0;
#pragma omp parallel for num_threads(nthreads) reduction(| : bad) schedule(static)
    for (long y = 0; y < ny; ++y)
      for (long x = 0; x < nx; ++x) {
        long c = cell(x, y);
        T Wc[4], uc[2], Qc[8], Pc, cc;
        for (int k = 0; k < NC; ++k) {
          T acc = 0.0;
          for (int i = 0; i < Q; ++i) acc = acc + f[fidx(i, k, c)];
          Wc[k] = acc;
          W[(size_t)k * N + c] = acc;
        }
        if (primitives_and_flux(D, eos, Wc, uc, &Pc, &cc, Qc)) {
          bad |= 1;
          continue;
        }
        for (int a = 0; a < D; ++a) u[(size_t)a * N + c] = uc[a];
        P[c] = Pc;
        cs2[c] = cc;
        for (int j = 0; j < D * NC; ++j) Qf[(size_t)j * N + c] = Qc[j];
      }
    return bad;
  }

  // s_max = max_x max_alpha (|u_alpha| + c_s) (Eq. 36).  The link speed is not differentiated,
  // so this works on values only.
  double smax() const {
    double m = 0.0;
#pragma omp parallel for num_threads(nthreads) reduction(max : m) schedule(static)
    for (long c = 0; c < N; ++c) {
      double cs = std::sqrt(val(cs2[c]));
      for (int a = 0; a < D; ++a) m = std::max(m, std::fabs(val(u[(size_t)a * N + c])) + cs);
    }
    return m;
  }

  // Shock sensor beta(x) (Sec. III D, Eqs. 28-35), or a constant beta.
  void sensor() {
    if (prm.beta_mode == BETA_CONST) {
      for (long c = 0; c < N; ++c) beta[c] = T(prm.beta_const);
      return;
    }
    // M_k = max_{x,alpha} |Q_alpha,k| (Eq. 30), scanned alpha-major, then y, then x; the first
    // maximal element wins (this fixes which element carries the derivative).
    T M[4];
    for (int k = 0; k < NC; ++k) {
      // per-row first maxima (in parallel), then combined in (alpha, y) order: the same element
      // as one serial scan
      std::vector<T> rowmax((size_t)D * ny, T(0.0));
#pragma omp parallel for num_threads(nthreads) schedule(static)
      for (long r = 0; r < (long)D * ny; ++r) {
        int a = (int)(r / ny);
        long y = r % ny;
        T m = 0.0;
        for (long x = 0; x < nx; ++x) {
          T q = fabs(Qf[(size_t)(a * NC + k) * N + cell(x, y)]);
          if (val(q) > val(m)) m = q;
        }
        rowmax[(size_t)r] = m;
      }
      T m = 0.0;
      for (long r = 0; r < (long)D * ny; ++r)
        if (val(rowmax[(size_t)r]) > val(m)) m = rowmax[(size_t)r];
      M[k] = m;
    }
    // Activity s (Eqs. 28-31) and, in 2D, the Ducros ratio theta (Eqs. 32-33) of every cell, and
    // of the ghost column x = -1 of a pinned-inflow side (read by the filter of column 0).
#pragma omp parallel for num_threads(nthreads) schedule(static)
    for (long y = 0; y < ny; ++y)
      for (long x = 0; x < nx; ++x) {
        long c = cell(x, y);
        s[c] = activity(x, y, M);
        if (D == 2) th[c] = ducros(x, y);
      }
    if (inflow) {
      s_gh.assign(ny, T(0.0));
      th_gh.assign(ny, T(0.0));
      for (long y = 0; y < ny; ++y) {
        s_gh[y] = activity(-1, y, M);
        if (D == 2) th_gh[y] = ducros(-1, y);
      }
    }
    if (keep_raw) {
      s_raw = s;
      th_raw = th;
    }
    box_filter(s, inflow ? s_gh.data() : nullptr);  // s_bar = S[s]
    if (D == 2) box_filter(th, inflow ? th_gh.data() : nullptr);  // theta_bar = S[theta]
    // Sensor A (1D, Eq. 34) / Sensor B (2D, Eq. 35).
#pragma omp parallel for num_threads(nthreads) schedule(static)
    for (long c = 0; c < N; ++c) {
      T arg = D == 2 ? prm.c_sensor * s[c] * th[c] : prm.c_sensor * s[c];
      T chi = clip01(arg);
      beta[c] = prm.beta_max - (prm.beta_max - prm.beta_min) * chi;
    }
  }

  // Separable one-cell box filter with weights (1/4, 1/2, 1/4), x first, then y (Sec. III D).
  // ghost_col: the values of the ghost column x = -1 of a pinned-inflow side (else nullptr).
  void box_filter(std::vector<T>& a, const T* ghost_col) {
#pragma omp parallel for num_threads(nthreads) schedule(static)
    for (long y = 0; y < ny; ++y)
      for (long x = 0; x < nx; ++x) {
        T left = (ghost_col && x == 0) ? ghost_col[y] : a[cell(xn(x, -1), y)];
        tmp[cell(x, y)] = 0.25 * left + 0.5 * a[cell(x, y)] + 0.25 * a[cell(xn(x, +1), y)];
      }
    if (D == 1) {
      a = tmp;
      return;
    }
#pragma omp parallel for num_threads(nthreads) schedule(static)
    for (long y = 0; y < ny; ++y)
      for (long x = 0; x < nx; ++x)
        a[cell(x, y)] = 0.25 * tmp[cell(x, yn(y, -1))] + 0.5 * tmp[cell(x, y)] + 0.25 * tmp[cell(x, yn(y, +1))];
  }

  // One time step, the cycle of Secs. III A and III E:
  //   1-2 W = sum_i f_i, EOS, flux;  3 s_max -> c_new, dt (Eqs. 36-37, final step shortened);
  //   4 reproject c_prev -> c_new (Eqs. 38-40);  5-6 sensor beta (Eqs. 28-35);
  //   7 relax towards f^eq(W; c_new) (Eqs. 20, 22);  8 stream (Eq. 21);  9 advance t.
  // last_out is set when the step landed on t_end.
  int step(double t_end, bool* last_out) {
    *last_out = false;
    if (moments_and_flux()) return E_NONPHYSICAL;
    double c_new, dt;
    bool last = false;
    if (!sched.empty()) {
      if ((size_t)n + 1 >= sched.size()) return E_NONPHYSICAL;
      c_new = sched[(size_t)n + 1];
      dt = dx / c_new;
    } else {
      bool retarget = prm.retarget_every <= 1 || (n % prm.retarget_every) == 0;
      c_new = retarget ? smax() / prm.cfl : c_prev;
      dt = dx / c_new;
      if (t_end > 0.0 && t + dt >= t_end) {  // final step shortened to land on t_end
        dt = t_end - t;
        c_new = dx / dt;
        last = true;
      }
    }
    if (!(c_new > 0.0) || !std::isfinite(c_new)) return E_NONPHYSICAL;
    // 4. reprojection, cell by cell.
#pragma omp parallel for num_threads(nthreads) schedule(static)
    for (long c = 0; c < N; ++c) {
      T fc[16];
      for (int i = 0; i < Q; ++i)
        for (int k = 0; k < NC; ++k) fc[i * NC + k] = f[fidx(i, k, c)];
      reproject(D, c_prev, c_new, fc);
      for (int i = 0; i < Q; ++i)
        for (int k = 0; k < NC; ++k) f[fidx(i, k, c)] = fc[i * NC + k];
    }
    // 5-6. sensor on the current W (flux already evaluated in step 1-2).
    sensor();
    // 7. relaxation (Eq. 22): f_i <- 2 beta f_i^eq(W) + (1 - 2 beta) f_i.
#pragma omp parallel for num_threads(nthreads) schedule(static)
    for (long c = 0; c < N; ++c) {
      T Wc[4], Qc[8], fe[4];
      for (int k = 0; k < NC; ++k) Wc[k] = W[(size_t)k * N + c];
      for (int j = 0; j < D * NC; ++j) Qc[j] = Qf[(size_t)j * N + c];
      T b2 = 2.0 * beta[c];
      for (int i = 0; i < Q; ++i) {
        feq(D, c_new, Wc, Qc, i, fe);
        for (int k = 0; k < NC; ++k) {
          T& fi = f[fidx(i, k, c)];
          fi = b2 * fe[k] + (1.0 - b2) * fi;
        }
      }
    }
    // 8. exact transport (Eq. 21): f_i(x) <- f_i(x - sigma_i), index rule at the boundary; from a
    // pinned-inflow ghost cell, the equilibrium of W_in at this step's link speed.
    std::vector<T>& g = fnext;
#pragma omp parallel for num_threads(nthreads) schedule(static)
    for (long y = 0; y < ny; ++y)
      for (long x = 0; x < nx; ++x)
        for (int i = 0; i < Q; ++i) {
          if (ghost(x - SIGMA[i][0])) {
            T fe[4];
            feq(D, c_new, win, qin, i, fe);
            for (int k = 0; k < NC; ++k) g[fidx(i, k, cell(x, y))] = fe[k];
            continue;
          }
          long src = cell(xn(x, -SIGMA[i][0]), D == 2 ? yn(y, -SIGMA[i][1]) : y);
          for (int k = 0; k < NC; ++k) g[fidx(i, k, cell(x, y))] = f[fidx(i, k, src)];
        }
    f.swap(g);
    // 9.
    t = last ? t_end : t + dt;
    c_prev = c_new;
    ++n;
    hist_dt.push_back(dt);
    hist_c.push_back(c_new);
    *last_out = last;
    return OK;
  }

  // Initial populations: equilibrium at the initial link speed c0 = s_max(W0)/CFL (Sec. III E).
  int init(const T* W0) {
    for (long c = 0; c < N; ++c)
      for (int k = 0; k < NC; ++k) W[(size_t)k * N + c] = W0[(size_t)k * N + c];
    int bad = 0;
    for (long c = 0; c < N; ++c) {
      T Wc[4], uc[2], Qc[8], Pc, cc;
      for (int k = 0; k < NC; ++k) Wc[k] = W[(size_t)k * N + c];
      if (primitives_and_flux(D, eos, Wc, uc, &Pc, &cc, Qc)) {
        bad = 1;
        break;
      }
      for (int a = 0; a < D; ++a) u[(size_t)a * N + c] = uc[a];
      cs2[c] = cc;
      for (int j = 0; j < D * NC; ++j) Qf[(size_t)j * N + c] = Qc[j];
    }
    if (bad) return E_NONPHYSICAL;
    double c0 = sched.empty() ? smax() / prm.cfl : sched[0];
    for (long c = 0; c < N; ++c) {
      T Wc[4], Qc[8], fe[4];
      for (int k = 0; k < NC; ++k) Wc[k] = W[(size_t)k * N + c];
      for (int j = 0; j < D * NC; ++j) Qc[j] = Qf[(size_t)j * N + c];
      for (int i = 0; i < Q; ++i) {
        feq(D, c0, Wc, Qc, i, fe);
        for (int k = 0; k < NC; ++k) f[fidx(i, k, c)] = fe[k];
      }
    }
    c_prev = c0;
    t = 0.0;
    n = 0;
    hist_dt.clear();
    hist_c.clear();
    return OK;
  }
};

}  // namespace orc

using namespace orc;

// ------------------------------------------------------------------------------------------
// C entry points for the Python test harness (ctypes).  eos6 = {kind, gamma, a, b, R, cv, cv1, cv2};
// prm8 = {cfl, beta_mode, beta_const, beta_min, beta_max, c_sensor, ducros_eps, retarget_every};
// field arrays are [component][y][x]; populations [i][k][y][x].
// ------------------------------------------------------------------------------------------
template <class T>
static Eos<T> make_eos(const double* e6, const double* de6) {
  Eos<T> q;
  q.kind = (int)e6[0];
  q.gamma = T(e6[1]);
  q.a = T(e6[2]);
  q.b = T(e6[3]);
  q.R = T(e6[4]);
  q.cv = T(e6[5]);
  q.cv1 = T(e6[6]);
  q.cv2 = T(e6[7]);
  if (de6) {
    if constexpr (std::is_same<T, Dual>::value) {
      q.gamma.d = de6[1];
      q.a.d = de6[2];
      q.b.d = de6[3];
      q.R.d = de6[4];
      q.cv.d = de6[5];
      q.cv1.d = de6[6];
      q.cv2.d = de6[7];
    }
  }
  return q;
}

static Params make_params(const double* p8) {
  Params p;
  p.cfl = p8[0];
  p.beta_mode = (int)p8[1];
  p.beta_const = p8[2];
  p.beta_min = p8[3];
  p.beta_max = p8[4];
  p.c_sensor = p8[5];
  p.ducros_eps = p8[6];
  p.retarget_every = (int)p8[7];
  return p;
}

template <class T>
static Solver<T>* create_solver(int dim, long nx, long ny, double dx, const int* bc4, const double* eos6,
                                const double* deos6, const double* prm8) {
  auto* s = new Solver<T>();
  s->D = dim;
  s->nx = nx;
  s->ny = dim == 1 ? 1 : ny;
  s->dx = dx;
  for (int j = 0; j < 4; ++j) s->bc[j] = bc4[j];
  s->eos = make_eos<T>(eos6, deos6);
  s->prm = make_params(prm8);
  s->alloc();
  return s;
}

extern "C" {

void orc_set_threads(void* h, int n) { static_cast<Solver<double>*>(h)->nthreads = n < 1 ? 1 : n; }
int orc_max_threads() {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void* orc_create(int dim, long nx, long ny, double dx, const int* bc4, const double* eos6, const double* prm8) {
  return create_solver<double>(dim, nx, ny, dx, bc4, eos6, nullptr, prm8);
}
void orc_destroy(void* h) { delete static_cast<Solver<double>*>(h); }
int orc_init(void* h, const double* W0) { return static_cast<Solver<double>*>(h)->init(W0); }

// Runs up to n_steps steps, stopping early once t reaches t_end (t_end <= 0: no end time).
int orc_step(void* h, long n_steps, double t_end, long* done) {
  auto* s = static_cast<Solver<double>*>(h);
  long k = 0;
  int st = OK;
  for (; k < n_steps; ++k) {
    if (t_end > 0.0 && s->t >= t_end) break;
    bool last;
    st = s->step(t_end, &last);
    if (st != OK) break;
  }
  if (done) *done = k;
  return st;
}

void orc_get_W(void* h, double* W) {
  auto* s = static_cast<Solver<double>*>(h);
  for (long c = 0; c < s->N; ++c)
    for (int k = 0; k < s->NC; ++k) {
      double acc = 0.0;
      for (int i = 0; i < s->Q; ++i) acc = acc + s->f[s->fidx(i, k, c)];
      W[(size_t)k * s->N + c] = acc;
    }
}
void orc_get_f(void* h, double* f) {
  auto* s = static_cast<Solver<double>*>(h);
  std::memcpy(f, s->f.data(), s->f.size() * sizeof(double));
}
void orc_set_state(void* h, const double* f, double c_prev, double t, long n) {
  auto* s = static_cast<Solver<double>*>(h);
  std::memcpy(s->f.data(), f, s->f.size() * sizeof(double));
  s->c_prev = c_prev;
  s->t = t;
  s->n = n;
}
void orc_get_beta(void* h, double* b) {
  auto* s = static_cast<Solver<double>*>(h);
  for (long c = 0; c < s->N; ++c) b[c] = s->beta[c];
}
// beta(x) of the current state at a given link speed, without advancing (diagnostic).
int orc_eval_beta(void* h, double* b) {
  auto* s = static_cast<Solver<double>*>(h);
  if (s->moments_and_flux()) return E_NONPHYSICAL;
  s->sensor();
  for (long c = 0; c < s->N; ++c) b[c] = s->beta[c];
  return OK;
}
// The shock sensor's fields of the current state (diagnostic for the pins): the activity s and
// the Ducros ratio theta before the box filter, their filtered values s_bar and theta_bar, and
// beta (Eqs. 31, 33-35).  1D: theta and theta_bar are returned as 0 (Sensor A has no gate).
int orc_eval_sensor_fields(void* h, double* s_out, double* th_out, double* sbar_out, double* thbar_out, double* b) {
  auto* s = static_cast<Solver<double>*>(h);
  if (s->moments_and_flux()) return E_NONPHYSICAL;
  s->keep_raw = true;
  s->sensor();
  s->keep_raw = false;
  for (long c = 0; c < s->N; ++c) {
    s_out[c] = s->s_raw[c];
    th_out[c] = s->D == 2 ? s->th_raw[c] : 0.0;
    sbar_out[c] = s->s[c];
    thbar_out[c] = s->D == 2 ? s->th[c] : 0.0;
    b[c] = s->beta[c];
  }
  return OK;
}
void orc_get_time(void* h, double* t, long* n, double* c_prev) {
  auto* s = static_cast<Solver<double>*>(h);
  *t = s->t;
  *n = s->n;
  *c_prev = s->c_prev;
}
long orc_get_hist(void* h, double* dt, double* c, long cap) {
  auto* s = static_cast<Solver<double>*>(h);
  long m = std::min<long>(cap, (long)s->hist_dt.size());
  for (long j = 0; j < m; ++j) {
    dt[j] = s->hist_dt[j];
    c[j] = s->hist_c[j];
  }
  return (long)s->hist_dt.size();
}
// State W_in (D+2 values) held by the ghost cells of a pinned-inflow x-lo side (Sec. IV H).
int orc_set_inflow(void* h, const double* w) { return static_cast<Solver<double>*>(h)->set_inflow(w); }
int orc_dual_set_inflow(void* h, const double* w) {
  auto* s = static_cast<Solver<Dual>*>(h);
  Dual wd[4];
  for (int k = 0; k < s->NC; ++k) wd[k] = Dual(w[k]);
  return s->set_inflow(wd);
}
// Replay a fixed link-speed sequence: entry 0 is the initial link speed c0, entry j >= 1 the
// link speed of step j-1 (a free run's history prefixed with its c0 replays that run).
void orc_set_schedule(void* h, const double* c, long n) {
  static_cast<Solver<double>*>(h)->sched.assign(c, c + n);
}

// --- point functions for the pins ---
void orc_eos_eval(const double* eos6, double rho, double e, double* P, double* cs2) {
  Eos<double> q = make_eos<double>(eos6, nullptr);
  eos_eval(q, rho, e, P, cs2);
}
double orc_fundamental_derivative(const double* eos6, double rho, double e) {
  return fundamental_derivative(make_eos<double>(eos6, nullptr), rho, e);
}
// Flux of one state W (length D+2) -> Qf[alpha*(D+2)+k]; returns nonzero if non-physical.
int orc_flux(int dim, const double* eos6, const double* W, double* Qf) {
  Eos<double> q = make_eos<double>(eos6, nullptr);
  double u[2], P, cs2;
  return primitives_and_flux(dim, q, W, u, &P, &cs2, Qf);
}
// f_i^eq of one state at link speed c -> out[i*(D+2)+k].
int orc_feq(int dim, const double* eos6, double c, const double* W, double* out) {
  Eos<double> q = make_eos<double>(eos6, nullptr);
  double u[2], P, cs2, Qf[8];
  if (primitives_and_flux(dim, q, W, u, &P, &cs2, Qf)) return E_NONPHYSICAL;
  for (int i = 0; i < 2 * dim; ++i) feq(dim, c, W, Qf, i, out + i * (dim + 2));
  return OK;
}
// Reprojection of one cell's populations f[i*(D+2)+k] in place.
void orc_reproject(int dim, double c_old, double c_new, double* f) { reproject(dim, c_old, c_new, f); }

// --- dual-number (forward-mode) solver: same code path in Dual arithmetic.  Requires a
// replayed link-speed schedule (the link speed is not differentiated).  deos6 seeds the EOS
// parameter derivatives, dW0 the initial-field direction.
void* orc_dual_create(int dim, long nx, long ny, double dx, const int* bc4, const double* eos6, const double* deos6,
                      const double* prm8) {
  return create_solver<Dual>(dim, nx, ny, dx, bc4, eos6, deos6, prm8);
}
void orc_dual_destroy(void* h) { delete static_cast<Solver<Dual>*>(h); }
void orc_dual_set_threads(void* h, int n) { static_cast<Solver<Dual>*>(h)->nthreads = n < 1 ? 1 : n; }
void orc_dual_set_schedule(void* h, const double* c, long n) { static_cast<Solver<Dual>*>(h)->sched.assign(c, c + n); }
int orc_dual_init(void* h, const double* W0, const double* dW0) {
  auto* s = static_cast<Solver<Dual>*>(h);
  std::vector<Dual> w((size_t)s->NC * s->N);
  for (size_t j = 0; j < w.size(); ++j) w[j] = Dual(W0[j], dW0 ? dW0[j] : 0.0);
  return s->init(w.data());
}
int orc_dual_step(void* h, long n_steps, long* done) {
  auto* s = static_cast<Solver<Dual>*>(h);
  long k = 0;
  int st = OK;
  for (; k < n_steps; ++k) {
    bool last;
    st = s->step(0.0, &last);
    if (st != OK) break;
  }
  if (done) *done = k;
  return st;
}
void orc_dual_get_W(void* h, double* W, double* dW) {
  auto* s = static_cast<Solver<Dual>*>(h);
  for (long c = 0; c < s->N; ++c)
    for (int k = 0; k < s->NC; ++k) {
      Dual acc = 0.0;
      for (int i = 0; i < s->Q; ++i) acc = acc + s->f[s->fidx(i, k, c)];
      W[(size_t)k * s->N + c] = acc.v;
      dW[(size_t)k * s->N + c] = acc.d;
    }
}
}
