// ORACLE: test infrastructure only.
//
// Independent reference solver for the one-dimensional benchmarks (Secs. IV B-IV D): a
// second-order finite-volume method unrelated to the lattice Boltzmann scheme, of the kind the
// paper validates against -- MUSCL reconstruction of the primitive variables (rho, u, P) with
// the minmod limiter (van Leer 1979), the Rusanov (local Lax-Friedrichs) interface flux
// (Rusanov 1961) and the two-stage second-order Runge-Kutta method of Heun (the strong-stability-
// preserving form of Shu & Osher 1988).  The closure is the oracle's own equation of state
// (orc_eos_eval, Eqs. 11-17), as the paper's reference solver uses the VLBM run's EOS routines.
//
// Readings (the paper names the method but not these details): the reference time step is
// dt = CFL dx / max_j(|u_j| + c_j) with CFL = cfl (0.4 by default), taken from the state at the
// start of the step, and the last step is shortened to land on t_end; boundaries are two ghost
// cells per side, copies of the edge cell (zero gradient) or the periodic images; the interface
// wave speed is max(|u_L| + c_L, |u_R| + c_R) of the two reconstructed states, with c^2 < 0 of a
// reconstructed state (possible near the van der Waals spinodal) counted as 0.
//
// Pins: tests/test_oracle_muscl.py (the exact Riemann solution of the Sod problem, the second-
// order convergence on a smooth periodic wave, conservation on a periodic domain).
#include <algorithm>
#include <cmath>
#include <vector>

extern "C" void orc_eos_eval(const double* eos6, double rho, double e, double* P, double* cs2);

namespace {

// Specific internal energy of (rho, P), the EOS solved for e: ideal gas e = P / ((gamma-1) rho)
// (Eq. 15); van der Waals T = (P + a rho^2)(1 - b rho) / (R rho) from Eq. (16), then
// e = cv T - a rho (Eq. 17), or e = cv T + cv1 T^2/2 + cv2 T^3/3 - a rho for c_v(T) = cv + cv1 T + cv2 T^2.
double energy_of(const double* e6, double rho, double P) {
  if (e6[0] == 0.0) return P / ((e6[1] - 1.0) * rho);
  const double a = e6[2], b = e6[3], R = e6[4], cv = e6[5], cv1 = e6[6], cv2 = e6[7];
  const double T = (P + a * rho * rho) * (1.0 - b * rho) / (R * rho);
  return cv * T + cv1 * T * T / 2.0 + cv2 * T * T * T / 3.0 - a * rho;
}

inline double minmod(double l, double r) {
  if (l * r <= 0.0) return 0.0;
  return std::fabs(l) < std::fabs(r) ? l : r;
}

struct Muscl {
  const double* e6;
  int n, bc;  // bc: 0 periodic, 1 zero gradient
  double dx;
  std::vector<double> V;  // primitives (rho, u, P) of n + 4 cells (two ghosts per side)

  int ghost(int j) const {  // cell index of padded position j (0..n+3)
    int i = j - 2;
    if (i < 0) return bc == 0 ? i + n : 0;
    if (i >= n) return bc == 0 ? i - n : n - 1;
    return i;
  }

  // Primitives of every cell of U (3 x n, conserved); returns the largest |u| + c, or -1 if a
  // cell is not physical (rho <= 0, c^2 <= 0 or non-finite).
  double primitives(const std::vector<double>& U) {
    double smax = 0.0;
    bool bad = false;
#pragma omp parallel for reduction(max : smax) reduction(|| : bad)
    for (int i = 0; i < n; ++i) {
      const double rho = U[i], m = U[n + i], E = U[2 * n + i];
      const double u = m / rho, e = E / rho - 0.5 * u * u;
      double P, c2;
      orc_eos_eval(e6, rho, e, &P, &c2);
      if (!(rho > 0.0) || !(c2 > 0.0) || !std::isfinite(P)) bad = true;
      V[3 * (i + 2) + 0] = rho;
      V[3 * (i + 2) + 1] = u;
      V[3 * (i + 2) + 2] = P;
      smax = std::max(smax, std::fabs(u) + std::sqrt(std::max(c2, 0.0)));
    }
    if (bad) return -1.0;
    for (int j : {0, 1, n + 2, n + 3})
      for (int k = 0; k < 3; ++k) V[3 * j + k] = V[3 * (ghost(j) + 2) + k];
    return smax;
  }

  // Conserved state, flux and |u| + c of one primitive state.
  void state(double rho, double u, double P, double* U, double* F, double* s) const {
    const double e = energy_of(e6, rho, P);
    double Pe, c2;
    orc_eos_eval(e6, rho, e, &Pe, &c2);
    const double E = rho * (e + 0.5 * u * u);
    U[0] = rho, U[1] = rho * u, U[2] = E;
    F[0] = rho * u, F[1] = rho * u * u + P, F[2] = (E + P) * u;
    *s = std::fabs(u) + std::sqrt(std::max(c2, 0.0));
  }

  // L(U) = -(F_{i+1/2} - F_{i-1/2}) / dx for the primitives in V.
  void rhs(std::vector<double>& L) const {
    std::vector<double> Fh(3 * (n + 1));
#pragma omp parallel for
    for (int f = 0; f <= n; ++f) {  // interface between padded cells f+1 and f+2
      const int jl = f + 1, jr = f + 2;
      double vl[3], vr[3];
      for (int k = 0; k < 3; ++k) {
        const double sl = minmod(V[3 * jl + k] - V[3 * (jl - 1) + k], V[3 * (jl + 1) + k] - V[3 * jl + k]);
        const double sr = minmod(V[3 * jr + k] - V[3 * (jr - 1) + k], V[3 * (jr + 1) + k] - V[3 * jr + k]);
        vl[k] = V[3 * jl + k] + 0.5 * sl;
        vr[k] = V[3 * jr + k] - 0.5 * sr;
      }
      double Ul[3], Ur[3], Fl[3], Fr[3], al, ar;
      state(vl[0], vl[1], vl[2], Ul, Fl, &al);
      state(vr[0], vr[1], vr[2], Ur, Fr, &ar);
      const double a = std::max(al, ar);
      for (int k = 0; k < 3; ++k) Fh[3 * f + k] = 0.5 * (Fl[k] + Fr[k]) - 0.5 * a * (Ur[k] - Ul[k]);
    }
#pragma omp parallel for
    for (int i = 0; i < n; ++i)
      for (int k = 0; k < 3; ++k) L[k * n + i] = -(Fh[3 * (i + 1) + k] - Fh[3 * i + k]) / dx;
  }
};

}  // namespace

extern "C" {

// Advances the conserved field W (3 x n, [rho, rho u, rho E][x]) of a 1D problem on a uniform
// grid of spacing dx from t = 0 to t_end.  Returns 0, or 1 if a non-physical state occurred
// (W then holds the last physical state).  *steps receives the number of steps taken.
int orc_muscl_1d(const double* e6, int n, double dx, int bc, double cfl, double t_end, double* W, long* steps) {
  Muscl m{e6, n, bc, dx, std::vector<double>(3 * (n + 4))};
  std::vector<double> U(W, W + 3 * n), U1(3 * n), L(3 * n);
  double t = 0.0;
  long s = 0;
  while (t < t_end) {
    const double smax = m.primitives(U);
    if (smax < 0.0) break;
    double dt = cfl * dx / smax;
    const bool last = t + dt >= t_end;
    if (last) dt = t_end - t;
    m.rhs(L);
    for (int j = 0; j < 3 * n; ++j) U1[j] = U[j] + dt * L[j];  // Heun stage 1
    if (m.primitives(U1) < 0.0) break;
    m.rhs(L);
    for (int j = 0; j < 3 * n; ++j) U[j] = 0.5 * U[j] + 0.5 * (U1[j] + dt * L[j]);  // stage 2
    t = last ? t_end : t + dt;
    ++s;
  }
  *steps = s;
  std::copy(U.begin(), U.end(), W);
  return t < t_end ? 1 : 0;
}

// Two-dimensional form on an nx x ny grid of square cells (spacing dx), zero-gradient on every
// side (two edge-copy ghost layers), without dimensional splitting: the same primitive minmod
// reconstruction and Rusanov flux across every x face (speed |u| + c) and every y face
// (|v| + c), summed into one update, Heun RK2 in time.  The step is
// dt = cfl dx / max_cells(|u| + |v| + 2c), the sum form of the unsplit stability limit.
// W is [rho, rho u, rho v, rho E][y][x].  bc4 = (x-lo, x-hi, y-lo, y-hi): 0 periodic, 1 zero-gradient
// (edge copy), 2 pinned (both ghost cells hold the conserved state win, the inflow boundary of
// Sec. IV H).  Returns 0, or 1 if a non-physical state occurred.
int orc_muscl_2d_bc(const double* e6, int nx, int ny, double dx, double cfl, double t_end, const int* bc4,
                    const double* win, double* W, long* steps) {
  const long N = (long)nx * ny;
  const int PX = nx + 4, PY = ny + 4;
  std::vector<double> V((size_t)4 * PX * PY), U(W, W + 4 * N), U1(4 * N), L(4 * N);
  double vpin[4] = {0.0, 0.0, 0.0, 0.0};  // primitives (rho, u, v, P) of the pinned state
  if (win) {
    const double rho = win[0], u = win[1] / rho, v = win[2] / rho, e = win[3] / rho - 0.5 * (u * u + v * v);
    double P, c2;
    orc_eos_eval(e6, rho, e, &P, &c2);
    vpin[0] = rho, vpin[1] = u, vpin[2] = v, vpin[3] = P;
  }
  auto vi = [&](int k, int y, int x) -> double& { return V[((size_t)k * PY + y) * PX + x]; };
  // primitives with ghosts; returns max(|u| + |v| + 2c) or -1 if not physical
  auto prim = [&](const std::vector<double>& Uc) -> double {
    double smax = 0.0;
    bool bad = false;
#pragma omp parallel for reduction(max : smax) reduction(|| : bad)
    for (int y = 0; y < ny; ++y)
      for (int x = 0; x < nx; ++x) {
        const long c = (long)y * nx + x;
        const double rho = Uc[c], u = Uc[N + c] / rho, v = Uc[2 * N + c] / rho;
        const double e = Uc[3 * N + c] / rho - 0.5 * (u * u + v * v);
        double P, c2;
        orc_eos_eval(e6, rho, e, &P, &c2);
        if (!(rho > 0.0) || !(c2 > 0.0) || !std::isfinite(P)) bad = true;
        vi(0, y + 2, x + 2) = rho, vi(1, y + 2, x + 2) = u, vi(2, y + 2, x + 2) = v, vi(3, y + 2, x + 2) = P;
        smax = std::max(smax, std::fabs(u) + std::fabs(v) + 2.0 * std::sqrt(std::max(c2, 0.0)));
      }
    if (bad) return -1.0;
    // ghost cells: periodic images, edge copies, or the pinned state
    for (int k = 0; k < 4; ++k)
      for (int y = 0; y < PY; ++y)
        for (int x = 0; x < PX; ++x) {
          int sy = y, sx = x, side = -1;
          if (x < 2) side = 0;
          if (x > nx + 1) side = 1;
          if (side >= 0) sx = bc4[side] == 0 ? (side == 0 ? x + nx : x - nx) : (side == 0 ? 2 : nx + 1);
          if (y < 2) sy = bc4[2] == 0 ? y + ny : 2;
          if (y > ny + 1) sy = bc4[3] == 0 ? y - ny : ny + 1;
          if (sy == y && sx == x) continue;
          vi(k, y, x) = (side >= 0 && bc4[side] == 2) ? vpin[k] : vi(k, sy, sx);
        }
    return smax;
  };
  // Rusanov flux across the face between padded cells a (left/below) and b, normal direction d
  // (0: x, 1: y); (ya, xa) and the step (oy, ox) towards b give the four-cell stencil
  auto face = [&](int ya, int xa, int oy, int ox, int d, double* F) {
    double vl[4], vr[4];
    for (int k = 0; k < 4; ++k) {
      const double a0 = vi(k, ya - oy, xa - ox), a1 = vi(k, ya, xa), a2 = vi(k, ya + oy, xa + ox),
                   a3 = vi(k, ya + 2 * oy, xa + 2 * ox);
      vl[k] = a1 + 0.5 * minmod(a1 - a0, a2 - a1);
      vr[k] = a2 - 0.5 * minmod(a2 - a1, a3 - a2);
    }
    double Ul[4], Ur[4], Fl[4], Fr[4], sl, sr;
    for (int side = 0; side < 2; ++side) {
      const double* q = side ? vr : vl;
      double* Uo = side ? Ur : Ul;
      double* Fo = side ? Fr : Fl;
      const double e = energy_of(e6, q[0], q[3]);
      double Pe, c2;
      orc_eos_eval(e6, q[0], e, &Pe, &c2);
      const double un = d == 0 ? q[1] : q[2];
      const double E = q[0] * (e + 0.5 * (q[1] * q[1] + q[2] * q[2]));
      Uo[0] = q[0], Uo[1] = q[0] * q[1], Uo[2] = q[0] * q[2], Uo[3] = E;
      Fo[0] = q[0] * un, Fo[1] = q[0] * q[1] * un, Fo[2] = q[0] * q[2] * un, Fo[3] = (E + q[3]) * un;
      Fo[1 + d] += q[3];
      (side ? sr : sl) = std::fabs(un) + std::sqrt(std::max(c2, 0.0));
    }
    const double a = std::max(sl, sr);
    for (int k = 0; k < 4; ++k) F[k] = 0.5 * (Fl[k] + Fr[k]) - 0.5 * a * (Ur[k] - Ul[k]);
  };
  // each face flux once: x faces (nx + 1 per row), y faces (ny + 1 per column)
  std::vector<double> Fx((size_t)4 * ny * (nx + 1)), Fy((size_t)4 * (ny + 1) * nx);
  auto rhs = [&]() {
#pragma omp parallel for
    for (int y = 0; y < ny; ++y)
      for (int f = 0; f <= nx; ++f) {
        double F[4];
        face(y + 2, f + 1, 0, 1, 0, F);  // between cells f - 1 and f of row y
        for (int k = 0; k < 4; ++k) Fx[((size_t)k * ny + y) * (nx + 1) + f] = F[k];
      }
#pragma omp parallel for
    for (int g = 0; g <= ny; ++g)
      for (int x = 0; x < nx; ++x) {
        double F[4];
        face(g + 1, x + 2, 1, 0, 1, F);  // between rows g - 1 and g of column x
        for (int k = 0; k < 4; ++k) Fy[((size_t)k * (ny + 1) + g) * nx + x] = F[k];
      }
#pragma omp parallel for
    for (int y = 0; y < ny; ++y)
      for (int x = 0; x < nx; ++x) {
        const long c = (long)y * nx + x;
        for (int k = 0; k < 4; ++k) {
          const double* fx = &Fx[((size_t)k * ny + y) * (nx + 1)];
          const double* fy = &Fy[(size_t)k * (ny + 1) * nx];
          L[k * N + c] = -((fx[x + 1] - fx[x]) + (fy[(size_t)(y + 1) * nx + x] - fy[(size_t)y * nx + x])) / dx;
        }
      }
  };
  double t = 0.0;
  long s = 0;
  while (t < t_end) {
    const double smax = prim(U);
    if (smax < 0.0) break;
    double dt = cfl * dx / smax;
    const bool last = t + dt >= t_end;
    if (last) dt = t_end - t;
    rhs();
    for (long j = 0; j < 4 * N; ++j) U1[j] = U[j] + dt * L[j];
    if (prim(U1) < 0.0) break;
    rhs();
    for (long j = 0; j < 4 * N; ++j) U[j] = 0.5 * U[j] + 0.5 * (U1[j] + dt * L[j]);
    t = last ? t_end : t + dt;
    ++s;
  }
  *steps = s;
  std::copy(U.begin(), U.end(), W);
  return t < t_end ? 1 : 0;
}

// Zero-gradient on every side.
int orc_muscl_2d(const double* e6, int nx, int ny, double dx, double cfl, double t_end, double* W, long* steps) {
  const int zg[4] = {1, 1, 1, 1};
  return orc_muscl_2d_bc(e6, nx, ny, dx, cfl, t_end, zg, nullptr, W, steps);
}

}  // extern "C"
