// Plain, slow FP64 CPU oracle for the lattice-Boltzmann step with
// velocity-interpolation bounce-back (Jin et al., arXiv:1903.01111).
//
// TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
// call this file; only the tests, the package smoke check and the benchmark's
// CPU-baseline leg do.  It shares no code, header or table with the CUDA
// library: the velocity sets, weights and every formula are written out here
// a second time, in the paper's order and notation.
//
// Form of the step (push form, whole-array passes, no fusion):
//   state at time t: post-collision populations f+_i(x,t) at every fluid node
//   and the moments rho(x,t), u(x,t) that the collision at t used.
//   1. open boundary columns at t (Sec. 4.3: non-equilibrium extrapolation
//      inlet, zero-gradient outlet)
//   2. streaming by push, Eq. (1):  f_i(x+e_i, t+1) = f+_i(x, t)
//   3. each cut link rebuilds its missing population (Sec. 3, Eqs. q_less,
//      q_larger, Yu's two equations, and the VIBB equations of Sec. 3.1);
//      momentum exchange force
//   4. moments (Sec. 2, density and velocity sums; velocity shifted by half the
//      body force, Guo forcing) and BGK collision (Sec. 2, Eq. feq), or the
//      MRT collision of Eq. (mrt) with the relaxation rates of Sec. 2.
//
// The scalar type is a template parameter so that a forward-mode (dual number)
// instantiation can be added without touching the arithmetic.
//
// Parity pins: see tests/test_oracle_pins.py (every function here is pinned
// there by a closed form, an invariant or a special case).
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

// ---------------------------------------------------------------- lattices --
// D2Q9 in the order fixed by the moment matrix M of Sec. 2:
// e1=(1,0) e2=(0,1) e3=(-1,0) e4=(0,-1) e5=(1,1) e6=(-1,1) e7=(-1,-1) e8=(1,-1).
const int kE2[9][3] = {{0, 0, 0},  {1, 0, 0},  {0, 1, 0},   {-1, 0, 0}, {0, -1, 0},
                       {1, 1, 0},  {-1, 1, 0}, {-1, -1, 0}, {1, -1, 0}};
const double kW2[9] = {4.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0, 1.0 / 9.0,
                       1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};
// D3Q19 (the paper is 2-D only): rest, 6 axis, 12 face-diagonal velocities,
// opposite directions adjacent.
const int kE3[19][3] = {{0, 0, 0},  {1, 0, 0},   {-1, 0, 0},  {0, 1, 0},  {0, -1, 0},
                        {0, 0, 1},  {0, 0, -1},  {1, 1, 0},   {-1, -1, 0}, {1, -1, 0},
                        {-1, 1, 0}, {1, 0, 1},   {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
                        {0, 1, 1},  {0, -1, -1}, {0, 1, -1},  {0, -1, 1}};
const double kW3[19] = {1.0 / 3.0,  1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0,
                        1.0 / 18.0, 1.0 / 18.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0,
                        1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0,
                        1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};

// The D2Q9 moment matrix M of Eq. (M), rows m0..m8 =
// (rho, e, epsilon, j_x, q_x, j_y, q_y, p_xx, p_xy).
const double kM[9][9] = {{1, 1, 1, 1, 1, 1, 1, 1, 1},     {-4, -1, -1, -1, -1, 2, 2, 2, 2},
                         {4, -2, -2, -2, -2, 1, 1, 1, 1}, {0, 1, 0, -1, 0, 1, -1, -1, 1},
                         {0, -2, 0, 2, 0, 1, -1, -1, 1},  {0, 0, 1, 0, -1, 1, 1, -1, -1},
                         {0, 0, -2, 0, 2, 1, 1, -1, -1},  {0, 1, -1, 1, -1, 0, 0, 0, 0},
                         {0, 0, 0, 0, 0, 1, -1, 1, -1}};

enum { BC_HALFWAY = 0, BC_BOUZIDI = 1, BC_VIBB = 2, BC_YU = 3 };
enum { NODE_FLUID = 0, NODE_SOLID = 1, NODE_INLET = 2, NODE_OUTLET = 3 };

}  // namespace

extern "C" {

// Own definition of the run configuration (same field order as the library's
// lbm_config; kept alike because both read the same test inputs).
struct oracle_config {
  int32_t stencil;    // 0 = D2Q9, 1 = D3Q19
  int32_t collision;  // 0 = BGK, 1 = MRT (D2Q9 only)
  int32_t bc;         // default link rule: 0 half-way, 1 Bouzidi, 2 VIBB, 3 Yu
  int32_t nx, ny, nz;
  int32_t periodic[3];
  int32_t inlet;   // 1: column x = 0 is a velocity inlet (D2Q9)
  int32_t outlet;  // 1: column x = nx-1 is a zero-gradient outlet (D2Q9)
  double tau, rho0;
  double g[3];                // body force per unit volume
  double inlet_umax;          // peak of the parabolic inflow
  double inlet_y0, inlet_y1;  // wall positions bounding the inflow parabola
  int32_t precision;          // unused by the oracle (always FP64)
  int32_t vibb_density;       // 0: rho_d as printed for every q; 1: rho_d = rho_f when q > 1/2
};

// Own definition of one cut link (same layout as the library's lbm_link).
struct oracle_link {
  int64_t node;  // fluid node x_f
  int32_t dir;   // i': direction from x_f towards the solid node
  int16_t bc;    // rule for this link, or -1 for the configuration default
  int16_t body;  // force accumulator index, or -1
  double q;      // |x_f - x_w| / |x_f - x_s|
  double uw[3];  // wall velocity at x_w
};

}  // extern "C"

namespace {

// Forward-mode dual number with K derivative components: every arithmetic
// operation applies the chain rule to the derivative part.
template <int K>
struct Dual {
  double v;
  double d[K];
  Dual(double x = 0.0) : v(x) {
    for (int k = 0; k < K; ++k) d[k] = 0.0;
  }
};
template <int K>
Dual<K> operator+(const Dual<K>& a, const Dual<K>& b) {
  Dual<K> r(a.v + b.v);
  for (int k = 0; k < K; ++k) r.d[k] = a.d[k] + b.d[k];
  return r;
}
template <int K>
Dual<K> operator-(const Dual<K>& a, const Dual<K>& b) {
  Dual<K> r(a.v - b.v);
  for (int k = 0; k < K; ++k) r.d[k] = a.d[k] - b.d[k];
  return r;
}
template <int K>
Dual<K> operator-(const Dual<K>& a) {
  Dual<K> r(-a.v);
  for (int k = 0; k < K; ++k) r.d[k] = -a.d[k];
  return r;
}
template <int K>
Dual<K> operator*(const Dual<K>& a, const Dual<K>& b) {
  Dual<K> r(a.v * b.v);
  for (int k = 0; k < K; ++k) r.d[k] = a.d[k] * b.v + a.v * b.d[k];
  return r;
}
template <int K>
Dual<K> operator/(const Dual<K>& a, const Dual<K>& b) {
  Dual<K> r(a.v / b.v);
  for (int k = 0; k < K; ++k) r.d[k] = (a.d[k] * b.v - a.v * b.d[k]) / (b.v * b.v);
  return r;
}
template <int K> Dual<K> operator+(const Dual<K>& a, double b) { return a + Dual<K>(b); }
template <int K> Dual<K> operator+(double a, const Dual<K>& b) { return Dual<K>(a) + b; }
template <int K> Dual<K> operator-(const Dual<K>& a, double b) { return a - Dual<K>(b); }
template <int K> Dual<K> operator-(double a, const Dual<K>& b) { return Dual<K>(a) - b; }
template <int K> Dual<K> operator*(const Dual<K>& a, double b) { return a * Dual<K>(b); }
template <int K> Dual<K> operator*(double a, const Dual<K>& b) { return Dual<K>(a) * b; }
template <int K> Dual<K> operator/(const Dual<K>& a, double b) { return a / Dual<K>(b); }
template <int K> Dual<K> operator/(double a, const Dual<K>& b) { return Dual<K>(a) / b; }
template <int K> bool operator<=(const Dual<K>& a, double b) { return a.v <= b; }
template <int K> bool operator>(const Dual<K>& a, double b) { return a.v > b; }

inline double value_of(double x) { return x; }
template <int K>
double value_of(const Dual<K>& x) {
  return x.v;
}

template <class T>
struct Oracle {
  oracle_config c;
  T tau;  // relaxation time (a scalar of type T so that it can carry derivatives)
  int Q, D;
  int e[19][3];
  double w[19];
  int opp[19];
  int64_t N;

  explicit Oracle(const oracle_config& cfg) : c(cfg), tau(cfg.tau) {
    if (c.stencil == 0) {
      Q = 9;
      D = 2;
      for (int i = 0; i < 9; ++i) {
        for (int a = 0; a < 3; ++a) e[i][a] = kE2[i][a];
        w[i] = kW2[i];
      }
    } else {
      Q = 19;
      D = 3;
      for (int i = 0; i < 19; ++i) {
        for (int a = 0; a < 3; ++a) e[i][a] = kE3[i][a];
        w[i] = kW3[i];
      }
    }
    for (int i = 0; i < Q; ++i)
      for (int j = 0; j < Q; ++j)
        if (e[j][0] == -e[i][0] && e[j][1] == -e[i][1] && e[j][2] == -e[i][2]) opp[i] = j;
    N = (int64_t)c.nx * c.ny * c.nz;
  }

  void coords(int64_t n, int64_t x[3]) const {
    x[0] = n % c.nx;
    x[1] = (n / c.nx) % c.ny;
    x[2] = n / ((int64_t)c.nx * c.ny);
  }
  // Neighbour x + s*e_i, wrapped on periodic axes; -1 if it leaves the
  // lattice through a non-periodic face.
  int64_t neighbour(int64_t n, int i, int s) const {
    int64_t x[3];
    coords(n, x);
    const int64_t len[3] = {c.nx, c.ny, c.nz};
    for (int a = 0; a < 3; ++a) {
      x[a] += s * e[i][a];
      if (x[a] < 0 || x[a] >= len[a]) {
        if (!c.periodic[a]) return -1;
        x[a] = (x[a] + len[a]) % len[a];
      }
    }
    return x[0] + (int64_t)c.nx * (x[1] + (int64_t)c.ny * x[2]);
  }

  // Eq. (feq) with C = 1.
  T feq(int i, const T& rho, const T u[3]) const {
    T eu = e[i][0] * u[0] + e[i][1] * u[1] + e[i][2] * u[2];
    T uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    return w[i] * rho * (1.0 + 3.0 * eu + 4.5 * eu * eu - 1.5 * uu);
  }

  // Guo body-force source without its relaxation prefactor (the paper names a
  // constant body force g but no forcing scheme):
  // w_i [3 (e_i - u) + 9 (e_i.u) e_i] . g
  T force_source(int i, const T u[3]) const {
    T eu = e[i][0] * u[0] + e[i][1] * u[1] + e[i][2] * u[2];
    T s = 0.0;
    for (int a = 0; a < 3; ++a) s = s + (3.0 * (e[i][a] - u[a]) + 9.0 * eu * e[i][a]) * c.g[a];
    return w[i] * s;
  }
  // BGK form of the Guo term: (1 - 1/(2 tau)) times the source.
  T force_term(int i, const T u[3]) const { return (1.0 - 0.5 / tau) * force_source(i, u); }

  // Moments of Sec. 2 plus the half-force velocity shift, then the collision:
  // BGK  f+ = f - (f - feq)/tau + F_i, or MRT  f+ = f - M^-1 S (m - meq) + F_i.
  void collide(const T* f, T* fp, T& rho, T u[3]) const {
    rho = 0.0;
    T j[3] = {0.0, 0.0, 0.0};
    for (int i = 0; i < Q; ++i) {
      rho = rho + f[i];
      for (int a = 0; a < 3; ++a) j[a] = j[a] + f[i] * e[i][a];
    }
    for (int a = 0; a < 3; ++a) u[a] = (j[a] + 0.5 * c.g[a]) / rho;
    if (c.collision == 0) {
      for (int i = 0; i < Q; ++i) fp[i] = f[i] - (f[i] - feq(i, rho, u)) / tau + force_term(i, u);
      return;
    }
    // MRT, Eq. (mrt): m = M f; equilibrium moments of Sec. 2 written with the
    // momentum j = rho u (force-shifted velocity, as for BGK); rates s_ii of
    // Sec. 2.  The printed list gives s = 0.3 for the conserved moments
    // 0, 3, 5, where m - meq vanishes (density) or is the half-force shift.
    T m[9], meq[9];
    for (int k = 0; k < 9; ++k) {
      m[k] = 0.0;
      for (int i = 0; i < 9; ++i) m[k] = m[k] + kM[k][i] * f[i];
    }
    T jx = rho * u[0], jy = rho * u[1];
    T jj = (jx * jx + jy * jy) / rho;
    meq[0] = rho;
    meq[1] = -2.0 * rho + 3.0 * jj;
    meq[2] = rho - 3.0 * jj;
    meq[3] = jx;
    meq[4] = -jx;
    meq[5] = jy;
    meq[6] = -jy;
    meq[7] = (jx * jx - jy * jy) / rho;
    meq[8] = jx * jy / rho;
    const T nu = (tau - 0.5) / 3.0;
    const T sv = 1.0 / (3.0 * nu + 0.5);
    const T s[9] = {0.3, 1.5, 1.5, 0.3, 1.2, 0.3, 1.2, sv, sv};
    // M^-1 = M^T diag(1/|row_k|^2) because the rows of M are orthogonal.
    double norm2[9];
    for (int k = 0; k < 9; ++k) {
      norm2[k] = 0.0;
      for (int i = 0; i < 9; ++i) norm2[k] += kM[k][i] * kM[k][i];
    }
    // Guo source in moment space, each moment scaled by (1 - s_k/2).
    T src[9], msrc[9];
    for (int i = 0; i < 9; ++i) src[i] = force_source(i, u);
    for (int k = 0; k < 9; ++k) {
      msrc[k] = 0.0;
      for (int i = 0; i < 9; ++i) msrc[k] = msrc[k] + kM[k][i] * src[i];
    }
    for (int i = 0; i < 9; ++i) {
      T delta = 0.0;
      for (int k = 0; k < 9; ++k)
        delta = delta + kM[k][i] / norm2[k] * (s[k] * (m[k] - meq[k]) - (1.0 - 0.5 * s[k]) * msrc[k]);
      fp[i] = f[i] - delta;
    }
  }

  // Parabolic inflow of Sec. 4.3, between walls at inlet_y0 and inlet_y1.
  double inflow(int64_t y) const {
    const double h = c.inlet_y1 - c.inlet_y0;
    return 4.0 * c.inlet_umax * ((double)y - c.inlet_y0) * (c.inlet_y1 - (double)y) / (h * h);
  }

  // Missing population f_i(x_f, t+1) of one link (i = opp(i')), from the
  // post-collision populations at x_f (fp_f) and x_ff (fp_ff), and the
  // moments at time t at both nodes.
  T link_value(int rule, int ip, const T& q, const double uw[3], const T* fp_f, const T* fp_ff, const T& rf,
               const T uf[3], const T& rff, const T uff[3]) const {
    const int i = opp[ip];
    // moving-wall momentum term 6 w_i' rho0 (e_i . u_w) / C^2 (Ladd)
    const double ew = e[i][0] * uw[0] + e[i][1] * uw[1] + e[i][2] * uw[2];
    const double wall = 6.0 * w[ip] * c.rho0 * ew;
    if (rule == BC_HALFWAY) return fp_f[ip] + wall;
    if (rule == BC_BOUZIDI) {
      if (q <= 0.5) return 2.0 * q * fp_f[ip] + (1.0 - 2.0 * q) * fp_ff[ip] + wall;  // Eq. (q_less)
      // Eq. (q_larger); its last term is read as the post-collision f+_i(x_f, t),
      // which is the population that reaches x_ff at t+1.
      return (fp_f[ip] + wall) / (2.0 * q) + (2.0 * q - 1.0) / (2.0 * q) * fp_f[i];
    }
    if (rule == BC_YU) {
      // Yu's unified interpolation (Sec. 3, the two displayed equations).
      // First the population that reaches the wall at t+1: it left x_w - e_i'
      // at t, which lies at q - 1 on the link (x_f at 0, x_ff at -1), so it is
      // interpolated linearly between f+_i'(x_f) and f+_i'(x_ff), and the
      // bounce-back at the wall adds the moving-wall term.
      const T f_wall = q * fp_f[ip] + (1.0 - q) * fp_ff[ip] + wall;
      // Then x_f lies between x_w (at q) and x_ff (at -1): the second
      // equation, read with its parenthesis closed after f_i(x_w, t+1), with
      // f_i(x_ff, t+1) = f+_i(x_f, t) (the population that streams from x_f
      // to x_ff).
      return f_wall / (1.0 + q) + q / (1.0 + q) * fp_f[i];
    }
    // VIBB (Sec. 3.1): f_i(x_f,t+1) = feq_i'(rho_d, u_d) + fneq_i'(x_d) + wall
    // Eq. (rhod) as printed extrapolates for q > 1/2; the optional reading
    // takes the density of x_f there (the O(Ma^2) approximation rho_s = rho_f
    // that Sec. 3.1 quotes from the non-equilibrium extrapolation scheme).
    const T rd = (c.vibb_density == 1 && q > 0.5) ? rf : 2.0 * q * rf + (1.0 - 2.0 * q) * rff;
    // non-equilibrium part at d, each term rescaled by its density ratio
    const T nd = 2.0 * q * (fp_f[ip] - feq(ip, rf, uf)) * (rd / rf) +
                 (1.0 - 2.0 * q) * (fp_ff[ip] - feq(ip, rff, uff)) * (rd / rff);
    T ud[3];
    for (int a = 0; a < 3; ++a) {
      T us;  // u*_d: linear between f and ff (q <= 1/2), or f and the wall
      if (q <= 0.5)
        us = 2.0 * q * uf[a] + (1.0 - 2.0 * q) * uff[a];
      else
        us = (1.0 - q) / q * uf[a] + (2.0 * q - 1.0) / q * uw[a];
      T uss = (1.0 - q) / (1.0 + q) * uff[a] + 2.0 * q / (1.0 + q) * uw[a];  // u**_d
      ud[a] = us / 3.0 + 2.0 * uss / 3.0;                                  // weighted average
    }
    return feq(ip, rd, ud) + nd + wall;
  }
};

thread_local char g_err[512];

template <class T>
std::vector<uint8_t> node_types(const Oracle<T>& o, const uint8_t* solid) {
  std::vector<uint8_t> type(o.N);
  for (int64_t n = 0; n < o.N; ++n) type[n] = solid[n] ? NODE_SOLID : NODE_FLUID;
  if (o.c.stencil == 0 && (o.c.inlet || o.c.outlet)) {
    for (int64_t n = 0; n < o.N; ++n) {
      int64_t x[3];
      o.coords(n, x);
      if (type[n] == NODE_SOLID) continue;
      if (o.c.inlet && x[0] == 0) type[n] = NODE_INLET;
      if (o.c.outlet && x[0] == o.c.nx - 1) type[n] = NODE_OUTLET;
    }
  }
  return type;
}

// One time step t -> t+1 on (fp, rho, u); force[nbody*3] gets the momentum
// exchange of this step per body.  Returns 0, or -1 with g_err set.
template <class T>
int step_once(const Oracle<T>& o, const std::vector<uint8_t>& type, const oracle_link* links, int64_t nl, T* fp,
              T* rho, T* u, std::vector<T>& fnew, T* force, int nbody, const T* qv) {
  const int Q = o.Q;
  const int64_t N = o.N;
  // 1. open boundary columns at time t (Sec. 4.3)
  if (o.c.inlet || o.c.outlet) {
    for (int64_t n = 0; n < N; ++n) {
      if (type[n] == NODE_INLET) {
        // non-equilibrium extrapolation from the first fluid column:
        // f+(0) = feq(rho(1), u_in) + [f+(1) - feq(rho(1), u(1))]
        const int64_t n1 = n + 1;
        int64_t x[3];
        o.coords(n, x);
        const T uin[3] = {o.inflow(x[1]), 0.0, 0.0};
        const T u1[3] = {u[3 * n1], u[3 * n1 + 1], u[3 * n1 + 2]};
        for (int i = 0; i < Q; ++i)
          fp[i * N + n] = o.feq(i, rho[n1], uin) + (fp[i * N + n1] - o.feq(i, rho[n1], u1));
      } else if (type[n] == NODE_OUTLET) {
        // zero gradient: every population equals that of the closest fluid node
        for (int i = 0; i < Q; ++i) fp[i * N + n] = fp[i * N + n - 1];
      }
    }
  }
  // 2. streaming by push into fluid nodes (Eq. 1).  The per-node passes run
  // on OpenMP threads: every node writes its own entries (push targets are
  // distinct), so the result does not depend on the thread count.
  const T nan = std::nan("");
#pragma omp parallel for schedule(static)
  for (int64_t k = 0; k < (int64_t)Q * N; ++k) fnew[k] = nan;
  const int64_t len[3] = {o.c.nx, o.c.ny, o.c.nz};
#pragma omp parallel for collapse(2) schedule(static)
  for (int64_t z = 0; z < len[2]; ++z)
    for (int64_t y = 0; y < len[1]; ++y)
      for (int64_t x = 0; x < len[0]; ++x) {
        const int64_t n = x + len[0] * (y + len[1] * z);
        if (type[n] == NODE_SOLID) continue;
        for (int i = 0; i < Q; ++i) {
          int64_t d[3] = {x + o.e[i][0], y + o.e[i][1], z + o.e[i][2]};
          bool inside = true;
          for (int a = 0; a < 3; ++a) {
            if (d[a] < 0 || d[a] >= len[a]) {
              if (!o.c.periodic[a]) inside = false;
              d[a] = (d[a] + len[a]) % len[a];
            }
          }
          if (!inside) continue;
          const int64_t m = d[0] + len[0] * (d[1] + len[1] * d[2]);
          if (type[m] == NODE_FLUID) fnew[i * N + m] = fp[i * N + n];
        }
      }
  // 3. cut links: each link's value (links write distinct entries), then the
  // momentum exchange summed over the links in order
  std::vector<T> val(nl);
#pragma omp parallel for schedule(static)
  for (int64_t k = 0; k < nl; ++k) {
    const oracle_link& L = links[k];
    const int ip = L.dir, i = o.opp[ip];
    const int64_t f = L.node;
    int64_t ff = o.neighbour(f, i, 1);              // x_ff = x_f - e_i' = x_f + e_i
    if (ff < 0 || type[ff] != NODE_FLUID) ff = f;  // no second fluid node: use f
    T fpf[19], fpff[19];
    for (int j = 0; j < Q; ++j) {
      fpf[j] = fp[j * N + f];
      fpff[j] = fp[j * N + ff];
    }
    const T uf[3] = {u[3 * f], u[3 * f + 1], u[3 * f + 2]};
    const T uff[3] = {u[3 * ff], u[3 * ff + 1], u[3 * ff + 2]};
    const int rule = L.bc >= 0 ? L.bc : o.c.bc;
    val[k] = o.link_value(rule, ip, qv[k], L.uw, fpf, fpff, rho[f], uf, rho[ff], uff);
  }
  for (int b = 0; b < nbody * 3; ++b) force[b] = 0.0;
  for (int64_t k = 0; k < nl; ++k) {
    const oracle_link& L = links[k];
    const int ip = L.dir, i = o.opp[ip];
    fnew[i * N + L.node] = val[k];
    // momentum exchange (Ladd): (f+_i'(x_f,t) + f_i(x_f,t+1)) e_i' on the solid
    if (L.body >= 0 && L.body < nbody)
      for (int a = 0; a < 3; ++a)
        force[3 * L.body + a] = force[3 * L.body + a] + (fp[ip * N + L.node] + val[k]) * (double)o.e[ip][a];
  }
  // 4. moments and collision at fluid nodes (a node that received no
  // population is reported: the first such node in node order)
  int64_t missing = N;
#pragma omp parallel for schedule(static) reduction(min : missing)
  for (int64_t n = 0; n < N; ++n) {
    if (type[n] != NODE_FLUID) continue;
    T f[19], fo[19];
    bool ok = true;
    for (int i = 0; i < Q; ++i) {
      f[i] = fnew[i * N + n];
      if (std::isnan(value_of(f[i]))) ok = false;
    }
    if (!ok) {
      missing = std::min(missing, n);
      continue;
    }
    T r, uu[3];
    o.collide(f, fo, r, uu);
    rho[n] = r;
    for (int a = 0; a < 3; ++a) u[3 * n + a] = uu[a];
    for (int i = 0; i < Q; ++i) fp[i * N + n] = fo[i];
  }
  if (missing < N) {
    int64_t x[3];
    o.coords(missing, x);
    int dir = 0;
    while (dir < Q && !std::isnan(value_of(fnew[dir * N + missing]))) ++dir;
    snprintf(g_err, sizeof g_err, "fluid node (%lld,%lld,%lld) received no population in direction %d: missing link",
             (long long)x[0], (long long)x[1], (long long)x[2], dir);
    return -1;
  }
  return 0;
}

bool check_config(const oracle_config* c) {
  if (c->stencil != 0 && c->stencil != 1) {
    snprintf(g_err, sizeof g_err, "bad stencil");
    return false;
  }
  if (c->nx < 1 || c->ny < 1 || c->nz < 1 || (c->stencil == 0 && c->nz != 1)) {
    snprintf(g_err, sizeof g_err, "bad lattice size");
    return false;
  }
  if (!(c->tau > 0.5)) {
    snprintf(g_err, sizeof g_err, "tau must exceed 1/2");
    return false;
  }
  if (c->collision == 1 && c->stencil != 0) {
    snprintf(g_err, sizeof g_err, "MRT is defined for D2Q9 only");
    return false;
  }
  return true;
}

}  // namespace

extern "C" {

const char* oracle_last_error() { return g_err; }

// OpenMP threads of the per-node passes (the results do not depend on it).
int oracle_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
  return omp_get_max_threads();
#else
  (void)n;
  return 1;
#endif
}

int oracle_num_velocities(int stencil) { return stencil == 0 ? 9 : 19; }

// Lattice velocities and weights of the oracle's own tables (e: Q*3 ints).
int oracle_velocity_set(int stencil, int32_t* e, double* w) {
  oracle_config c{};
  c.stencil = stencil;
  c.nx = c.ny = c.nz = 1;
  Oracle<double> o(c);
  for (int i = 0; i < o.Q; ++i) {
    for (int a = 0; a < 3; ++a) e[3 * i + a] = o.e[i][a];
    w[i] = o.w[i];
  }
  return o.Q;
}

// Equilibrium of Eq. (feq) for one (rho, u); out has Q entries.
int oracle_feq(int stencil, double rho, const double* u, double* out) {
  oracle_config c{};
  c.stencil = stencil;
  c.nx = c.ny = c.nz = 1;
  Oracle<double> o(c);
  const double uu[3] = {u[0], u[1], stencil == 0 ? 0.0 : u[2]};
  for (int i = 0; i < o.Q; ++i) out[i] = o.feq(i, rho, uu);
  return o.Q;
}

// Collision of one node: pre-collision f (Q) -> post-collision fp (Q), and the
// moments it used.  cfg supplies tau, g and the collision operator.
int oracle_collide(const oracle_config* cfg, const double* f, double* fp, double* rho, double* u) {
  if (!check_config(cfg)) return -1;
  Oracle<double> o(*cfg);
  double uu[3];
  o.collide(f, fp, *rho, uu);
  for (int a = 0; a < 3; ++a) u[a] = uu[a];
  return 0;
}

// The missing population f_i(x_f, t+1) of one link from explicit data at its
// two fluid nodes.  fp_f, fp_ff: post-collision populations (Q each); rho and
// u (3 each) at time t at x_f and x_ff.
double oracle_link_value(const oracle_config* cfg, int rule, int dir, double q, const double* uw, const double* fp_f,
                         const double* fp_ff, double rho_f, const double* u_f, double rho_ff, const double* u_ff) {
  Oracle<double> o(*cfg);
  return o.link_value(rule, dir, q, uw, fp_f, fp_ff, rho_f, u_f, rho_ff, u_ff);
}

// Initial state: f(x,0) = feq(rho_in, u_in) at every fluid node, followed by
// the collision at t = 0 -> fp (Q*N), rho (N), u (3*N).  rho_in (N) and u_in
// (3*N, xyz interleaved) may be NULL for rho0 and rest.  Non-fluid entries are
// set to zero.
int oracle_init(const oracle_config* cfg, const uint8_t* solid, const double* rho_in, const double* u_in, double* fp,
                double* rho, double* u) {
  if (!check_config(cfg)) return -1;
  Oracle<double> o(*cfg);
  const std::vector<uint8_t> type = node_types(o, solid);
  const int64_t N = o.N;
  for (int64_t k = 0; k < (int64_t)o.Q * N; ++k) fp[k] = 0.0;
  for (int64_t n = 0; n < N; ++n) {
    rho[n] = 0.0;
    u[3 * n] = u[3 * n + 1] = u[3 * n + 2] = 0.0;
    if (type[n] != NODE_FLUID) continue;
    const double r0 = rho_in ? rho_in[n] : cfg->rho0;
    const double u0[3] = {u_in ? u_in[3 * n] : 0.0, u_in ? u_in[3 * n + 1] : 0.0, u_in ? u_in[3 * n + 2] : 0.0};
    double f[19], fo[19], uu[3], r;
    for (int i = 0; i < o.Q; ++i) f[i] = o.feq(i, r0, u0);
    o.collide(f, fo, r, uu);
    rho[n] = r;
    for (int a = 0; a < 3; ++a) u[3 * n + a] = uu[a];
    for (int i = 0; i < o.Q; ++i) fp[i * N + n] = fo[i];
  }
  return 0;
}

// Advance the state (fp, rho, u as produced by oracle_init) by nsteps.
// force (nbody*3) receives the momentum-exchange force of the last step.
int oracle_run(const oracle_config* cfg, const uint8_t* solid, const oracle_link* links, int64_t nl, double* fp,
               double* rho, double* u, int64_t nsteps, double* force, int nbody) {
  if (!check_config(cfg)) return -1;
  Oracle<double> o(*cfg);
  const std::vector<uint8_t> type = node_types(o, solid);
  for (int64_t k = 0; k < nl; ++k) {
    const oracle_link& L = links[k];
    if (L.node < 0 || L.node >= o.N || L.dir <= 0 || L.dir >= o.Q || !(L.q > 0.0 && L.q <= 1.0) ||
        type[L.node] != NODE_FLUID) {
      snprintf(g_err, sizeof g_err, "link %lld is invalid", (long long)k);
      return -1;
    }
  }
  std::vector<double> fnew((size_t)o.Q * o.N);
  std::vector<double> fbuf(nbody > 0 ? nbody * 3 : 3);
  std::vector<double> qv(nl);
  for (int64_t k = 0; k < nl; ++k) qv[k] = links[k].q;
  for (int64_t s = 0; s < nsteps; ++s) {
    if (step_once(o, type, links, nl, fp, rho, u, fnew, fbuf.data(), nbody, qv.data()) != 0) return -1;
  }
  if (force)
    for (int b = 0; b < nbody * 3; ++b) force[b] = fbuf[b];
  return 0;
}

// Macroscopic fields of a post-collision state: rho = sum f+,
// u = (sum f+ e - g/2) / rho (the collision conserves mass and adds g to the
// momentum, so this equals the velocity the collision used).
int oracle_moments(const oracle_config* cfg, const uint8_t* solid, const double* fp, double* rho, double* u) {
  if (!check_config(cfg)) return -1;
  Oracle<double> o(*cfg);
  const std::vector<uint8_t> type = node_types(o, solid);
  const int64_t N = o.N;
  for (int64_t n = 0; n < N; ++n) {
    rho[n] = 0.0;
    u[3 * n] = u[3 * n + 1] = u[3 * n + 2] = 0.0;
    if (type[n] != NODE_FLUID) continue;
    double r = 0.0, j[3] = {0.0, 0.0, 0.0};
    for (int i = 0; i < o.Q; ++i) {
      r += fp[i * N + n];
      for (int a = 0; a < 3; ++a) j[a] += fp[i * N + n] * o.e[i][a];
    }
    rho[n] = r;
    for (int a = 0; a < 3; ++a) u[3 * n + a] = (j[a] - 0.5 * cfg->g[a]) / r;
  }
  return 0;
}

// Forward-mode derivatives (dual numbers, K = 4 parameters) of the
// momentum-exchange force of the last of nsteps steps from the initial state
// of oracle_init.  dq: n_links x 4 derivatives of each link's q; dtau: 4
// derivatives of tau.  F: nbody x 3 forces; dF: nbody x 3 x 4 derivatives.
int oracle_run_dual(const oracle_config* cfg, const uint8_t* solid, const oracle_link* links, int64_t nl,
                    const double* dq, const double* dtau, const double* rho_in, const double* u_in, int64_t nsteps,
                    double* F, double* dF, int nbody) {
  constexpr int K = 4;
  using D = Dual<K>;
  if (!check_config(cfg)) return -1;
  Oracle<D> o(*cfg);
  for (int k = 0; k < K; ++k) o.tau.d[k] = dtau[k];
  const std::vector<uint8_t> type = node_types(o, solid);
  const int64_t N = o.N;
  for (int64_t k = 0; k < nl; ++k) {
    const oracle_link& L = links[k];
    if (L.node < 0 || L.node >= N || L.dir <= 0 || L.dir >= o.Q || !(L.q > 0.0 && L.q <= 1.0) ||
        type[L.node] != NODE_FLUID) {
      snprintf(g_err, sizeof g_err, "link %lld is invalid", (long long)k);
      return -1;
    }
  }
  std::vector<D> qv(nl);
  for (int64_t k = 0; k < nl; ++k) {
    qv[k] = D(links[k].q);
    for (int j = 0; j < K; ++j) qv[k].d[j] = dq[k * K + j];
  }
  std::vector<D> fp((size_t)o.Q * N), rho(N), u(3 * N), fnew((size_t)o.Q * N);
  for (int64_t n = 0; n < N; ++n) {
    if (type[n] != NODE_FLUID) continue;
    const D r0(rho_in ? rho_in[n] : cfg->rho0);
    const D u0[3] = {D(u_in ? u_in[3 * n] : 0.0), D(u_in ? u_in[3 * n + 1] : 0.0), D(u_in ? u_in[3 * n + 2] : 0.0)};
    D f[19], fo[19], uu[3], r;
    for (int i = 0; i < o.Q; ++i) f[i] = o.feq(i, r0, u0);
    o.collide(f, fo, r, uu);
    rho[n] = r;
    for (int a = 0; a < 3; ++a) u[3 * n + a] = uu[a];
    for (int i = 0; i < o.Q; ++i) fp[i * N + n] = fo[i];
  }
  std::vector<D> fbuf(nbody > 0 ? nbody * 3 : 3);
  for (int64_t s = 0; s < nsteps; ++s)
    if (step_once(o, type, links, nl, fp.data(), rho.data(), u.data(), fnew, fbuf.data(), nbody, qv.data()) != 0)
      return -1;
  for (int b = 0; b < nbody * 3; ++b) {
    F[b] = fbuf[b].v;
    for (int k = 0; k < K; ++k) dF[b * K + k] = fbuf[b].d[k];
  }
  return 0;
}

}  // extern "C"
