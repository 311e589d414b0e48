// Lattice constants and the parameter block shared by the kernels and the
// host side of liblbm.so.  Velocity sets:
//   D2Q9  in the order of the moment matrix M (Sec. 2 of arXiv:1903.01111):
//         e1=(1,0) e2=(0,1) e3=(-1,0) e4=(0,-1) e5=(1,1) e6=(-1,1) e7=(-1,-1)
//         e8=(1,-1), weights 4/9, 1/9, 1/36;
//   D3Q19 rest, +-x, +-y, +-z, (+-1,+-1,0), (+-1,0,+-1), (0,+-1,+-1) with
//         opposite directions adjacent, weights 1/3, 1/18, 1/36.
// Everything is constexpr so that unrolled loops fold the velocities.
#pragma once
#include <cstdint>

namespace lbm {

// Largest number of force accumulators (bodies) of a lattice.
constexpr int MAX_BODIES = 32768;

struct D2Q9 {
  static constexpr int Q = 9, D = 2;
  __host__ __device__ static constexpr int cx(int i) {
    return (i == 1 || i == 5 || i == 8) ? 1 : (i == 3 || i == 6 || i == 7) ? -1 : 0;
  }
  __host__ __device__ static constexpr int cy(int i) {
    return (i == 2 || i == 5 || i == 6) ? 1 : (i == 4 || i == 7 || i == 8) ? -1 : 0;
  }
  __host__ __device__ static constexpr int cz(int) { return 0; }
  __host__ __device__ static constexpr double w(int i) { return i == 0 ? 4.0 / 9.0 : (i < 5 ? 1.0 / 9.0 : 1.0 / 36.0); }
  __host__ __device__ static constexpr int opp(int i) { return i == 0 ? 0 : (i < 5 ? 1 + ((i + 1) & 3) : 5 + ((i - 3) & 3)); }
};

// D2Q9 moment matrix of Sec. 2, Eq. (M): rows m0..m8 = (rho, e, epsilon, j_x,
// q_x, j_y, q_y, p_xx, p_xy), columns = directions in the order above; rows
// are orthogonal, so M^-1 = M^T diag(1 / |row_k|^2).
__host__ __device__ constexpr int mrt_m(int k, int i) {
  constexpr int M[9][9] = {{1, 1, 1, 1, 1, 1, 1, 1, 1},     {-4, -1, -1, -1, -1, 2, 2, 2, 2},
                           {4, -2, -2, -2, -2, 1, 1, 1, 1}, {0, 1, 0, -1, 0, 1, -1, -1, 1},
                           {0, -2, 0, 2, 0, 1, -1, -1, 1},  {0, 0, 1, 0, -1, 1, 1, -1, -1},
                           {0, 0, -2, 0, 2, 1, 1, -1, -1},  {0, 1, -1, 1, -1, 0, 0, 0, 0},
                           {0, 0, 0, 0, 0, 1, -1, 1, -1}};
  return M[k][i];
}
__host__ __device__ constexpr int mrt_norm2(int k) {
  return k == 0 ? 9 : (k == 1 || k == 2) ? 36 : (k == 3 || k == 5) ? 6 : (k == 4 || k == 6) ? 12 : 4;
}

struct D3Q19 {
  static constexpr int Q = 19, D = 3;
  __host__ __device__ static constexpr int cx(int i) {
    return (i == 1 || i == 7 || i == 9 || i == 11 || i == 13) ? 1
           : (i == 2 || i == 8 || i == 10 || i == 12 || i == 14) ? -1
                                                                  : 0;
  }
  __host__ __device__ static constexpr int cy(int i) {
    return (i == 3 || i == 7 || i == 10 || i == 15 || i == 17) ? 1
           : (i == 4 || i == 8 || i == 9 || i == 16 || i == 18) ? -1
                                                                 : 0;
  }
  __host__ __device__ static constexpr int cz(int i) {
    return (i == 5 || i == 11 || i == 14 || i == 15 || i == 18) ? 1
           : (i == 6 || i == 12 || i == 13 || i == 16 || i == 17) ? -1
                                                                   : 0;
  }
  __host__ __device__ static constexpr double w(int i) { return i == 0 ? 1.0 / 3.0 : (i < 7 ? 1.0 / 18.0 : 1.0 / 36.0); }
  __host__ __device__ static constexpr int opp(int i) { return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1); }
};

// Collision constants folded on the host from omega, fpre3 and g for a
// stencil's weights, the same for every node of a domain: per weight class
// c (0 rest, 1 |e| = 1, 2 diagonal) ko = omega w_c, kh = 4.5 omega w_c,
// kb = 3 omega w_c, kf = fpre3 w_c; per direction kt = 3 fpre3 w_i (e_i.g),
// ke = fpre3 w_i (e_i.g); om1 = 1 - omega; hg = g/2.  The float copies
// serve the FP32 kernels.  One function (fold) fills them for a lattice and
// for each domain of a batch, so that a domain collides with the same bits
// alone and in a batch.
struct Folded {
  double ko[3], kh[3], kb[3], kf[3], kt[19], ke[19], om1, hg[3];
  float ko_f[3], kh_f[3], kb_f[3], kf_f[3], kt_f[19], ke_f[19], om1_f, hg_f[3];
};

template <class L>
inline void fold(Folded& k, double omega, double fpre3, const double g[3]) {
  const double wc[3] = {L::w(0), L::w(1), L::w(L::Q == 9 ? 5 : 7)};
  for (int c = 0; c < 3; ++c) {
    k.ko[c] = omega * wc[c];
    k.kh[c] = 4.5 * omega * wc[c];
    k.kb[c] = 3.0 * omega * wc[c];
    k.kf[c] = fpre3 * wc[c];
    k.ko_f[c] = (float)k.ko[c];
    k.kh_f[c] = (float)k.kh[c];
    k.kb_f[c] = (float)k.kb[c];
    k.kf_f[c] = (float)k.kf[c];
  }
  for (int i = 0; i < 19; ++i) {
    // e_i.g with integer e_i: every product exact, whatever the contraction
    const double eg = i < L::Q ? L::cx(i) * g[0] + L::cy(i) * g[1] + L::cz(i) * g[2] : 0.0;
    const double fw = i < L::Q ? fpre3 * L::w(i) : 0.0;
    k.kt[i] = 3.0 * fw * eg;
    k.ke[i] = fw * eg;
    k.kt_f[i] = (float)k.kt[i];
    k.ke_f[i] = (float)k.ke[i];
  }
  k.om1 = 1.0 - omega;
  k.om1_f = (float)k.om1;
  for (int a = 0; a < 3; ++a) {
    k.hg[a] = 0.5 * g[a];
    k.hg_f[a] = (float)k.hg[a];
  }
}

// Run parameters handed to every kernel by value.
struct Params {
  int nx, ny, nz;
  int64_t N;            // nx*ny*nz
  double tau, rho0;
  double omega;         // 1/tau
  double fpre3;         // 3 (1 - 1/(2 tau)), Guo source prefactor
  double g[3];
  int has_force;        // g != 0
  int collision;        // 0 BGK, 1 MRT
  double inlet_umax, inlet_y0, inlet_y1;
  int inlet, outlet;
  int vibb_local_rho;   // rho_d = rho_f when q > 1/2
  int periodic[3];
  int nbody;            // force accumulators per slot (max body id + 1, >= 1)
  // rho0, omega, fpre3, g, g/2 and omega^2 rounded once to float: the FP32
  // kernels read these copies (set by round_params), because a double ->
  // float conversion on every node or link costs FP64-pipe time
  float rho0_f, omega_f, fpre3_f, g_f[3], hg_f[3], omega2_f;
  Folded kc;            // collision constants (fold_params)
};

// Fills the float copies of Params from its doubles (after any change).
inline void round_params(Params& p) {
  p.rho0_f = (float)p.rho0;
  p.omega_f = (float)p.omega;
  p.fpre3_f = (float)p.fpre3;
  p.omega2_f = (float)(p.omega * p.omega);
  for (int a = 0; a < 3; ++a) {
    p.g_f[a] = (float)p.g[a];
    p.hg_f[a] = (float)(0.5 * p.g[a]);
  }
}

// Fills the folded collision constants and every float copy of Params for
// stencil L (after any change of omega, fpre3 or g).
template <class L>
inline void fold_params(Params& p) {
  fold<L>(p.kc, p.omega, p.fpre3, p.g);
  round_params(p);
}

// Error message shared by every translation unit of the library (set by a
// failing entry point, read through lbm_last_error).
void set_last_error(const char* msg);

}  // namespace lbm
