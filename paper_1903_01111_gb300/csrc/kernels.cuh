// CUDA kernels of the lattice-Boltzmann step with velocity-interpolation
// bounce-back (arXiv:1903.01111), templated on the velocity set (D2Q9,
// D3Q19) and the storage precision:
//   F64  -- populations f_i stored in double;
//   F32S -- populations stored in float as h_i = f_i - w_i rho0 ("shifted"),
//           so the O(1) rest part w_i rho0 never enters a float rounding.
//
// Storage: SoA  f[i*N + n], n = x + nx*(y + ny*z).  The buffer read by a
// step holds the post-collision populations f+(t) of every fluid node; the
// solid nodes' slots serve as ghost cells that the link kernel fills with
// the missing populations before the bulk kernel pulls them.
//
// Step t -> t+1 (three launches on one stream):
//   k_links: per cut link (x_f, i'), the missing f_i(x_f, t+1), i = opp(i'),
//            from f+ and the moment cache at x_f and x_ff (Sec. 3 and 3.1),
//            written to f[i][x_f + e_i'] (the solid neighbour's slot, read
//            only by x_f); momentum exchange force in FP64.
//   k_open:  inlet/outlet columns (Sec. 4.3), D2Q9 only.
//   k_bulk:  pull streaming f_i(x, t+1) = f+_i(x - e_i, t) (Eq. 1), moments,
//            Guo-forced BGK (Sec. 2, Eq. feq) -> f+(t+1) into the other
//            buffer; rho, u(t+1) into the moment cache where flagged.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "lattice.cuh"

namespace lbm {

struct F64 {
  using T = double;
  static constexpr bool shifted = false;
};
struct F32S {
  using T = float;
  static constexpr bool shifted = true;
};

// One moment-cache record per node: (r, ux, uy, uz) with r = rho (F64) or
// rho - rho0 (F32S); 16 B (FP32) or 32 B (FP64), loaded in one piece.
template <class T>
struct __align__(4 * sizeof(T)) Mom4 {
  T r, ux, uy, uz;
};

// --------------------------------------------------------------- helpers --

// Equilibrium of Eq. (feq), C = 1, in storage form: r is rho (F64) or
// rho - rho0 (F32S); rho is the full density.
template <class L, class P>
__device__ __forceinline__ typename P::T equilibrium(int i, typename P::T r, typename P::T rho, typename P::T ux,
                                                      typename P::T uy, typename P::T uz) {
  using T = typename P::T;
  const T eu = (T)L::cx(i) * ux + (T)L::cy(i) * uy + (T)L::cz(i) * uz;
  const T uu = ux * ux + uy * uy + uz * uz;
  const T w = (T)L::w(i);
  const T poly = (T)3 * eu + (T)4.5 * eu * eu - (T)1.5 * uu;
  if (P::shifted) return w * (r + rho * poly);
  return w * rho * ((T)1 + poly);
}

// Pull source coordinate x - c along one axis, with periodic wrap.
__device__ __forceinline__ int src_coord(int c, int x, int xm, int xp) { return c == 0 ? x : (c > 0 ? xm : xp); }

// Moments, collision and store of one fluid node.  f holds the pre-collision
// populations f(x, t+1) in storage form; n < 2^31.
template <class L, class P>
__device__ __forceinline__ void collide_store(typename P::T (&f)[L::Q], const Params& p, typename P::T* __restrict__ fout,
                                              uint32_t n, Mom4<typename P::T>* __restrict__ mom, bool cache) {
  using T = typename P::T;
  T r = 0, jx = 0, jy = 0, jz = 0;
#pragma unroll
  for (int i = 0; i < L::Q; ++i) {
    r += f[i];
    if (L::cx(i) > 0) jx += f[i];
    if (L::cx(i) < 0) jx -= f[i];
    if (L::cy(i) > 0) jy += f[i];
    if (L::cy(i) < 0) jy -= f[i];
    if (L::cz(i) > 0) jz += f[i];
    if (L::cz(i) < 0) jz -= f[i];
  }
  const T rho = P::shifted ? (T)p.rho0 + r : r;
  const T gx = (T)p.g[0], gy = (T)p.g[1], gz = (T)p.g[2];
  const T inv = (T)1 / rho;
  // Guo forcing: velocity shifted by half the body force
  const T ux = (jx + (T)0.5 * gx) * inv, uy = (jy + (T)0.5 * gy) * inv, uz = (jz + (T)0.5 * gz) * inv;
  if (cache) mom[n] = Mom4<T>{r, ux, uy, L::D == 3 ? uz : (T)0};
  const T omega = (T)(1.0 / p.tau);
  const T uu15 = (T)1.5 * (ux * ux + uy * uy + uz * uz);
  // Guo source (1 - 1/(2 tau)) w_i [3 (e_i - u).g + 9 (e_i.u)(e_i.g)]
  //   = 3 (1 - 1/(2 tau)) w_i [(e_i.g)(1 + 3 e_i.u) - u.g]
  const T fpre3 = (T)(3.0 * (1.0 - 0.5 / p.tau));
  const T ug = ux * gx + uy * gy + uz * gz;
#pragma unroll
  for (int i = 0; i < L::Q; ++i) {
    const T eu = (T)L::cx(i) * ux + (T)L::cy(i) * uy + (T)L::cz(i) * uz;
    const T w = (T)L::w(i);
    const T poly = (T)3 * eu + (T)4.5 * eu * eu - uu15;
    const T feq = P::shifted ? w * (r + rho * poly) : w * rho * ((T)1 + poly);
    T out = f[i] + omega * (feq - f[i]);
    if (p.has_force) {
      const T eg = (T)L::cx(i) * gx + (T)L::cy(i) * gy + (T)L::cz(i) * gz;
      out += fpre3 * w * (eg * ((T)1 + (T)3 * eu) - ug);
    }
    fout[(size_t)i * p.N + n] = out;
  }
}

// ------------------------------------------------------------------ bulk --

// One thread per node of an x-row segment; grid (ceil(nx/bx), ny, nz).
// Block (0,0,0) also clears the force slot of the next step.
template <class L, class P>
__global__ void __launch_bounds__(256) k_bulk(const typename P::T* __restrict__ fin, typename P::T* __restrict__ fout,
                                              const uint8_t* __restrict__ mask, Mom4<typename P::T>* __restrict__ mom,
                                              double* __restrict__ force_next, Params p) {
  using T = typename P::T;
  if (force_next && blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0)
    for (int t = threadIdx.x; t < 3 * MAX_BODIES; t += blockDim.x) force_next[t] = 0.0;
  const uint32_t x = blockIdx.x * blockDim.x + threadIdx.x;
  const uint32_t y = blockIdx.y, z = blockIdx.z;
  const uint32_t nx = p.nx, nxy = (uint32_t)p.nx * (uint32_t)p.ny;
  if (x >= nx) return;
  const uint32_t row = nx * y + nxy * z;
  const uint32_t n = x + row;
  const uint8_t m = mask[n];
  if (m & (M_SOLID | M_OPEN)) return;
  // wrapped neighbour coordinates as row/plane offsets (32-bit)
  const uint32_t xm = x == 0 ? nx - 1 : x - 1, xp = x == nx - 1 ? 0 : x + 1;
  const uint32_t ym = (y == 0 ? p.ny - 1 : y - 1) * nx, y0 = y * nx, yp = (y == (uint32_t)p.ny - 1 ? 0 : y + 1) * nx;
  const uint32_t zm = (z == 0 ? p.nz - 1 : z - 1) * nxy, z0 = z * nxy, zp = (z == (uint32_t)p.nz - 1 ? 0 : z + 1) * nxy;
  T f[L::Q];
#pragma unroll
  for (int i = 0; i < L::Q; ++i) {
    const uint32_t sx = L::cx(i) == 0 ? x : (L::cx(i) > 0 ? xm : xp);
    const uint32_t sy = L::cy(i) == 0 ? y0 : (L::cy(i) > 0 ? ym : yp);
    const uint32_t sz = L::cz(i) == 0 ? z0 : (L::cz(i) > 0 ? zm : zp);
    f[i] = __ldg(fin + (size_t)i * p.N + (sx + sy + sz));
  }
  collide_store<L, P>(f, p, fout, n, mom, (m & M_CACHE) != 0);
}

// ----------------------------------------------------------------- links --

// Per-direction data of the link kernel, staged in shared memory so that
// lanes holding different directions read it without serialisation.
template <class T, int Q>
struct DirTable {
  int off[Q];   // cx + nx (cy + ny cz): node offset of e_d (32-bit)
  int opp[Q];
  T w[Q];
  T e[Q][3];
};

// Equilibrium of direction d from table values (storage form, see above).
template <class P>
__device__ __forceinline__ typename P::T eq_dir(typename P::T w, typename P::T ex, typename P::T ey, typename P::T ez,
                                                typename P::T r, typename P::T rho, typename P::T ux, typename P::T uy,
                                                typename P::T uz) {
  using T = typename P::T;
  const T eu = ex * ux + ey * uy + ez * uz;
  const T poly = (T)3 * eu + (T)4.5 * eu * eu - (T)1.5 * (ux * ux + uy * uy + uz * uz);
  return P::shifted ? w * (r + rho * poly) : w * rho * ((T)1 + poly);
}

// One thread per link.  keys: packed (node, dir, rule, ff fallback, wrap,
// body); qv: q in storage precision; uw: [D][nl] wall velocities or null.
// force: the step's accumulator slot [MAX_BODIES][3] (FP64).
//
// Rules (storage form; the rest part w rho0 cancels because every rule's
// weights sum to one):
//   half-way  f_i = f+_i'(x_f) + wall
//   Bouzidi   q <= 1/2: 2q f+_i'(x_f) + (1-2q) f+_i'(x_ff) + wall   (Eq. q_less)
//             q >  1/2: (f+_i'(x_f) + wall)/(2q) + (2q-1)/(2q) f+_i(x_f)  (Eq. q_larger)
//   VIBB      feq_i'(rho_d, u_d) + fneq_i'(x_d) + wall                 (Sec. 3.1)
// with wall = 6 w rho0 (e_i . u_w).
template <class L, class P>
__global__ void __launch_bounds__(256) k_links(typename P::T* __restrict__ f, const Mom4<typename P::T>* __restrict__ mom,
                                               const uint64_t* __restrict__ keys, const typename P::T* __restrict__ qv,
                                               const typename P::T* __restrict__ uwv, int64_t nl,
                                               double* __restrict__ force, Params p) {
  using T = typename P::T;
  __shared__ DirTable<T, L::Q> tab;
  if (threadIdx.x < L::Q) {
    const int d = threadIdx.x;
    tab.off[d] = L::cx(d) + p.nx * (L::cy(d) + p.ny * L::cz(d));
    tab.opp[d] = L::opp(d);
    tab.w[d] = (T)L::w(d);
    tab.e[d][0] = (T)L::cx(d);
    tab.e[d][1] = (T)L::cy(d);
    tab.e[d][2] = (T)L::cz(d);
  }
  __syncthreads();
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  double F0 = 0.0, F1 = 0.0, F2 = 0.0;
  int body = -1;
  if (k < nl) {
    const uint64_t key = keys[k];
    const int ip = (int)(key & 31);
    const int rule = (int)((key >> 5) & 3);
    const int fb = (int)((key >> 7) & 1);
    const int wrap = (int)((key >> 8) & 1);
    body = (int)((key >> 9) & 127) - 1;
    const uint32_t node = (uint32_t)(key >> KEY_NODE_SHIFT);
    const int i = tab.opp[ip];
    const T ex = tab.e[ip][0], ey = tab.e[ip][1], ez = tab.e[ip][2];
    const T w = tab.w[ip];
    const size_t N = (size_t)p.N;
    uint32_t s, ff;
    if (!wrap) {
      const uint32_t o = (uint32_t)tab.off[ip];
      s = node + o;
      ff = node - o;
    } else {
      const uint32_t nx = p.nx, ny = p.ny, nz = p.nz;
      const uint32_t x = node % nx, y = (node / nx) % ny, z = node / (nx * ny);
      const int cx = (int)ex, cy = (int)ey, cz = (int)ez;
      const uint32_t xs = (x + cx + nx) % nx, ys = (y + cy + ny) % ny, zs = (z + cz + nz) % nz;
      const uint32_t xf = (x - cx + nx) % nx, yf = (y - cy + ny) % ny, zf = (z - cz + nz) % nz;
      s = xs + nx * (ys + ny * zs);
      ff = xf + nx * (yf + ny * zf);
    }
    if (fb) ff = node;
    const T q = qv[k];
    T uw0 = 0, uw1 = 0, uw2 = 0;
    if (uwv) {
      uw0 = uwv[k];
      uw1 = uwv[nl + k];
      if (L::D == 3) uw2 = uwv[2 * nl + k];
    }
    // 6 w_i' rho0 (e_i . u_w) with e_i = -e_i'
    const T wall = -(T)6 * w * (T)p.rho0 * (ex * uw0 + ey * uw1 + ez * uw2);
    const T fpf = f[(size_t)ip * N + node];
    const T two_q = (T)2 * q;
    T val;
    if (rule == 0) {
      val = fpf + wall;
    } else if (rule == 1) {
      if (q <= (T)0.5) {
        val = two_q * fpf + ((T)1 - two_q) * f[(size_t)ip * N + ff] + wall;
      } else {
        const T fpi = f[(size_t)i * N + node];
        const T inv2q = (T)1 / two_q;
        val = (fpf + wall) * inv2q + (two_q - (T)1) * inv2q * fpi;
      }
    } else {
      const T fpff = f[(size_t)ip * N + ff];
      const Mom4<T> mf = mom[node], mff = mom[ff];
      const T rhof = P::shifted ? (T)p.rho0 + mf.r : mf.r;
      const T rhoff = P::shifted ? (T)p.rho0 + mff.r : mff.r;
      // Eq. (rhod) in storage form; optionally rho_d = rho_f when q > 1/2
      const T rd = (p.vibb_local_rho && q > (T)0.5) ? mf.r : two_q * mf.r + ((T)1 - two_q) * mff.r;
      const T rhod = P::shifted ? (T)p.rho0 + rd : rd;
      const T neq_f = fpf - eq_dir<P>(w, ex, ey, ez, mf.r, rhof, mf.ux, mf.uy, mf.uz);
      const T neq_ff = fpff - eq_dir<P>(w, ex, ey, ez, mff.r, rhoff, mff.ux, mff.uy, mff.uz);
      // fneq at d, each term rescaled by its density ratio
      const T nd = rhod * (two_q * neq_f / rhof + ((T)1 - two_q) * neq_ff / rhoff);
      // u*_d (piecewise linear), u**_d (between x_ff and the wall), weighted 1/3 : 2/3
      T af, aff, aw;
      if (q <= (T)0.5) {
        af = two_q;
        aff = (T)1 - two_q;
        aw = 0;
      } else {
        const T iq = (T)1 / q;
        af = ((T)1 - q) * iq;
        aff = 0;
        aw = (two_q - (T)1) * iq;
      }
      const T i1q = (T)1 / ((T)1 + q);
      const T bff = ((T)1 - q) * i1q, bw = two_q * i1q;
      const T third = (T)(1.0 / 3.0), two_thirds = (T)(2.0 / 3.0);
      const T cf = third * af, cff = third * aff + two_thirds * bff, cw = third * aw + two_thirds * bw;
      const T udx = cf * mf.ux + cff * mff.ux + cw * uw0;
      const T udy = cf * mf.uy + cff * mff.uy + cw * uw1;
      const T udz = cf * mf.uz + cff * mff.uz + cw * uw2;
      val = eq_dir<P>(w, ex, ey, ez, rd, rhod, udx, udy, udz) + nd + wall;
    }
    f[(size_t)i * N + s] = val;
    if (body >= 0) {
      // momentum exchange (f+_i'(x_f,t) + f_i(x_f,t+1)) e_i', FP64; shifted
      // storage adds back the two rest parts w rho0
      const double t = (double)fpf + (double)val + (P::shifted ? 2.0 * (double)w * p.rho0 : 0.0);
      F0 = t * (double)ex;
      F1 = t * (double)ey;
      F2 = t * (double)ez;
    }
  }
  // block reduction: one atomic per component when the block has one body
  __shared__ double red[3][32];
  __shared__ int b_first;
  if (threadIdx.x == 0) b_first = body;
  __syncthreads();
  const int b0 = b_first;
  const int uniform = __syncthreads_and(body == b0 || body < 0);
  if (!uniform) {
    if (body >= 0) {
      atomicAdd(&force[3 * body + 0], F0);
      atomicAdd(&force[3 * body + 1], F1);
      atomicAdd(&force[3 * body + 2], F2);
    }
    return;
  }
  if (b0 < 0) return;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    F0 += __shfl_down_sync(0xffffffffu, F0, o);
    F1 += __shfl_down_sync(0xffffffffu, F1, o);
    F2 += __shfl_down_sync(0xffffffffu, F2, o);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) {
    red[0][warp] = F0;
    red[1][warp] = F1;
    red[2][warp] = F2;
  }
  __syncthreads();
  if (warp == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    F0 = lane < nw ? red[0][lane] : 0.0;
    F1 = lane < nw ? red[1][lane] : 0.0;
    F2 = lane < nw ? red[2][lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      F0 += __shfl_down_sync(0xffffffffu, F0, o);
      F1 += __shfl_down_sync(0xffffffffu, F1, o);
      F2 += __shfl_down_sync(0xffffffffu, F2, o);
    }
    if (lane == 0) {
      atomicAdd(&force[3 * b0 + 0], F0);
      atomicAdd(&force[3 * b0 + 1], F1);
      atomicAdd(&force[3 * b0 + 2], F2);
    }
  }
}

// ------------------------------------------------------------ open sides --

// Sec. 4.3: inlet column x = 0 by non-equilibrium extrapolation from x = 1
// with the parabolic velocity u_in(y); outlet column x = nx-1 copies x = nx-2.
// One thread per row (D2Q9).
template <class L, class P>
__global__ void k_open(typename P::T* __restrict__ f, const Mom4<typename P::T>* __restrict__ mom,
                       const uint8_t* __restrict__ mask, Params p) {
  using T = typename P::T;
  const int y = blockIdx.x * blockDim.x + threadIdx.x;
  if (y >= p.ny) return;
  const size_t N = (size_t)p.N;
  if (p.inlet) {
    const uint32_t n0 = (uint32_t)p.nx * y, n1 = n0 + 1;
    if (mask[n0] & M_OPEN) {
      const double h = p.inlet_y1 - p.inlet_y0;
      const T uin = (T)(4.0 * p.inlet_umax * ((double)y - p.inlet_y0) * (p.inlet_y1 - (double)y) / (h * h));
      const Mom4<T> m1 = mom[n1];
      const T rho1 = P::shifted ? (T)p.rho0 + m1.r : m1.r;
#pragma unroll
      for (int i = 0; i < L::Q; ++i)
        f[i * N + n0] = equilibrium<L, P>(i, m1.r, rho1, uin, (T)0, (T)0) +
                        (f[i * N + n1] - equilibrium<L, P>(i, m1.r, rho1, m1.ux, m1.uy, (T)0));
    }
  }
  if (p.outlet) {
    const uint32_t n = (uint32_t)p.nx * y + p.nx - 1;
    if (mask[n] & M_OPEN) {
#pragma unroll
      for (int i = 0; i < L::Q; ++i) f[i * N + n] = f[i * N + n - 1];
    }
  }
}

// ------------------------------------------------------- init and fields --

// f(x,0) = feq(rho_in, u_in) followed by the collision at t = 0 (fluid
// nodes); zero elsewhere.  rho_in (N) and u_in (N x 3, interleaved) may be
// null for rho0 and rest.
template <class L, class P>
__global__ void k_init(typename P::T* __restrict__ f, Mom4<typename P::T>* __restrict__ mom, const uint8_t* __restrict__ mask,
                       const double* __restrict__ rho_in, const double* __restrict__ u_in, Params p) {
  using T = typename P::T;
  const int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (n >= p.N) return;
  const uint8_t m = mask[n];
  if (m & (M_SOLID | M_OPEN)) {
#pragma unroll
    for (int i = 0; i < L::Q; ++i) f[(int64_t)i * p.N + n] = (T)0;
    return;
  }
  const double rho = rho_in ? rho_in[n] : p.rho0;
  const double ux = u_in ? u_in[3 * n] : 0.0, uy = u_in ? u_in[3 * n + 1] : 0.0;
  const double uz = (u_in && L::D == 3) ? u_in[3 * n + 2] : 0.0;
  T fl[L::Q];
#pragma unroll
  for (int i = 0; i < L::Q; ++i) {
    const double eu = L::cx(i) * ux + L::cy(i) * uy + L::cz(i) * uz;
    const double poly = 3.0 * eu + 4.5 * eu * eu - 1.5 * (ux * ux + uy * uy + uz * uz);
    fl[i] = P::shifted ? (T)(L::w(i) * ((rho - p.rho0) + rho * poly)) : (T)(L::w(i) * rho * (1.0 + poly));
  }
  collide_store<L, P>(fl, p, f, (uint32_t)n, mom, (m & M_CACHE) != 0);
}

// rho = sum f+, u = (sum f+ e - g/2)/rho of the post-collision state (the
// collision conserves mass and adds g to the momentum); FP64 output, zero
// at solid and open nodes.  u: [D][N].
template <class L, class P>
__global__ void k_moments(const typename P::T* __restrict__ f, const uint8_t* __restrict__ mask,
                          double* __restrict__ rho_out, double* __restrict__ u_out, Params p) {
  using T = typename P::T;
  const int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (n >= p.N) return;
  const int64_t N = p.N;
  if (mask[n] & (M_SOLID | M_OPEN)) {
    rho_out[n] = 0.0;
    for (int a = 0; a < L::D; ++a) u_out[a * N + n] = 0.0;
    return;
  }
  T r = 0, jx = 0, jy = 0, jz = 0;
#pragma unroll
  for (int i = 0; i < L::Q; ++i) {
    const T v = f[(int64_t)i * N + n];
    r += v;
    jx += (T)L::cx(i) * v;
    jy += (T)L::cy(i) * v;
    jz += (T)L::cz(i) * v;
  }
  const double rho = P::shifted ? p.rho0 + (double)r : (double)r;
  rho_out[n] = rho;
  u_out[n] = ((double)jx - 0.5 * p.g[0]) / rho;
  u_out[N + n] = ((double)jy - 0.5 * p.g[1]) / rho;
  if (L::D == 3) u_out[2 * N + n] = ((double)jz - 0.5 * p.g[2]) / rho;
}

// Moment cache refresh from a post-collision state (after the caller sets
// the populations): same formula as k_moments, storage precision.
template <class L, class P>
__global__ void k_refresh(const typename P::T* __restrict__ f, const uint8_t* __restrict__ mask,
                          Mom4<typename P::T>* __restrict__ mom, Params p) {
  using T = typename P::T;
  const int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (n >= p.N || !(mask[n] & M_CACHE)) return;
  const int64_t N = p.N;
  T r = 0, jx = 0, jy = 0, jz = 0;
#pragma unroll
  for (int i = 0; i < L::Q; ++i) {
    const T v = f[(int64_t)i * N + n];
    r += v;
    jx += (T)L::cx(i) * v;
    jy += (T)L::cy(i) * v;
    jz += (T)L::cz(i) * v;
  }
  const T rho = P::shifted ? (T)p.rho0 + r : r;
  mom[n] = Mom4<T>{r, (jx - (T)(0.5 * p.g[0])) / rho, (jy - (T)(0.5 * p.g[1])) / rho,
                   L::D == 3 ? (jz - (T)(0.5 * p.g[2])) / rho : (T)0};
}

// One direction of the state to/from FP64 unshifted populations.
template <class L, class P>
__global__ void k_get_dir(const typename P::T* __restrict__ f, const uint8_t* __restrict__ mask, int i,
                          double* __restrict__ out, Params p) {
  const int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (n >= p.N) return;
  if (mask[n] & (M_SOLID | M_OPEN)) {
    out[n] = 0.0;
    return;
  }
  double w = 0.0;
#pragma unroll
  for (int k = 0; k < L::Q; ++k)
    if (k == i) w = L::w(k);
  out[n] = (double)f[(int64_t)i * p.N + n] + (P::shifted ? w * p.rho0 : 0.0);
}

template <class L, class P>
__global__ void k_set_dir(typename P::T* __restrict__ f, const uint8_t* __restrict__ mask, int i,
                          const double* __restrict__ in, Params p) {
  using T = typename P::T;
  const int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (n >= p.N) return;
  double w = 0.0;
#pragma unroll
  for (int k = 0; k < L::Q; ++k)
    if (k == i) w = L::w(k);
  f[(int64_t)i * p.N + n] = (mask[n] & (M_SOLID | M_OPEN)) ? (T)0 : (T)(in[n] - (P::shifted ? w * p.rho0 : 0.0));
}

// Populations of listed nodes (FP64 unshifted), out[k*Q + i].
template <class L, class P>
__global__ void k_gather(const typename P::T* __restrict__ f, const uint8_t* __restrict__ mask,
                         const int64_t* __restrict__ nodes, int64_t n, double* __restrict__ out, Params p) {
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= n) return;
  const int64_t node = nodes[k];
  const bool off = (mask[node] & (M_SOLID | M_OPEN)) != 0;
#pragma unroll
  for (int i = 0; i < L::Q; ++i)
    out[k * L::Q + i] = off ? 0.0 : (double)f[(int64_t)i * p.N + node] + (P::shifted ? L::w(i) * p.rho0 : 0.0);
}

// Failure detection: flag any non-finite population or non-positive density.
template <class L, class P>
__global__ void k_check(const typename P::T* __restrict__ f, const uint8_t* __restrict__ mask, int* __restrict__ flag,
                        Params p) {
  using T = typename P::T;
  const int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (n >= p.N || (mask[n] & (M_SOLID | M_OPEN))) return;
  T r = 0;
  bool bad = false;
#pragma unroll
  for (int i = 0; i < L::Q; ++i) {
    const T v = f[(int64_t)i * p.N + n];
    bad |= !isfinite(v);
    r += v;
  }
  const double rho = P::shifted ? p.rho0 + (double)r : (double)r;
  if (bad || !(rho > 0.0)) atomicOr(flag, 1);
}

// ------------------------------------------------------------- launchers --

struct KernelOps {
  int Q, D;
  size_t real_bytes;
  void (*bulk)(const void* fin, void* fout, const uint8_t* mask, void* mom, double* force_next, const Params& p,
               cudaStream_t s);
  void (*links)(void* f, const void* mom, const uint64_t* keys, const void* q, const void* uw, int64_t nl, double* force,
                const Params& p, cudaStream_t s);
  void (*open)(void* f, const void* mom, const uint8_t* mask, const Params& p, cudaStream_t s);
  void (*init)(void* f, void* mom, const uint8_t* mask, const double* rho, const double* u, const Params& p,
               cudaStream_t s);
  void (*moments)(const void* f, const uint8_t* mask, double* rho, double* u, const Params& p, cudaStream_t s);
  void (*refresh)(const void* f, const uint8_t* mask, void* mom, const Params& p, cudaStream_t s);
  void (*get_dir)(const void* f, const uint8_t* mask, int i, double* out, const Params& p, cudaStream_t s);
  void (*set_dir)(void* f, const uint8_t* mask, int i, const double* in, const Params& p, cudaStream_t s);
  void (*check)(const void* f, const uint8_t* mask, int* flag, const Params& p, cudaStream_t s);
  void (*gather)(const void* f, const uint8_t* mask, const int64_t* nodes, int64_t n, double* out, const Params& p,
                 cudaStream_t s);
};

inline unsigned blocks_for(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

template <class L, class P>
struct Launch {
  using T = typename P::T;
  static void bulk(const void* fin, void* fout, const uint8_t* mask, void* mom, double* force_next, const Params& p,
                   cudaStream_t s) {
    const int bx = p.nx >= 256 ? 256 : ((p.nx + 31) / 32) * 32;
    dim3 grid(blocks_for(p.nx, bx), p.ny, p.nz);
    k_bulk<L, P><<<grid, bx, 0, s>>>((const T*)fin, (T*)fout, mask, (Mom4<T>*)mom, force_next, p);
  }
  static void links(void* f, const void* mom, const uint64_t* keys, const void* q, const void* uw, int64_t nl,
                    double* force, const Params& p, cudaStream_t s) {
    if (nl == 0) return;
    k_links<L, P><<<blocks_for(nl, 256), 256, 0, s>>>((T*)f, (const Mom4<T>*)mom, keys, (const T*)q, (const T*)uw, nl,
                                                     force, p);
  }
  static void open(void* f, const void* mom, const uint8_t* mask, const Params& p, cudaStream_t s) {
    k_open<L, P><<<blocks_for(p.ny, 128), 128, 0, s>>>((T*)f, (const Mom4<T>*)mom, mask, p);
  }
  static void init(void* f, void* mom, const uint8_t* mask, const double* rho, const double* u, const Params& p,
                   cudaStream_t s) {
    k_init<L, P><<<blocks_for(p.N, 256), 256, 0, s>>>((T*)f, (Mom4<T>*)mom, mask, rho, u, p);
  }
  static void moments(const void* f, const uint8_t* mask, double* rho, double* u, const Params& p, cudaStream_t s) {
    k_moments<L, P><<<blocks_for(p.N, 256), 256, 0, s>>>((const T*)f, mask, rho, u, p);
  }
  static void refresh(const void* f, const uint8_t* mask, void* mom, const Params& p, cudaStream_t s) {
    k_refresh<L, P><<<blocks_for(p.N, 256), 256, 0, s>>>((const T*)f, mask, (Mom4<T>*)mom, p);
  }
  static void get_dir(const void* f, const uint8_t* mask, int i, double* out, const Params& p, cudaStream_t s) {
    k_get_dir<L, P><<<blocks_for(p.N, 256), 256, 0, s>>>((const T*)f, mask, i, out, p);
  }
  static void set_dir(void* f, const uint8_t* mask, int i, const double* in, const Params& p, cudaStream_t s) {
    k_set_dir<L, P><<<blocks_for(p.N, 256), 256, 0, s>>>((T*)f, mask, i, in, p);
  }
  static void check(const void* f, const uint8_t* mask, int* flag, const Params& p, cudaStream_t s) {
    k_check<L, P><<<blocks_for(p.N, 256), 256, 0, s>>>((const T*)f, mask, flag, p);
  }
  static void gather(const void* f, const uint8_t* mask, const int64_t* nodes, int64_t n, double* out, const Params& p,
                     cudaStream_t s) {
    if (n == 0) return;
    k_gather<L, P><<<blocks_for(n, 256), 256, 0, s>>>((const T*)f, mask, nodes, n, out, p);
  }
  static KernelOps ops() {
    return KernelOps{L::Q, L::D, sizeof(T), bulk, links, open, init, moments, refresh, get_dir, set_dir, check, gather};
  }
};

KernelOps ops_d2q9_f64();
KernelOps ops_d2q9_f32s();
KernelOps ops_d3q19_f64();
KernelOps ops_d3q19_f32s();

}  // namespace lbm
