// Discrete adjoint of one lattice-Boltzmann step (BGK + Guo forcing, pull
// streaming, half-way / Bouzidi / VIBB links, open columns): the transpose of
// the step's Jacobian applied to lambda(s+1) = dJ/df+(s+1), giving
// lambda(s) = dJ/df+(s), plus the explicit derivatives of the step with
// respect to tau (summed in FP64) and to every link's q (accumulated per link
// in FP64 over time).
//
// The state of a step is f+(s); the moments a link rule uses are the
// functions rho = sum f+, u = (sum f+ e - g/2)/rho of it (refreshed from
// f+(s) before the adjoint step), so that every dependence is through f+(s).
//
// Per step (one stream, in this order):
//   k_adj_bulk   per fluid node x: pre-collision f(s+1) from the pull sources
//                (ghost slots hold the link values of step s), the collision
//                transpose mu = (dC/df)^T lambda(s+1)(x), and mu_i scattered to
//                the pull source of direction i -- streaming is a permutation,
//                so these writes never collide; the ghost slot of a cut link
//                receives the adjoint weight of its link value.  Cached nodes
//                also refresh their moments from f+(s) for the link kernel.
//   k_adj_links  per link: the link value's transpose into x_f and x_ff
//                (populations and, through the moments, all directions), by
//                atomics; dJ/dq accumulated per link.
//   k_adj_open   inlet (non-equilibrium extrapolation) and outlet (copy)
//                transposes into the first and last fluid columns.
// The buffer of lambda(s+1) becomes the output of the next step back.  There
// k_adj_bulk assigns every entry (j, m) of a fluid node m whose neighbour
// m + e_j is a fluid node (each such entry is the pull source of exactly one
// node), so only the entries that the pass does not assign have to be zero
// when the link and open kernels add into them: (i', x_f) of every cut link
// and (j, m) with m + e_j an open node.  The link and open kernels clear
// those of lambda(s+1) once k_adj_bulk has read it, and clear the ghost and
// open entries of lambda(s) they consume; no pass clears whole nodes.
#pragma once
#include "kernels.cuh"

namespace lbm {

template <class T>
__device__ __forceinline__ void atomic_add_real(T* p, T v) {
  atomicAdd(p, v);
}

// Collision transpose at one node.  f: pre-collision populations (storage
// form); lam: lambda(s+1) of this node; mu: output.  Returns the node's
// sum_i lam_i dC_i/dtau.
template <class L, class P>
__device__ __forceinline__ typename P::T collide_adjoint(const typename P::T (&f)[L::Q], const typename P::T (&lam)[L::Q],
                                                  typename P::T (&mu)[L::Q], const Params& p, const Relax& rx) {
  using T = typename P::T;
  T r = 0, jx = 0, jy = 0, jz = 0;
#pragma unroll
  for (int i = 0; i < L::Q; ++i) {
    r += f[i];
    jx += (T)L::cx(i) * f[i];
    jy += (T)L::cy(i) * f[i];
    jz += (T)L::cz(i) * f[i];
  }
  const T rho = P::shifted ? par<T>(p.rho0, p.rho0_f) + r : r;
  const T gx = par<T>(rx.g[0], rx.g_f[0]), gy = par<T>(rx.g[1], rx.g_f[1]), gz = par<T>(rx.g[2], rx.g_f[2]);
  // the velocity as the forward collision forms it (one reciprocal of rho)
  const T ir = (T)1 / rho;
  const T ux = (jx + (T)0.5 * gx) * ir, uy = (jy + (T)0.5 * gy) * ir, uz = (jz + (T)0.5 * gz) * ir;
  const T omega = par<T>(rx.omega, rx.omega_f);
  const T uu15 = (T)1.5 * (ux * ux + uy * uy + uz * uz);
  const T ug = ux * gx + uy * gy + uz * gz;
  // The u-derivatives of the equilibrium and of the source, and f - feq +
  // src/2, sum to zero over the directions (mass is conserved and the source
  // carries no mass), so the B and dtau sums may use lambda minus its mean:
  // the same values in exact arithmetic, without the rounding of a large
  // common part of lambda that cancels.
  T lbar = 0;
#pragma unroll
  for (int i = 0; i < L::Q; ++i) lbar += lam[i];
  lbar *= (T)(1.0 / L::Q);
  // Every sum over the directions below is a polynomial in e_i of degree
  // <= 2 weighted by w_i (lam_i - lbar), so it is formed from the moments
  //   S0 = sum w_i d_i,  S_a = sum w_i d_i e_ia,  T_ab = sum w_i d_i e_ia e_ib
  // (d_i = lam_i - lbar) and from lf = sum d_i f_i:
  //   A   = sum lam_i w_i (1 + poly_i) = S0 (1 - 1.5 u.u) + lbar + 3 u.S + 4.5 u.T.u
  //   B_a = omega rho (3 S_a + 9 (T u)_a - 3 u_a S0) + (1 - omega/2) (9 (T g)_a - 3 g_a S0)
  //   dtau sum = lf - sum d_i feq_i + sum d_i src_i / 2
  T S0 = 0, Sx = 0, Sy = 0, Sz = 0, Txx = 0, Tyy = 0, Tzz = 0, Txy = 0, Txz = 0, Tyz = 0, lf = 0;
#pragma unroll
  for (int i = 0; i < L::Q; ++i) {
    const T d = lam[i] - lbar;
    const T wd = (T)L::w(i) * d;
    const int cx = L::cx(i), cy = L::cy(i), cz = L::cz(i);
    S0 += wd;
    if (cx > 0) Sx += wd;
    if (cx < 0) Sx -= wd;
    if (cy > 0) Sy += wd;
    if (cy < 0) Sy -= wd;
    if (cz > 0) Sz += wd;
    if (cz < 0) Sz -= wd;
    if (cx != 0) Txx += wd;
    if (cy != 0) Tyy += wd;
    if (cz != 0) Tzz += wd;
    if (cx * cy > 0) Txy += wd;
    if (cx * cy < 0) Txy -= wd;
    if (cx * cz > 0) Txz += wd;
    if (cx * cz < 0) Txz -= wd;
    if (cy * cz > 0) Tyz += wd;
    if (cy * cz < 0) Tyz -= wd;
    lf += d * f[i];
  }
  const T Tux = Txx * ux + Txy * uy + Txz * uz, Tuy = Txy * ux + Tyy * uy + Tyz * uz,
          Tuz = Txz * ux + Tyz * uy + Tzz * uz;
  const T Tgx = Txx * gx + Txy * gy + Txz * gz, Tgy = Txy * gx + Tyy * gy + Tyz * gz,
          Tgz = Txz * gx + Tyz * gy + Tzz * gz;
  const T uS = ux * Sx + uy * Sy + uz * Sz, uTu = ux * Tux + uy * Tuy + uz * Tuz;
  const T A = S0 * ((T)1 - uu15) + lbar + (T)3 * uS + (T)4.5 * uTu;
  const T orho = omega * rho, c2 = (T)1 - (T)0.5 * omega;
  const T B0 = orho * ((T)3 * Sx + (T)9 * Tux - (T)3 * ux * S0) + c2 * ((T)9 * Tgx - (T)3 * gx * S0);
  const T B1 = orho * ((T)3 * Sy + (T)9 * Tuy - (T)3 * uy * S0) + c2 * ((T)9 * Tgy - (T)3 * gy * S0);
  const T B2 = orho * ((T)3 * Sz + (T)9 * Tuz - (T)3 * uz * S0) + c2 * ((T)9 * Tgz - (T)3 * gz * S0);
  // sum d_i feq_i (storage form: feq_i = w_i (r + rho poly_i) shifted, w_i rho (1 + poly_i) else)
  const T dpoly = (T)3 * uS + (T)4.5 * uTu - uu15 * S0;
  const T dfeq = P::shifted ? r * S0 + rho * dpoly : rho * (S0 + dpoly);
  // sum d_i src_i, src_i = w_i (3 (e_i.g - u.g) + 9 (e_i.u)(e_i.g))
  const T dsrc = rx.has_force ? (T)3 * (gx * Sx + gy * Sy + gz * Sz) - (T)3 * ug * S0 +
                                    (T)9 * (ux * Tgx + uy * Tgy + uz * Tgz)
                              : (T)0;
  const T dtau = lf - dfeq + (T)0.5 * dsrc;
#pragma unroll
  for (int j = 0; j < L::Q; ++j) {
    const T ex = (T)L::cx(j), ey = (T)L::cy(j), ez = (T)L::cz(j);
    mu[j] = ((T)1 - omega) * lam[j] + omega * A + (B0 * (ex - ux) + B1 * (ey - uy) + B2 * (ez - uz)) * ir;
  }
  return dtau * par<T>(rx.omega * rx.omega, rx.omega2_f);
}

// Adds v to target[key] over the block (key < 0: nothing to add): a warp
// whose contributing lanes share one key sums in the value's own precision
// by shuffles (any other warp adds per thread with FP64 atomics); after one
// barrier the first thread adds the warp sums in FP64, one atomic per run of
// equal keys.
template <class T>
__device__ __forceinline__ void block_add_keyed(T v, int key, double* target) {
  __shared__ double red[32];
  __shared__ int rkey[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int wk = __reduce_max_sync(0xffffffffu, key);
  const bool uniform = __all_sync(0xffffffffu, key < 0 || key == wk);
  if (!uniform) {
    if (key >= 0 && v != (T)0) atomicAdd(target + key, (double)v);
    v = (T)0;
  } else if (key < 0) {
    v = (T)0;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if (lane == 0) {
    red[warp] = (double)v;
    rkey[warp] = uniform ? wk : -1;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int cur = -1;
    double acc = 0.0;
    for (int wi = 0; wi < (int)((blockDim.x + 31) >> 5); ++wi) {
      const int kk = rkey[wi];
      if (kk < 0) continue;
      if (kk != cur) {
        if (cur >= 0) atomicAdd(target + cur, acc);
        cur = kk;
        acc = 0.0;
      }
      acc += red[wi];
    }
    if (cur >= 0) atomicAdd(target + cur, acc);
  }
}

// Resident 256-thread blocks per SM of the adjoint bulk kernel: 5 (48
// registers, a few spilled words) for FP32 D2Q9 — measured faster than 4 at
// 64 registers on the channel batch (backward 0.667 -> 0.641 ms per step) —,
// 2 (up to 128 registers) for FP64 D2Q9 and FP32 D3Q19, 1 for FP64 D3Q19.
template <class L, class P>
constexpr int adj_bulk_blocks_per_sm() {
  return L::Q == 9 ? (P::shifted ? 5 : 2) : (P::shifted ? 2 : 1);
}

template <class L, class P>
__global__ void __launch_bounds__(256, (adj_bulk_blocks_per_sm<L, P>())) k_adj_bulk(const typename P::T* __restrict__ fin,
                                                  typename P::T* __restrict__ lam_next,
                                                  typename P::T* __restrict__ lam_out, Layout lay, Params p,
                                                  double* __restrict__ dtau, Mom4<typename P::T>* __restrict__ mom) {
  using T = typename P::T;
  const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
  const size_t S = (size_t)lay.S;
  T dt = 0;
  int key = -1;
  if (k < (uint64_t)lay.S) {
    const uint32_t w = lay.word[k];
    if (!(w & (W_GHOST | W_OPEN))) {
      const RunRec run = lay.runs[w & W_RUN];
      key = lay.ndom > 1 ? run.dom : 0;
      const Relax rx = lay.ndom > 1 ? relax_domain(lay.dom, key) : relax_params(p);
      int d[L::Q];
      pull_offsets<L>(k, run, lay, p, d);
      T f[L::Q], lam[L::Q], mu[L::Q];
#pragma unroll
      for (int i = 0; i < L::Q; ++i) {
        f[i] = fin[(ptrdiff_t)i * (ptrdiff_t)S + (ptrdiff_t)k + d[i]];
        lam[i] = lam_next[(size_t)i * S + k];
      }
      if (w & W_CACHE) {
        // moments of f+(s) at this node (the k_refresh formula)
        T r = 0, jx = 0, jy = 0, jz = 0;
#pragma unroll
        for (int i = 0; i < L::Q; ++i) {
          const T v = fin[(size_t)i * S + k];
          r += v;
          jx += (T)L::cx(i) * v;
          jy += (T)L::cy(i) * v;
          jz += (T)L::cz(i) * v;
        }
        const T rho = P::shifted ? par<T>(p.rho0, p.rho0_f) + r : r;
        mom[k] = Mom4<T>{r, (jx - par<T>(0.5 * rx.g[0], rx.hg_f[0])) / rho,
                         (jy - par<T>(0.5 * rx.g[1], rx.hg_f[1])) / rho,
                         L::D == 3 ? (jz - par<T>(0.5 * rx.g[2], rx.hg_f[2])) / rho : (T)0};
      }
      dt = collide_adjoint<L, P>(f, lam, mu, p, rx);
#pragma unroll
      for (int i = 0; i < L::Q; ++i) lam_out[(ptrdiff_t)i * (ptrdiff_t)S + (ptrdiff_t)k + d[i]] = mu[i];
    }
  }
  block_add_keyed<T>(dt, key, dtau);
}

// Adds (a_r, a_u) -- adjoints of a node's moments rho and u -- to all
// directions of that node: d rho/df+_j = 1, d u_a/df+_j = (e_ja - u_a)/rho.
template <class L, class T>
__device__ __forceinline__ void scatter_moment_adjoint(T* __restrict__ lam, size_t S, uint32_t k, T ar, T a0, T a1,
                                                       T a2, const Mom4<T>& m, T rho) {
  const T ir = (T)1 / rho;
#pragma unroll
  for (int j = 0; j < L::Q; ++j) {
    const T v = ar + (a0 * ((T)L::cx(j) - m.ux) + a1 * ((T)L::cy(j) - m.uy) + a2 * ((T)L::cz(j) - m.uz)) * ir;
    atomic_add_real(lam + (size_t)j * S + k, v);
  }
}

// One thread per link.  lam: lambda(s) under construction (ghost slots hold
// the weights of the link values); lam_in: lambda(s+1), already read by
// k_adj_bulk, whose entry (i', x_f) is cleared here.  final_step: add the
// objective's direct terms J = sum_b wbody[b] . F_b(step) (wbody: [nbody][3]
// FP64).
// Adjoint of the moments (rho, u) of one node (a_r, a_u) that a link
// leaves to be spread over the node's directions; key = the node's storage
// index, or ~0 for none.
template <class T>
struct MomAdj {
  uint32_t key;
  T ar, a0, a1, a2;
  Mom4<T> m;
  T rho;
};

// Spreads each warp's pending moment adjoints: lanes holding the same node
// (links of one node are consecutive in the link order) are summed by a
// segmented scan and the segment's last lane adds the sum to the node's
// directions (one set of atomics per node instead of one per link).  All 32
// lanes of the warp take part.
template <class L, class T>
__device__ __forceinline__ void spread_moment_adjoints(T* __restrict__ lam, size_t S, MomAdj<T> a) {
  const int lane = threadIdx.x & 31;
  const uint32_t prev = __shfl_up_sync(0xffffffffu, a.key, 1);
  const uint32_t next = __shfl_down_sync(0xffffffffu, a.key, 1);
  const bool head = lane == 0 || prev != a.key;
  const bool tail = lane == 31 || next != a.key;
  const unsigned heads = __ballot_sync(0xffffffffu, head);
  const int start = 31 - __clz(heads & (0xffffffffu >> (31 - lane)));  // head of this lane's segment
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const T r = __shfl_up_sync(0xffffffffu, a.ar, o), x = __shfl_up_sync(0xffffffffu, a.a0, o),
            y = __shfl_up_sync(0xffffffffu, a.a1, o), z = __shfl_up_sync(0xffffffffu, a.a2, o);
    if (lane - o >= start) {
      a.ar += r;
      a.a0 += x;
      a.a1 += y;
      a.a2 += z;
    }
  }
  if (tail && a.key != ~0u) scatter_moment_adjoint<L, T>(lam, S, a.key, a.ar, a.a0, a.a1, a.a2, a.m, a.rho);
}

// The adjoint of link k (k < nl) with the direction table tab; the
// adjoint of x_f's moments is left in ma (spread by the caller).
template <class L, class P>
__device__ __forceinline__ void adj_link(int64_t k, const DirTable<typename P::T, L::Q>& tab,
                                         const typename P::T* __restrict__ f,
                                         const Mom4<typename P::T>* __restrict__ mom, typename P::T* __restrict__ lam,
                                         typename P::T* __restrict__ lam_in, const LinkRec* __restrict__ recs,
                                         const typename P::T* __restrict__ qv, const typename P::T* __restrict__ uwv,
                                         int64_t nl, const Params& p, int64_t S_, double* __restrict__ dq_acc,
                                         int final_step, const double* __restrict__ wbody,
                                         MomAdj<typename P::T>& ma) {
  using T = typename P::T;
  const size_t S = (size_t)S_;
  const LinkRec rec = recs[k];
  const int ip = (int)(rec.meta & 31);
  const int rule = (int)((rec.meta >> 5) & 3);
  const int body = (int)(rec.meta >> 7) - 1;
  const uint32_t kf = rec.kf, kff = rec.kff, ks = rec.ks;
  const int i = tab.opp[ip];
  const T ex = tab.e[ip][0], ey = tab.e[ip][1], ez = tab.e[ip][2];
  const T w = tab.w[ip];
  const T q = qv[k];
  T uw0 = 0, uw1 = 0, uw2 = 0;
  if (uwv) {
    uw0 = uwv[k];
    uw1 = uwv[nl + k];
    if (L::D == 3) uw2 = uwv[2 * nl + k];
  }
  T om = lam[(size_t)i * S + ks];  // weight of this link's value (consumed here)
  if (final_step && body >= 0) {
    // J = w_b . sum (f+_i'(x_f) + L) e_i'
    const double* wb = wbody + 3 * body;
    const T c = (T)(wb[0] * (double)ex + wb[1] * (double)ey + wb[2] * (double)ez);
    om += c;
    atomic_add_real(lam + (size_t)ip * S + kf, c);
  }
  const T rho0 = par<T>(p.rho0, p.rho0_f);
  const T wall = -(T)6 * w * rho0 * (ex * uw0 + ey * uw1 + ez * uw2);
  const T fpf = f[(size_t)ip * S + kf];
  const T two_q = (T)2 * q;
  double dLdq = 0.0;
  if (rule == 0) {
    atomic_add_real(lam + (size_t)ip * S + kf, om);
  } else if (rule == 1) {
    if (q <= (T)0.5) {
      const T fpff = f[(size_t)ip * S + kff];
      atomic_add_real(lam + (size_t)ip * S + kf, two_q * om);
      atomic_add_real(lam + (size_t)ip * S + kff, ((T)1 - two_q) * om);
      dLdq = 2.0 * ((double)fpf - (double)fpff);
    } else {
      const T fpi = f[(size_t)i * S + kf];
      const T inv2q = (T)1 / two_q;
      atomic_add_real(lam + (size_t)ip * S + kf, om * inv2q);
      atomic_add_real(lam + (size_t)i * S + kf, om * ((T)1 - inv2q));
      dLdq = -((double)fpf + (double)wall - (double)fpi) / (2.0 * (double)q * (double)q);
    }
  } else if (rule == 3) {
    // Yu: L = (q f+_i'(x_f) + (1-q) f+_i'(x_ff) + wall)/(1+q) + q/(1+q) f+_i(x_f)
    const T fpff = f[(size_t)ip * S + kff];
    const T fpi = f[(size_t)i * S + kf];
    const T i1q = (T)1 / ((T)1 + q);
    atomic_add_real(lam + (size_t)ip * S + kf, om * q * i1q);
    atomic_add_real(lam + (size_t)ip * S + kff, om * ((T)1 - q) * i1q);
    atomic_add_real(lam + (size_t)i * S + kf, om * q * i1q);
    const double q1 = 1.0 + (double)q;
    dLdq = ((double)fpf - 2.0 * (double)fpff - (double)wall + (double)fpi) / (q1 * q1);
  } else {
    const T fpff = f[(size_t)ip * S + kff];
    const Mom4<T> mf = mom[kf], mff = mom[kff];
    const T rhof = P::shifted ? rho0 + mf.r : mf.r;
    const T rhoff = P::shifted ? rho0 + mff.r : mff.r;
    const bool local = p.vibb_local_rho && q > (T)0.5;
    const T rd = local ? mf.r : two_q * mf.r + ((T)1 - two_q) * mff.r;
    const T rhod = P::shifted ? rho0 + rd : rd;
    const T euf = ex * mf.ux + ey * mf.uy + ez * mf.uz;
    const T euff = ex * mff.ux + ey * mff.uy + ez * mff.uz;
    const T polyf = (T)3 * euf + (T)4.5 * euf * euf - (T)1.5 * (mf.ux * mf.ux + mf.uy * mf.uy + mf.uz * mf.uz);
    const T polyff =
        (T)3 * euff + (T)4.5 * euff * euff - (T)1.5 * (mff.ux * mff.ux + mff.uy * mff.uy + mff.uz * mff.uz);
    const T neq_f = fpf - (P::shifted ? w * (mf.r + rhof * polyf) : w * rhof * ((T)1 + polyf));
    const T neq_ff = fpff - (P::shifted ? w * (mff.r + rhoff * polyff) : w * rhoff * ((T)1 + polyff));
    const T nd = rhod * (two_q * neq_f / rhof + ((T)1 - two_q) * neq_ff / rhoff);
    T af, aff, aw, daf, daff, daw;
    if (q <= (T)0.5) {
      af = two_q;
      aff = (T)1 - two_q;
      aw = 0;
      daf = 2;
      daff = -2;
      daw = 0;
    } else {
      const T iq = (T)1 / q;
      af = ((T)1 - q) * iq;
      aff = 0;
      aw = (two_q - (T)1) * iq;
      daf = -iq * iq;
      daff = 0;
      daw = iq * iq;
    }
    const T i1q = (T)1 / ((T)1 + q);
    const T bff = ((T)1 - q) * i1q, bw = two_q * i1q;
    const T dbff = (T)-2 * i1q * i1q, dbw = (T)2 * i1q * i1q;
    const T third = (T)(1.0 / 3.0), two_thirds = (T)(2.0 / 3.0);
    const T cf = third * af, cff = third * aff + two_thirds * bff, cw = third * aw + two_thirds * bw;
    const T dcf = third * daf, dcff = third * daff + two_thirds * dbff, dcw = third * daw + two_thirds * dbw;
    const T udx = cf * mf.ux + cff * mff.ux + cw * uw0;
    const T udy = cf * mf.uy + cff * mff.uy + cw * uw1;
    const T udz = cf * mf.uz + cff * mff.uz + cw * uw2;
    const T eud = ex * udx + ey * udy + ez * udz;
    const T polyd = (T)3 * eud + (T)4.5 * eud * eud - (T)1.5 * (udx * udx + udy * udy + udz * udz);
    // partial derivatives of L = feq_i'(rd, ud) + nd + wall
    const T gd = w * ((T)1 + polyd) + nd / rhod;                     // d/d rd
    const T aud0 = w * rhod * ((T)3 * ex + (T)9 * eud * ex - (T)3 * udx);  // d/d ud
    const T aud1 = w * rhod * ((T)3 * ey + (T)9 * eud * ey - (T)3 * udy);
    const T aud2 = w * rhod * ((T)3 * ez + (T)9 * eud * ez - (T)3 * udz);
    const T dn_f = rhod * two_q / rhof;                               // d nd / d neq_f
    const T dn_ff = rhod * ((T)1 - two_q) / rhoff;
    const T drd_f = local ? (T)1 : two_q, drd_ff = local ? (T)0 : (T)1 - two_q;
    const T a_rf = gd * drd_f - dn_f * w * ((T)1 + polyf) - rhod * two_q * neq_f / (rhof * rhof);
    const T a_rff = gd * drd_ff - dn_ff * w * ((T)1 + polyff) - rhod * ((T)1 - two_q) * neq_ff / (rhoff * rhoff);
    const T wf = dn_f * w * rhof, wff = dn_ff * w * rhoff;
    const T a_uf0 = aud0 * cf - wf * ((T)3 * ex + (T)9 * euf * ex - (T)3 * mf.ux);
    const T a_uf1 = aud1 * cf - wf * ((T)3 * ey + (T)9 * euf * ey - (T)3 * mf.uy);
    const T a_uf2 = aud2 * cf - wf * ((T)3 * ez + (T)9 * euf * ez - (T)3 * mf.uz);
    const T a_uff0 = aud0 * cff - wff * ((T)3 * ex + (T)9 * euff * ex - (T)3 * mff.ux);
    const T a_uff1 = aud1 * cff - wff * ((T)3 * ey + (T)9 * euff * ey - (T)3 * mff.uy);
    const T a_uff2 = aud2 * cff - wff * ((T)3 * ez + (T)9 * euff * ez - (T)3 * mff.uz);
    atomic_add_real(lam + (size_t)ip * S + kf, om * dn_f);
    atomic_add_real(lam + (size_t)ip * S + kff, om * dn_ff);
    ma = MomAdj<T>{kf, om * a_rf, om * a_uf0, om * a_uf1, om * a_uf2, mf, rhof};
    scatter_moment_adjoint<L, T>(lam, S, kff, om * a_rff, om * a_uff0, om * a_uff1, om * a_uff2, mff, rhoff);
    const double drd_q = local ? 0.0 : 2.0 * ((double)mf.r - (double)mff.r);
    dLdq = (double)gd * drd_q + (double)rhod * (2.0 * (double)neq_f / (double)rhof - 2.0 * (double)neq_ff / (double)rhoff) +
           (double)aud0 * (double)(dcf * mf.ux + dcff * mff.ux + dcw * uw0) +
           (double)aud1 * (double)(dcf * mf.uy + dcff * mff.uy + dcw * uw1) +
           (double)aud2 * (double)(dcf * mf.uz + dcff * mff.uz + dcw * uw2);
  }
  dq_acc[k] += (double)om * dLdq;
  lam[(size_t)i * S + ks] = (T)0;
  lam_in[(size_t)ip * S + kf] = (T)0;
}

// One thread per link.  lam: lambda(s) under construction (ghost slots hold
// the weights of the link values); lam_in: lambda(s+1), already read by
// k_adj_bulk, whose entry (i', x_f) is cleared here.  final_step: add the
// objective's direct terms J = sum_b wbody[b] . F_b(step) (wbody: [nbody][3]
// FP64).
template <class L, class P>
__global__ void __launch_bounds__(256) k_adj_links(const typename P::T* __restrict__ f,
                                                   const Mom4<typename P::T>* __restrict__ mom,
                                                   typename P::T* __restrict__ lam, typename P::T* __restrict__ lam_in,
                                                   const LinkRec* __restrict__ recs,
                                                   const typename P::T* __restrict__ qv,
                                                   const typename P::T* __restrict__ uwv, int64_t nl, Params p,
                                                   int64_t S_, double* __restrict__ dq_acc, int final_step,
                                                   const double* __restrict__ wbody) {
  __shared__ DirTable<typename P::T, L::Q> tab;
  fill_dir_table<L>(tab);
  __syncthreads();
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  MomAdj<typename P::T> ma{~0u, 0, 0, 0, 0, {0, 0, 0, 0}, 1};
  if (k < nl) adj_link<L, P>(k, tab, f, mom, lam, lam_in, recs, qv, uwv, nl, p, S_, dq_acc, final_step, wbody, ma);
  spread_moment_adjoints<L>(lam, (size_t)S_, ma);
}

// Clears in lam_in the entries (j, m) whose neighbour m + e_j is the open
// node of row y, for the directions j with cx(j) = cx: m is the fluid node
// next to the open column in row y - cy(j) (table: row_in1 for the inlet,
// cx = -1; row_out1 for the outlet, cx = +1).
template <class L, class T>
__device__ __forceinline__ void clear_open_neighbours(T* __restrict__ lam_in, const Layout& lay, const Params& p, int y,
                                                      int cx) {
  const int32_t* __restrict__ next = cx < 0 ? lay.row_in1 : lay.row_out1;
#pragma unroll
  for (int j = 0; j < L::Q; ++j) {
    if (L::cx(j) != cx) continue;
    int yy = y - L::cy(j);
    if (yy < 0 || yy >= p.ny) {
      if (!p.periodic[1]) continue;
      yy = (yy + p.ny) % p.ny;
    }
    const int32_t m = next[yy];
    if (m >= 0) lam_in[(size_t)j * lay.S + m] = (T)0;
  }
}

// Open columns (D2Q9): inlet f+(0) = feq(rho1, u_in) + f+(1) - feq(rho1, u1)
// and outlet f+(nx-1) = f+(nx-2), transposed into columns 1 and nx-2 (by
// atomics: cut links of the channel walls add into the same nodes); the open
// nodes' entries are then cleared (they are not state), and so are the
// entries of lambda(s+1) (lam_in, read by k_adj_bulk) that point into an
// open node.  t < ny: inlet of row t; ny <= t < 2 ny: outlet of row t - ny.
template <class L, class P>
__device__ __forceinline__ void adj_open_row(int t, typename P::T* __restrict__ lam, typename P::T* __restrict__ lam_in,
                                             const Mom4<typename P::T>* __restrict__ mom, const Layout& lay,
                                             const Params& p) {
  using T = typename P::T;
  if (t >= 2 * p.ny) return;
  const bool inlet_side = t < p.ny;
  const int y = inlet_side ? t : t - p.ny;
  const size_t S = (size_t)lay.S;
  if (inlet_side && p.inlet) {
    // the inflow velocity does not depend on the row's storage: issued first
    const T uin = (T)inlet_velocity(p, lay, y);
    const int32_t k0 = lay.row_first[y];
    if (k0 >= 0 && (lay.word[k0] & W_OPEN)) {
      const uint32_t k1 = (uint32_t)k0 + 1;
      const Mom4<T> m1 = mom[k1];
      T l0[L::Q];
      T sp = 0, B0 = 0, B1 = 0;
#pragma unroll
      for (int i = 0; i < L::Q; ++i) {
        l0[i] = lam[(size_t)i * S + k0];
        const T ex = (T)L::cx(i), ey = (T)L::cy(i), w = (T)L::w(i);
        const T ein = ex * uin;
        const T e1 = ex * m1.ux + ey * m1.uy;
        const T pin = (T)3 * ein + (T)4.5 * ein * ein - (T)1.5 * uin * uin;
        const T p1 = (T)3 * e1 + (T)4.5 * e1 * e1 - (T)1.5 * (m1.ux * m1.ux + m1.uy * m1.uy);
        sp += l0[i] * w * (pin - p1);
        B0 += l0[i] * w * ((T)3 * ex + (T)9 * e1 * ex - (T)3 * m1.ux);
        B1 += l0[i] * w * ((T)3 * ey + (T)9 * e1 * ey - (T)3 * m1.uy);
      }
#pragma unroll
      for (int j = 0; j < L::Q; ++j)
        atomic_add_real(lam + (size_t)j * S + k1, l0[j] + sp - (B0 * ((T)L::cx(j) - m1.ux) + B1 * ((T)L::cy(j) - m1.uy)));
#pragma unroll
      for (int j = 0; j < L::Q; ++j) lam[(size_t)j * S + k0] = (T)0;
      clear_open_neighbours<L, T>(lam_in, lay, p, y, -1);
    }
  }
  if (!inlet_side && p.outlet) {
    const int32_t kl = lay.row_last[y];
    if (kl >= 0 && (lay.word[kl] & W_OPEN)) {
      T a[L::Q];
#pragma unroll
      for (int i = 0; i < L::Q; ++i) a[i] = lam[(size_t)i * S + kl];
#pragma unroll
      for (int i = 0; i < L::Q; ++i) atomic_add_real(lam + (size_t)i * S + kl - 1, a[i]);
#pragma unroll
      for (int i = 0; i < L::Q; ++i) lam[(size_t)i * S + kl] = (T)0;
      clear_open_neighbours<L, T>(lam_in, lay, p, y, 1);
    }
  }
}

template <class L, class P>
__global__ void k_adj_open(typename P::T* __restrict__ lam, typename P::T* __restrict__ lam_in,
                           const Mom4<typename P::T>* __restrict__ mom, Layout lay, Params p) {
  adj_open_row<L, P>(blockIdx.x * blockDim.x + threadIdx.x, lam, lam_in, mom, lay, p);
}

// The link and open-column transposes of one step in one launch: blocks
// [0, nbo) take the open rows (as k_adj_open; first, so that their scattered
// accesses overlap the link blocks), the others the links (as
// k_adj_links); the two parts touch common entries only through atomics.
template <class L, class P>
__global__ void __launch_bounds__(256) k_adj_links_open(const typename P::T* __restrict__ f,
                                                        const Mom4<typename P::T>* __restrict__ mom,
                                                        typename P::T* __restrict__ lam,
                                                        typename P::T* __restrict__ lam_in,
                                                        const LinkRec* __restrict__ recs,
                                                        const typename P::T* __restrict__ qv,
                                                        const typename P::T* __restrict__ uwv, int64_t nl, Params p,
                                                        int64_t S_, double* __restrict__ dq_acc, int final_step,
                                                        const double* __restrict__ wbody, Layout lay, int nbo) {
  if ((int)blockIdx.x >= nbo) {
    __shared__ DirTable<typename P::T, L::Q> tab;
    fill_dir_table<L>(tab);
    __syncthreads();
    const int64_t k = (blockIdx.x - nbo) * (int64_t)blockDim.x + threadIdx.x;
    MomAdj<typename P::T> ma{~0u, 0, 0, 0, 0, {0, 0, 0, 0}, 1};
    if (k < nl) adj_link<L, P>(k, tab, f, mom, lam, lam_in, recs, qv, uwv, nl, p, S_, dq_acc, final_step, wbody, ma);
    spread_moment_adjoints<L>(lam, (size_t)S_, ma);
  } else {
    adj_open_row<L, P>((int)(blockIdx.x * blockDim.x + threadIdx.x), lam, lam_in, mom, lay, p);
  }
}

// tau-dependence of the initial collision f+(0) = C(feq(rho, u_in)), with
// rho and u_in recovered from f+(0): rho = sum f+, u_in = (sum f+ e - g)/rho.
template <class L, class P>
__global__ void __launch_bounds__(256) k_adj_init(const typename P::T* __restrict__ f0,
                                                  const typename P::T* __restrict__ lam, Layout lay, Params p,
                                                  double* __restrict__ dtau) {
  using T = typename P::T;
  const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
  const size_t S = (size_t)lay.S;
  double dt = 0.0;
  int key = -1;
  if (k < (uint64_t)lay.S && !(lay.word[k] & (W_GHOST | W_OPEN))) {
    const uint32_t run = lay.word[k] & W_RUN;
    key = lay.ndom > 1 ? lay.runs[run].dom : 0;
    const Relax rx = relax_of_run(p, lay, run);
    const double g[3] = {rx.g[0], rx.g[1], rx.g[2]};
    double r = 0.0, j[3] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int i = 0; i < L::Q; ++i) {
      const double v = (double)f0[(size_t)i * S + k] + (P::shifted ? L::w(i) * p.rho0 : 0.0);
      r += v;
      j[0] += L::cx(i) * v;
      j[1] += L::cy(i) * v;
      j[2] += L::cz(i) * v;
    }
    const double uin[3] = {(j[0] - g[0]) / r, (j[1] - g[1]) / r, (j[2] - g[2]) / r};
    const double u[3] = {uin[0] + 0.5 * g[0] / r, uin[1] + 0.5 * g[1] / r, uin[2] + 0.5 * g[2] / r};
    const double uu_in = uin[0] * uin[0] + uin[1] * uin[1] + uin[2] * uin[2];
    const double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    const double ug = u[0] * g[0] + u[1] * g[1] + u[2] * g[2];
#pragma unroll
    for (int i = 0; i < L::Q; ++i) {
      const double ein = L::cx(i) * uin[0] + L::cy(i) * uin[1] + L::cz(i) * uin[2];
      const double eu = L::cx(i) * u[0] + L::cy(i) * u[1] + L::cz(i) * u[2];
      const double eg = L::cx(i) * g[0] + L::cy(i) * g[1] + L::cz(i) * g[2];
      const double f0i = L::w(i) * r * (1.0 + 3.0 * ein + 4.5 * ein * ein - 1.5 * uu_in);
      const double feq = L::w(i) * r * (1.0 + 3.0 * eu + 4.5 * eu * eu - 1.5 * uu);
      const double src = L::w(i) * (3.0 * (eg - ug) + 9.0 * eu * eg);
      dt += (double)lam[(size_t)i * S + k] * (f0i - feq + 0.5 * src);
    }
    dt *= rx.omega * rx.omega;
  }
  block_add_keyed<double>(dt, key, dtau);
}

struct AdjointOps {
  void (*bulk)(const void* fin, void* lam_next, void* lam_out, const Layout& lay, const Params& p, double* dtau,
               void* mom, cudaStream_t s);
  // lam: lambda(s) (output); lam_in: lambda(s+1), read by bulk before
  void (*links)(const void* f, const void* mom, void* lam, void* lam_in, const LinkRec* recs, const void* q,
                const void* uw, int64_t nl, const Params& p, int64_t S, double* dq_acc, int final_step,
                const double* wbody, cudaStream_t s);
  void (*open)(void* lam, void* lam_in, const void* mom, const Layout& lay, const Params& p, cudaStream_t s);
  // links and open columns in one launch (lattices with open columns)
  void (*links_open)(const void* f, const void* mom, void* lam, void* lam_in, const LinkRec* recs, const void* q,
                     const void* uw, int64_t nl, const Params& p, int64_t S, double* dq_acc, int final_step,
                     const double* wbody, const Layout& lay, cudaStream_t s);
  void (*init)(const void* f0, const void* lam, const Layout& lay, const Params& p, double* dtau, cudaStream_t s);
};

template <class L, class P>
struct AdjointLaunch {
  using T = typename P::T;
  static void bulk(const void* fin, void* lam_next, void* lam_out, const Layout& lay, const Params& p, double* dtau,
                   void* mom, cudaStream_t s) {
    if (lay.S == 0) return;
    k_adj_bulk<L, P><<<blocks_for(lay.S, 256), 256, 0, s>>>((const T*)fin, (T*)lam_next, (T*)lam_out, lay, p, dtau,
                                                           (Mom4<T>*)mom);
  }
  static void links(const void* f, const void* mom, void* lam, void* lam_in, const LinkRec* recs, const void* q,
                    const void* uw, int64_t nl, const Params& p, int64_t S, double* dq_acc, int final_step,
                    const double* wbody, cudaStream_t s) {
    if (nl == 0) return;
    k_adj_links<L, P><<<blocks_for(nl, 256), 256, 0, s>>>((const T*)f, (const Mom4<T>*)mom, (T*)lam, (T*)lam_in,
                                                         recs, (const T*)q, (const T*)uw, nl, p, S, dq_acc,
                                                         final_step, wbody);
  }
  static void links_open(const void* f, const void* mom, void* lam, void* lam_in, const LinkRec* recs, const void* q,
                         const void* uw, int64_t nl, const Params& p, int64_t S, double* dq_acc, int final_step,
                         const double* wbody, const Layout& lay, cudaStream_t s) {
    const int nbl = (int)blocks_for(nl, 256);
    const int nbo = (int)blocks_for(2 * (int64_t)p.ny, 256);
    k_adj_links_open<L, P><<<nbl + nbo, 256, 0, s>>>((const T*)f, (const Mom4<T>*)mom, (T*)lam, (T*)lam_in, recs,
                                                     (const T*)q, (const T*)uw, nl, p, S, dq_acc, final_step, wbody,
                                                     lay, nbo);
  }
  static void open(void* lam, void* lam_in, const void* mom, const Layout& lay, const Params& p, cudaStream_t s) {
    k_adj_open<L, P><<<blocks_for(2 * (int64_t)p.ny, 128), 128, 0, s>>>((T*)lam, (T*)lam_in, (const Mom4<T>*)mom, lay, p);
  }
  static void init(const void* f0, const void* lam, const Layout& lay, const Params& p, double* dtau,
                   cudaStream_t s) {
    if (lay.S == 0) return;
    k_adj_init<L, P><<<blocks_for(lay.S, 256), 256, 0, s>>>((const T*)f0, (const T*)lam, lay, p, dtau);
  }
  static AdjointOps ops() { return AdjointOps{bulk, links, open, links_open, init}; }
};

AdjointOps adj_d2q9_f64();
AdjointOps adj_d2q9_f32s();
AdjointOps adj_d3q19_f64();
AdjointOps adj_d3q19_f32s();

}  // namespace lbm
