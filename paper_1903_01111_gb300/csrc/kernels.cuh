// CUDA kernels of the lattice-Boltzmann step with velocity-interpolation
// bounce-back (arXiv:1903.01111), templated on the velocity set (D2Q9,
// D3Q19) and the storage precision:
//   F64  -- populations f_i stored in double;
//   F32S -- populations stored in float as h_i = f_i - w_i rho0 ("shifted"),
//           so the O(1) rest part w_i rho0 never enters a float rounding.
//
// Storage (compacted): only fluid nodes, open-column nodes and ghost nodes
// (solid nodes that receive a link's missing population) are stored, in
// x-row order; k is the storage index, S their number.  SoA f[i*S + k].
// A fluid run (maximal x-run of fluid nodes in one row) has every node of
// its neighbour rows over [x0 - 1, x_end + 1] stored and contiguous, so one
// run record (the storage index of (x0, row') for each neighbour row)
// addresses every pull; pulls across the periodic x seam use the row's first
// and last storage index.  The buffer read by a step holds f+(t) of every
// fluid node; ghost slots are filled by the link kernel before the bulk
// kernel pulls them.
//
// Step t -> t+1, on one stream, in one of two forms.  Fused (the default on
// lattices with cut links): k_fused stages each block's pulls in shared
// memory, evaluates the block's link rules into the staged slots and
// collides (after k_open where there are open columns).  Split (the
// adjoint's recompute, and wherever the autotuner finds it faster):
//   k_links: per cut link (x_f, i'), the missing f_i(x_f, t+1), i = opp(i'),
//            from f+ and the moment cache at x_f and x_ff (Sec. 3 and 3.1),
//            written to the ghost slot f[i][k_s] (read only by x_f);
//            momentum exchange force in FP64.
//   k_open:  inlet/outlet columns (Sec. 4.3), D2Q9 only.
//   k_bulk:  pull streaming f_i(x, t+1) = f+_i(x - e_i, t) (Eq. 1), moments,
//            Guo-forced BGK (Sec. 2, Eq. feq) -> f+(t+1) into the other
//            buffer; rho, u(t+1) into the moment cache where flagged.  Ghost
//            and open slots of the output get zeros (through the same store
//            instructions as the fluid slots) so that every written sector
//            is complete.  FP64 one-node shapes run k_bulk_list instead, over
//            the fluid nodes alone.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "lattice.cuh"

namespace lbm {

// bulk_min_blocks: resident 256-thread blocks per SM the bulk kernel is
// compiled for (FP32: 5, FP64: 2; 6 for FP32 forces spills and ran slower on
// the porous workload).
struct F64 {
  using T = double;
  static constexpr bool shifted = false;
  static constexpr int bulk_min_blocks = 2;
};
struct F32S {
  using T = float;
  static constexpr bool shifted = true;
  static constexpr int bulk_min_blocks = 5;
};

// One moment-cache record per node: (r, ux, uy, uz) with r = rho (F64) or
// rho - rho0 (F32S); 16 B (FP32) or 32 B (FP64), loaded in one piece.
template <class T>
struct __align__(4 * sizeof(T)) Mom4 {
  T r, ux, uy, uz;
};

// Per stored node word: run id of a fluid node and its cache flag, or the
// open / ghost bit.
constexpr uint32_t W_RUN = (1u << 29) - 1;
constexpr uint32_t W_CACHE = 1u << 29;
constexpr uint32_t W_OPEN = 1u << 30;
constexpr uint32_t W_GHOST = 1u << 31;

// One fluid run starting at x0 with storage index k0: xk = x0 - k0 (so that
// node k of the run sits at x = k + xk), its row (y, z), the domain the row
// belongs to, and for each neighbour row (slot order below) dbase = the
// storage index of (x0, row') minus k0 (so that the pull from (x + dx, row')
// is k + dbase + dx).  48 B.
struct __align__(16) RunRec {
  int32_t xk, y, z, dom;
  int32_t dbase[8];
};

// Run parameters of one domain of a batch (several independent flows
// stacked along the last axis of one lattice, each with its own relaxation
// time, body force and inlet profile).  A lattice of one domain reads Params.
struct DomPar {
  double omega, fpre3;    // 1/tau, 3 (1 - 1/(2 tau))
  double g[3];
  double inlet_umax, inlet_y0, inlet_y1;  // inlet rows relative to lo
  int32_t lo, has_force;  // first row (y in 2-D, z in 3-D) of the domain
  float omega_f, fpre3_f, g_f[3], hg_f[3], omega2_f;  // float copies, as in Params
  Folded kc;              // collision constants, as in Params
};

// Collision parameters of one node, from Params or from its domain.
struct Relax {
  double omega, fpre3, g[3];
  int has_force;
  float omega_f, fpre3_f, g_f[3], hg_f[3], omega2_f;
};

// A run parameter in the storage precision: the double, or its float copy
// rounded on the host (the same value as a conversion on the device).
template <class T>
__host__ __device__ __forceinline__ T par(double d, float f) {
  if constexpr (sizeof(T) == sizeof(float))
    return f;
  else
    return d;
}

// Neighbour-row slots by source-row offset (dy, dz).  D2Q9: (1,0), (-1,0).
// D3Q19: (1,0), (-1,0), (0,1), (0,-1), (1,1), (-1,-1), (1,-1), (-1,1).
__host__ __device__ constexpr int row_slot(int dy, int dz) {
  return dz == 0 ? (dy > 0 ? 0 : 1)
                 : (dy == 0 ? (dz > 0 ? 2 : 3) : (dy == dz ? (dy > 0 ? 4 : 5) : (dy > 0 ? 6 : 7)));
}

struct Layout {
  int64_t S;                   // stored nodes
  const uint32_t* word;        // [S]
  const int32_t* node_of;      // [S] dense node index
  const RunRec* runs;
  const int32_t* row_first;    // [ny*nz] storage index of the row's first stored node (-1: none)
  const int32_t* row_last;     // [ny*nz] ... last stored node
  const int32_t* row_in1;      // [ny*nz] storage index of the fluid node at x = 1 (open inlet rows), else -1
  const int32_t* row_out1;     // [ny*nz] ... at x = width - 2 (open outlet rows), else -1
  const DomPar* dom;           // [ndom] when ndom > 1, else null
  const int32_t* row_dom;      // [ny*nz] domain of each row when ndom > 1
  int32_t ndom;
  const uint32_t* fluid;       // [nfluid] storage indices of the fluid nodes (FP64 lattices), else null
  int64_t nfluid;
};

__device__ __forceinline__ Relax relax_params(const Params& p) {
  return Relax{p.omega,   p.fpre3,   {p.g[0], p.g[1], p.g[2]},          p.has_force,
               p.omega_f, p.fpre3_f, {p.g_f[0], p.g_f[1], p.g_f[2]}, {p.hg_f[0], p.hg_f[1], p.hg_f[2]},
               p.omega2_f};
}

__device__ __forceinline__ Relax relax_domain(const DomPar* __restrict__ dp, int d) {
  const DomPar& q = dp[d];
  return Relax{q.omega,   q.fpre3,   {q.g[0], q.g[1], q.g[2]},          q.has_force,
               q.omega_f, q.fpre3_f, {q.g_f[0], q.g_f[1], q.g_f[2]}, {q.hg_f[0], q.hg_f[1], q.hg_f[2]},
               q.omega2_f};
}

// Relaxation of a node of fluid run `run` (any kernel but the bulk one,
// which resolves the single-domain case at compile time).
__device__ __forceinline__ Relax relax_of_run(const Params& p, const Layout& lay, uint32_t run) {
  return lay.ndom > 1 ? relax_domain(lay.dom, lay.runs[run].dom) : relax_params(p);
}

// One link: storage indices of x_f, x_ff (x_f if no second fluid node) and
// the ghost x_s; meta = dir | rule << 5 | (body + 1) << 7 (25 bits of body).
struct __align__(16) LinkRec {
  uint32_t kf, kff, ks, meta;
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
// populations f(x, t+1) in storage form; n < 2^31.  keep == false (a ghost
// or open slot in the bulk pass): the same instructions store zeros and the
// moment cache is not written, so that a warp mixing fluid and ghost slots
// issues one store per direction instead of two divergent store sequences.
// Weight class of direction i: 0 rest, 1 |e| = 1, 2 diagonal.
template <class L>
__host__ __device__ constexpr int weight_class(int i) {
  return i == 0 ? 0 : (L::w(i) == L::w(1) ? 1 : 2);
}

// The node's collision constants folded on the host: the lattice's (Params)
// or its domain's (DomPar), both filled by fold.
template <bool MULTI>
__device__ __forceinline__ const Folded& folded_of(const Params& p, const Layout& lay, int dom) {
  if constexpr (MULTI)
    return lay.dom[dom].kc;
  else
    return p.kc;
}

// Collision and store of one node: moments of f, Guo-forced BGK (or D2Q9
// MRT) with the run parameters rx and the folded constants kc, the node's
// moment cache entry when flagged.
#define LBM_K(name) par<T>(kc.name, kc.name##_f)
#define LBM_KI(name, i) par<T>(kc.name[i], kc.name##_f[i])
template <class L, class P>
__device__ __forceinline__ void collide_store(typename P::T (&f)[L::Q], const Params& p, const Relax& rx,
                                              const Folded& kc,
                                              typename P::T* __restrict__ fout, size_t S, uint32_t n_,
                                              Mom4<typename P::T>* __restrict__ mom, bool cache, bool keep = true) {
  using T = typename P::T;
  T r = 0, jx = 0, jy = 0, jz = 0;
  if constexpr (!P::shifted) {
    // FP64 (bound by the FP64 pipe, where every add, multiply or FMA takes
    // one issue slot): density and momentum from the sums and differences of
    // opposite directions, Q - 1 operations fewer than summing the
    // directions into each moment
    r = f[0];
#pragma unroll
    for (int i = 1; i < L::Q; ++i) {
      const int j = L::opp(i);
      if (j < i) continue;
      r += f[i] + f[j];
      const T d = f[i] - f[j];
      if (L::cx(i) > 0) jx += d;
      if (L::cx(i) < 0) jx -= d;
      if (L::cy(i) > 0) jy += d;
      if (L::cy(i) < 0) jy -= d;
      if (L::cz(i) > 0) jz += d;
      if (L::cz(i) < 0) jz -= d;
    }
  } else {
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
  }
  const T rho = P::shifted ? par<T>(p.rho0, p.rho0_f) + r : r;
  const T gx = par<T>(rx.g[0], rx.g_f[0]), gy = par<T>(rx.g[1], rx.g_f[1]), gz = par<T>(rx.g[2], rx.g_f[2]);
  const T inv = (T)1 / rho;
  // Guo forcing: velocity shifted by half the body force
  const T hx = LBM_KI(hg, 0), hy = LBM_KI(hg, 1), hz = LBM_KI(hg, 2);
  const T ux = (jx + hx) * inv, uy = (jy + hy) * inv, uz = (jz + hz) * inv;
  if (cache && keep) mom[n_] = Mom4<T>{r, ux, uy, L::D == 3 ? uz : (T)0};
  const T omega = par<T>(rx.omega, rx.omega_f);
  const T uu15 = (T)1.5 * (ux * ux + uy * uy + uz * uz);
  if constexpr (L::Q == 9) {
    if (p.collision == 1) {
      // MRT (Sec. 2, Eq. mrt) on the non-equilibrium part n = f - feq, whose
      // moments are m - meq (meq = M feq, the moments of the BGK
      // equilibrium); Guo source in moment space scaled by (1 - s_k/2).
      const T gx_ = gx, gy_ = gy;
      const T ug2 = ux * gx_ + uy * gy_;
      T n[9], src[9];
#pragma unroll
      for (int i = 0; i < 9; ++i) {
        const T eu = (T)L::cx(i) * ux + (T)L::cy(i) * uy;
        const T w = (T)L::w(i);
        const T poly = (T)3 * eu + (T)4.5 * eu * eu - uu15;
        const T feq = P::shifted ? w * (r + rho * poly) : (w * rho) * ((T)1 + poly);
        n[i] = f[i] - feq;
        const T eg = (T)L::cx(i) * gx_ + (T)L::cy(i) * gy_;
        src[i] = rx.has_force ? w * ((T)3 * (eg - ug2) + (T)9 * eu * eg) : (T)0;
      }
      T dm[9];
#pragma unroll
      for (int k = 0; k < 9; ++k) {
        T mn = 0, ms = 0;
#pragma unroll
        for (int i = 0; i < 9; ++i) {
          if (mrt_m(k, i) != 0) {
            mn += (T)mrt_m(k, i) * n[i];
            ms += (T)mrt_m(k, i) * src[i];
          }
        }
        const T sk = (k == 7 || k == 8) ? omega : (T)((k == 0 || k == 3 || k == 5) ? 0.3 : (k == 1 || k == 2) ? 1.5 : 1.2);
        dm[k] = (sk * mn - ((T)1 - (T)0.5 * sk) * ms) / (T)mrt_norm2(k);
      }
#pragma unroll
      for (int i = 0; i < 9; ++i) {
        T d = 0;
#pragma unroll
        for (int k = 0; k < 9; ++k)
          if (mrt_m(k, i) != 0) d += (T)mrt_m(k, i) * dm[k];
        fout[(size_t)i * S + n_] = keep ? f[i] - d : (T)0;
      }
      return;
    }
  }
  // BGK with the Guo source (1 - 1/(2 tau)) w_i [3 (e_i - u).g + 9 (e_i.u)(e_i.g)]
  //   = 3 (1 - 1/(2 tau)) w_i [(e_i.g)(1 + 3 e_i.u) - u.g].
  const T ug = rx.has_force ? ux * gx + uy * gy + uz * gz : (T)0;
  if constexpr (P::shifted) {
    // Shifted FP32 storage: each direction keeps its own equilibrium
    // feq_i = w (r + rho poly_i) and relaxes in the difference form
    // f + omega (feq - f), so that rounding falls on the small
    // non-equilibrium part; opposite directions (i, j = opp(i), e_j = -e_i)
    // share e.u, the symmetric part 4.5 (e.u)^2 - 1.5 u.u of the polynomial
    // and the two parts of the source, Sc +- So with Sc = kt_i (e_i.u) -
    // kf_c (u.g) and So = ke_i from the folded constants.  (Relaxing the
    // pair's symmetric and antisymmetric parts separately, as FP64 does,
    // measured 5x larger FP32 errors in drag and in the adjoint's dJ/dtau.)
    T sc[3] = {0, 0, 0};
    if (rx.has_force) {
#pragma unroll
      for (int c = 0; c < 3; ++c) sc[c] = LBM_KI(kf, c) * ug;
    }
#pragma unroll
    for (int i = 0; i < L::Q; ++i) {
      const int j = L::opp(i);
      if (i != 0 && j < i) continue;
      const T eu = (T)L::cx(i) * ux + (T)L::cy(i) * uy + (T)L::cz(i) * uz;
      const T w = (T)L::w(i);
      const T sym = (T)4.5 * eu * eu - uu15;
      const T feqi = w * (r + rho * (sym + (T)3 * eu));
      T oi = f[i] + omega * (feqi - f[i]);
      T Sc = 0, So = 0;
      if (rx.has_force) {
        Sc = LBM_KI(kt, i) * eu - sc[weight_class<L>(i)];
        So = LBM_KI(ke, i);
        oi += Sc + So;
      }
      fout[(size_t)i * S + n_] = keep ? oi : (T)0;
      if (i != 0) {
        const T feqj = w * (r + rho * (sym - (T)3 * eu));
        T oj = f[j] + omega * (feqj - f[j]);
        if (rx.has_force) oj += Sc - So;
        fout[(size_t)j * S + n_] = keep ? oj : (T)0;
      }
    }
  } else {
    // FP64 (bound by the FP64 pipe, where every add, multiply or FMA takes
    // one issue slot): per pair of opposite directions (i, j = opp(i)),
    // e_j = -e_i turns the equilibria into A +- B and the sources into
    // Sc +- So, so that with the folded constants
    //   a_c = ko_c rho (1 - 1.5 u.u) - kf_c (u.g),  h_c = kh_c rho,  b_c = kb_c rho,
    //   P = (h_c eu + kt_i) eu + a_c = omega A + Sc,  M = b_c eu + ke_i = omega B + So,
    //   f+_i,j = (1 - omega) f_i,j + (P +- M):
    // the source's symmetric part joins the FMAs of the equilibrium's, its
    // antisymmetric part the FMA of M, and a pair costs an FMA and a multiply
    // for P, an FMA for M and two adds and two FMAs for the outputs.
    const T om1 = LBM_K(om1);
    const T c0 = (T)1 - uu15;
    {
      const T out = om1 * f[0] + ((LBM_KI(ko, 0) * rho) * c0 - LBM_KI(kf, 0) * ug);
      fout[n_] = keep ? out : (T)0;
    }
    T a[3], h[3], b[3];
#pragma unroll
    for (int c = 1; c < 3; ++c) {
      a[c] = (LBM_KI(ko, c) * rho) * c0 - LBM_KI(kf, c) * ug;
      h[c] = LBM_KI(kh, c) * rho;
      b[c] = LBM_KI(kb, c) * rho;
    }
#pragma unroll
    for (int i = 1; i < L::Q; ++i) {
      const int j = L::opp(i);
      if (j < i) continue;
      const int c = weight_class<L>(i);
      const T eu = (T)L::cx(i) * ux + (T)L::cy(i) * uy + (T)L::cz(i) * uz;
      const T Pv = (h[c] * eu + LBM_KI(kt, i)) * eu + a[c];
      const T Mv = b[c] * eu + LBM_KI(ke, i);
      fout[(size_t)i * S + n_] = keep ? om1 * f[i] + (Pv + Mv) : (T)0;
      fout[(size_t)j * S + n_] = keep ? om1 * f[j] + (Pv - Mv) : (T)0;
    }
  }
}

#undef LBM_K
#undef LBM_KI

// Storage indices of the pull sources x - e_i of fluid node k of run `run`.
template <class L>
__device__ __forceinline__ void pull_sources(uint32_t k, const RunRec& run, const Layout& lay, const Params& p,
                                             uint32_t (&src)[L::Q]) {
  const int nx = p.nx;
  const int x = (int)k + run.xk;
  const bool left = x == 0, right = x == nx - 1;
#pragma unroll
  for (int i = 0; i < L::Q; ++i) {
    // source x - e_i: offsets (dx, dy, dz) = -(cx, cy, cz)
    const int dx = -L::cx(i), dy = -L::cy(i), dz = -L::cz(i);
    if (dy == 0 && dz == 0) {
      if (dx == 0) {
        src[i] = k;
      } else if ((dx < 0 && left) || (dx > 0 && right)) {
        const int row = run.y + p.ny * run.z;
        src[i] = (uint32_t)(dx < 0 ? lay.row_last[row] : lay.row_first[row]);
      } else {
        src[i] = k + dx;
      }
    } else {
      if ((dx < 0 && left) || (dx > 0 && right)) {
        int yy = run.y + dy, zz = run.z + dz;
        yy = yy < 0 ? yy + p.ny : (yy >= p.ny ? yy - p.ny : yy);
        zz = zz < 0 ? zz + p.nz : (zz >= p.nz ? zz - p.nz : zz);
        const int row = yy + p.ny * zz;
        src[i] = (uint32_t)(dx < 0 ? lay.row_last[row] : lay.row_first[row]);
      } else {
        src[i] = (uint32_t)((int)k + run.dbase[row_slot(dy, dz)] + dx);
      }
    }
  }
}

// Offsets src_i - k of the pull sources of fluid node k (run `run`): away
// from the periodic x seam every offset is a per-run constant (dx in the
// node's own row, base - k0 + dx in a neighbour row); at the seam (x = 0 or
// nx - 1 of a periodic row) they come from pull_sources.
template <class L>
__device__ __forceinline__ void pull_offsets(uint32_t k, const RunRec& run, const Layout& lay, const Params& p,
                                             int (&d)[L::Q]) {
  const int x = (int)k + run.xk;
  if (x > 0 && x < p.nx - 1) {
#pragma unroll
    for (int i = 0; i < L::Q; ++i) {
      const int dx = -L::cx(i), dy = -L::cy(i), dz = -L::cz(i);
      d[i] = (dy == 0 && dz == 0) ? dx : run.dbase[row_slot(dy, dz)] + dx;
    }
    return;
  }
  uint32_t src[L::Q];
  pull_sources<L>(k, run, lay, p, src);
#pragma unroll
  for (int i = 0; i < L::Q; ++i) d[i] = (int)(src[i] - k);
}

// ------------------------------------------------------------------ bulk --

// Shapes of the bulk kernel the autotuner chooses from: threads per block,
// nodes per thread in parallel (a thread with two nodes takes k and
// k + ceil(S/2), both ranges coalesced, and has 2Q loads in flight) and nodes
// per thread in sequence (a thread walks k, k + G, k + 2G, ... over the grid
// G and loads the next node's word and run while the current node's pulls
// are in flight).  Two nodes per thread and the sequential walk are built
// for D2Q9 only (D3Q19 threads already have 19 loads in flight).
struct BulkShape {
  int threads, npt, seq;
};
constexpr BulkShape kBulkShapes[] = {{256, 1, 1}, {128, 1, 1}, {512, 1, 1}, {256, 2, 1},
                                     {128, 2, 1}, {512, 2, 1}, {128, 1, 4}, {128, 1, 8}};
constexpr int kNumBulkShapes = 8;

template <class L>
constexpr int bulk_max_npt() {
  return L::Q == 9 ? 2 : 1;
}

// Shapes built for a stencil, one bit per shape.
template <class L>
constexpr unsigned bulk_shape_mask() {
  return L::Q == 9 ? 0xffu : 0x07u;
}

// Default shape: two nodes per thread in 256-thread blocks for D2Q9; one
// node per thread in 128-thread blocks for D3Q19 (the autotuner's choice on
// dense and porous D3Q19 lattices in both precisions, and the fused step's
// best block: 1.30 ms per step on a 384^3 pack against 1.37 at 256).
template <class L>
constexpr int bulk_default_shape() {
  return L::Q == 9 ? 3 : 1;
}

// Resident blocks per SM a shape is compiled for, from a register budget per
// 256 threads: FP32 D2Q9 6 blocks with one node per thread (40 registers) and
// 4 with two; FP32 D3Q19 5 (48 registers); FP64 2.  Measured: one block more
// spills (D3Q19) or runs slower (D2Q9 two nodes); one fewer leaves too few
// loads in flight.
template <class L, class P, int BT, int NPT>
constexpr int bulk_blocks_per_sm() {
  constexpr int base = !P::shifted ? 2 : (L::Q == 9 ? (NPT == 1 ? 6 : 4) : 5);
  return base * 256 / BT < 1 ? 1 : base * 256 / BT;
}

// MULTI: the lattice holds several domains; each node's collision reads its
// run's domain parameters.  Block (0) also clears the force slot of the
// next step.
template <class L, class P, bool MULTI, int BT, int NPT>
__global__ void __launch_bounds__(BT, (bulk_blocks_per_sm<L, P, BT, NPT>())) k_bulk(const typename P::T* __restrict__ fin,
                                                                       typename P::T* __restrict__ fout, Layout lay,
                                                                       Mom4<typename P::T>* __restrict__ mom,
                                                                       double* __restrict__ force_next, Params p) {
  using T = typename P::T;
  if (force_next && blockIdx.x == 0)
    for (int t = threadIdx.x; t < 3 * p.nbody; t += BT) force_next[t] = 0.0;
  const uint32_t t = blockIdx.x * BT + threadIdx.x;
  const size_t S = (size_t)lay.S;
  const uint32_t stride = (uint32_t)((S + NPT - 1) / NPT);
  uint32_t k[NPT], w[NPT];
  int dom[NPT];
  bool live[NPT];
  T f[NPT][L::Q];
#pragma unroll
  for (int j = 0; j < NPT; ++j) {
    k[j] = t + (uint32_t)j * stride;
    live[j] = t < stride && (uint64_t)k[j] < S;
    w[j] = live[j] ? __ldg(lay.word + k[j]) : W_GHOST;
    dom[j] = 0;
    if (live[j] && !(w[j] & (W_GHOST | W_OPEN))) {
      const RunRec run = lay.runs[w[j] & W_RUN];
      if (MULTI) dom[j] = run.dom;
      int d[L::Q];
      pull_offsets<L>(k[j], run, lay, p, d);
      const T* __restrict__ fk = fin + k[j];
#pragma unroll
      for (int i = 0; i < L::Q; ++i) f[j][i] = __ldg(fk + ((ptrdiff_t)i * (ptrdiff_t)S + d[i]));
    }
  }
#pragma unroll
  for (int j = 0; j < NPT; ++j) {
    if (!live[j]) continue;
    // ghost and open slots: zeros through the same stores (inputs at rest)
    const bool fl = !(w[j] & (W_GHOST | W_OPEN));
    if (!fl) {
#pragma unroll
      for (int i = 0; i < L::Q; ++i) f[j][i] = P::shifted ? (T)0 : (T)L::w(i);
    }
    const Relax rx = MULTI ? relax_domain(lay.dom, dom[j]) : relax_params(p);
    collide_store<L, P>(f[j], p, rx, folded_of<MULTI>(p, lay, dom[j]), fout, S, k[j], mom, (w[j] & W_CACHE) != 0,
                        fl);
  }
}

// FP64 bulk pass over the fluid nodes alone, one thread per entry of the
// layout's fluid list, otherwise as k_bulk.  An FP64 warp instruction holds
// the FP64 pipe for the same time whatever its active lanes, so the ghost
// and open slots that k_bulk's warps carry (23 % of a porous pack's storage)
// cost as much as fluid nodes there; this pass has no such lanes.  It leaves
// the ghost and open slots of the output unwritten: a ghost slot is read
// only in its link's direction after the link kernel of the next step has
// written it, and the open-column kernel rewrites the open slots before they
// are pulled.
template <class L, class P, bool MULTI, int BT>
__global__ void __launch_bounds__(BT, (bulk_blocks_per_sm<L, P, BT, 1>())) k_bulk_list(
    const typename P::T* __restrict__ fin, typename P::T* __restrict__ fout, Layout lay,
    Mom4<typename P::T>* __restrict__ mom, double* __restrict__ force_next, Params p) {
  using T = typename P::T;
  if (force_next && blockIdx.x == 0)
    for (int t = threadIdx.x; t < 3 * p.nbody; t += BT) force_next[t] = 0.0;
  const int64_t t = (int64_t)blockIdx.x * BT + threadIdx.x;
  if (t >= lay.nfluid) return;
  const size_t S = (size_t)lay.S;
  const uint32_t k = __ldg(lay.fluid + t);
  const uint32_t w = __ldg(lay.word + k);
  const RunRec run = lay.runs[w & W_RUN];
  int d[L::Q];
  pull_offsets<L>(k, run, lay, p, d);
  T f[L::Q];
  const T* __restrict__ fk = fin + k;
#pragma unroll
  for (int i = 0; i < L::Q; ++i) f[i] = __ldg(fk + ((ptrdiff_t)i * (ptrdiff_t)S + d[i]));
  const Relax rx = MULTI ? relax_domain(lay.dom, run.dom) : relax_params(p);
  collide_store<L, P>(f, p, rx, folded_of<MULTI>(p, lay, run.dom), fout, S, k, mom, (w & W_CACHE) != 0);
}

// Resident blocks per SM of the sequential walk (it keeps the next node's
// word and run live): 4 per 256 threads in FP32 (64 registers, no spill;
// at 40 registers the spills cost more than the prefetch wins), 2 in FP64.
template <class P, int BT>
constexpr int bulk_seq_blocks_per_sm() {
  return (P::shifted ? 4 : 2) * 256 / BT;
}

// The fields of a run record that the pull offsets use away from the seam.
template <class L>
struct RunLite {
  int32_t xk, dom;
  int32_t dbase[L::D == 2 ? 2 : 8];
};

template <class L, bool MULTI>
__device__ __forceinline__ RunLite<L> load_run_lite(const RunRec* __restrict__ runs, uint32_t r) {
  RunLite<L> v;
  v.xk = runs[r].xk;
  v.dom = MULTI ? runs[r].dom : 0;
#pragma unroll
  for (int sl = 0; sl < (L::D == 2 ? 2 : 8); ++sl) v.dbase[sl] = runs[r].dbase[sl];
  return v;
}

// Sequential walk over the grid: the word of the node after next is loaded
// while the current node's pulls are in flight, and the next node's run
// record right after the current node's stores (D2Q9).
template <class L, class P, bool MULTI, int BT, int SEQ>
__global__ void __launch_bounds__(BT, (bulk_seq_blocks_per_sm<P, BT>())) k_bulk_seq(
    const typename P::T* __restrict__ fin, typename P::T* __restrict__ fout, Layout lay,
    Mom4<typename P::T>* __restrict__ mom, double* __restrict__ force_next, Params p) {
  using T = typename P::T;
  if (force_next && blockIdx.x == 0)
    for (int t = threadIdx.x; t < 3 * p.nbody; t += BT) force_next[t] = 0.0;
  const size_t S = (size_t)lay.S;
  const uint32_t G = gridDim.x * BT;
  uint32_t k = blockIdx.x * BT + threadIdx.x;
  uint32_t w = k < S ? __ldg(lay.word + k) : W_GHOST;
  RunLite<L> run{};
  if (!(w & (W_GHOST | W_OPEN))) run = load_run_lite<L, MULTI>(lay.runs, w & W_RUN);
  uint32_t w2 = ((uint64_t)k + G < S) ? __ldg(lay.word + k + G) : W_GHOST;
#pragma unroll 1
  for (int it = 0; it < SEQ && (uint64_t)k < S; ++it, k += G) {
    T f[L::Q];
    const bool fluid = !(w & (W_GHOST | W_OPEN));
    if (fluid) {
      int d[L::Q];
      const int x = (int)k + run.xk;
      if (x > 0 && x < p.nx - 1) {
#pragma unroll
        for (int i = 0; i < L::Q; ++i) {
          const int dx = -L::cx(i), dy = -L::cy(i), dz = -L::cz(i);
          d[i] = (dy == 0 && dz == 0) ? dx : run.dbase[row_slot(dy, dz)] + dx;
        }
      } else {
        pull_offsets<L>(k, lay.runs[w & W_RUN], lay, p, d);
      }
      const T* __restrict__ fk = fin + k;
#pragma unroll
      for (int i = 0; i < L::Q; ++i) f[i] = __ldg(fk + ((ptrdiff_t)i * (ptrdiff_t)S + d[i]));
    }
    const uint32_t w3 = ((uint64_t)k + 2ull * G < S) ? __ldg(lay.word + k + 2 * G) : W_GHOST;
    // (a separate zero-store branch here: the walk serves dense lattices,
    // where selecting zeros in every store measured about 2 % slower)
    if (!fluid) {
#pragma unroll
      for (int i = 0; i < L::Q; ++i) fout[(size_t)i * S + k] = (T)0;
    } else {
      const Relax rx = MULTI ? relax_domain(lay.dom, run.dom) : relax_params(p);
      collide_store<L, P>(f, p, rx, folded_of<MULTI>(p, lay, run.dom), fout, S, k, mom, (w & W_CACHE) != 0);
    }
    // the next node's run record, loaded before its pulls are needed
    w = w2;
    if ((uint64_t)k + G < S && !(w & (W_GHOST | W_OPEN))) run = load_run_lite<L, MULTI>(lay.runs, w & W_RUN);
    w2 = w3;
  }
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

// Missing population f_i(x_f, t+1) of one link in storage form (see the
// rule list below).  fpf = f+_i'(x_f), fpff = f+_i'(x_ff), fpi = f+_i(x_f)
// (only read by the rule that needs it, through the callbacks' values);
// mf, mff: moments at time t at x_f and x_ff; (w, ex, ey, ez) of i'.
template <class P>
__device__ __forceinline__ typename P::T link_value(int rule, typename P::T q, typename P::T w, typename P::T ex,
                                                    typename P::T ey, typename P::T ez, typename P::T fpf,
                                                    typename P::T fpff, typename P::T fpi, const Mom4<typename P::T>& mf,
                                                    const Mom4<typename P::T>& mff, typename P::T uw0,
                                                    typename P::T uw1, typename P::T uw2, typename P::T rho0,
                                                    int local_rho, bool moving = true) {
  using T = typename P::T;
  // 6 w_i' rho0 (e_i . u_w) with e_i = -e_i'.  FP64 skips it when no wall
  // of the lattice moves (the same for every link of a launch: five FP64
  // instructions of about a hundred per link); FP32 forms it always (the
  // branch moved registers of the fused kernel into spills and cost 2 %)
  const T wall = (P::shifted || moving) ? -(T)6 * w * rho0 * (ex * uw0 + ey * uw1 + ez * uw2) : (T)0;
  const T two_q = (T)2 * q;
  if (rule == 0) return fpf + wall;
  if (rule == 1) {
    if (q <= (T)0.5) return two_q * fpf + ((T)1 - two_q) * fpff + wall;
    const T inv2q = (T)1 / two_q;
    return (fpf + wall) * inv2q + (two_q - (T)1) * inv2q * fpi;
  }
  if (rule == 3) {
    // Yu: the population reaching the wall, linear between x_f and x_ff at
    // q - 1 along e_i', bounced back; then x_f linear between x_w (at q)
    // and x_ff (at -1), whose f_i(x_ff, t+1) is f+_i(x_f, t) in pull form
    const T i1q = (T)1 / ((T)1 + q);
    return (q * fpf + ((T)1 - q) * fpff + wall) * i1q + q * i1q * fpi;
  }
  const T rhof = P::shifted ? rho0 + mf.r : mf.r;
  const T rhoff = P::shifted ? rho0 + mff.r : mff.r;
  // Eq. (rhod) in storage form; optionally rho_d = rho_f when q > 1/2
  const T rd = (local_rho && q > (T)0.5) ? mf.r : two_q * mf.r + ((T)1 - two_q) * mff.r;
  const T rhod = P::shifted ? rho0 + rd : rd;
  const T neq_f = fpf - eq_dir<P>(w, ex, ey, ez, mf.r, rhof, mf.ux, mf.uy, mf.uz);
  const T neq_ff = fpff - eq_dir<P>(w, ex, ey, ez, mff.r, rhoff, mff.ux, mff.uy, mff.uz);
  // every quotient of the rule from one reciprocal, r = 1/(rho_f rho_ff D)
  // with D = q (1 + q) (q > 1/2) or 1 + q: 1/(rho_f rho_ff) = D r,
  // 1/D = rho_f rho_ff r, 1/(1 + q) and 1/q from 1/D
  const bool far = q > (T)0.5;
  const T D = far ? q * ((T)1 + q) : (T)1 + q;
  const T rr = rhof * rhoff;
  const T r = (T)1 / (rr * D);
  const T iD = rr * r;
  const T i1q = far ? q * iD : iD;
  // fneq at d, each term rescaled by its density ratio
  const T nd = rhod * (two_q * neq_f * rhoff + ((T)1 - two_q) * neq_ff * rhof) * (D * r);
  // u*_d (piecewise linear), u**_d (between x_ff and the wall), weighted 1/3 : 2/3
  T af, aff, aw;
  if (!far) {
    af = two_q;
    aff = (T)1 - two_q;
    aw = 0;
  } else {
    const T iq = ((T)1 + q) * iD;
    af = ((T)1 - q) * iq;
    aff = 0;
    aw = (two_q - (T)1) * iq;
  }
  const T bff = ((T)1 - q) * i1q, bw = two_q * i1q;
  const T third = (T)(1.0 / 3.0), two_thirds = (T)(2.0 / 3.0);
  const T cf = third * af, cff = third * aff + two_thirds * bff, cw = third * aw + two_thirds * bw;
  const T udx = cf * mf.ux + cff * mff.ux + cw * uw0;
  const T udy = cf * mf.uy + cff * mff.uy + cw * uw1;
  const T udz = cf * mf.uz + cff * mff.uz + cw * uw2;
  return eq_dir<P>(w, ex, ey, ez, rd, rhod, udx, udy, udz) + nd + wall;
}

// Direction table of the link kernels in shared memory (filled by the
// block's first Q threads; the caller synchronises).
template <class L, class T>
__device__ __forceinline__ void fill_dir_table(DirTable<T, L::Q>& tab) {
  if (threadIdx.x < L::Q) {
    const int d = threadIdx.x;
    tab.off[d] = 0;
    tab.opp[d] = L::opp(d);
    tab.w[d] = (T)L::w(d);
    tab.e[d][0] = (T)L::cx(d);
    tab.e[d][1] = (T)L::cy(d);
    tab.e[d][2] = (T)L::cz(d);
  }
}

// Missing population f_i(x_f, t+1) of the link (x_f = node, i' = ip) from
// the post-collision state f (storage form, [Q][N]) and the moment cache at
// time t; x_ff = ff (x_f when there is no second fluid node).  fpf receives
// f+_i'(x_f, t), the link's other term of the momentum exchange.  Each rule
// loads only what it reads.
template <class L, class P>
__device__ __forceinline__ typename P::T eval_link(const DirTable<typename P::T, L::Q>& tab,
                                                   const typename P::T* __restrict__ f,
                                                   const Mom4<typename P::T>* __restrict__ mom, size_t N, int ip,
                                                   int rule, typename P::T q, uint32_t node, uint32_t ff,
                                                   typename P::T uw0, typename P::T uw1, typename P::T uw2,
                                                   const Params& p, typename P::T& fpf, bool moving) {
  using T = typename P::T;
  const int i = tab.opp[ip];
  const T ex = tab.e[ip][0], ey = tab.e[ip][1], ez = tab.e[ip][2];
  const T w = tab.w[ip];
  fpf = f[(size_t)ip * N + node];
  T fpff = 0, fpi = 0;
  Mom4<T> mf{0, 0, 0, 0}, mff{0, 0, 0, 0};
  if (rule == 1) {
    if (q <= (T)0.5)
      fpff = f[(size_t)ip * N + ff];
    else
      fpi = f[(size_t)i * N + node];
  } else if (rule == 2) {
    fpff = f[(size_t)ip * N + ff];
    mf = mom[node];
    mff = mom[ff];
  } else if (rule == 3) {
    fpff = f[(size_t)ip * N + ff];
    fpi = f[(size_t)i * N + node];
  }
  return link_value<P>(rule, q, w, ex, ey, ez, fpf, fpff, fpi, mf, mff, uw0, uw1, uw2, par<T>(p.rho0, p.rho0_f),
                       p.vibb_local_rho, moving);
}

// VIBB (Sec. 3.1) with the velocity interpolation weights of the link given:
// u_d = cf u_f + cff u_ff + cw u_w, where (cf, cff, cw) are the 1/3 : 2/3
// blend of u*_d and u**_d and depend on q alone (the FP64 link kernel takes
// them from a per-link array the host fills, instead of forming them from
// 1/q and 1/(1+q) per link and step).  Otherwise as link_value's VIBB branch.
template <class L, class P>
__device__ __forceinline__ typename P::T vibb_weighted(const DirTable<typename P::T, L::Q>& tab,
                                                       const typename P::T* __restrict__ f,
                                                       const Mom4<typename P::T>* __restrict__ mom, size_t N, int ip,
                                                       typename P::T q, uint32_t node, uint32_t ff, typename P::T uw0,
                                                       typename P::T uw1, typename P::T uw2, const Params& p,
                                                       typename P::T& fpf, bool moving, typename P::T cf,
                                                       typename P::T cff, typename P::T cw) {
  using T = typename P::T;
  const T ex = tab.e[ip][0], ey = tab.e[ip][1], ez = tab.e[ip][2];
  const T w = tab.w[ip];
  fpf = f[(size_t)ip * N + node];
  const T fpff = f[(size_t)ip * N + ff];
  const Mom4<T> mf = mom[node], mff = mom[ff];
  const T rho0 = par<T>(p.rho0, p.rho0_f);
  const T wall = (P::shifted || moving) ? -(T)6 * w * rho0 * (ex * uw0 + ey * uw1 + ez * uw2) : (T)0;
  const T two_q = (T)2 * q;
  const T rhof = P::shifted ? rho0 + mf.r : mf.r;
  const T rhoff = P::shifted ? rho0 + mff.r : mff.r;
  const T rd = (p.vibb_local_rho && q > (T)0.5) ? mf.r : two_q * mf.r + ((T)1 - two_q) * mff.r;
  const T rhod = P::shifted ? rho0 + rd : rd;
  const T neq_f = fpf - eq_dir<P>(w, ex, ey, ez, mf.r, rhof, mf.ux, mf.uy, mf.uz);
  const T neq_ff = fpff - eq_dir<P>(w, ex, ey, ez, mff.r, rhoff, mff.ux, mff.uy, mff.uz);
  // fneq at d, each term rescaled by its density ratio
  const T nd = rhod * (two_q * neq_f * rhoff + ((T)1 - two_q) * neq_ff * rhof) / (rhof * rhoff);
  const T udx = cf * mf.ux + cff * mff.ux + cw * uw0;
  const T udy = cf * mf.uy + cff * mff.uy + cw * uw1;
  const T udz = cf * mf.uz + cff * mff.uz + cw * uw2;
  return eq_dir<P>(w, ex, ey, ez, rd, rhod, udx, udy, udz) + nd + wall;
}

// One thread per link.  recs: storage indices and metadata; qv: q in
// storage precision; uw: [D][nl] wall velocities or null.  force: the step's
// accumulator slot [MAX_BODIES][3] (FP64).
//
// Rules (storage form; the rest part w rho0 cancels because every rule's
// weights sum to one):
//   half-way  f_i = f+_i'(x_f) + wall
//   Bouzidi   q <= 1/2: 2q f+_i'(x_f) + (1-2q) f+_i'(x_ff) + wall   (Eq. q_less)
//             q >  1/2: (f+_i'(x_f) + wall)/(2q) + (2q-1)/(2q) f+_i(x_f)  (Eq. q_larger)
//   VIBB      feq_i'(rho_d, u_d) + fneq_i'(x_d) + wall                 (Sec. 3.1)
//   Yu        (q f+_i'(x_f) + (1-q) f+_i'(x_ff) + wall)/(1+q) + q/(1+q) f+_i(x_f)  (Sec. 3)
// with wall = 6 w rho0 (e_i . u_w).
template <class L, class P, int SEQ>
__global__ void __launch_bounds__(256) k_links(typename P::T* __restrict__ f, const Mom4<typename P::T>* __restrict__ mom,
                                               const LinkRec* __restrict__ recs, const typename P::T* __restrict__ qv,
                                               const typename P::T* __restrict__ uwv,
                                               const typename P::T* __restrict__ qcv, int64_t nl,
                                               double* __restrict__ force, Params p, int64_t S_) {
  using T = typename P::T;
  __shared__ DirTable<T, L::Q> tab;
  fill_dir_table<L>(tab);
  __syncthreads();
  // the block takes SEQ rounds of blockDim consecutive links; the next
  // round's record and q are loaded while the current link is processed
  const int64_t base = (int64_t)blockIdx.x * blockDim.x * SEQ;
  // body of the block's first link: the block's links of that body are
  // summed per lane (storage precision), per warp and per block (FP64);
  // links of any other body (a body boundary inside the block) add their
  // terms with FP64 atomics directly
  const int b0 = (int)(__ldg(&recs[base].meta) >> 7) - 1;
  const size_t N = (size_t)S_;
  T F0 = 0, F1 = 0, F2 = 0;
  int64_t k = base + threadIdx.x;
  bool live = k < nl;
  LinkRec rec{0, 0, 0, 0};
  T q = 0;
  if (live) {
    rec = recs[k];
    q = qv[k];
  }
#pragma unroll 1
  for (int r = 0; r < SEQ; ++r) {
    const int64_t kn = k + blockDim.x;
    const bool liven = (r + 1 < SEQ) && kn < nl;
    LinkRec recn{0, 0, 0, 0};
    T qn = 0;
    if (liven) {
      recn = recs[kn];
      qn = qv[kn];
    }
    if (live) {
      const int ip = (int)(rec.meta & 31);
      const int rule = (int)((rec.meta >> 5) & 3);
      const int body = (int)(rec.meta >> 7) - 1;
      T uw0 = 0, uw1 = 0, uw2 = 0;
      if (uwv) {
        uw0 = uwv[k];
        uw1 = uwv[nl + k];
        if (L::D == 3) uw2 = uwv[2 * nl + k];
      }
      T fpf, val;
      // FP64 VIBB links take their velocity weights from qcv; the FP32 kernel
      // keeps the one evaluation path (its rounding of the rule is what the
      // FP32 adjoint's accuracy was measured with)
      if constexpr (!P::shifted) {
        if (qcv && rule == 2)
          val = vibb_weighted<L, P>(tab, f, mom, N, ip, q, rec.kf, rec.kff, uw0, uw1, uw2, p, fpf, uwv != nullptr,
                                    qcv[k], qcv[nl + k], qcv[2 * nl + k]);
        else
          val = eval_link<L, P>(tab, f, mom, N, ip, rule, q, rec.kf, rec.kff, uw0, uw1, uw2, p, fpf,
                                uwv != nullptr);
      } else {
        val = eval_link<L, P>(tab, f, mom, N, ip, rule, q, rec.kf, rec.kff, uw0, uw1, uw2, p, fpf,
                              uwv != nullptr);
      }
      f[(size_t)tab.opp[ip] * N + rec.ks] = val;
      if (body >= 0) {
        // momentum exchange (f+_i'(x_f,t) + f_i(x_f,t+1)) e_i'.  In shifted
        // storage this sums (h+_i' + h_i) e_i'; the rest part 2 w_i' rho0 e_i'
        // of every link is a geometric constant that the host adds in FP64.
        const T t = fpf + val;
        const T ex = tab.e[ip][0], ey = tab.e[ip][1], ez = tab.e[ip][2];
        if (body == b0) {
          F0 += t * ex;
          F1 += t * ey;
          F2 += t * ez;
        } else {
          atomicAdd(&force[3 * body + 0], (double)(t * ex));
          atomicAdd(&force[3 * body + 1], (double)(t * ey));
          atomicAdd(&force[3 * body + 2], (double)(t * ez));
        }
      }
    }
    k = kn;
    rec = recn;
    q = qn;
    live = liven;
  }
  if (b0 < 0) return;
  __shared__ double red[3][32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    F0 += __shfl_down_sync(0xffffffffu, F0, o);
    F1 += __shfl_down_sync(0xffffffffu, F1, o);
    F2 += __shfl_down_sync(0xffffffffu, F2, o);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) {
    red[0][warp] = (double)F0;
    red[1][warp] = (double)F1;
    red[2][warp] = (double)F2;
  }
  __syncthreads();
  if (threadIdx.x < 3) {
    const int nw = (blockDim.x + 31) >> 5;
    double acc = 0.0;
    for (int wi = 0; wi < nw; ++wi) acc += red[threadIdx.x][wi];
    atomicAdd(&force[3 * b0 + threadIdx.x], acc);
  }
}

// ------------------------------------------------------------ fused step --

// Links of the fused step kernel, in (node, direction) order: the links of
// the stored nodes 32 g .. 32 g + 31 are first[g] .. first[g+1] - 1, and
// mask[k] has bit d set when stored node k has a link in direction d.  One
// 16-B record per link: the storage indices of x_f and x_ff (x_f when there
// is no second fluid node), meta = dir | rule << 5 | (body + 1) << 8, and
// q as FP32 bits (FP32 storage; FP64 keeps q in qd).
struct __align__(16) FusedRec {
  uint32_t kf, kff, meta, q32;
};

template <class T>
struct FusedLinks {
  const int32_t* first;    // [ngroups + 1]
  const uint32_t* mask;    // [S]
  const FusedRec* rec;     // [nl]
  const double* qd;        // [nl] (FP64 storage) or null
  const T* uw;             // [D][nl] wall velocities or null
  int64_t nl;
  int64_t ngroups;         // ceil(S / 32)
};

// Asynchronous global -> shared copies of one real (cp.async, cached in L1;
// no register holds the value while it is in flight).
template <class T>
__device__ __forceinline__ void cp_async_real(T* smem, const T* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  if constexpr (sizeof(T) == 8)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Resident blocks per SM of the fused kernel, per 256 threads: FP32 D2Q9 4
// (64 registers: the link phase spills at the bulk kernel's 40), FP32
// D3Q19 5 (48), FP64 2.
template <class L, class P, int BT>
constexpr int fused_blocks_per_sm() {
  constexpr int base = !P::shifted ? 2 : (L::Q == 9 ? 4 : 5);
  return base * 256 / BT < 1 ? 1 : base * 256 / BT;
}

// One time step with the link rules fused into the pull pass, one thread
// per stored node (as k_bulk):
//  1. each fluid node issues the pulls of its non-link directions as
//     asynchronous copies into its column of the block's shared-memory
//     stage (ghost and open slots put the rest state there);
//  2. meanwhile the block evaluates the cut links of its nodes, spread over
//     all its threads (the same rule code as k_links, on f+(t) and the
//     moment cache at t, mom_in), and writes each link value into the
//     stage at its node and direction i = opp(i');
//  3. after one barrier every node collides from its staged column.
// The link values never go through HBM and no ghost slot is read or written
// by the link rules; ghost and open slots of fout get zeros as in k_bulk.
// The moments at t+1 go to mom_out (a second cache buffer: other blocks'
// link phases still read mom_in).  Momentum exchange: per thread in storage
// precision, per warp by shuffles, per block in FP64 and one atomic per
// block and component for the body of the block's first link; links of
// other bodies add their terms with FP64 atomics directly.
template <class L, class P, bool MULTI, int BT>
__global__ void __launch_bounds__(BT, (fused_blocks_per_sm<L, P, BT>())) k_fused(
    const typename P::T* __restrict__ fin, typename P::T* __restrict__ fout, Layout lay,
    FusedLinks<typename P::T> fl, const Mom4<typename P::T>* __restrict__ mom_in,
    Mom4<typename P::T>* __restrict__ mom_out, double* __restrict__ force, double* __restrict__ force_next,
    Params p) {
  using T = typename P::T;
  constexpr int NW = BT / 32;
  __shared__ T stage[NW][L::Q][32];
  __shared__ DirTable<T, L::Q> tab;
  __shared__ double red[3][NW];
  fill_dir_table<L>(tab);
  if (force_next && blockIdx.x == 0)
    for (int t = threadIdx.x; t < 3 * p.nbody; t += BT) force_next[t] = 0.0;
  __syncthreads();  // the direction table (every thread arrives here at once)
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t base = blockIdx.x * BT;
  const uint32_t k = base + threadIdx.x;
  const size_t S = (size_t)lay.S;
  const bool live = (uint64_t)k < S;
  const uint32_t w = live ? __ldg(lay.word + k) : W_GHOST;
  const uint32_t mask = live ? __ldg(fl.mask + k) : 0u;
  // the block's range of the link list (the same two words in every thread)
  const int64_t g0 = base >> 5, g1 = g0 + NW < fl.ngroups ? g0 + NW : fl.ngroups;
  const int64_t l0 = __ldg(fl.first + g0), l1 = __ldg(fl.first + g1);
  const int total = (int)(l1 - l0);
  // this thread's first link record, requested before the run record and
  // the pulls so that the link phase does not wait behind them
  FusedRec r_first{0, 0, 0, 0};
  T q_first = 0;
  if ((int)threadIdx.x < total) {
    r_first = fl.rec[l0 + threadIdx.x];
    q_first = P::shifted ? (T)__uint_as_float(r_first.q32) : (T)__ldg(fl.qd + l0 + threadIdx.x);
  }
  const bool fluid = live && !(w & (W_GHOST | W_OPEN));
  T(&col)[L::Q][32] = stage[warp];
  int dom = 0;
  if (fluid) {
    const RunRec run = lay.runs[w & W_RUN];
    if (MULTI) dom = run.dom;
    int d[L::Q];
    pull_offsets<L>(k, run, lay, p, d);
    const T* __restrict__ fk = fin + k;
#pragma unroll
    for (int i = 0; i < L::Q; ++i)
      // direction i comes from the solid side when its opposite is a link
      if (!((mask >> L::opp(i)) & 1u)) cp_async_real(&col[i][lane], fk + ((ptrdiff_t)i * (ptrdiff_t)S + d[i]));
  } else if (live) {
    // ghost and open slots: zeros through the same stores (inputs at rest)
#pragma unroll
    for (int i = 0; i < L::Q; ++i) col[i][lane] = P::shifted ? (T)0 : (T)L::w(i);
  }
  cp_async_commit();
  const int wb = total > 0 ? (int)(__ldg(&fl.rec[l0].meta) >> 8) - 1 : -1;
  T F0 = 0, F1 = 0, F2 = 0;
  for (int j = threadIdx.x; j < total; j += BT) {
    const int64_t li = l0 + j;
    const bool first_round = j == (int)threadIdx.x;
    const FusedRec r = first_round ? r_first : fl.rec[li];
    const T q = first_round ? q_first : (P::shifted ? (T)__uint_as_float(r.q32) : (T)__ldg(fl.qd + li));
    const int ip = (int)(r.meta & 31);
    const int rule = (int)((r.meta >> 5) & 7);
    const int body = (int)(r.meta >> 8) - 1;
    T uw0 = 0, uw1 = 0, uw2 = 0;
    if (fl.uw) {
      uw0 = fl.uw[li];
      uw1 = fl.uw[fl.nl + li];
      if (L::D == 3) uw2 = fl.uw[2 * fl.nl + li];
    }
    T fpf;
    const T val = eval_link<L, P>(tab, fin, mom_in, S, ip, rule, q, r.kf, r.kff, uw0, uw1, uw2, p, fpf,
                                  fl.uw != nullptr);
    const uint32_t o = r.kf - base;  // the node's place in the block
    stage[o >> 5][tab.opp[ip]][o & 31] = val;
    if (body >= 0) {
      // momentum exchange as in k_links
      const T t = fpf + val;
      const T ex = tab.e[ip][0], ey = tab.e[ip][1], ez = tab.e[ip][2];
      if (body == wb) {
        F0 += t * ex;
        F1 += t * ey;
        F2 += t * ez;
      } else {
        atomicAdd(&force[3 * body + 0], (double)(t * ex));
        atomicAdd(&force[3 * body + 1], (double)(t * ey));
        atomicAdd(&force[3 * body + 2], (double)(t * ez));
      }
    }
  }
  if (wb >= 0) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      F0 += __shfl_down_sync(0xffffffffu, F0, o);
      F1 += __shfl_down_sync(0xffffffffu, F1, o);
      F2 += __shfl_down_sync(0xffffffffu, F2, o);
    }
    if (lane == 0) {
      red[0][warp] = (double)F0;
      red[1][warp] = (double)F1;
      red[2][warp] = (double)F2;
    }
  }
  cp_async_wait_all();
  __syncthreads();  // staged pulls, link values and warp sums of the whole block
  if (wb >= 0 && threadIdx.x < 3) {
    double acc = 0.0;
#pragma unroll
    for (int wi = 0; wi < NW; ++wi) acc += red[threadIdx.x][wi];
    atomicAdd(&force[3 * wb + threadIdx.x], acc);
  }
  if (live) {
    T f[L::Q];
#pragma unroll
    for (int i = 0; i < L::Q; ++i) f[i] = col[i][lane];
    const Relax rx = MULTI ? relax_domain(lay.dom, dom) : relax_params(p);
    collide_store<L, P>(f, p, rx, folded_of<MULTI>(p, lay, dom), fout, S, k, mom_out, (w & W_CACHE) != 0, fluid);
  }
}

// ------------------------------------------------------------ open sides --

// Inlet velocity of row y: 4 u_max (y - y0)(y1 - y)/(y1 - y0)^2, with y
// counted from the first row of the row's domain.
__device__ __forceinline__ double inlet_velocity(const Params& p, const Layout& lay, int y) {
  double umax = p.inlet_umax, y0 = p.inlet_y0, y1 = p.inlet_y1, yy = (double)y;
  if (lay.ndom > 1) {
    const DomPar& d = lay.dom[lay.row_dom[y]];
    umax = d.inlet_umax;
    y0 = d.inlet_y0;
    y1 = d.inlet_y1;
    yy = (double)(y - d.lo);
  }
  const double h = y1 - y0;
  return 4.0 * umax * (yy - y0) * (y1 - yy) / (h * h);
}

// Sec. 4.3: inlet column x = 0 by non-equilibrium extrapolation from x = 1
// with the parabolic velocity u_in(y); outlet column x = nx-1 copies x = nx-2.
// One thread per row and side (D2Q9); the open node is the first (inlet) or
// last (outlet) stored node of its row and its fluid neighbour is adjacent.
template <class L, class P>
__global__ void k_open(typename P::T* __restrict__ f, const Mom4<typename P::T>* __restrict__ mom, Layout lay,
                       Params p) {
  using T = typename P::T;
  // threads 0 .. ny-1: inlet rows; ny .. 2 ny - 1: outlet rows
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
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
      const T rho1 = P::shifted ? par<T>(p.rho0, p.rho0_f) + m1.r : m1.r;
      T v[L::Q];
#pragma unroll
      for (int i = 0; i < L::Q; ++i) v[i] = f[i * S + k1];
#pragma unroll
      for (int i = 0; i < L::Q; ++i)
        f[i * S + k0] = equilibrium<L, P>(i, m1.r, rho1, uin, (T)0, (T)0) +
                        (v[i] - equilibrium<L, P>(i, m1.r, rho1, m1.ux, m1.uy, (T)0));
    }
  }
  if (!inlet_side && p.outlet) {
    const int32_t kl = lay.row_last[y];
    if (kl >= 0 && (lay.word[kl] & W_OPEN)) {
      T v[L::Q];
#pragma unroll
      for (int i = 0; i < L::Q; ++i) v[i] = f[i * S + kl - 1];
#pragma unroll
      for (int i = 0; i < L::Q; ++i) f[i * S + kl] = v[i];
    }
  }
}

// ------------------------------------------------------- init and fields --

__device__ __forceinline__ bool is_fluid(uint32_t w) { return (w & (W_GHOST | W_OPEN)) == 0; }

// f(x,0) = feq(rho_in, u_in) followed by the collision at t = 0 (fluid
// nodes); zero elsewhere.  rho_in (N) and u_in (N x 3, interleaved), dense
// indices, may be null for rho0 and rest.
template <class L, class P>
__global__ void k_init(typename P::T* __restrict__ f, Mom4<typename P::T>* __restrict__ mom, Layout lay,
                       const double* __restrict__ rho_in, const double* __restrict__ u_in, Params p) {
  using T = typename P::T;
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= lay.S) return;
  const size_t S = (size_t)lay.S;
  const uint32_t w = lay.word[k];
  if (!is_fluid(w)) {
#pragma unroll
    for (int i = 0; i < L::Q; ++i) f[(size_t)i * S + k] = (T)0;
    return;
  }
  const int64_t n = lay.node_of[k];
  const Relax rx = relax_of_run(p, lay, w & W_RUN);
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
  // one inlined collision for both cases (the lattice's constants or the
  // domain's), so that a domain's initial state has the same bits alone and
  // in a batch
  const Folded* kc = lay.ndom > 1 ? &lay.dom[lay.runs[w & W_RUN].dom].kc : &p.kc;
  collide_store<L, P>(fl, p, rx, *kc, f, S, (uint32_t)k, mom, (w & W_CACHE) != 0);
}

// rho = sum f+, u = (sum f+ e - g/2)/rho of the post-collision state (the
// collision conserves mass and adds g to the momentum); FP64 output at dense
// indices (the caller zeroes the outputs first).  u: [D][N].
template <class L, class P>
__global__ void k_moments(const typename P::T* __restrict__ f, Layout lay, double* __restrict__ rho_out,
                          double* __restrict__ u_out, Params p) {
  using T = typename P::T;
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= lay.S || !is_fluid(lay.word[k])) return;
  const size_t S = (size_t)lay.S;
  const int64_t N = p.N, n = lay.node_of[k];
  const Relax rx = relax_of_run(p, lay, lay.word[k] & W_RUN);
  T r = 0, jx = 0, jy = 0, jz = 0;
#pragma unroll
  for (int i = 0; i < L::Q; ++i) {
    const T v = f[(size_t)i * S + k];
    r += v;
    jx += (T)L::cx(i) * v;
    jy += (T)L::cy(i) * v;
    jz += (T)L::cz(i) * v;
  }
  const double rho = P::shifted ? p.rho0 + (double)r : (double)r;
  rho_out[n] = rho;
  u_out[n] = ((double)jx - 0.5 * rx.g[0]) / rho;
  u_out[N + n] = ((double)jy - 0.5 * rx.g[1]) / rho;
  if (L::D == 3) u_out[2 * N + n] = ((double)jz - 0.5 * rx.g[2]) / rho;
}

// Moment cache refresh from a post-collision state (after the caller sets
// the populations): same formula as k_moments, storage precision.
template <class L, class P>
__global__ void k_refresh(const typename P::T* __restrict__ f, Layout lay, Mom4<typename P::T>* __restrict__ mom,
                          Params p) {
  using T = typename P::T;
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= lay.S || !(lay.word[k] & W_CACHE) || !is_fluid(lay.word[k])) return;
  const size_t S = (size_t)lay.S;
  const Relax rx = relax_of_run(p, lay, lay.word[k] & W_RUN);
  T r = 0, jx = 0, jy = 0, jz = 0;
#pragma unroll
  for (int i = 0; i < L::Q; ++i) {
    const T v = f[(size_t)i * S + k];
    r += v;
    jx += (T)L::cx(i) * v;
    jy += (T)L::cy(i) * v;
    jz += (T)L::cz(i) * v;
  }
  const T rho = P::shifted ? par<T>(p.rho0, p.rho0_f) + r : r;
  mom[k] = Mom4<T>{r, (jx - par<T>(0.5 * rx.g[0], rx.hg_f[0])) / rho, (jy - par<T>(0.5 * rx.g[1], rx.hg_f[1])) / rho,
                   L::D == 3 ? (jz - par<T>(0.5 * rx.g[2], rx.hg_f[2])) / rho : (T)0};
}

template <class L>
__device__ __forceinline__ double weight_of(int i) {
  double w = 0.0;
#pragma unroll
  for (int k = 0; k < L::Q; ++k)
    if (k == i) w = L::w(k);
  return w;
}

// One direction of the state to (k_get_dir, dense FP64 unshifted output,
// zeroed by the caller) or from (k_set_dir) the caller's layout.
template <class L, class P>
__global__ void k_get_dir(const typename P::T* __restrict__ f, Layout lay, int i, double* __restrict__ out, Params p) {
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= lay.S || !is_fluid(lay.word[k])) return;
  out[lay.node_of[k]] = (double)f[(size_t)i * lay.S + k] + (P::shifted ? weight_of<L>(i) * p.rho0 : 0.0);
}

template <class L, class P>
__global__ void k_set_dir(typename P::T* __restrict__ f, Layout lay, int i, const double* __restrict__ in, Params p) {
  using T = typename P::T;
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= lay.S) return;
  f[(size_t)i * lay.S + k] =
      is_fluid(lay.word[k]) ? (T)(in[lay.node_of[k]] - (P::shifted ? weight_of<L>(i) * p.rho0 : 0.0)) : (T)0;
}

// Populations of listed storage indices (-1: not a fluid node -> 0), FP64
// unshifted, out[k*Q + i].
template <class L, class P>
__global__ void k_gather(const typename P::T* __restrict__ f, Layout lay, const int64_t* __restrict__ sk, int64_t n,
                         double* __restrict__ out, Params p) {
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= n) return;
  const int64_t s = sk[k];
  const bool off = s < 0 || !is_fluid(lay.word[s]);
#pragma unroll
  for (int i = 0; i < L::Q; ++i)
    out[k * L::Q + i] = off ? 0.0 : (double)f[(size_t)i * lay.S + s] + (P::shifted ? L::w(i) * p.rho0 : 0.0);
}

// Failure detection: flag any non-finite population or non-positive density.
template <class L, class P>
__global__ void k_check(const typename P::T* __restrict__ f, Layout lay, int* __restrict__ flag, Params p) {
  using T = typename P::T;
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= lay.S || !is_fluid(lay.word[k])) return;
  T r = 0;
  bool bad = false;
#pragma unroll
  for (int i = 0; i < L::Q; ++i) {
    const T v = f[(size_t)i * lay.S + k];
    bad |= !isfinite(v);
    r += v;
  }
  const double rho = P::shifted ? p.rho0 + (double)r : (double)r;
  if (bad || !(rho > 0.0)) atomicOr(flag, 1);
}

// ------------------------------------------------------------- launchers --

// Link arrays of the fused step kernel without the storage type (the
// launchers cast q and uw).
struct FusedRaw {
  const int32_t* first;
  const uint32_t* mask;
  const FusedRec* rec;
  const double* qd;
  const void* uw;
  int64_t nl, ngroups;
};

struct KernelOps {
  int Q, D;
  size_t real_bytes;
  int default_shape;
  unsigned shape_mask;  // bit b: kBulkShapes[b] is built for this stencil
  // shape: index into kBulkShapes; threads: link kernel block size (64, 128 or
  // 256); seq: links per thread of the link kernel (1 or 4)
  void (*bulk)(const void* fin, void* fout, const Layout& lay, void* mom, double* force_next, const Params& p,
               int shape, cudaStream_t s);
  void (*links)(void* f, const void* mom, const LinkRec* recs, const void* q, const void* uw, const void* qc,
                int64_t nl, double* force, const Params& p, int64_t S, int threads, int seq, cudaStream_t s);
  // fused step (threads per block 128, 256 or 512; 512 runs as 256 for
  // FP64 D3Q19, whose link buffer would not fit the static shared memory)
  void (*fused)(const void* fin, void* fout, const Layout& lay, const FusedRaw& fl, const void* mom_in,
                void* mom_out, double* force, double* force_next, const Params& p, int threads, cudaStream_t s);
  void (*open)(void* f, const void* mom, const Layout& lay, const Params& p, cudaStream_t s);
  void (*init)(void* f, void* mom, const Layout& lay, const double* rho, const double* u, const Params& p,
               cudaStream_t s);
  void (*moments)(const void* f, const Layout& lay, double* rho, double* u, const Params& p, cudaStream_t s);
  void (*refresh)(const void* f, const Layout& lay, void* mom, const Params& p, cudaStream_t s);
  void (*get_dir)(const void* f, const Layout& lay, int i, double* out, const Params& p, cudaStream_t s);
  void (*set_dir)(void* f, const Layout& lay, int i, const double* in, const Params& p, cudaStream_t s);
  void (*check)(const void* f, const Layout& lay, int* flag, const Params& p, cudaStream_t s);
  void (*gather)(const void* f, const Layout& lay, const int64_t* sk, int64_t n, double* out, const Params& p,
                 cudaStream_t s);
};

inline unsigned blocks_for(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

template <class L, class P>
struct Launch {
  using T = typename P::T;
  template <bool M, int BT, int NPT>
  static void bulk_shape(const void* fin, void* fout, const Layout& lay, void* mom, double* force_next,
                         const Params& p, cudaStream_t s) {
    if constexpr (!P::shifted && NPT == 1) {
      if (lay.fluid) {
        k_bulk_list<L, P, M, BT><<<blocks_for(lay.nfluid > 0 ? lay.nfluid : 1, BT), BT, 0, s>>>(
            (const T*)fin, (T*)fout, lay, (Mom4<T>*)mom, force_next, p);
        return;
      }
    }
    k_bulk<L, P, M, BT, NPT><<<blocks_for((lay.S + NPT - 1) / NPT, BT), BT, 0, s>>>((const T*)fin, (T*)fout, lay,
                                                                                   (Mom4<T>*)mom, force_next, p);
  }
  template <bool M, int BT, int SEQ>
  static void bulk_seq(const void* fin, void* fout, const Layout& lay, void* mom, double* force_next,
                       const Params& p, cudaStream_t s) {
    k_bulk_seq<L, P, M, BT, SEQ><<<blocks_for((lay.S + SEQ - 1) / SEQ, BT), BT, 0, s>>>(
        (const T*)fin, (T*)fout, lay, (Mom4<T>*)mom, force_next, p);
  }
  template <bool M>
  static void bulk_m(const void* fin, void* fout, const Layout& lay, void* mom, double* fn, const Params& p,
                     int shape, cudaStream_t s) {
    switch (shape) {
      case 1: return bulk_shape<M, 128, 1>(fin, fout, lay, mom, fn, p, s);
      case 2: return bulk_shape<M, 512, 1>(fin, fout, lay, mom, fn, p, s);
      default: break;
    }
    if constexpr (bulk_max_npt<L>() >= 2) {
      switch (shape) {
        case 3: return bulk_shape<M, 256, 2>(fin, fout, lay, mom, fn, p, s);
        case 4: return bulk_shape<M, 128, 2>(fin, fout, lay, mom, fn, p, s);
        case 5: return bulk_shape<M, 512, 2>(fin, fout, lay, mom, fn, p, s);
        case 6: return bulk_seq<M, 128, 4>(fin, fout, lay, mom, fn, p, s);
        case 7: return bulk_seq<M, 128, 8>(fin, fout, lay, mom, fn, p, s);
        default: break;
      }
    }
    bulk_shape<M, 256, 1>(fin, fout, lay, mom, fn, p, s);
  }
  static void bulk(const void* fin, void* fout, const Layout& lay, void* mom, double* force_next, const Params& p,
                   int shape, cudaStream_t s) {
    if (lay.S == 0) return;
    if (lay.ndom > 1)
      bulk_m<true>(fin, fout, lay, mom, force_next, p, shape, s);
    else
      bulk_m<false>(fin, fout, lay, mom, force_next, p, shape, s);
  }
  static void links(void* f, const void* mom, const LinkRec* recs, const void* q, const void* uw, const void* qc,
                    int64_t nl, double* force, const Params& p, int64_t S, int threads, int seq, cudaStream_t s) {
    if (nl == 0) return;
    const int bt = (threads == 64 || threads == 128) ? threads : 256;
    if (seq == 4)
      k_links<L, P, 4><<<blocks_for(nl, 4 * bt), bt, 0, s>>>((T*)f, (const Mom4<T>*)mom, recs, (const T*)q,
                                                             (const T*)uw, (const T*)qc, nl, force, p, S);
    else
      k_links<L, P, 1><<<blocks_for(nl, bt), bt, 0, s>>>((T*)f, (const Mom4<T>*)mom, recs, (const T*)q,
                                                         (const T*)uw, (const T*)qc, nl, force, p, S);
  }
  template <bool M, int BT>
  static void fused_shape(const void* fin, void* fout, const Layout& lay, const FusedRaw& r, const void* mom_in,
                          void* mom_out, double* force, double* force_next, const Params& p, cudaStream_t s) {
    const FusedLinks<T> fl{r.first, r.mask, r.rec, r.qd, (const T*)r.uw, r.nl, r.ngroups};
    k_fused<L, P, M, BT><<<blocks_for(lay.S, BT), BT, 0, s>>>((const T*)fin, (T*)fout, lay, fl,
                                                              (const Mom4<T>*)mom_in, (Mom4<T>*)mom_out, force,
                                                              force_next, p);
  }
  template <bool M>
  static void fused_m(const void* fin, void* fout, const Layout& lay, const FusedRaw& r, const void* mom_in,
                      void* mom_out, double* force, double* force_next, const Params& p, int threads,
                      cudaStream_t s) {
    constexpr bool big_ok = P::shifted || L::Q == 9;
    if (threads == 128) return fused_shape<M, 128>(fin, fout, lay, r, mom_in, mom_out, force, force_next, p, s);
    if (big_ok && threads == 512)
      return fused_shape<M, big_ok ? 512 : 256>(fin, fout, lay, r, mom_in, mom_out, force, force_next, p, s);
    fused_shape<M, 256>(fin, fout, lay, r, mom_in, mom_out, force, force_next, p, s);
  }
  static void fused(const void* fin, void* fout, const Layout& lay, const FusedRaw& r, const void* mom_in,
                    void* mom_out, double* force, double* force_next, const Params& p, int threads,
                    cudaStream_t s) {
    if (lay.S == 0) return;
    if (lay.ndom > 1)
      fused_m<true>(fin, fout, lay, r, mom_in, mom_out, force, force_next, p, threads, s);
    else
      fused_m<false>(fin, fout, lay, r, mom_in, mom_out, force, force_next, p, threads, s);
  }
  static void open(void* f, const void* mom, const Layout& lay, const Params& p, cudaStream_t s) {
    k_open<L, P><<<blocks_for(2 * (int64_t)p.ny, 128), 128, 0, s>>>((T*)f, (const Mom4<T>*)mom, lay, p);
  }
  static void init(void* f, void* mom, const Layout& lay, const double* rho, const double* u, const Params& p,
                   cudaStream_t s) {
    if (lay.S == 0) return;
    k_init<L, P><<<blocks_for(lay.S, 256), 256, 0, s>>>((T*)f, (Mom4<T>*)mom, lay, rho, u, p);
  }
  static void moments(const void* f, const Layout& lay, double* rho, double* u, const Params& p, cudaStream_t s) {
    if (lay.S == 0) return;
    k_moments<L, P><<<blocks_for(lay.S, 256), 256, 0, s>>>((const T*)f, lay, rho, u, p);
  }
  static void refresh(const void* f, const Layout& lay, void* mom, const Params& p, cudaStream_t s) {
    if (lay.S == 0) return;
    k_refresh<L, P><<<blocks_for(lay.S, 256), 256, 0, s>>>((const T*)f, lay, (Mom4<T>*)mom, p);
  }
  static void get_dir(const void* f, const Layout& lay, int i, double* out, const Params& p, cudaStream_t s) {
    if (lay.S == 0) return;
    k_get_dir<L, P><<<blocks_for(lay.S, 256), 256, 0, s>>>((const T*)f, lay, i, out, p);
  }
  static void set_dir(void* f, const Layout& lay, int i, const double* in, const Params& p, cudaStream_t s) {
    if (lay.S == 0) return;
    k_set_dir<L, P><<<blocks_for(lay.S, 256), 256, 0, s>>>((T*)f, lay, i, in, p);
  }
  static void check(const void* f, const Layout& lay, int* flag, const Params& p, cudaStream_t s) {
    if (lay.S == 0) return;
    k_check<L, P><<<blocks_for(lay.S, 256), 256, 0, s>>>((const T*)f, lay, flag, p);
  }
  static void gather(const void* f, const Layout& lay, const int64_t* sk, int64_t n, double* out, const Params& p,
                     cudaStream_t s) {
    if (n == 0) return;
    k_gather<L, P><<<blocks_for(n, 256), 256, 0, s>>>((const T*)f, lay, sk, n, out, p);
  }
  static KernelOps ops() {
    return KernelOps{L::Q,   L::D,    sizeof(T), bulk_default_shape<L>(), bulk_shape_mask<L>(), bulk, links, fused,
                     open,   init,    moments,   refresh, get_dir, set_dir, check, gather};
  }
};

KernelOps ops_d2q9_f64();
KernelOps ops_d2q9_f32s();
KernelOps ops_d3q19_f64();
KernelOps ops_d3q19_f32s();

}  // namespace lbm
