// lbm_force_noalloc: the momentum-exchange force of one step, for callers
// that cannot allocate device memory.
//
// Some callers may not call cudaMalloc at all: code on a real-time path, or
// a framework that owns every byte of device memory through its own pool.  lbm_create_lattice allocates the
// whole lattice state, so it is of no use to them.  This entry point needs
// only memory the caller already owns (populations, mask, links, output).
// Its one piece of scratch -- one FP64 partial sum per thread block -- lives
// in the file-scope array below, which every GPU that loads liblbm.so holds
// (1.5 MiB) until the process exits.
//
// The computation is the force part of k_links: for every link of the body,
// the link rule's missing population f_i(x_f, t+1) from the caller's FP64
// post-collision state f+(t) (moments recomputed from f+), and the exchange
// (f+_i'(x_f, t) + f_i(x_f, t+1)) e_i'.  Block sums go to the scratch array;
// a second one-block kernel adds them in a fixed order, so the result is the
// same bit for bit on every call.
#include <cuda_runtime.h>

#include <cstdio>
#include <mutex>

#include "kernels.cuh"
#include "lbm.h"

namespace {

constexpr int kBlock = 256;
constexpr int kMaxBlocks = LBM_NOALLOC_MAX_LINKS / kBlock;
static_assert(kMaxBlocks * kBlock == LBM_NOALLOC_MAX_LINKS, "limit must be a whole number of blocks");

// Block partial sums (3 doubles per block).  In host code this name is only
// a stand-in for the device array: the kernels receive the address that
// cudaGetSymbolAddress returns for the current device.
static __device__ __align__(256) double lbm_noalloc_scratch[3 * kMaxBlocks];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
double* g_scratch[kMaxDevices] = {};

lbm_status fail(lbm_status st, const char* msg) {
  lbm::set_last_error(msg);
  return st;
}

template <class L>
__global__ void __launch_bounds__(kBlock) k_force_partial(const double* __restrict__ f, const uint8_t* __restrict__ solid,
                                                          const lbm_link* __restrict__ links, int64_t nl, int body,
                                                          int default_rule, lbm::Params p, double* __restrict__ partial) {
  using P = lbm::F64;
  __shared__ lbm::DirTable<double, L::Q> tab;
  __shared__ double red[3][kBlock / 32];
  if (threadIdx.x < L::Q) {
    const int d = threadIdx.x;
    tab.off[d] = 0;
    tab.opp[d] = L::opp(d);
    tab.w[d] = L::w(d);
    tab.e[d][0] = L::cx(d);
    tab.e[d][1] = L::cy(d);
    tab.e[d][2] = L::cz(d);
  }
  __syncthreads();
  const int64_t k = blockIdx.x * (int64_t)kBlock + threadIdx.x;
  double F0 = 0.0, F1 = 0.0, F2 = 0.0;
  const lbm_link lk = k < nl ? links[k] : lbm_link{};
  // the caller's records are not validated on the host: one that would read
  // outside f or solid (direction outside [1, Q), node outside [0, N) or on
  // a solid node) or names an unknown rule contributes nothing
  const bool valid = k < nl && lk.dir >= 1 && lk.dir < L::Q && lk.node >= 0 && lk.node < p.N &&
                     !solid[lk.node] && lk.bc >= LBM_BC_DEFAULT && lk.bc <= LBM_BC_YU;
  if (valid && lk.body == body) {
    const int64_t N = p.N, nx = p.nx, ny = p.ny, nz = p.nz;
    const int ip = lk.dir, i = tab.opp[ip];
    const double ex = tab.e[ip][0], ey = tab.e[ip][1], ez = tab.e[ip][2];
    const int64_t node = lk.node;
    // x_ff = x_f - e_i', wrapped on periodic axes; x_f when it is not a fluid node
    const int64_t x = node % nx, y = (node / nx) % ny, z = node / (nx * ny);
    int64_t c[3] = {x - (int64_t)ex, y - (int64_t)ey, z - (int64_t)ez};
    const int64_t len[3] = {nx, ny, nz};
    const int per[3] = {p.periodic[0], p.periodic[1], p.periodic[2]};
    bool inside = true;
    for (int a = 0; a < 3; ++a)
      if (c[a] < 0 || c[a] >= len[a]) {
        if (!per[a]) inside = false;
        c[a] = (c[a] + len[a]) % len[a];
      }
    int64_t ff = c[0] + nx * (c[1] + ny * c[2]);
    const bool open = (p.inlet && c[0] == 0) || (p.outlet && c[0] == nx - 1);
    if (!inside || solid[ff] || open) ff = node;
    // moments at time t from the post-collision state
    lbm::Mom4<double> m[2];
    const int64_t nodes[2] = {node, ff};
    for (int s = 0; s < 2; ++s) {
      double r = 0.0, jx = 0.0, jy = 0.0, jz = 0.0;
#pragma unroll
      for (int d = 0; d < L::Q; ++d) {
        const double v = f[d * N + nodes[s]];
        r += v;
        jx += L::cx(d) * v;
        jy += L::cy(d) * v;
        jz += L::cz(d) * v;
      }
      m[s] = lbm::Mom4<double>{r, (jx - 0.5 * p.g[0]) / r, (jy - 0.5 * p.g[1]) / r,
                               L::D == 3 ? (jz - 0.5 * p.g[2]) / r : 0.0};
    }
    const int rule = lk.bc >= 0 ? lk.bc : default_rule;
    const double fpf = f[ip * N + node];
    const double val = lbm::link_value<P>(rule, lk.q, tab.w[ip], ex, ey, ez, fpf, f[ip * N + ff], f[i * N + node], m[0],
                                          m[1], lk.uw[0], lk.uw[1], L::D == 3 ? lk.uw[2] : 0.0, p.rho0,
                                          p.vibb_local_rho);
    const double t = fpf + val;
    F0 = t * ex;
    F1 = t * ey;
    F2 = t * ez;
  }
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
  if (threadIdx.x < 3) {
    double s = 0.0;
    for (int w = 0; w < kBlock / 32; ++w) s += red[threadIdx.x][w];
    partial[3 * blockIdx.x + threadIdx.x] = s;
  }
}

// One block: sum the first nb partials in a fixed order into F (3 doubles).
__global__ void __launch_bounds__(kBlock) k_force_total(const double* __restrict__ partial, int nb,
                                                        double* __restrict__ F) {
  __shared__ double red[3][kBlock];
  for (int c = 0; c < 3; ++c) {
    double s = 0.0;
    for (int b = threadIdx.x; b < nb; b += kBlock) s += partial[3 * b + c];
    red[c][threadIdx.x] = s;
  }
  __syncthreads();
  for (int h = kBlock / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h)
      for (int c = 0; c < 3; ++c) red[c][threadIdx.x] += red[c][threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x < 3) F[threadIdx.x] = red[threadIdx.x][0];
}

// Address of the scratch array on the current device, looked up once per
// device (the first call on a device does this set-up).
lbm_status scratch_for_current_device(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(LBM_ERR_CUDA, cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return fail(LBM_ERR_UNSUPPORTED, "device index beyond 63");
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_scratch[dev]) {
    void* ptr = nullptr;
    e = cudaGetSymbolAddress(&ptr, lbm_noalloc_scratch);
    if (e != cudaSuccess || !ptr) {
      cudaGetLastError();
      return fail(LBM_ERR_CUDA, "cudaGetSymbolAddress of the no-alloc scratch failed");
    }
    g_scratch[dev] = (double*)ptr;
  }
  *out = g_scratch[dev];
  return LBM_OK;
}

}  // namespace

extern "C" lbm_status lbm_force_noalloc(const lbm_config* cfg, const double* f_post, const uint8_t* solid,
                                        const lbm_link* links, int64_t n_links, int32_t body, double* F) {
  lbm::set_last_error("");
  if (!cfg || !f_post || !solid || !F || n_links < 0 || (n_links > 0 && !links))
    return fail(LBM_ERR_INVALID_ARG, "null or negative argument");
  if (n_links > LBM_NOALLOC_MAX_LINKS)
    return fail(LBM_ERR_INVALID_ARG, "n_links exceeds LBM_NOALLOC_MAX_LINKS (16,777,216): use lbm_force on a lattice");
  if (body < 0 || body >= LBM_MAX_BODIES) return fail(LBM_ERR_INVALID_ARG, "body out of range");
  const lbm_config& c = *cfg;
  if (c.stencil != LBM_D2Q9 && c.stencil != LBM_D3Q19) return fail(LBM_ERR_INVALID_ARG, "unknown stencil");
  if (c.nx < 1 || c.ny < 1 || c.nz < 1 || (c.stencil == LBM_D2Q9 && c.nz != 1))
    return fail(LBM_ERR_INVALID_ARG, "bad lattice size");
  if (c.bc < LBM_BC_HALFWAY || c.bc > LBM_BC_YU) return fail(LBM_ERR_INVALID_ARG, "unknown default rule");
  if (!(c.rho0 > 0.0)) return fail(LBM_ERR_INVALID_ARG, "rho0 must be positive");
  double* scratch = nullptr;
  lbm_status st = scratch_for_current_device(&scratch);
  if (st != LBM_OK) return st;
  lbm::Params p{};
  p.nx = c.nx;
  p.ny = c.ny;
  p.nz = c.nz;
  p.N = (int64_t)c.nx * c.ny * c.nz;
  for (int a = 0; a < 3; ++a) p.periodic[a] = c.periodic[a] ? 1 : 0;
  p.rho0 = c.rho0;
  const int D = c.stencil == LBM_D2Q9 ? 2 : 3;
  for (int a = 0; a < 3; ++a) p.g[a] = a < D ? c.g[a] : 0.0;
  p.inlet = c.inlet ? 1 : 0;
  p.outlet = c.outlet ? 1 : 0;
  p.vibb_local_rho = c.vibb_density == LBM_VIBB_RHO_LOCAL ? 1 : 0;
  lbm::round_params(p);
  cudaStream_t s = (cudaStream_t)c.cuda_stream;
  const int nb = (int)((n_links + kBlock - 1) / kBlock);
  if (nb > 0) {
    if (c.stencil == LBM_D2Q9)
      k_force_partial<lbm::D2Q9><<<nb, kBlock, 0, s>>>(f_post, solid, links, n_links, body, c.bc, p, scratch);
    else
      k_force_partial<lbm::D3Q19><<<nb, kBlock, 0, s>>>(f_post, solid, links, n_links, body, c.bc, p, scratch);
  }
  k_force_total<<<1, kBlock, 0, s>>>(scratch, nb, F);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(LBM_ERR_CUDA, cudaGetErrorString(e));
  return LBM_OK;
}
