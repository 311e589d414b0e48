// Host side of liblbm.so: the C ABI declared in include/lbm.h.
//
// A lattice owns two population buffers (ping-pong), the moment cache, the
// node mask, the compacted link arrays and two FP64 force slots.  lbm_step
// replays a captured CUDA graph of two steps (one per buffer parity) and
// launches single steps directly for an odd remainder; with profiling on it
// launches kernel by kernel between CUDA events.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "kernels.cuh"
#include "lbm.h"

using namespace lbm;

namespace {

thread_local char g_msg[1024] = "";

lbm_status fail(lbm_status st, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_msg, sizeof g_msg, fmt, ap);
  va_end(ap);
  return st;
}

#define CUDA_TRY(call)                                                                               \
  do {                                                                                               \
    cudaError_t e_ = (call);                                                                         \
    if (e_ != cudaSuccess)                                                                           \
      return fail(e_ == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA, "%s: %s (%s:%d)", #call, \
                  cudaGetErrorString(e_), __FILE__, __LINE__);                                       \
  } while (0)

constexpr int kMaxTimedKernels = 3;

}  // namespace

struct lbm_lattice_s {
  lbm_config cfg{};
  KernelOps ops{};
  Params p{};
  int Q = 0, D = 0;
  int64_t N = 0;
  size_t rb = 0;  // bytes per stored real
  void* f[2] = {nullptr, nullptr};
  void* mom = nullptr;
  uint8_t* mask = nullptr;
  double* force = nullptr;  // [2][MAX_BODIES][3]
  uint64_t* keys = nullptr;
  void* q = nullptr;
  void* uw = nullptr;
  int64_t n_links = 0, n_fluid = 0, n_cached = 0;
  int cur = 0;        // buffer holding f+(t)
  int64_t step = 0;
  bool has_geometry = false, has_state = false;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  cudaGraphExec_t graph[2] = {nullptr, nullptr};  // two steps starting at parity 0 / 1
  // profiling
  bool profiling = false;
  std::vector<cudaEvent_t> ev;  // pairs, kernel id in ev_kernel
  std::vector<int> ev_kernel;
  size_t ev_used = 0;
  int64_t prof_launches[kMaxTimedKernels] = {0, 0, 0};
  double prof_ms[kMaxTimedKernels] = {0, 0, 0};
  int64_t device_bytes = 0;
};

namespace {

lbm_status dev_alloc(lbm_handle h, void** p, size_t bytes) {
  if (bytes == 0) {
    *p = nullptr;
    return LBM_OK;
  }
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    *p = nullptr;
    cudaGetLastError();
    return fail(LBM_ERR_OOM, "cudaMalloc(%zu bytes): %s", bytes, cudaGetErrorString(e));
  }
  h->device_bytes += (int64_t)bytes;
  return LBM_OK;
}

void drop_graphs(lbm_handle h) {
  for (int k = 0; k < 2; ++k)
    if (h->graph[k]) {
      cudaGraphExecDestroy(h->graph[k]);
      h->graph[k] = nullptr;
    }
}

void free_links(lbm_handle h) {
  if (h->keys) cudaFree(h->keys);
  if (h->q) cudaFree(h->q);
  if (h->uw) cudaFree(h->uw);
  h->keys = nullptr;
  h->q = h->uw = nullptr;
}

int cx_of(const lbm_handle h, int i) { return h->Q == 9 ? D2Q9::cx(i) : D3Q19::cx(i); }
int cy_of(const lbm_handle h, int i) { return h->Q == 9 ? D2Q9::cy(i) : D3Q19::cy(i); }
int cz_of(const lbm_handle h, int i) { return h->Q == 9 ? D2Q9::cz(i) : D3Q19::cz(i); }

// Enqueue one time step on the stream (parity = buffer holding f+(t)).
lbm_status enqueue_step(lbm_handle h, int parity, int64_t step_index, bool timed) {
  void* fc = h->f[parity];
  void* fn = h->f[parity ^ 1];
  double* slot = h->force + 3 * MAX_BODIES * (step_index & 1);
  double* next = h->force + 3 * MAX_BODIES * ((step_index + 1) & 1);
  auto timed_launch = [&](int kid, auto&& fn_launch) -> lbm_status {
    if (!timed) {
      fn_launch();
      return LBM_OK;
    }
    if (h->ev_used + 2 > h->ev.size()) {
      for (int k = 0; k < 64; ++k) {
        cudaEvent_t e;
        CUDA_TRY(cudaEventCreate(&e));
        h->ev.push_back(e);
        h->ev_kernel.push_back(0);
      }
    }
    const size_t a = h->ev_used;
    h->ev_kernel[a] = kid;
    CUDA_TRY(cudaEventRecord(h->ev[a], h->stream));
    fn_launch();
    CUDA_TRY(cudaEventRecord(h->ev[a + 1], h->stream));
    h->ev_used += 2;
    return LBM_OK;
  };
  lbm_status st;
  st = timed_launch(0, [&] { h->ops.links(fc, h->mom, h->keys, h->q, h->uw, h->n_links, slot, h->p, h->stream); });
  if (st != LBM_OK) return st;
  if (h->p.inlet || h->p.outlet) {
    st = timed_launch(1, [&] { h->ops.open(fc, h->mom, h->mask, h->p, h->stream); });
    if (st != LBM_OK) return st;
  }
  st = timed_launch(2, [&] { h->ops.bulk(fc, fn, h->mask, h->mom, next, h->p, h->stream); });
  if (st != LBM_OK) return st;
  CUDA_TRY(cudaGetLastError());
  return LBM_OK;
}

lbm_status harvest_events(lbm_handle h) {
  if (h->ev_used == 0) return LBM_OK;
  CUDA_TRY(cudaStreamSynchronize(h->stream));
  for (size_t a = 0; a + 1 < h->ev_used; a += 2) {
    float ms = 0.f;
    CUDA_TRY(cudaEventElapsedTime(&ms, h->ev[a], h->ev[a + 1]));
    h->prof_launches[h->ev_kernel[a]] += 1;
    h->prof_ms[h->ev_kernel[a]] += ms;
  }
  h->ev_used = 0;
  return LBM_OK;
}

lbm_status build_graph(lbm_handle h, int parity) {
  cudaGraph_t g = nullptr;
  CUDA_TRY(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
  // graphs are replayed from even step counts only: force slots 0 then 1
  lbm_status st = enqueue_step(h, parity, 0, false);
  if (st == LBM_OK) st = enqueue_step(h, parity ^ 1, 1, false);
  cudaError_t e = cudaStreamEndCapture(h->stream, &g);
  if (st != LBM_OK) {
    if (g) cudaGraphDestroy(g);
    return st;
  }
  if (e != cudaSuccess) return fail(LBM_ERR_CUDA, "stream capture: %s", cudaGetErrorString(e));
  e = cudaGraphInstantiate(&h->graph[parity], g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return fail(LBM_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(e));
  return LBM_OK;
}

bool is_device_pointer(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" {

const char* lbm_last_error(void) { return g_msg; }

lbm_status lbm_create_lattice(const lbm_config* cfg, lbm_handle* out) {
  g_msg[0] = 0;
  if (!cfg || !out) return fail(LBM_ERR_INVALID_ARG, "null argument");
  *out = nullptr;
  const lbm_config& c = *cfg;
  if (c.stencil != LBM_D2Q9 && c.stencil != LBM_D3Q19) return fail(LBM_ERR_INVALID_ARG, "unknown stencil %d", c.stencil);
  if (c.precision != LBM_FP64 && c.precision != LBM_FP32_SHIFTED)
    return fail(LBM_ERR_INVALID_ARG, "unknown precision %d", c.precision);
  if (c.collision == LBM_MRT) return fail(LBM_ERR_UNSUPPORTED, "MRT collision is not built");
  if (c.collision != LBM_BGK) return fail(LBM_ERR_INVALID_ARG, "unknown collision %d", c.collision);
  if (c.bc < LBM_BC_HALFWAY || c.bc > LBM_BC_VIBB) return fail(LBM_ERR_INVALID_ARG, "unknown default rule %d", c.bc);
  if (c.vibb_density != LBM_VIBB_RHO_PRINTED && c.vibb_density != LBM_VIBB_RHO_LOCAL)
    return fail(LBM_ERR_INVALID_ARG, "unknown vibb_density %d", c.vibb_density);
  if (c.nx < 1 || c.ny < 1 || c.nz < 1) return fail(LBM_ERR_INVALID_ARG, "lattice size must be positive");
  if (c.stencil == LBM_D2Q9 && c.nz != 1) return fail(LBM_ERR_INVALID_ARG, "D2Q9 needs nz == 1");
  if (c.ny > 65535 || c.nz > 65535) return fail(LBM_ERR_UNSUPPORTED, "ny and nz are limited to 65535");
  if (!(c.tau > 0.5) || !std::isfinite(c.tau)) return fail(LBM_ERR_INVALID_ARG, "tau must be finite and > 1/2");
  if (!(c.rho0 > 0.0) || !std::isfinite(c.rho0)) return fail(LBM_ERR_INVALID_ARG, "rho0 must be positive");
  for (int a = 0; a < 3; ++a)
    if (!std::isfinite(c.g[a])) return fail(LBM_ERR_INVALID_ARG, "g must be finite");
  if ((c.inlet || c.outlet) && c.stencil != LBM_D2Q9)
    return fail(LBM_ERR_UNSUPPORTED, "open inlet/outlet columns are built for D2Q9 only");
  if ((c.inlet || c.outlet) && c.periodic[0]) return fail(LBM_ERR_INVALID_ARG, "open columns need a non-periodic x axis");
  if (c.inlet && !(c.inlet_y1 > c.inlet_y0)) return fail(LBM_ERR_INVALID_ARG, "inlet needs inlet_y1 > inlet_y0");
  const int64_t N = (int64_t)c.nx * c.ny * c.nz;
  if (N >= ((int64_t)1 << 31)) return fail(LBM_ERR_UNSUPPORTED, "lattices are limited to 2^31 nodes");

  lbm_handle h = new (std::nothrow) lbm_lattice_s;
  if (!h) return fail(LBM_ERR_OOM, "host allocation failed");
  h->cfg = c;
  if (c.stencil == LBM_D2Q9)
    h->ops = c.precision == LBM_FP64 ? ops_d2q9_f64() : ops_d2q9_f32s();
  else
    h->ops = c.precision == LBM_FP64 ? ops_d3q19_f64() : ops_d3q19_f32s();
  h->Q = h->ops.Q;
  h->D = h->ops.D;
  h->N = N;
  h->rb = h->ops.real_bytes;
  Params& p = h->p;
  p.nx = c.nx;
  p.ny = c.ny;
  p.nz = c.nz;
  p.N = N;
  p.tau = c.tau;
  p.rho0 = c.rho0;
  for (int a = 0; a < 3; ++a) p.g[a] = (a < h->D) ? c.g[a] : 0.0;
  p.has_force = (p.g[0] != 0.0 || p.g[1] != 0.0 || p.g[2] != 0.0);
  p.collision = c.collision;
  p.inlet = c.inlet ? 1 : 0;
  p.outlet = c.outlet ? 1 : 0;
  p.inlet_umax = c.inlet_umax;
  p.inlet_y0 = c.inlet_y0;
  p.inlet_y1 = c.inlet_y1;
  p.vibb_local_rho = c.vibb_density == LBM_VIBB_RHO_LOCAL ? 1 : 0;

  lbm_status st = LBM_OK;
  if (c.cuda_stream) {
    h->stream = (cudaStream_t)c.cuda_stream;
  } else {
    cudaError_t e = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      delete h;
      return fail(LBM_ERR_CUDA, "cudaStreamCreate: %s", cudaGetErrorString(e));
    }
    h->own_stream = true;
  }
  const size_t fb = (size_t)h->Q * N * h->rb;
  for (int k = 0; k < 2 && st == LBM_OK; ++k) st = dev_alloc(h, &h->f[k], fb);
  if (st == LBM_OK) st = dev_alloc(h, &h->mom, (size_t)4 * N * h->rb);
  if (st == LBM_OK) st = dev_alloc(h, (void**)&h->mask, (size_t)N);
  if (st == LBM_OK) st = dev_alloc(h, (void**)&h->force, sizeof(double) * 2 * 3 * MAX_BODIES);
  if (st == LBM_OK) {
    cudaError_t e = cudaMemsetAsync(h->force, 0, sizeof(double) * 2 * 3 * MAX_BODIES, h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->mom, 0, (size_t)4 * N * h->rb, h->stream);
    if (e != cudaSuccess) st = fail(LBM_ERR_CUDA, "cudaMemsetAsync: %s", cudaGetErrorString(e));
  }
  if (st != LBM_OK) {
    char keep[sizeof g_msg];
    memcpy(keep, g_msg, sizeof keep);
    lbm_destroy(h);
    memcpy(g_msg, keep, sizeof keep);
    return st;
  }
  *out = h;
  return LBM_OK;
}

lbm_status lbm_destroy(lbm_handle h) {
  if (!h) return LBM_OK;
  if (h->stream) cudaStreamSynchronize(h->stream);
  drop_graphs(h);
  for (auto e : h->ev) cudaEventDestroy(e);
  for (int k = 0; k < 2; ++k)
    if (h->f[k]) cudaFree(h->f[k]);
  if (h->mom) cudaFree(h->mom);
  if (h->mask) cudaFree(h->mask);
  if (h->force) cudaFree(h->force);
  free_links(h);
  if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
  delete h;
  return LBM_OK;
}

lbm_status lbm_set_geometry(lbm_handle h, const uint8_t* solid, const lbm_link* links, int64_t n_links) {
  g_msg[0] = 0;
  if (!h || !solid || n_links < 0 || (n_links > 0 && !links)) return fail(LBM_ERR_INVALID_ARG, "null or negative argument");
  const lbm_config& c = h->cfg;
  const int64_t N = h->N, nx = c.nx, ny = c.ny, nz = c.nz;
  const int Q = h->Q, D = h->D;
  // node classes: mask bits
  std::vector<uint8_t> m(N);
  for (int64_t n = 0; n < N; ++n) m[n] = solid[n] ? M_SOLID : 0;
  if (c.inlet || c.outlet)
    for (int64_t z = 0; z < nz; ++z)
      for (int64_t y = 0; y < ny; ++y) {
        const int64_t row = nx * (y + ny * z);
        if (c.inlet && !(m[row] & M_SOLID)) m[row] |= M_OPEN;
        if (c.outlet && !(m[row + nx - 1] & M_SOLID)) m[row + nx - 1] |= M_OPEN;
      }
  // faces of non-periodic axes must be solid (or open columns)
  const int64_t len[3] = {nx, ny, nz};
  for (int a = 0; a < 3; ++a) {
    if (c.periodic[a] || (a == 2 && D == 2)) continue;
    for (int64_t n = 0; n < N; ++n) {
      const int64_t x[3] = {n % nx, (n / nx) % ny, n / (nx * ny)};
      if ((x[a] == 0 || x[a] == len[a] - 1) && !(m[n] & (M_SOLID | M_OPEN)))
        return fail(LBM_ERR_INVALID_ARG,
                    "node (%lld,%lld,%lld) on a face of non-periodic axis %d is fluid: add a solid layer",
                    (long long)x[0], (long long)x[1], (long long)x[2], a);
    }
  }
  auto coords = [&](int64_t n, int64_t x[3]) {
    x[0] = n % nx;
    x[1] = (n / nx) % ny;
    x[2] = n / (nx * ny);
  };
  // neighbour n + s e_d with wrap; -1 if it leaves through a non-periodic face
  auto neighbour = [&](int64_t n, int d, int s, bool* wrapped) -> int64_t {
    int64_t x[3];
    coords(n, x);
    const int e[3] = {cx_of(h, d), cy_of(h, d), cz_of(h, d)};
    for (int a = 0; a < 3; ++a) {
      x[a] += s * e[a];
      if (x[a] < 0 || x[a] >= len[a]) {
        if (!c.periodic[a]) return -1;
        x[a] = (x[a] + len[a]) % len[a];
        if (wrapped) *wrapped = true;
      }
    }
    return x[0] + nx * (x[1] + ny * x[2]);
  };
  // links
  std::vector<uint64_t> keys(n_links);
  std::vector<double> qs(n_links);
  bool moving = false;
  for (int64_t k = 0; k < n_links; ++k) {
    const lbm_link& L = links[k];
    if (L.node < 0 || L.node >= N) return fail(LBM_ERR_INVALID_ARG, "link %lld: node out of range", (long long)k);
    if (m[L.node] & (M_SOLID | M_OPEN))
      return fail(LBM_ERR_INVALID_ARG, "link %lld: node %lld is not a fluid node", (long long)k, (long long)L.node);
    if (L.dir < 1 || L.dir >= Q) return fail(LBM_ERR_INVALID_ARG, "link %lld: dir %d out of range", (long long)k, L.dir);
    if (!(L.q > 0.0 && L.q <= 1.0)) return fail(LBM_ERR_INVALID_ARG, "link %lld: q = %g not in (0,1]", (long long)k, L.q);
    if (L.bc < LBM_BC_DEFAULT || L.bc > LBM_BC_VIBB)
      return fail(LBM_ERR_INVALID_ARG, "link %lld: unknown rule %d", (long long)k, L.bc);
    if (L.body < -1 || L.body >= MAX_BODIES)
      return fail(LBM_ERR_INVALID_ARG, "link %lld: body %d out of range", (long long)k, L.body);
    for (int a = 0; a < 3; ++a)
      if (!std::isfinite(L.uw[a])) return fail(LBM_ERR_INVALID_ARG, "link %lld: non-finite wall velocity", (long long)k);
    bool wrapped = false;
    const int64_t s = neighbour(L.node, L.dir, 1, &wrapped);
    if (s < 0 || !(m[s] & M_SOLID))
      return fail(LBM_ERR_INVALID_ARG, "link %lld: neighbour of node %lld in direction %d is not a solid node",
                  (long long)k, (long long)L.node, L.dir);
    const int64_t ff = neighbour(L.node, L.dir, -1, &wrapped);
    const int fallback = (ff < 0 || (m[ff] & (M_SOLID | M_OPEN))) ? 1 : 0;
    const int rule = L.bc >= 0 ? L.bc : c.bc;
    if (rule == LBM_BC_VIBB) {
      m[L.node] |= M_CACHE;
      if (!fallback) m[ff] |= M_CACHE;
    }
    for (int a = 0; a < D; ++a) moving |= L.uw[a] != 0.0;
    keys[k] = pack_key(L.node, L.dir, rule, fallback, wrapped ? 1 : 0, L.body);
    qs[k] = L.q;
  }
  // open inlet reads the moments of the first fluid column
  if (c.inlet)
    for (int64_t y = 0; y < ny; ++y)
      if ((m[nx * y] & M_OPEN) && nx > 1) {
        if (m[nx * y + 1] & (M_SOLID | M_OPEN))
          return fail(LBM_ERR_INVALID_ARG, "inlet node (0,%lld) has no fluid node at x = 1", (long long)y);
        m[nx * y + 1] |= M_CACHE;
      }
  // order by (node, dir) -- the usual input order already -- then stably
  // by body; reject duplicate (node, dir)
  std::vector<int64_t> order(n_links);
  for (int64_t k = 0; k < n_links; ++k) order[k] = k;
  auto nodedir = [&](int64_t k) { return (keys[k] >> KEY_NODE_SHIFT) * 32 + (keys[k] & 31); };
  bool sorted = true;
  for (int64_t k = 1; k < n_links && sorted; ++k) sorted = nodedir(k - 1) < nodedir(k);
  if (!sorted) {
    std::vector<std::pair<uint64_t, int64_t>> tmp(n_links);
    for (int64_t k = 0; k < n_links; ++k) tmp[k] = {nodedir(k), k};
    std::sort(tmp.begin(), tmp.end());
    for (int64_t k = 0; k < n_links; ++k) order[k] = tmp[k].second;
  }
  for (int64_t k = 1; k < n_links; ++k)
    if (nodedir(order[k]) == nodedir(order[k - 1]))
      return fail(LBM_ERR_INVALID_ARG, "duplicate link at node %lld direction %d",
                  (long long)(nodedir(order[k]) / 32), (int)(nodedir(order[k]) % 32));
  {
    std::vector<int64_t> count(MAX_BODIES + 2, 0);
    for (int64_t k = 0; k < n_links; ++k) count[links[k].body + 2]++;
    for (int b = 1; b < MAX_BODIES + 2; ++b) count[b] += count[b - 1];
    std::vector<int64_t> byb(n_links);
    for (int64_t k = 0; k < n_links; ++k) byb[count[links[order[k]].body + 1]++] = order[k];
    order.swap(byb);
  }
  // completeness: count (fluid node, dir) pairs with a solid neighbour
  int64_t expected = 0, n_fluid = 0;
  for (int64_t n = 0; n < N; ++n) {
    if (m[n] & (M_SOLID | M_OPEN)) continue;
    ++n_fluid;
    int64_t x[3];
    coords(n, x);
    for (int d = 1; d < Q; ++d) {
      int64_t y[3] = {x[0] + cx_of(h, d), x[1] + cy_of(h, d), x[2] + cz_of(h, d)};
      bool out = false;
      for (int a = 0; a < 3; ++a)
        if (y[a] < 0 || y[a] >= len[a]) {
          if (!c.periodic[a]) out = true;
          y[a] = (y[a] + len[a]) % len[a];
        }
      if (out) continue;  // only open columns can sit there (faces are solid otherwise)
      if (m[y[0] + nx * (y[1] + ny * y[2])] & M_SOLID) ++expected;
    }
  }
  if (expected != n_links)
    return fail(LBM_ERR_INVALID_ARG, "%lld fluid-to-solid neighbour pairs but %lld links: every cut link needs a record",
                (long long)expected, (long long)n_links);
  int64_t n_cached = 0;
  for (int64_t n = 0; n < N; ++n) n_cached += (m[n] & M_CACHE) ? 1 : 0;

  // device arrays
  CUDA_TRY(cudaStreamSynchronize(h->stream));
  drop_graphs(h);
  free_links(h);
  std::vector<uint64_t> skeys(n_links);
  for (int64_t k = 0; k < n_links; ++k) skeys[k] = keys[order[k]];
  lbm_status st = LBM_OK;
  const size_t rb = h->rb;
  if (n_links > 0) {
    st = dev_alloc(h, (void**)&h->keys, sizeof(uint64_t) * n_links);
    if (st == LBM_OK) st = dev_alloc(h, &h->q, rb * n_links);
    if (st == LBM_OK && moving) st = dev_alloc(h, &h->uw, rb * D * n_links);
    if (st != LBM_OK) {
      free_links(h);
      return st;
    }
    CUDA_TRY(cudaMemcpy(h->keys, skeys.data(), sizeof(uint64_t) * n_links, cudaMemcpyHostToDevice));
    if (rb == 8) {
      std::vector<double> tq(n_links), tw(moving ? D * n_links : 0);
      for (int64_t k = 0; k < n_links; ++k) {
        tq[k] = qs[order[k]];
        if (moving)
          for (int a = 0; a < D; ++a) tw[a * n_links + k] = links[order[k]].uw[a];
      }
      CUDA_TRY(cudaMemcpy(h->q, tq.data(), 8 * n_links, cudaMemcpyHostToDevice));
      if (moving) CUDA_TRY(cudaMemcpy(h->uw, tw.data(), 8 * D * n_links, cudaMemcpyHostToDevice));
    } else {
      std::vector<float> tq(n_links), tw(moving ? D * n_links : 0);
      for (int64_t k = 0; k < n_links; ++k) {
        tq[k] = (float)qs[order[k]];
        if (moving)
          for (int a = 0; a < D; ++a) tw[a * n_links + k] = (float)links[order[k]].uw[a];
      }
      CUDA_TRY(cudaMemcpy(h->q, tq.data(), 4 * n_links, cudaMemcpyHostToDevice));
      if (moving) CUDA_TRY(cudaMemcpy(h->uw, tw.data(), 4 * D * n_links, cudaMemcpyHostToDevice));
    }
  }
  CUDA_TRY(cudaMemcpy(h->mask, m.data(), (size_t)N, cudaMemcpyHostToDevice));
  h->n_links = n_links;
  h->n_fluid = n_fluid;
  h->n_cached = n_cached;
  h->has_geometry = true;
  h->has_state = false;
  return LBM_OK;
}

lbm_status lbm_init_equilibrium(lbm_handle h, const double* rho, const double* u) {
  g_msg[0] = 0;
  if (!h) return fail(LBM_ERR_INVALID_ARG, "null handle");
  if (!h->has_geometry) return fail(LBM_ERR_STATE, "set the geometry first");
  const int64_t N = h->N;
  double *drho = nullptr, *du = nullptr;
  if (rho) CUDA_TRY(cudaMalloc(&drho, sizeof(double) * N));
  if (u) {
    cudaError_t e = cudaMalloc(&du, sizeof(double) * 3 * N);
    if (e != cudaSuccess) {
      cudaFree(drho);
      return fail(LBM_ERR_OOM, "cudaMalloc: %s", cudaGetErrorString(e));
    }
  }
  cudaError_t e = cudaSuccess;
  if (rho) e = cudaMemcpyAsync(drho, rho, sizeof(double) * N, cudaMemcpyHostToDevice, h->stream);
  if (u && e == cudaSuccess) e = cudaMemcpyAsync(du, u, sizeof(double) * 3 * N, cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) {
    CUDA_TRY(cudaMemsetAsync(h->mom, 0, (size_t)4 * N * h->rb, h->stream));
    h->ops.init(h->f[0], h->mom, h->mask, drho, du, h->p, h->stream);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemsetAsync(h->force, 0, sizeof(double) * 2 * 3 * MAX_BODIES, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  cudaFree(drho);
  cudaFree(du);
  if (e != cudaSuccess) return fail(LBM_ERR_CUDA, "init: %s", cudaGetErrorString(e));
  h->cur = 0;
  h->step = 0;
  h->has_state = true;
  return LBM_OK;
}

lbm_status lbm_step(lbm_handle h, int64_t n) {
  g_msg[0] = 0;
  if (!h) return fail(LBM_ERR_INVALID_ARG, "null handle");
  if (n < 0) return fail(LBM_ERR_INVALID_ARG, "negative step count");
  if (!h->has_state) return fail(LBM_ERR_STATE, "initialise the state first");
  if (h->profiling) {
    for (int64_t k = 0; k < n; ++k) {
      lbm_status st = enqueue_step(h, h->cur, h->step, true);
      if (st != LBM_OK) return st;
      h->cur ^= 1;
      ++h->step;
      if (h->ev_used > (1u << 16)) {
        st = harvest_events(h);
        if (st != LBM_OK) return st;
      }
    }
    return LBM_OK;
  }
  int64_t left = n;
  // graphs run two steps and keep the force slot parity; align first
  if (left > 0 && (h->step & 1)) {
    lbm_status st = enqueue_step(h, h->cur, h->step, false);
    if (st != LBM_OK) return st;
    h->cur ^= 1;
    ++h->step;
    --left;
  }
  if (left >= 2) {
    if (!h->graph[h->cur]) {
      lbm_status st = build_graph(h, h->cur);
      if (st != LBM_OK) return st;
    }
    for (; left >= 2; left -= 2) {
      CUDA_TRY(cudaGraphLaunch(h->graph[h->cur], h->stream));
      h->step += 2;
    }
  }
  if (left == 1) {
    lbm_status st = enqueue_step(h, h->cur, h->step, false);
    if (st != LBM_OK) return st;
    h->cur ^= 1;
    ++h->step;
  }
  return LBM_OK;
}

lbm_status lbm_moments(lbm_handle h, double* rho, double* u) {
  g_msg[0] = 0;
  if (!h || !rho || !u) return fail(LBM_ERR_INVALID_ARG, "null argument");
  if (!h->has_state) return fail(LBM_ERR_STATE, "no state");
  const bool drho = is_device_pointer(rho), du = is_device_pointer(u);
  if (drho != du) return fail(LBM_ERR_INVALID_ARG, "rho and u must both be host or both device pointers");
  const int64_t N = h->N;
  if (drho) {
    h->ops.moments(h->f[h->cur], h->mask, rho, u, h->p, h->stream);
    CUDA_TRY(cudaGetLastError());
    return LBM_OK;
  }
  double* tmp = nullptr;
  CUDA_TRY(cudaMalloc(&tmp, sizeof(double) * (1 + h->D) * N));
  h->ops.moments(h->f[h->cur], h->mask, tmp, tmp + N, h->p, h->stream);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(rho, tmp, sizeof(double) * N, cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(u, tmp + N, sizeof(double) * h->D * N, cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  cudaFree(tmp);
  if (e != cudaSuccess) return fail(LBM_ERR_CUDA, "moments: %s", cudaGetErrorString(e));
  return LBM_OK;
}

lbm_status lbm_force(lbm_handle h, int32_t body, double F[3]) {
  g_msg[0] = 0;
  if (!h || !F) return fail(LBM_ERR_INVALID_ARG, "null argument");
  if (body < 0 || body >= MAX_BODIES) return fail(LBM_ERR_INVALID_ARG, "body %d out of range", body);
  if (!h->has_state || h->step == 0) return fail(LBM_ERR_STATE, "no step has run");
  const double* slot = h->force + 3 * MAX_BODIES * ((h->step - 1) & 1) + 3 * body;
  CUDA_TRY(cudaMemcpyAsync(F, slot, sizeof(double) * 3, cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(cudaStreamSynchronize(h->stream));
  return LBM_OK;
}

lbm_status lbm_get_distributions(lbm_handle h, double* f) {
  g_msg[0] = 0;
  if (!h || !f) return fail(LBM_ERR_INVALID_ARG, "null argument");
  if (!h->has_state) return fail(LBM_ERR_STATE, "no state");
  const int64_t N = h->N;
  double* tmp = nullptr;
  CUDA_TRY(cudaMalloc(&tmp, sizeof(double) * N));
  cudaError_t e = cudaSuccess;
  for (int i = 0; i < h->Q && e == cudaSuccess; ++i) {
    h->ops.get_dir(h->f[h->cur], h->mask, i, tmp, h->p, h->stream);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(f + (int64_t)i * N, tmp, sizeof(double) * N, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  }
  cudaFree(tmp);
  if (e != cudaSuccess) return fail(LBM_ERR_CUDA, "get_distributions: %s", cudaGetErrorString(e));
  return LBM_OK;
}

lbm_status lbm_set_distributions(lbm_handle h, const double* f) {
  g_msg[0] = 0;
  if (!h || !f) return fail(LBM_ERR_INVALID_ARG, "null argument");
  if (!h->has_geometry) return fail(LBM_ERR_STATE, "set the geometry first");
  const int64_t N = h->N;
  double* tmp = nullptr;
  CUDA_TRY(cudaMalloc(&tmp, sizeof(double) * N));
  cudaError_t e = cudaStreamSynchronize(h->stream);
  for (int i = 0; i < h->Q && e == cudaSuccess; ++i) {
    e = cudaMemcpyAsync(tmp, f + (int64_t)i * N, sizeof(double) * N, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) {
      h->ops.set_dir(h->f[h->cur], h->mask, i, tmp, h->p, h->stream);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  }
  if (e == cudaSuccess) {
    h->ops.refresh(h->f[h->cur], h->mask, h->mom, h->p, h->stream);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  cudaFree(tmp);
  if (e != cudaSuccess) return fail(LBM_ERR_CUDA, "set_distributions: %s", cudaGetErrorString(e));
  h->has_state = true;
  return LBM_OK;
}

lbm_status lbm_gather(lbm_handle h, const int64_t* nodes, int64_t n, double* out) {
  g_msg[0] = 0;
  if (!h || n < 0 || (n > 0 && (!nodes || !out))) return fail(LBM_ERR_INVALID_ARG, "null or negative argument");
  if (!h->has_state) return fail(LBM_ERR_STATE, "no state");
  for (int64_t k = 0; k < n; ++k)
    if (nodes[k] < 0 || nodes[k] >= h->N) return fail(LBM_ERR_INVALID_ARG, "node %lld out of range", (long long)nodes[k]);
  if (n == 0) return LBM_OK;
  int64_t* dn = nullptr;
  double* dout = nullptr;
  CUDA_TRY(cudaMalloc(&dn, sizeof(int64_t) * n));
  cudaError_t e = cudaMalloc(&dout, sizeof(double) * h->Q * n);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dn, nodes, sizeof(int64_t) * n, cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) {
    h->ops.gather(h->f[h->cur], h->mask, dn, n, dout, h->p, h->stream);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(out, dout, sizeof(double) * h->Q * n, cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  cudaFree(dn);
  cudaFree(dout);
  if (e != cudaSuccess) return fail(LBM_ERR_CUDA, "gather: %s", cudaGetErrorString(e));
  return LBM_OK;
}

lbm_status lbm_check(lbm_handle h) {
  g_msg[0] = 0;
  if (!h) return fail(LBM_ERR_INVALID_ARG, "null handle");
  if (!h->has_state) return fail(LBM_ERR_STATE, "no state");
  int* flag = nullptr;
  CUDA_TRY(cudaMalloc(&flag, sizeof(int)));
  int hv = 0;
  cudaError_t e = cudaMemsetAsync(flag, 0, sizeof(int), h->stream);
  if (e == cudaSuccess) {
    h->ops.check(h->f[h->cur], h->mask, flag, h->p, h->stream);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hv, flag, sizeof(int), cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  cudaFree(flag);
  if (e != cudaSuccess) return fail(LBM_ERR_CUDA, "check: %s", cudaGetErrorString(e));
  if (hv) return fail(LBM_ERR_DIVERGED, "non-finite population or non-positive density at step %lld", (long long)h->step);
  return LBM_OK;
}

lbm_status lbm_synchronize(lbm_handle h) {
  if (!h) return fail(LBM_ERR_INVALID_ARG, "null handle");
  CUDA_TRY(cudaStreamSynchronize(h->stream));
  return LBM_OK;
}

lbm_status lbm_query(lbm_handle h, lbm_info* info) {
  if (!h || !info) return fail(LBM_ERR_INVALID_ARG, "null argument");
  info->n_nodes = h->N;
  info->n_fluid = h->n_fluid;
  info->n_links = h->n_links;
  info->n_cached = h->n_cached;
  info->step = h->step;
  info->device_bytes = h->device_bytes;
  info->Q = h->Q;
  info->D = h->D;
  info->precision = h->cfg.precision;
  info->real_bytes = (int32_t)h->rb;
  return LBM_OK;
}

lbm_status lbm_set_profiling(lbm_handle h, int32_t on) {
  g_msg[0] = 0;
  if (!h) return fail(LBM_ERR_INVALID_ARG, "null handle");
  lbm_status st = harvest_events(h);
  if (st != LBM_OK) return st;
  h->profiling = on != 0;
  for (int k = 0; k < kMaxTimedKernels; ++k) {
    h->prof_launches[k] = 0;
    h->prof_ms[k] = 0.0;
  }
  return LBM_OK;
}

lbm_status lbm_kernel_times(lbm_handle h, int64_t launches[3], double ms[3]) {
  g_msg[0] = 0;
  if (!h || !launches || !ms) return fail(LBM_ERR_INVALID_ARG, "null argument");
  lbm_status st = harvest_events(h);
  if (st != LBM_OK) return st;
  for (int k = 0; k < kMaxTimedKernels; ++k) {
    launches[k] = h->prof_launches[k];
    ms[k] = h->prof_ms[k];
  }
  return LBM_OK;
}

}  // extern "C"
