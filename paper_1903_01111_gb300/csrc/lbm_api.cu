// Host side of liblbm.so: the C ABI declared in include/lbm.h.
//
// A lattice owns two population buffers (ping-pong) over the stored nodes of
// the compacted layout (fluid, open-column and ghost nodes, see
// kernels.cuh), two moment caches (the moments of buffer c live in cache c),
// the layout tables, the link records (in the link kernel's order and in the
// fused step kernel's (node, direction) order), the domain table of a batch
// and two FP64 force slots.  lbm_step replays
// captured CUDA graphs (graph_steps steps, then two) and launches single
// steps directly for an odd remainder; with profiling on it launches kernel
// by kernel between CUDA events.  lbm_autotune picks the launch shapes.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <type_traits>
#include <utility>
#include <vector>

#include "adjoint.cuh"
#include "kernels.cuh"
#include "lbm.h"

using namespace lbm;

namespace {

thread_local char g_msg[1024] = "";

// NVTX range over a scope (host-side annotation for timeline profilers;
// without a profiler attached the calls return at once).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

lbm_status fail(lbm_status st, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_msg, sizeof g_msg, fmt, ap);
  va_end(ap);
  return st;
}

#define CUDA_TRY(call)                                                                                    \
  do {                                                                                                    \
    cudaError_t e_ = (call);                                                                              \
    if (e_ != cudaSuccess)                                                                                \
      return fail(e_ == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA, "%s: %s (%s:%d)", #call, \
                  cudaGetErrorString(e_), __FILE__, __LINE__);                                            \
  } while (0)

constexpr int kMaxTimedKernels = 3;

// Host arrays of the layout build: elements are not value-initialised on
// construction (a serial zero fill of a few GB took a large part of
// lbm_set_geometry); each array is filled or written in full by parallel
// loops, which also spread the first-touch page faults over the threads.
template <class T>
struct RawAlloc {
  using value_type = T;
  RawAlloc() = default;
  template <class U>
  RawAlloc(const RawAlloc<U>&) {}
  T* allocate(size_t n) { return std::allocator<T>().allocate(n); }
  void deallocate(T* p, size_t n) { std::allocator<T>().deallocate(p, n); }
  template <class U>
  void construct(U* p) noexcept(std::is_nothrow_default_constructible<U>::value) {
    ::new ((void*)p) U;
  }
  template <class U, class... A>
  void construct(U* p, A&&... a) {
    ::new ((void*)p) U(std::forward<A>(a)...);
  }
  template <class U>
  bool operator==(const RawAlloc<U>&) const { return true; }
  template <class U>
  bool operator!=(const RawAlloc<U>&) const { return false; }
};
template <class T>
using raw_vec = std::vector<T, RawAlloc<T>>;

template <class V, class T>
void par_fill(V& v, const T& x) {
  const int64_t n = (int64_t)v.size();
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) v[i] = x;
}

// host mask bits used while building the layout
enum : uint8_t { H_SOLID = 1, H_CACHE = 2, H_OPEN = 4, H_GHOST = 8 };

}  // namespace

void lbm::set_last_error(const char* msg) { snprintf(g_msg, sizeof g_msg, "%s", msg); }

// One owned device buffer.
struct DeviceBuf {
  void* p = nullptr;
  size_t bytes = 0;
};

struct lbm_lattice_s {
  lbm_config cfg{};
  KernelOps ops{};
  AdjointOps adj{};
  Params p{};
  int Q = 0, D = 0;
  int64_t N = 0;
  size_t rb = 0;  // bytes per stored real
  // state over stored nodes: f[c] and its moment cache mom[c]
  DeviceBuf f[2], mom[2];
  // layout
  DeviceBuf word, node_of, runs, row_first, row_last, row_in1, row_out1;
  Layout lay{};
  // batch: domains along the last axis (empty: one domain run by cfg)
  std::vector<lbm_domain> domains;
  DeviceBuf dom, row_dom;
  int nbody = 1;  // force accumulators per slot
  lbm_tuning tune{-1, 256, 2, 1, 1};
  raw_vec<int32_t> sidx;  // dense -> storage index (-1: not stored), host
  // links, in the link kernel's order (body, node, dir)
  DeviceBuf recs, q, uw;
  // links of the fused step kernel, in (node, dir) order (FusedLinks)
  DeviceBuf lfirst, lmask, lrec, lqd, luw;
  DeviceBuf fidx;  // FP64: storage indices of the fluid nodes (the bulk pass's thread map)
  DeviceBuf lqc;   // FP64: per-link VIBB velocity weights [3][n_links] in the link kernel's order
  int64_t n_links = 0, n_fluid = 0, n_cached = 0, n_runs = 0;
  DeviceBuf force;  // [2][nbody][3]
  // shifted storage: sum over each body's links of 2 w_i' rho0 e_i' (FP64),
  // the rest part of the momentum exchange that the link kernel leaves out
  std::vector<double> force_rest = std::vector<double>(3, 0.0);
  // pinned host copy of the force slot read by lbm_force / lbm_forces (a
  // device-to-host copy into pageable memory is staged by the driver)
  double* force_host = nullptr;
  size_t force_host_n = 0;
  raw_vec<int64_t> link_order;  // device link j = caller's link link_order[j]
  bool from_init = false;           // state is the one lbm_init_equilibrium made
  int cur = 0;      // buffer holding f+(t)
  int64_t step = 0;
  bool has_geometry = false, has_state = false;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  cudaGraphExec_t graph[2] = {nullptr, nullptr};   // two steps, per parity of the buffer
  cudaGraphExec_t graphG[2] = {nullptr, nullptr};  // tune.graph_steps steps
  // profiling
  bool profiling = false;
  std::vector<cudaEvent_t> ev;
  std::vector<int> ev_kernel;
  size_t ev_used = 0;
  int64_t prof_launches[kMaxTimedKernels] = {0, 0, 0};
  double prof_ms[kMaxTimedKernels] = {0, 0, 0};
};

namespace {

int64_t device_bytes(const lbm_handle h) {
  const DeviceBuf* all[] = {&h->f[0],     &h->f[1],     &h->mom[0],   &h->mom[1], &h->word,  &h->node_of,
                            &h->runs,     &h->row_first, &h->row_last, &h->row_in1, &h->row_out1, &h->recs,
                            &h->q,        &h->uw,       &h->lfirst, &h->lmask, &h->lrec,
                            &h->lqd,      &h->luw,      &h->force,    &h->dom,    &h->row_dom, &h->fidx, &h->lqc};
  int64_t s = 0;
  for (auto* b : all) s += (int64_t)b->bytes;
  return s;
}

void release(DeviceBuf& b) {
  if (b.p) cudaFree(b.p);
  b.p = nullptr;
  b.bytes = 0;
}

lbm_status acquire(DeviceBuf& b, size_t bytes) {
  release(b);
  if (bytes == 0) return LBM_OK;
  cudaError_t e = cudaMalloc(&b.p, bytes);
  if (e != cudaSuccess) {
    b.p = nullptr;
    cudaGetLastError();
    return fail(LBM_ERR_OOM, "cudaMalloc(%zu bytes): %s", bytes, cudaGetErrorString(e));
  }
  b.bytes = bytes;
  return LBM_OK;
}

lbm_status upload(DeviceBuf& b, const void* src, size_t bytes) {
  lbm_status st = acquire(b, bytes);
  if (st != LBM_OK || bytes == 0) return st;
  CUDA_TRY(cudaMemcpy(b.p, src, bytes, cudaMemcpyHostToDevice));
  return LBM_OK;
}

// First touch of a host output buffer, spread over the host cores: pages a
// caller allocated but never wrote are mapped by the copy that fills them,
// one fault at a time on the thread that drives the copy (a fresh 1.8 GB
// destination took 67 ms that way against 9 ms once mapped).  Writes one
// byte per 4 KB, which the copy then overwrites.
void touch_host_output(void* p, size_t bytes) {
  char* c = (char*)p;
  const int64_t n = (int64_t)((bytes + 4095) / 4096);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) ((volatile char*)c)[i * 4096] = 0;
}

void drop_graphs(lbm_handle h) {
  for (int k = 0; k < 2; ++k) {
    if (h->graph[k]) cudaGraphExecDestroy(h->graph[k]);
    if (h->graphG[k]) cudaGraphExecDestroy(h->graphG[k]);
    h->graph[k] = h->graphG[k] = nullptr;
  }
}

void release_geometry(lbm_handle h) {
  DeviceBuf* all[] = {&h->f[0],     &h->f[1],      &h->mom[0],   &h->mom[1], &h->word,  &h->node_of,
                      &h->runs,     &h->row_first, &h->row_last, &h->row_in1, &h->row_out1, &h->recs,
                      &h->q,        &h->uw,        &h->lfirst, &h->lmask, &h->lrec,
                      &h->lqd,      &h->luw,       &h->dom,      &h->row_dom, &h->fidx, &h->lqc};
  for (auto* b : all) release(*b);
  h->lay = Layout{};
}

int cx_of(const lbm_handle h, int i) { return h->Q == 9 ? D2Q9::cx(i) : D3Q19::cx(i); }
int cy_of(const lbm_handle h, int i) { return h->Q == 9 ? D2Q9::cy(i) : D3Q19::cy(i); }
int cz_of(const lbm_handle h, int i) { return h->Q == 9 ? D2Q9::cz(i) : D3Q19::cz(i); }

// Enqueue one time step from buffer fc (f+(t), moments mc) into fn (moments
// at t+1 into mn), adding the force to `slot` and clearing `next`.  fused:
// the link rules run inside the pull pass (k_fused; mn must differ from mc),
// else the link kernel writes the ghost slots of fc and the bulk kernel
// pulls them (mn may equal mc: the link kernel reads mc before the bulk
// kernel writes it).
lbm_status enqueue_step_buf(lbm_handle h, void* fc, void* fn, void* mc, void* mn, double* slot, double* next,
                            bool timed, bool fused);

// Whether lbm_step runs the fused kernel: chosen by the tuning, and only
// where there are links (without them the bulk kernel is the same pass).
bool use_fused(const lbm_handle h) { return h->tune.fused && h->n_links > 0; }

// Threads per block of the fused kernel: those of the bulk shape when it
// has one node per thread, else 256.
int fused_threads(const lbm_handle h) {
  const BulkShape& b = kBulkShapes[h->tune.bulk_shape < 0 ? 0 : h->tune.bulk_shape];
  return (b.npt == 1 && b.seq == 1) ? b.threads : 256;
}

// Enqueue one time step on the stream (parity = buffer holding f+(t)).
lbm_status enqueue_step(lbm_handle h, int parity, int64_t step_index, bool timed) {
  double* force = (double*)h->force.p;
  const int64_t nb3 = 3 * (int64_t)h->nbody;
  return enqueue_step_buf(h, h->f[parity].p, h->f[parity ^ 1].p, h->mom[parity].p, h->mom[parity ^ 1].p,
                          force + nb3 * (step_index & 1), force + nb3 * ((step_index + 1) & 1), timed, use_fused(h));
}

lbm_status enqueue_step_buf(lbm_handle h, void* fc, void* fn, void* mc, void* mn, double* slot, double* next,
                            bool timed, bool fused) {
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
  if (!fused) {
    st = timed_launch(0, [&] {
      h->ops.links(fc, mc, (const LinkRec*)h->recs.p, h->q.p, h->uw.p, h->lqc.p, h->n_links, slot, h->p, h->lay.S,
                   h->tune.link_threads, h->tune.link_seq, h->stream);
    });
    if (st != LBM_OK) return st;
  }
  if (h->p.inlet || h->p.outlet) {
    st = timed_launch(1, [&] { h->ops.open(fc, mc, h->lay, h->p, h->stream); });
    if (st != LBM_OK) return st;
  }
  if (fused) {
    const FusedRaw fl{(const int32_t*)h->lfirst.p, (const uint32_t*)h->lmask.p, (const FusedRec*)h->lrec.p,
                      (const double*)h->lqd.p, h->luw.p, h->n_links, (h->lay.S + 31) / 32};
    st = timed_launch(2, [&] {
      h->ops.fused(fc, fn, h->lay, fl, mc, mn, slot, next, h->p, fused_threads(h), h->stream);
    });
  } else {
    st = timed_launch(2, [&] { h->ops.bulk(fc, fn, h->lay, mn, next, h->p, h->tune.bulk_shape, h->stream); });
  }
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

// A graph of `steps` (even) steps from the buffer `parity`; graphs are
// replayed from even step counts only, so the force slots alternate 0, 1.
lbm_status build_graph(lbm_handle h, int parity, int steps, cudaGraphExec_t* out) {
  cudaGraph_t g = nullptr;
  CUDA_TRY(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
  lbm_status st = LBM_OK;
  for (int k = 0; k < steps && st == LBM_OK; ++k) st = enqueue_step(h, parity ^ (k & 1), k, false);
  cudaError_t e = cudaStreamEndCapture(h->stream, &g);
  if (st != LBM_OK) {
    if (g) cudaGraphDestroy(g);
    return st;
  }
  if (e != cudaSuccess) return fail(LBM_ERR_CUDA, "stream capture: %s", cudaGetErrorString(e));
  e = cudaGraphInstantiate(out, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return fail(LBM_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(e));
  return LBM_OK;
}

// Pinned host buffer of at least n doubles for reading force slots.
lbm_status force_host_buffer(lbm_handle h, size_t n, double** out) {
  if (h->force_host_n < n) {
    if (h->force_host) cudaFreeHost(h->force_host);
    h->force_host = nullptr;
    h->force_host_n = 0;
    CUDA_TRY(cudaMallocHost(&h->force_host, sizeof(double) * n));
    h->force_host_n = n;
  }
  *out = h->force_host;
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
  if (c.collision != LBM_BGK && c.collision != LBM_MRT) return fail(LBM_ERR_INVALID_ARG, "unknown collision %d", c.collision);
  if (c.collision == LBM_MRT && c.stencil != LBM_D2Q9)
    return fail(LBM_ERR_UNSUPPORTED, "MRT is defined for D2Q9 (the moment matrix of the paper)");
  if (c.bc < LBM_BC_HALFWAY || c.bc > LBM_BC_YU) return fail(LBM_ERR_INVALID_ARG, "unknown default rule %d", c.bc);
  if (c.vibb_density != LBM_VIBB_RHO_PRINTED && c.vibb_density != LBM_VIBB_RHO_LOCAL)
    return fail(LBM_ERR_INVALID_ARG, "unknown vibb_density %d", c.vibb_density);
  if (c.nx < 1 || c.ny < 1 || c.nz < 1) return fail(LBM_ERR_INVALID_ARG, "lattice size must be positive");
  if (c.stencil == LBM_D2Q9 && c.nz != 1) return fail(LBM_ERR_INVALID_ARG, "D2Q9 needs nz == 1");
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
  if (c.stencil == LBM_D2Q9)
    h->adj = c.precision == LBM_FP64 ? adj_d2q9_f64() : adj_d2q9_f32s();
  else
    h->adj = c.precision == LBM_FP64 ? adj_d3q19_f64() : adj_d3q19_f32s();
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
  p.omega = 1.0 / c.tau;
  p.fpre3 = 3.0 * (1.0 - 0.5 / c.tau);
  for (int a = 0; a < 3; ++a) p.g[a] = (a < h->D) ? c.g[a] : 0.0;
  p.has_force = (p.g[0] != 0.0 || p.g[1] != 0.0 || p.g[2] != 0.0);
  if (h->Q == 9)
    fold_params<D2Q9>(p);
  else
    fold_params<D3Q19>(p);
  p.collision = c.collision;
  p.inlet = c.inlet ? 1 : 0;
  p.outlet = c.outlet ? 1 : 0;
  p.inlet_umax = c.inlet_umax;
  p.inlet_y0 = c.inlet_y0;
  p.inlet_y1 = c.inlet_y1;
  p.vibb_local_rho = c.vibb_density == LBM_VIBB_RHO_LOCAL ? 1 : 0;
  for (int a = 0; a < 3; ++a) p.periodic[a] = c.periodic[a] ? 1 : 0;
  p.nbody = 1;
  h->tune.bulk_shape = h->ops.default_shape;

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
  lbm_status st = acquire(h->force, sizeof(double) * 2 * 3);
  if (st == LBM_OK) {
    cudaError_t e = cudaMemsetAsync(h->force.p, 0, h->force.bytes, h->stream);
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
  release_geometry(h);
  release(h->force);
  if (h->force_host) cudaFreeHost(h->force_host);
  if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
  delete h;
  return LBM_OK;
}

lbm_status lbm_set_domains(lbm_handle h, const lbm_domain* d, int32_t n) {
  g_msg[0] = 0;
  if (!h || n < 0 || (n > 0 && !d)) return fail(LBM_ERR_INVALID_ARG, "null or negative argument");
  if (h->has_geometry) return fail(LBM_ERR_STATE, "set the domains before the geometry");
  const lbm_config& c = h->cfg;
  const int64_t len = h->D == 2 ? c.ny : c.nz;
  int64_t next = 0;
  for (int32_t k = 0; k < n; ++k) {
    const lbm_domain& q = d[k];
    if (q.lo != next) return fail(LBM_ERR_INVALID_ARG, "domain %d starts at row %d, expected %lld", k, q.lo, (long long)next);
    if (q.n < 3) return fail(LBM_ERR_INVALID_ARG, "domain %d has %d rows (at least 3)", k, q.n);
    if (q.nx < 1 || q.nx > c.nx) return fail(LBM_ERR_INVALID_ARG, "domain %d: width %d not in 1..%d", k, q.nx, c.nx);
    if (c.periodic[0] && q.nx != c.nx)
      return fail(LBM_ERR_INVALID_ARG, "domain %d: a periodic x axis needs the full width %d", k, c.nx);
    if (!(q.tau > 0.5) || !std::isfinite(q.tau)) return fail(LBM_ERR_INVALID_ARG, "domain %d: tau must be > 1/2", k);
    for (int a = 0; a < 3; ++a)
      if (!std::isfinite(q.g[a])) return fail(LBM_ERR_INVALID_ARG, "domain %d: g must be finite", k);
    if (c.inlet && !(q.inlet_y1 > q.inlet_y0))
      return fail(LBM_ERR_INVALID_ARG, "domain %d: the inlet needs inlet_y1 > inlet_y0", k);
    next = (int64_t)q.lo + q.n;
  }
  if (n > 0 && next != len)
    return fail(LBM_ERR_INVALID_ARG, "domains cover %lld of %lld rows", (long long)next, (long long)len);
  h->domains.assign(d, d + n);
  return LBM_OK;
}

lbm_status lbm_set_geometry(lbm_handle h, const uint8_t* solid, const lbm_link* links, int64_t n_links) {
  g_msg[0] = 0;
  NvtxRange range("lbm_set_geometry");
  if (!h || !solid || n_links < 0 || (n_links > 0 && !links)) return fail(LBM_ERR_INVALID_ARG, "null or negative argument");
  const lbm_config& c = h->cfg;
  const int64_t N = h->N, nx = c.nx, ny = c.ny, nz = c.nz;
  const int Q = h->Q, D = h->D;
  if (n_links >= ((int64_t)1 << 31)) return fail(LBM_ERR_UNSUPPORTED, "at most 2^31 - 1 links");
  // domains: row r = y + ny z belongs to domain rdom[r]; width of each row
  const int ndom = (int)h->domains.size();
  const int64_t rows = ny * nz;
  std::vector<int32_t> rdom(rows, 0);
  std::vector<int64_t> rwidth(rows, nx);
  for (int k = 0; k < ndom; ++k) {
    const lbm_domain& q = h->domains[k];
    for (int64_t r = 0; r < rows; ++r) {
      const int64_t a = D == 2 ? r % ny : r / ny;  // stacking axis: y (2-D) or z (3-D)
      if (a >= q.lo && a < (int64_t)q.lo + q.n) {
        rdom[r] = k;
        rwidth[r] = q.nx;
      }
    }
  }
  // node classes
  raw_vec<uint8_t> m(N);
#pragma omp parallel for schedule(static)
  for (int64_t n = 0; n < N; ++n) m[n] = solid[n] ? H_SOLID : 0;
  if (ndom > 0) {
    for (int64_t r = 0; r < rows; ++r)
      for (int64_t x = rwidth[r]; x < nx; ++x)
        if (!(m[x + nx * r] & H_SOLID))
          return fail(LBM_ERR_INVALID_ARG, "node (%lld, row %lld) lies beyond the width %lld of domain %d: it must be solid",
                      (long long)x, (long long)r, (long long)rwidth[r], rdom[r]);
    for (int k = 0; k < ndom; ++k) {
      const lbm_domain& q = h->domains[k];
      for (int64_t r = 0; r < rows; ++r) {
        const int64_t a = D == 2 ? r % ny : r / ny;
        if (a != q.lo && a != (int64_t)q.lo + q.n - 1) continue;
        for (int64_t x = 0; x < nx; ++x)
          if (!(m[x + nx * r] & H_SOLID))
            return fail(LBM_ERR_INVALID_ARG,
                        "domain %d: its first and last rows must be solid (node %lld of row %lld is not)", k,
                        (long long)x, (long long)r);
      }
    }
  }
  if (c.inlet || c.outlet)
    for (int64_t r = 0; r < rows; ++r) {
      const int64_t row = nx * r;
      if (c.inlet && !(m[row] & H_SOLID)) m[row] |= H_OPEN;
      if (c.outlet && !(m[row + rwidth[r] - 1] & H_SOLID)) m[row + rwidth[r] - 1] |= H_OPEN;
    }
  // faces of non-periodic axes must be solid (or open columns)
  const int64_t len[3] = {nx, ny, nz};
  for (int a = 0; a < 3; ++a) {
    if (c.periodic[a] || (a == 2 && D == 2)) continue;
    // the two faces x_a = 0 and x_a = len_a - 1, node by node
    const int b = a == 0 ? 1 : 0, e = a == 2 ? 1 : 2;  // the other two axes
    for (int64_t side : {(int64_t)0, len[a] - 1})
      for (int64_t v = 0; v < len[e]; ++v)
        for (int64_t u = 0; u < len[b]; ++u) {
          int64_t x[3];
          x[a] = side;
          x[b] = u;
          x[e] = v;
          const int64_t n = x[0] + nx * (x[1] + ny * x[2]);
          if (!(m[n] & (H_SOLID | H_OPEN)))
            return fail(LBM_ERR_INVALID_ARG,
                        "node (%lld,%lld,%lld) on a face of non-periodic axis %d is fluid: add a solid layer",
                        (long long)x[0], (long long)x[1], (long long)x[2], a);
        }
  }
  // the neighbours n + e_d and n - e_d with wrap (-1 where one leaves through
  // a non-periodic face): one split of n into coordinates for both
  auto neighbours = [&](int64_t n, int d, int64_t& plus, int64_t& minus) {
    const int64_t xy = nx * ny;
    const int64_t z = n / xy, rem = n - z * xy, y = rem / nx;
    const int64_t x[3] = {rem - y * nx, y, z};
    const int e[3] = {cx_of(h, d), cy_of(h, d), cz_of(h, d)};
    int64_t p[3], q[3];
    bool pout = false, qout = false;
    for (int a = 0; a < 3; ++a) {
      p[a] = x[a] + e[a];
      q[a] = x[a] - e[a];
      if (p[a] < 0 || p[a] >= len[a]) {
        pout |= !c.periodic[a];
        p[a] = (p[a] + len[a]) % len[a];
      }
      if (q[a] < 0 || q[a] >= len[a]) {
        qout |= !c.periodic[a];
        q[a] = (q[a] + len[a]) % len[a];
      }
    }
    plus = pout ? -1 : p[0] + nx * (p[1] + ny * p[2]);
    minus = qout ? -1 : q[0] + nx * (q[1] + ny * q[2]);
  };
  // links: checks, second fluid node, cache flags.  The checks run in
  // parallel; the first failing link is reported.
  raw_vec<int64_t> lk_s(n_links), lk_ff(n_links);  // written for every link that passes
  raw_vec<int> lk_rule(n_links);
  auto check_link = [&](int64_t k, int64_t& s, int64_t& ff, int& rule) -> int {
    const lbm_link& L = links[k];
    if (L.node < 0 || L.node >= N) return 1;
    if (m[L.node] & (H_SOLID | H_OPEN)) return 2;
    if (L.dir < 1 || L.dir >= Q) return 3;
    if (!(L.q > 0.0 && L.q <= 1.0)) return 4;
    if (L.bc < LBM_BC_DEFAULT || L.bc > LBM_BC_YU) return 5;
    if (L.body < -1 || L.body >= MAX_BODIES) return 6;
    for (int a = 0; a < 3; ++a)
      if (!std::isfinite(L.uw[a])) return 7;
    neighbours(L.node, L.dir, s, ff);
    if (s < 0 || !(m[s] & H_SOLID)) return 8;
    if (ff < 0 || (m[ff] & (H_SOLID | H_OPEN))) ff = L.node;  // no second fluid node: use x_f
    rule = L.bc >= 0 ? L.bc : c.bc;
    return 0;
  };
  // moment-cache nodes (x_f, x_ff of VIBB links: fluid) and ghost nodes
  // (x_s: solid) are disjoint, so one mark per node records both: every
  // writer stores the same byte (an atomic write, no read-modify-write), and
  // the class of the node tells which flag the mark stands for.  The marks
  // are written by the check pass (they matter only if every link passes).
  raw_vec<uint8_t> mark(N);
  par_fill(mark, (uint8_t)0);
  auto nodedir = [&](int64_t k) { return (uint64_t)links[k].node * 32 + (uint64_t)links[k].dir; };
  int64_t first_bad = n_links, unsorted = 0, first_eq = n_links;
  int nbody = 1, moving_i = 0, min_body = MAX_BODIES, max_body = -1;
#pragma omp parallel for schedule(static) reduction(min : first_bad, min_body, first_eq) \
    reduction(max : nbody, max_body) reduction(| : moving_i) reduction(+ : unsorted)
  for (int64_t k = 0; k < n_links; ++k) {
    int64_t s = 0, ff = 0;
    int rule = 0;
    if (check_link(k, s, ff, rule)) {
      first_bad = std::min(first_bad, k);
      continue;
    }
    const lbm_link& L = links[k];
    nbody = std::max(nbody, (int)L.body + 1);
    min_body = std::min(min_body, (int)L.body);
    max_body = std::max(max_body, (int)L.body);
    for (int a = 0; a < D; ++a) moving_i |= L.uw[a] != 0.0 ? 1 : 0;
    lk_s[k] = s;
    lk_ff[k] = ff;
    lk_rule[k] = rule;
    if (rule == LBM_BC_VIBB) {
#pragma omp atomic write
      mark[L.node] = 1;
#pragma omp atomic write
      mark[ff] = 1;
    }
#pragma omp atomic write
    mark[s] = 1;
    // input order: (node, dir) increasing, and equal neighbours (duplicates
    // when it is)
    if (k > 0) {
      const uint64_t a = nodedir(k - 1), b = nodedir(k);
      unsorted += a < b ? 0 : 1;
      if (a == b) first_eq = std::min(first_eq, k);
    }
  }
  if (first_bad < n_links) {
    const int64_t k = first_bad;
    const lbm_link& L = links[k];
    int64_t s = 0, ff = 0;
    int rule = 0;
    switch (check_link(k, s, ff, rule)) {
      case 1: return fail(LBM_ERR_INVALID_ARG, "link %lld: node out of range", (long long)k);
      case 2: return fail(LBM_ERR_INVALID_ARG, "link %lld: node %lld is not a fluid node", (long long)k, (long long)L.node);
      case 3: return fail(LBM_ERR_INVALID_ARG, "link %lld: dir %d out of range", (long long)k, L.dir);
      case 4: return fail(LBM_ERR_INVALID_ARG, "link %lld: q = %g not in (0,1]", (long long)k, L.q);
      case 5: return fail(LBM_ERR_INVALID_ARG, "link %lld: unknown rule %d", (long long)k, L.bc);
      case 6: return fail(LBM_ERR_INVALID_ARG, "link %lld: body %d out of range", (long long)k, L.body);
      case 7: return fail(LBM_ERR_INVALID_ARG, "link %lld: non-finite wall velocity", (long long)k);
      default:
        return fail(LBM_ERR_INVALID_ARG, "link %lld: neighbour of node %lld in direction %d is not a solid node",
                    (long long)k, (long long)L.node, L.dir);
    }
  }
  const bool moving = moving_i != 0;
#pragma omp parallel for schedule(static)
  for (int64_t n = 0; n < N; ++n)
    if (mark[n]) m[n] |= (m[n] & H_SOLID) ? H_GHOST : H_CACHE;
  // open inlet reads the moments of the first fluid column
  if (c.inlet)
    for (int64_t y = 0; y < ny; ++y)
      if ((m[nx * y] & H_OPEN) && nx > 1) {
        if (m[nx * y + 1] & (H_SOLID | H_OPEN))
          return fail(LBM_ERR_INVALID_ARG, "inlet node (0,%lld) has no fluid node at x = 1", (long long)y);
        m[nx * y + 1] |= H_CACHE;
      }
  // the outlet copies the fluid node before it
  if (c.outlet)
    for (int64_t r = 0; r < rows; ++r) {
      const int64_t xo = rwidth[r] - 1;
      if (!(m[nx * r + xo] & H_OPEN)) continue;
      if (xo < 1 || (m[nx * r + xo - 1] & (H_SOLID | H_OPEN)))
        return fail(LBM_ERR_INVALID_ARG, "outlet node (%lld, row %lld) has no fluid node before it", (long long)xo,
                    (long long)r);
    }
  // link order: (node, dir) -- usually the input order already -- then
  // stably by body; reject duplicate (node, dir)
  raw_vec<int64_t> order(n_links);
#pragma omp parallel for schedule(static)
  for (int64_t k = 0; k < n_links; ++k) order[k] = k;
  const bool sorted = unsorted == 0;
  // sorted input: a duplicate is an equal neighbour (found by the check pass)
  int64_t first_dup = sorted ? first_eq : n_links;
  if (!sorted) {
    std::vector<std::pair<uint64_t, int64_t>> tmp(n_links);
    for (int64_t k = 0; k < n_links; ++k) tmp[k] = {nodedir(k), k};
    std::sort(tmp.begin(), tmp.end());
    for (int64_t k = 0; k < n_links; ++k) order[k] = tmp[k].second;
#pragma omp parallel for schedule(static) reduction(min : first_dup)
    for (int64_t k = 1; k < n_links; ++k)
      if (nodedir(order[k]) == nodedir(order[k - 1])) first_dup = std::min(first_dup, k);
  }
  if (first_dup < n_links)
    return fail(LBM_ERR_INVALID_ARG, "duplicate link at node %lld direction %d",
                (long long)(nodedir(order[first_dup]) / 32), (int)(nodedir(order[first_dup]) % 32));
  // (node, dir) order of the fused kernel's link arrays: `order` before the
  // body sort below (ond points into whichever vector holds it)
  raw_vec<int64_t> byb;
  const int64_t* ond = order.data();
  if (min_body < max_body) {  // (one body for every link: the order stands)
    std::vector<int64_t> count(nbody + 2, 0);
    for (int64_t k = 0; k < n_links; ++k) count[links[k].body + 2]++;
    for (int b = 1; b < nbody + 2; ++b) count[b] += count[b - 1];
    byb.resize(n_links);
    for (int64_t k = 0; k < n_links; ++k) byb[count[links[order[k]].body + 1]++] = order[k];
    order.swap(byb);
    ond = byb.data();
  }
  // completeness: count (fluid node, dir) pairs with a solid neighbour, row
  // by row (each direction's neighbour row is found once per row).  A
  // neighbour outside a non-periodic face is skipped: only open columns can
  // sit there (faces are solid otherwise).
  int64_t expected = 0, n_fluid = 0;
  {
    // a row with no solid node stands for a neighbour row outside a
    // non-periodic face; nodes away from the x ends need no wrap
    raw_vec<uint8_t> open_row(nx);
    par_fill(open_row, (uint8_t)0);
    auto count_row = [&](auto stencil, int64_t r, int64_t& exp, int64_t& nf) {
      using L = decltype(stencil);
      const int64_t y = r % ny, z = r / ny;
      const uint8_t* nrow[L::Q];
      nrow[0] = nullptr;
      for (int d = 1; d < L::Q; ++d) {
        int64_t yy = y + L::cy(d), zz = z + L::cz(d);
        bool out = false;
        if (yy < 0 || yy >= ny) {
          if (!c.periodic[1]) out = true;
          yy = (yy + ny) % ny;
        }
        if (zz < 0 || zz >= nz) {
          if (!c.periodic[2]) out = true;
          zz = (zz + nz) % nz;
        }
        nrow[d] = out ? open_row.data() : m.data() + nx * (yy + ny * zz);
      }
      const uint8_t* mr = m.data() + nx * r;
      for (int64_t x = 0; x < nx; ++x) {
        if (mr[x] & (H_SOLID | H_OPEN)) continue;
        ++nf;
        if (x > 0 && x < nx - 1) {
          for (int d = 1; d < L::Q; ++d) exp += (nrow[d][x + L::cx(d)] & H_SOLID) ? 1 : 0;
        } else {
          for (int d = 1; d < L::Q; ++d) {
            int64_t xx = x + L::cx(d);
            if (xx < 0 || xx >= nx) {
              if (!c.periodic[0]) continue;
              xx = (xx + nx) % nx;
            }
            exp += (nrow[d][xx] & H_SOLID) ? 1 : 0;
          }
        }
      }
    };
    if (Q == 9) {
#pragma omp parallel for schedule(static) reduction(+ : expected, n_fluid)
      for (int64_t r = 0; r < rows; ++r) count_row(D2Q9{}, r, expected, n_fluid);
    } else {
#pragma omp parallel for schedule(static) reduction(+ : expected, n_fluid)
      for (int64_t r = 0; r < rows; ++r) count_row(D3Q19{}, r, expected, n_fluid);
    }
  }
  if (expected != n_links)
    return fail(LBM_ERR_INVALID_ARG, "%lld fluid-to-solid neighbour pairs but %lld links: every cut link needs a record",
                (long long)expected, (long long)n_links);

  // ---- compacted layout: stored = fluid, open and ghost nodes, in row order
  // storage indices in node order: per-chunk counts, prefix sums, fill
  auto stored = [&](int64_t n) { return !(m[n] & H_SOLID) || (m[n] & H_GHOST); };
  const int64_t nchunk = std::max<int64_t>(1, std::min<int64_t>(1024, N / 65536));
  std::vector<int64_t> chunk_start(nchunk + 1, 0);
#pragma omp parallel for schedule(static)
  for (int64_t ch = 0; ch < nchunk; ++ch) {
    int64_t cnt = 0;
    for (int64_t n = N * ch / nchunk; n < N * (ch + 1) / nchunk; ++n) cnt += stored(n) ? 1 : 0;
    chunk_start[ch + 1] = cnt;
  }
  for (int64_t ch = 0; ch < nchunk; ++ch) chunk_start[ch + 1] += chunk_start[ch];
  const int64_t S = chunk_start[nchunk];
  raw_vec<int32_t> sidx(N);
  par_fill(sidx, (int32_t)-1);
  raw_vec<int32_t> node_of((size_t)S);  // written for every stored node
#pragma omp parallel for schedule(static)
  for (int64_t ch = 0; ch < nchunk; ++ch) {
    int64_t k = chunk_start[ch];
    for (int64_t n = N * ch / nchunk; n < N * (ch + 1) / nchunk; ++n)
      if (stored(n)) {
        sidx[n] = (int32_t)k;
        node_of[k++] = (int32_t)n;
      }
  }
  std::vector<int32_t> row_first(rows, -1), row_last(rows, -1);
#pragma omp parallel for schedule(static)
  for (int64_t r = 0; r < rows; ++r)
    for (int64_t x = 0; x < nx; ++x) {
      const int32_t k = sidx[x + nx * r];
      if (k < 0) continue;
      if (row_first[r] < 0) row_first[r] = k;
      row_last[r] = k;
    }
  // open columns: the fluid node next to the inlet (x = 1) and to the outlet
  // (x = width - 2) of every row, -1 where there is none
  std::vector<int32_t> row_in1(rows, -1), row_out1(rows, -1);
  if (c.inlet || c.outlet)
    for (int64_t r = 0; r < rows; ++r) {
      const int64_t a = nx * r + 1, b = nx * r + rwidth[r] - 2;
      if (c.inlet && nx > 1 && !(m[a] & (H_SOLID | H_OPEN))) row_in1[r] = sidx[a];
      if (c.outlet && rwidth[r] > 1 && !(m[b] & (H_SOLID | H_OPEN))) row_out1[r] = sidx[b];
    }
  // neighbour-row slots in use: source-row offsets (dy, dz) = -(cy, cz)
  // and the range of x offsets pulled from each such row
  int nslots = 0;
  int slot_dy[8] = {0}, slot_dz[8] = {0}, slot_dxlo[8], slot_dxhi[8];
  for (int sl = 0; sl < 8; ++sl) {
    slot_dxlo[sl] = 1;
    slot_dxhi[sl] = -1;
  }
  for (int d = 1; d < Q; ++d) {
    const int dy = -cy_of(h, d), dz = -cz_of(h, d), dx = -cx_of(h, d);
    if (dy == 0 && dz == 0) continue;
    const int sl = row_slot(dy, dz);
    slot_dy[sl] = dy;
    slot_dz[sl] = dz;
    slot_dxlo[sl] = std::min(slot_dxlo[sl], dx);
    slot_dxhi[sl] = std::max(slot_dxhi[sl], dx);
    nslots = std::max(nslots, sl + 1);
  }
  // fluid runs and their neighbour-row bases, row by row in parallel: count
  // the runs of every row and check that the pulled part of each neighbour
  // row is stored and contiguous (x0 + min dx .. x_end + max dx, inside the
  // row), then fill the records with their global run ids.
  std::vector<int64_t> row_runs(rows + 1, 0);
  // walks row r; out == nullptr: count and check (returns false and the run
  // at fault on a contiguity error); else write records from run id rid0
  auto walk_row = [&](int64_t r, RunRec* out, uint32_t rid0, uint32_t* word_out, int64_t* bad) -> bool {
    const int64_t y = r % ny, z = r / ny;
    int64_t x = 0, count = 0;
    while (x < nx) {
      const int64_t n = x + nx * r;
      if (m[n] & (H_SOLID | H_OPEN)) {
        ++x;
        continue;
      }
      int64_t xe = x;
      while (xe + 1 < nx && !(m[xe + 1 + nx * r] & (H_SOLID | H_OPEN))) ++xe;
      RunRec rec{};
      rec.xk = (int32_t)(x - sidx[n]);
      rec.y = (int32_t)y;
      rec.z = (int32_t)z;
      rec.dom = rdom[r];
      for (int sl = 0; sl < nslots; ++sl) {
        const int64_t yy = (y + slot_dy[sl] + ny) % ny, zz = (z + slot_dz[sl] + nz) % nz;
        const int64_t rr = yy + ny * zz;
        const int32_t base = sidx[x + nx * rr];
        if (!out)
          for (int64_t xx = std::max<int64_t>(x + slot_dxlo[sl], 0);
               xx <= std::min<int64_t>(xe + slot_dxhi[sl], nx - 1); ++xx)
            if (base < 0 || sidx[xx + nx * rr] != base + (int32_t)(xx - x)) {
              bad[0] = x;
              bad[1] = xe;
              return false;
            }
        rec.dbase[sl] = base - sidx[n];
      }
      if (out) {
        const uint32_t rid = rid0 + (uint32_t)count;
        for (int64_t xx = x; xx <= xe; ++xx) {
          const int64_t nn = xx + nx * r;
          word_out[sidx[nn]] = rid | ((m[nn] & H_CACHE) ? W_CACHE : 0u);
        }
        out[count] = rec;
      }
      ++count;
      x = xe + 1;
    }
    if (!out) row_runs[r + 1] = count;
    return true;
  };
  int64_t bad_row = rows;
#pragma omp parallel for schedule(dynamic, 64) reduction(min : bad_row)
  for (int64_t r = 0; r < rows; ++r) {
    int64_t bad[2];
    if (!walk_row(r, nullptr, 0, nullptr, bad)) bad_row = std::min(bad_row, r);
  }
  if (bad_row < rows) {
    int64_t bad[2] = {0, 0};
    walk_row(bad_row, nullptr, 0, nullptr, bad);
    return fail(LBM_ERR_INVALID_ARG,
                "layout: neighbour row of the fluid run at (%lld..%lld, %lld, %lld) is not fully stored",
                (long long)bad[0], (long long)bad[1], (long long)(bad_row % ny), (long long)(bad_row / ny));
  }
  for (int64_t r = 0; r < rows; ++r) row_runs[r + 1] += row_runs[r];
  if (row_runs[rows] > (int64_t)W_RUN + 1) return fail(LBM_ERR_UNSUPPORTED, "too many fluid runs");
  raw_vec<RunRec> runs((size_t)row_runs[rows]);
  par_fill(runs, RunRec{});
  raw_vec<uint32_t> word(S);
  par_fill(word, 0u);
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t r = 0; r < rows; ++r) {
    int64_t bad[2];
    walk_row(r, runs.data() + row_runs[r], (uint32_t)row_runs[r], word.data(), bad);
  }
  int64_t n_cached = 0;
#pragma omp parallel for schedule(static) reduction(+ : n_cached)
  for (int64_t n = 0; n < N; ++n) {
    if (sidx[n] < 0) continue;
    if (m[n] & H_OPEN)
      word[sidx[n]] = W_OPEN;
    else if (m[n] & H_SOLID)
      word[sidx[n]] = W_GHOST;
    else
      n_cached += (m[n] & H_CACHE) ? 1 : 0;
  }
  // FP64: the fluid nodes' storage indices in order (the FP64 bulk pass
  // maps its threads onto these; per-chunk counts, prefix sums, fill)
  raw_vec<uint32_t> flist(h->rb == 8 ? (size_t)S : 0);
  int64_t nflist = 0;
  if (h->rb == 8 && S > 0) {
    const int64_t nch = std::max<int64_t>(1, std::min<int64_t>(1024, S / 65536));
    std::vector<int64_t> cs(nch + 1, 0);
#pragma omp parallel for schedule(static)
    for (int64_t ch = 0; ch < nch; ++ch) {
      int64_t cnt = 0;
      for (int64_t k = S * ch / nch; k < S * (ch + 1) / nch; ++k) cnt += (word[k] & (W_GHOST | W_OPEN)) ? 0 : 1;
      cs[ch + 1] = cnt;
    }
    for (int64_t ch = 0; ch < nch; ++ch) cs[ch + 1] += cs[ch];
    nflist = cs[nch];
#pragma omp parallel for schedule(static)
    for (int64_t ch = 0; ch < nch; ++ch) {
      int64_t j = cs[ch];
      for (int64_t k = S * ch / nch; k < S * (ch + 1) / nch; ++k)
        if (!(word[k] & (W_GHOST | W_OPEN))) flist[j++] = (uint32_t)k;
    }
  }
  // rest part of the momentum exchange per body (shifted storage):
  // sum over the body's links of 2 w_i' rho0 e_i', from the exact count of
  // its links per direction (counted in parallel, summed in a fixed order)
  std::vector<double> rest(3 * (size_t)nbody, 0.0);
  if (c.precision == LBM_FP32_SHIFTED && n_links > 0 && max_body >= 0) {
    const size_t nc = (size_t)(max_body + 1) * Q;
    std::vector<int64_t> cnt(nc, 0);
#pragma omp parallel
    {
      std::vector<int64_t> mine(nc, 0);
#pragma omp for schedule(static) nowait
      for (int64_t k = 0; k < n_links; ++k)
        if (links[k].body >= 0) ++mine[(size_t)links[k].body * Q + links[k].dir];
#pragma omp critical
      for (size_t j = 0; j < nc; ++j) cnt[j] += mine[j];
    }
    for (int b = 0; b <= max_body; ++b)
      for (int d = 1; d < Q; ++d) {
        const int64_t n = cnt[(size_t)b * Q + d];
        if (n == 0) continue;
        const double t = (double)n * 2.0 * (Q == 9 ? D2Q9::w(d) : D3Q19::w(d)) * c.rho0;
        rest[3 * b + 0] += t * cx_of(h, d);
        rest[3 * b + 1] += t * cy_of(h, d);
        rest[3 * b + 2] += t * cz_of(h, d);
      }
  }
  // link records: the split form's in `order`, the fused kernel's in
  // (node, dir) order (`ond`); with one body the two orders are the same and
  // one pass fills both
  raw_vec<LinkRec> recs(n_links);  // these three: written in full below
  raw_vec<double> qs(n_links);
  raw_vec<double> uws(moving ? (size_t)D * n_links : 0);
  const int64_t ngroups = (S + 31) / 32;
  raw_vec<int32_t> ffirst((size_t)ngroups + 1);
  raw_vec<uint32_t> fmask((size_t)S);
  par_fill(fmask, 0u);
  raw_vec<FusedRec> frec(n_links);  // written in full below
  raw_vec<double> fq(h->rb == 8 ? n_links : 0);
  raw_vec<double> fuw(moving ? (size_t)D * n_links : 0);
  const bool same_order = ond == order.data();
  auto split_rec = [&](int64_t j, int64_t k, uint32_t kf, uint32_t kff) {
    const lbm_link& L = links[k];
    recs[j].kf = kf;
    recs[j].kff = kff;
    recs[j].ks = (uint32_t)sidx[lk_s[k]];
    recs[j].meta = (uint32_t)L.dir | ((uint32_t)lk_rule[k] << 5) | ((uint32_t)(L.body + 1) << 7);
    qs[j] = L.q;
    if (moving)
      for (int a = 0; a < D; ++a) uws[a * n_links + j] = L.uw[a];
  };
#pragma omp parallel for schedule(static)
  for (int64_t j = 0; j < n_links; ++j) {
    const int64_t k = ond[j];
    const lbm_link& L = links[k];
    const uint32_t kf = (uint32_t)sidx[L.node], kff = (uint32_t)sidx[lk_ff[k]];
#pragma omp atomic update
    fmask[kf] |= 1u << L.dir;
    const float q32 = (float)L.q;
    uint32_t qbits;
    memcpy(&qbits, &q32, 4);
    frec[j] = FusedRec{kf, kff, (uint32_t)L.dir | ((uint32_t)lk_rule[k] << 5) | ((uint32_t)(L.body + 1) << 8), qbits};
    if (h->rb == 8) fq[j] = L.q;
    if (moving)
      for (int a = 0; a < D; ++a) fuw[a * n_links + j] = L.uw[a];
    if (same_order) split_rec(j, k, kf, kff);
  }
  if (!same_order) {
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < n_links; ++j) {
      const int64_t k = order[j];
      split_rec(j, k, (uint32_t)sidx[links[k].node], (uint32_t)sidx[lk_ff[k]]);
    }
  }
  // FP64: the VIBB velocity weights of each link in the link kernel's order
  // (u*_d's and u**_d's weights of Sec. 3.1 blended 1/3 : 2/3; q alone
  // fixes them)
  raw_vec<double> qcw(h->rb == 8 ? 3 * (size_t)n_links : 0);
  if (h->rb == 8) {
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < n_links; ++j) {
      const double q = links[order[j]].q, two_q = 2.0 * q;
      double af, aff, aw;
      if (q <= 0.5) {
        af = two_q;
        aff = 1.0 - two_q;
        aw = 0.0;
      } else {
        const double iq = 1.0 / q;
        af = (1.0 - q) * iq;
        aff = 0.0;
        aw = (two_q - 1.0) * iq;
      }
      const double i1q = 1.0 / (1.0 + q);
      const double bff = (1.0 - q) * i1q, bw = two_q * i1q;
      const double third = 1.0 / 3.0, two_thirds = 2.0 / 3.0;
      qcw[j] = third * af;
      qcw[n_links + j] = third * aff + two_thirds * bff;
      qcw[2 * n_links + j] = third * aw + two_thirds * bw;
    }
  }
  // first link of each 32-node group: storage indices of x_f are
  // non-decreasing along (node, dir) order, so ffirst[g] (the first j with
  // kf_j >= 32 g) is j for every g in (kf_{j-1} / 32, kf_j / 32], and n_links
  // after the last link's group
#pragma omp parallel for schedule(static)
  for (int64_t j = 0; j < n_links; ++j) {
    const int64_t g = frec[j].kf >> 5, gp = j > 0 ? (int64_t)(frec[j - 1].kf >> 5) : -1;
    for (int64_t t = gp + 1; t <= g; ++t) ffirst[t] = (int32_t)j;
  }
  {
    const int64_t glast = n_links > 0 ? (int64_t)(frec[n_links - 1].kf >> 5) : -1;
#pragma omp parallel for schedule(static)
    for (int64_t t = glast + 1; t <= ngroups; ++t) ffirst[t] = (int32_t)n_links;
  }

  // ---- device
  CUDA_TRY(cudaStreamSynchronize(h->stream));
  drop_graphs(h);
  release_geometry(h);
  h->has_geometry = h->has_state = false;
  lbm_status st = LBM_OK;
  const size_t rb = h->rb;
  for (int k = 0; k < 2 && st == LBM_OK; ++k) st = acquire(h->f[k], (size_t)Q * S * rb);
  for (int k = 0; k < 2 && st == LBM_OK; ++k) st = acquire(h->mom[k], (size_t)S * 4 * rb);
  if (st == LBM_OK) st = upload(h->word, word.data(), sizeof(uint32_t) * S);
  if (st == LBM_OK) st = upload(h->node_of, node_of.data(), sizeof(int32_t) * S);
  if (st == LBM_OK) st = upload(h->runs, runs.data(), sizeof(RunRec) * runs.size());
  if (st == LBM_OK) st = upload(h->row_first, row_first.data(), sizeof(int32_t) * rows);
  if (st == LBM_OK) st = upload(h->row_last, row_last.data(), sizeof(int32_t) * rows);
  if (st == LBM_OK) st = upload(h->row_in1, row_in1.data(), sizeof(int32_t) * rows);
  if (st == LBM_OK) st = upload(h->row_out1, row_out1.data(), sizeof(int32_t) * rows);
  if (st == LBM_OK) st = upload(h->recs, recs.data(), sizeof(LinkRec) * n_links);
  if (st == LBM_OK && n_links > 0) st = upload(h->lfirst, ffirst.data(), sizeof(int32_t) * (ngroups + 1));
  if (st == LBM_OK && n_links > 0) st = upload(h->lmask, fmask.data(), sizeof(uint32_t) * S);
  if (st == LBM_OK) st = upload(h->lrec, frec.data(), sizeof(FusedRec) * n_links);
  if (st == LBM_OK) st = upload(h->lqd, fq.data(), sizeof(double) * fq.size());
  if (st == LBM_OK && nflist > 0) st = upload(h->fidx, flist.data(), sizeof(uint32_t) * nflist);
  if (st == LBM_OK && h->rb == 8 && n_links > 0) st = upload(h->lqc, qcw.data(), sizeof(double) * 3 * n_links);
  if (st == LBM_OK && ndom > 0) {
    std::vector<DomPar> dp(ndom);
    for (int k = 0; k < ndom; ++k) {
      const lbm_domain& q = h->domains[k];
      dp[k].omega = 1.0 / q.tau;
      dp[k].fpre3 = 3.0 * (1.0 - 0.5 / q.tau);
      for (int a = 0; a < 3; ++a) dp[k].g[a] = a < D ? q.g[a] : 0.0;
      dp[k].has_force = (dp[k].g[0] != 0.0 || dp[k].g[1] != 0.0 || dp[k].g[2] != 0.0) ? 1 : 0;
      if (Q == 9)
        fold<D2Q9>(dp[k].kc, dp[k].omega, dp[k].fpre3, dp[k].g);
      else
        fold<D3Q19>(dp[k].kc, dp[k].omega, dp[k].fpre3, dp[k].g);
      dp[k].omega_f = (float)dp[k].omega;
      dp[k].fpre3_f = (float)dp[k].fpre3;
      dp[k].omega2_f = (float)(dp[k].omega * dp[k].omega);
      for (int a = 0; a < 3; ++a) {
        dp[k].g_f[a] = (float)dp[k].g[a];
        dp[k].hg_f[a] = (float)(0.5 * dp[k].g[a]);
      }
      dp[k].inlet_umax = q.inlet_umax;
      dp[k].inlet_y0 = q.inlet_y0;
      dp[k].inlet_y1 = q.inlet_y1;
      dp[k].lo = q.lo;
    }
    st = upload(h->dom, dp.data(), sizeof(DomPar) * ndom);
    if (st == LBM_OK) st = upload(h->row_dom, rdom.data(), sizeof(int32_t) * rows);
  }
  if (st == LBM_OK && h->force.bytes != sizeof(double) * 6 * (size_t)nbody) {
    st = acquire(h->force, sizeof(double) * 6 * (size_t)nbody);
    if (st == LBM_OK) {
      cudaError_t e = cudaMemsetAsync(h->force.p, 0, h->force.bytes, h->stream);
      if (e != cudaSuccess) st = fail(LBM_ERR_CUDA, "cudaMemsetAsync: %s", cudaGetErrorString(e));
    }
  }
  if (st == LBM_OK) {
    // q and u_w in storage precision, for both link orders
    auto put = [&](DeviceBuf& b, const raw_vec<double>& v) -> lbm_status {
      if (rb == 8) return upload(b, v.data(), 8 * v.size());
      raw_vec<float> t(v.size());
#pragma omp parallel for schedule(static)
      for (int64_t j = 0; j < (int64_t)v.size(); ++j) t[j] = (float)v[j];
      return upload(b, t.data(), 4 * t.size());
    };
    st = put(h->q, qs);
    if (st == LBM_OK && moving) st = put(h->uw, uws);
    if (st == LBM_OK && moving) st = put(h->luw, fuw);
  }
  for (int k = 0; k < 2 && st == LBM_OK; ++k)
    if (h->mom[k].bytes) {
      cudaError_t e = cudaMemsetAsync(h->mom[k].p, 0, h->mom[k].bytes, h->stream);
      if (e != cudaSuccess) st = fail(LBM_ERR_CUDA, "cudaMemsetAsync: %s", cudaGetErrorString(e));
    }
  if (st != LBM_OK) {
    release_geometry(h);
    return st;
  }
  h->lay.S = S;
  h->lay.word = (const uint32_t*)h->word.p;
  h->lay.node_of = (const int32_t*)h->node_of.p;
  h->lay.runs = (const RunRec*)h->runs.p;
  h->lay.row_first = (const int32_t*)h->row_first.p;
  h->lay.row_last = (const int32_t*)h->row_last.p;
  h->lay.row_in1 = (const int32_t*)h->row_in1.p;
  h->lay.row_out1 = (const int32_t*)h->row_out1.p;
  h->lay.dom = ndom > 0 ? (const DomPar*)h->dom.p : nullptr;
  h->lay.row_dom = ndom > 0 ? (const int32_t*)h->row_dom.p : nullptr;
  h->lay.ndom = std::max(ndom, 1);
  h->lay.fluid = nflist > 0 ? (const uint32_t*)h->fidx.p : nullptr;
  h->lay.nfluid = nflist;
  // a single domain runs through Params like an unsplit lattice
  Params& p = h->p;
  const lbm_domain one{0, 0, 0, 0, c.tau, {c.g[0], c.g[1], c.g[2]}, c.inlet_umax, c.inlet_y0, c.inlet_y1};
  const lbm_domain& d0 = ndom == 1 ? h->domains[0] : one;
  p.tau = d0.tau;
  p.omega = 1.0 / d0.tau;
  p.fpre3 = 3.0 * (1.0 - 0.5 / d0.tau);
  for (int a = 0; a < 3; ++a) p.g[a] = a < D ? d0.g[a] : 0.0;
  p.has_force = (p.g[0] != 0.0 || p.g[1] != 0.0 || p.g[2] != 0.0);
  if (h->Q == 9)
    fold_params<D2Q9>(p);
  else
    fold_params<D3Q19>(p);
  p.inlet_umax = d0.inlet_umax;
  p.inlet_y0 = d0.inlet_y0;
  p.inlet_y1 = d0.inlet_y1;
  h->nbody = nbody;
  h->p.nbody = nbody;
  h->sidx.swap(sidx);
  h->n_links = n_links;
  h->n_fluid = n_fluid;
  h->n_cached = n_cached;
  h->n_runs = (int64_t)runs.size();
  h->force_rest.swap(rest);
  h->link_order.swap(order);
  h->has_geometry = true;
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
  if (e == cudaSuccess && h->mom[0].bytes) e = cudaMemsetAsync(h->mom[0].p, 0, h->mom[0].bytes, h->stream);
  if (e == cudaSuccess) {
    h->ops.init(h->f[0].p, h->mom[0].p, h->lay, drho, du, h->p, h->stream);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemsetAsync(h->force.p, 0, h->force.bytes, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  cudaFree(drho);
  cudaFree(du);
  if (e != cudaSuccess) return fail(LBM_ERR_CUDA, "init: %s", cudaGetErrorString(e));
  h->cur = 0;
  h->step = 0;
  h->has_state = true;
  h->from_init = true;
  return LBM_OK;
}

lbm_status lbm_step(lbm_handle h, int64_t n) {
  g_msg[0] = 0;
  NvtxRange range("lbm_step");
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
  // graphs run an even number of steps and keep the force slot parity;
  // align first
  if (left > 0 && (h->step & 1)) {
    lbm_status st = enqueue_step(h, h->cur, h->step, false);
    if (st != LBM_OK) return st;
    h->cur ^= 1;
    ++h->step;
    --left;
  }
  const int G = h->tune.graph_steps;
  if (G > 2 && left >= G) {
    if (!h->graphG[h->cur]) {
      lbm_status st = build_graph(h, h->cur, G, &h->graphG[h->cur]);
      if (st != LBM_OK) return st;
    }
    for (; left >= G; left -= G) {
      CUDA_TRY(cudaGraphLaunch(h->graphG[h->cur], h->stream));
      h->step += G;
    }
  }
  if (left >= 2) {
    if (!h->graph[h->cur]) {
      lbm_status st = build_graph(h, h->cur, 2, &h->graph[h->cur]);
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
    CUDA_TRY(cudaMemsetAsync(rho, 0, sizeof(double) * N, h->stream));
    CUDA_TRY(cudaMemsetAsync(u, 0, sizeof(double) * h->D * N, h->stream));
    h->ops.moments(h->f[h->cur].p, h->lay, rho, u, h->p, h->stream);
    CUDA_TRY(cudaGetLastError());
    return LBM_OK;
  }
  double* tmp = nullptr;
  CUDA_TRY(cudaMalloc(&tmp, sizeof(double) * (1 + h->D) * N));
  cudaError_t e = cudaMemsetAsync(tmp, 0, sizeof(double) * (1 + h->D) * N, h->stream);
  if (e == cudaSuccess) {
    h->ops.moments(h->f[h->cur].p, h->lay, tmp, tmp + N, h->p, h->stream);
    e = cudaGetLastError();
  }
  // while the device computes
  touch_host_output(rho, sizeof(double) * N);
  touch_host_output(u, sizeof(double) * h->D * N);
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
  if (body >= h->nbody) {
    F[0] = F[1] = F[2] = 0.0;
    return LBM_OK;
  }
  const double* slot = (const double*)h->force.p + 3 * (int64_t)h->nbody * ((h->step - 1) & 1) + 3 * body;
  double* pinned = nullptr;
  lbm_status st = force_host_buffer(h, 3, &pinned);
  if (st != LBM_OK) return st;
  CUDA_TRY(cudaMemcpyAsync(pinned, slot, sizeof(double) * 3, cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(cudaStreamSynchronize(h->stream));
  for (int a = 0; a < 3; ++a) F[a] = pinned[a] + h->force_rest[3 * body + a];
  return LBM_OK;
}

lbm_status lbm_forces(lbm_handle h, int32_t n, double* F) {
  g_msg[0] = 0;
  if (!h || n < 0 || (n > 0 && !F)) return fail(LBM_ERR_INVALID_ARG, "null or negative argument");
  if (n > MAX_BODIES) return fail(LBM_ERR_INVALID_ARG, "%d bodies requested, at most %d", n, MAX_BODIES);
  if (!h->has_state || h->step == 0) return fail(LBM_ERR_STATE, "no step has run");
  const int m = std::min(n, h->nbody);
  const double* slot = (const double*)h->force.p + 3 * (int64_t)h->nbody * ((h->step - 1) & 1);
  double* pinned = nullptr;
  lbm_status st = force_host_buffer(h, 3 * (size_t)std::max(m, 1), &pinned);
  if (st != LBM_OK) return st;
  if (m > 0) CUDA_TRY(cudaMemcpyAsync(pinned, slot, sizeof(double) * 3 * m, cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(cudaStreamSynchronize(h->stream));
  for (int64_t k = 0; k < 3 * (int64_t)m; ++k) F[k] = pinned[k] + h->force_rest[k];
  for (int64_t k = 3 * (int64_t)m; k < 3 * (int64_t)n; ++k) F[k] = 0.0;
  return LBM_OK;
}

lbm_status lbm_step_forces(lbm_handle h, int64_t n, int32_t body, double* F) {
  g_msg[0] = 0;
  NvtxRange range("lbm_step_forces");
  if (!h || n < 0 || (n > 0 && !F)) return fail(LBM_ERR_INVALID_ARG, "null or negative argument");
  if (body < 0 || body >= MAX_BODIES) return fail(LBM_ERR_INVALID_ARG, "body %d out of range", body);
  if (!h->has_state) return fail(LBM_ERR_STATE, "initialise the state first");
  constexpr int64_t kChunk = 4096;
  const bool has = body < h->nbody;
  double* pinned = nullptr;
  if (n > 0) {
    lbm_status st = force_host_buffer(h, 3 * (size_t)std::min(n, kChunk), &pinned);
    if (st != LBM_OK) return st;
  }
  for (int64_t k0 = 0; k0 < n; k0 += kChunk) {
    const int64_t m = std::min(kChunk, n - k0);
    for (int64_t k = 0; k < m; ++k) {
      lbm_status st = enqueue_step(h, h->cur, h->step, h->profiling);
      if (st != LBM_OK) return st;
      h->cur ^= 1;
      ++h->step;
      // this step's slot: the next step clears the other one, the step
      // after it this one, so the copy (queued before both) reads it whole
      if (has) {
        const double* slot = (const double*)h->force.p + 3 * (int64_t)h->nbody * ((h->step - 1) & 1) + 3 * body;
        CUDA_TRY(cudaMemcpyAsync(pinned + 3 * k, slot, sizeof(double) * 3, cudaMemcpyDeviceToHost, h->stream));
      }
      if (h->profiling && h->ev_used > (1u << 16)) {
        st = harvest_events(h);
        if (st != LBM_OK) return st;
      }
    }
    CUDA_TRY(cudaStreamSynchronize(h->stream));
    for (int64_t k = 0; k < m; ++k)
      for (int a = 0; a < 3; ++a)
        F[3 * (k0 + k) + a] = has ? pinned[3 * k + a] + h->force_rest[3 * body + a] : 0.0;
  }
  return LBM_OK;
}

lbm_status lbm_get_distributions(lbm_handle h, double* f) {
  g_msg[0] = 0;
  if (!h || !f) return fail(LBM_ERR_INVALID_ARG, "null argument");
  if (!h->has_state) return fail(LBM_ERR_STATE, "no state");
  const int64_t N = h->N;
  double* tmp = nullptr;
  CUDA_TRY(cudaMalloc(&tmp, sizeof(double) * N));
  if (!is_device_pointer(f)) touch_host_output(f, sizeof(double) * h->Q * N);
  cudaError_t e = cudaSuccess;
  for (int i = 0; i < h->Q && e == cudaSuccess; ++i) {
    e = cudaMemsetAsync(tmp, 0, sizeof(double) * N, h->stream);
    if (e == cudaSuccess) {
      h->ops.get_dir(h->f[h->cur].p, h->lay, i, tmp, h->p, h->stream);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(f + (int64_t)i * N, tmp, sizeof(double) * N, cudaMemcpyDeviceToHost, h->stream);
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
      h->ops.set_dir(h->f[h->cur].p, h->lay, i, tmp, h->p, h->stream);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  }
  if (e == cudaSuccess) {
    h->ops.refresh(h->f[h->cur].p, h->lay, h->mom[h->cur].p, h->p, h->stream);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  cudaFree(tmp);
  if (e != cudaSuccess) return fail(LBM_ERR_CUDA, "set_distributions: %s", cudaGetErrorString(e));
  h->has_state = true;
  h->from_init = false;
  return LBM_OK;
}

lbm_status lbm_gather(lbm_handle h, const int64_t* nodes, int64_t n, double* out) {
  g_msg[0] = 0;
  if (!h || n < 0 || (n > 0 && (!nodes || !out))) return fail(LBM_ERR_INVALID_ARG, "null or negative argument");
  if (!h->has_state) return fail(LBM_ERR_STATE, "no state");
  std::vector<int64_t> sk(n);
  for (int64_t k = 0; k < n; ++k) {
    if (nodes[k] < 0 || nodes[k] >= h->N) return fail(LBM_ERR_INVALID_ARG, "node %lld out of range", (long long)nodes[k]);
    sk[k] = h->sidx[nodes[k]];
  }
  if (n == 0) return LBM_OK;
  int64_t* dn = nullptr;
  double* dout = nullptr;
  CUDA_TRY(cudaMalloc(&dn, sizeof(int64_t) * n));
  cudaError_t e = cudaMalloc(&dout, sizeof(double) * h->Q * n);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dn, sk.data(), sizeof(int64_t) * n, cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) {
    h->ops.gather(h->f[h->cur].p, h->lay, dn, n, dout, h->p, h->stream);
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
    h->ops.check(h->f[h->cur].p, h->lay, flag, h->p, h->stream);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hv, flag, sizeof(int), cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  cudaFree(flag);
  if (e != cudaSuccess) return fail(LBM_ERR_CUDA, "check: %s", cudaGetErrorString(e));
  if (hv) return fail(LBM_ERR_DIVERGED, "non-finite population or non-positive density at step %lld", (long long)h->step);
  return LBM_OK;
}

lbm_status lbm_adjoint_step(lbm_handle h, int32_t body, const double dJ_dF[3], int64_t n_steps,
                            int64_t checkpoint_every, double* J, double* dJ_dq, double* dJ_dtau, double seconds[3]) {
  g_msg[0] = 0;
  NvtxRange range("lbm_adjoint_step");
  if (!h || !dJ_dF || !J || !dJ_dtau || (h && h->n_links > 0 && !dJ_dq))
    return fail(LBM_ERR_INVALID_ARG, "null argument");
  if (!h->has_state) return fail(LBM_ERR_STATE, "initialise the state first");
  if (h->cfg.collision != LBM_BGK) return fail(LBM_ERR_UNSUPPORTED, "the adjoint is built for BGK collision");
  if (n_steps < 1 || checkpoint_every < 1) return fail(LBM_ERR_INVALID_ARG, "n_steps and checkpoint_every must be >= 1");
  if (body < -1 || body >= MAX_BODIES) return fail(LBM_ERR_INVALID_ARG, "body %d out of range", body);
  const bool from_init = h->from_init && h->step == 0;
  const int nb = h->nbody;
  const int ndom = std::max<int>((int)h->domains.size(), 1);
  // objective weights per body
  std::vector<double> wbody(3 * (size_t)nb, 0.0);
  if (body >= 0) {
    if (body < nb)
      for (int a = 0; a < 3; ++a) wbody[3 * body + a] = dJ_dF[a];
  } else {
    for (size_t k = 0; k < wbody.size(); ++k) wbody[k] = dJ_dF[k];
  }
  const int64_t S = h->lay.S, Q = h->Q, nl = h->n_links;
  const size_t sb = (size_t)Q * S * h->rb;  // bytes of one state
  const int64_t K = std::min(checkpoint_every, n_steps);
  const int64_t nck = (n_steps + K - 1) / K;
  DeviceBuf ck, seg, lam[2], dq, scr;
  lbm_status st = acquire(ck, sb * nck);
  if (st == LBM_OK) st = acquire(seg, sb * K);
  if (st == LBM_OK) st = acquire(lam[0], sb);
  if (st == LBM_OK) st = acquire(lam[1], sb);
  if (st == LBM_OK) st = acquire(dq, sizeof(double) * std::max<int64_t>(nl, 1));
  if (st == LBM_OK) st = acquire(scr, sizeof(double) * (ndom + 9 * (size_t)nb));
  auto cleanup = [&]() {
    release(ck);
    release(seg);
    release(lam[0]);
    release(lam[1]);
    release(dq);
    release(scr);
  };
  if (st != LBM_OK) {
    cleanup();
    return st;
  }
  char* ckp = (char*)ck.p;
  char* segp = (char*)seg.p;
  double* dtau = (double*)scr.p;       // [ndom]
  double* fslot = dtau + ndom;         // scratch force slots of the recomputed steps, [2][nb][3]
  double* wdev = fslot + 6 * (size_t)nb;  // objective weights [nb][3]
  cudaEvent_t ev[2];
  cudaEventCreate(&ev[0]);
  cudaEventCreate(&ev[1]);
  double t_fwd = 0.0, t_rec = 0.0, t_adj = 0.0;
  auto timed = [&](double& acc, auto&& work) -> lbm_status {
    cudaEventRecord(ev[0], h->stream);
    lbm_status r = work();
    cudaEventRecord(ev[1], h->stream);
    cudaEventSynchronize(ev[1]);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ev[0], ev[1]);
    acc += ms * 1e-3;
    return r;
  };
  cudaError_t e = cudaMemsetAsync(dq.p, 0, dq.bytes, h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(scr.p, 0, scr.bytes, h->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(wdev, wbody.data(), sizeof(double) * wbody.size(), cudaMemcpyHostToDevice, h->stream);
  if (e != cudaSuccess) st = fail(LBM_ERR_CUDA, "adjoint set-up: %s", cudaGetErrorString(e));
  // forward with checkpoints
  if (st == LBM_OK)
    st = timed(t_fwd, [&]() -> lbm_status {
      for (int64_t c = 0; c < nck; ++c) {
        CUDA_TRY(cudaMemcpyAsync(ckp + sb * c, h->f[h->cur].p, sb, cudaMemcpyDeviceToDevice, h->stream));
        const lbm_status r = lbm_step(h, std::min(K, n_steps - c * K));
        if (r != LBM_OK) return r;
      }
      return LBM_OK;
    });
  std::vector<double> F(3 * (size_t)nb, 0.0);
  if (st == LBM_OK) st = lbm_forces(h, nb, F.data());
  if (st == LBM_OK) {
    double Jv = 0.0;
    for (size_t k = 0; k < F.size(); ++k) Jv += wbody[k] * F[k];
    *J = Jv;
  }
  // backward: lambda(n) = 0 in both buffers; every adjoint step leaves the
  // buffer it read zero again
  int la = 0;
  if (st == LBM_OK) {
    e = cudaMemsetAsync(lam[0].p, 0, sb, h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(lam[1].p, 0, sb, h->stream);
    if (e != cudaSuccess) st = fail(LBM_ERR_CUDA, "adjoint: %s", cudaGetErrorString(e));
  }
  const bool open = h->p.inlet || h->p.outlet;
  // moment cache of the recomputed and transposed states: the cache of the
  // buffer that does not hold the current state (the current state and its
  // moments stay as they are)
  void* am = h->mom[h->cur ^ 1].p;
  // the states f+(s0) .. f+(s0 + m - 1) of a segment from its first state
  // (copied into seg[0]); the link and open kernels leave the link values
  // of step s0 + j in the ghost slots of seg[j] for j < m - 1
  auto enqueue_recompute = [&](int64_t m) -> lbm_status {
    h->ops.refresh(segp, h->lay, am, h->p, h->stream);
    for (int64_t j = 0; j + 1 < m; ++j) {
      const lbm_status r = enqueue_step_buf(h, segp + sb * j, segp + sb * (j + 1), am, am, fslot,
                                            fslot + 3 * (size_t)nb, false, false);
      if (r != LBM_OK) return r;
    }
    CUDA_TRY(cudaGetLastError());
    return LBM_OK;
  };
  // the transposed steps s0 + m - 1 .. s0 of a segment; lambda(s0 + m) in
  // lam[l0]; `last`: the segment ends with the objective's step
  auto enqueue_adjoint = [&](int64_t m, int l0, bool last) -> lbm_status {
    int l = l0;
    for (int64_t j = m - 1; j >= 0; --j) {
      void* state = segp + sb * j;
      if (j == m - 1) {
        // the last state of the segment has no link values yet; the moment
        // cache holds the moments the recompute's last step wrote for it,
        // those its forward step used (a one-state segment: the refresh of
        // the recompute)
        h->ops.links(state, am, (const LinkRec*)h->recs.p, h->q.p, h->uw.p, h->lqc.p, nl, fslot, h->p, S,
                     h->tune.link_threads, h->tune.link_seq, h->stream);
        if (open) h->ops.open(state, am, h->lay, h->p, h->stream);
      }
      h->adj.bulk(state, lam[l].p, lam[l ^ 1].p, h->lay, h->p, dtau, am, h->stream);
      if (open)
        h->adj.links_open(state, am, lam[l ^ 1].p, lam[l].p, (const LinkRec*)h->recs.p, h->q.p, h->uw.p, nl, h->p, S,
                          (double*)dq.p, (last && j == m - 1) ? 1 : 0, wdev, h->lay, h->stream);
      else
        h->adj.links(state, am, lam[l ^ 1].p, lam[l].p, (const LinkRec*)h->recs.p, h->q.p, h->uw.p, nl, h->p, S,
                     (double*)dq.p, (last && j == m - 1) ? 1 : 0, wdev, h->stream);
      l ^= 1;
    }
    CUDA_TRY(cudaGetLastError());
    return LBM_OK;
  };
  // segments other than the last replay captured graphs (keyed by length
  // and the lambda buffer they start from)
  struct SegGraph {
    int kind;
    int64_t m;
    int l0;
    cudaGraphExec_t g;
  };
  std::vector<SegGraph> seg_graphs;
  auto replay = [&](int kind, int64_t m, int l0, auto&& enqueue) -> lbm_status {
    for (const SegGraph& sg : seg_graphs)
      if (sg.kind == kind && sg.m == m && sg.l0 == l0) {
        CUDA_TRY(cudaGraphLaunch(sg.g, h->stream));
        return LBM_OK;
      }
    cudaGraph_t g = nullptr;
    CUDA_TRY(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
    const lbm_status r = enqueue();
    const cudaError_t ec = cudaStreamEndCapture(h->stream, &g);
    if (r != LBM_OK) {
      if (g) cudaGraphDestroy(g);
      return r;
    }
    if (ec != cudaSuccess) return fail(LBM_ERR_CUDA, "adjoint capture: %s", cudaGetErrorString(ec));
    cudaGraphExec_t x = nullptr;
    const cudaError_t ei = cudaGraphInstantiate(&x, g, 0);
    cudaGraphDestroy(g);
    if (ei != cudaSuccess) return fail(LBM_ERR_CUDA, "adjoint graph: %s", cudaGetErrorString(ei));
    seg_graphs.push_back(SegGraph{kind, m, l0, x});
    CUDA_TRY(cudaGraphLaunch(x, h->stream));
    return LBM_OK;
  };
  for (int64_t c = nck - 1; c >= 0 && st == LBM_OK; --c) {
    const int64_t s0 = c * K, m = std::min(K, n_steps - s0);
    const bool last = c == nck - 1;
    NvtxRange seg_range("adjoint segment");
    st = timed(t_rec, [&]() -> lbm_status {
      CUDA_TRY(cudaMemcpyAsync(segp, ckp + sb * c, sb, cudaMemcpyDeviceToDevice, h->stream));
      if (last) return enqueue_recompute(m);
      return replay(0, m, 0, [&] { return enqueue_recompute(m); });
    });
    if (st != LBM_OK) break;
    const int l0 = la;
    st = timed(t_adj, [&]() -> lbm_status {
      if (last) return enqueue_adjoint(m, l0, true);
      return replay(1, m, l0, [&] { return enqueue_adjoint(m, l0, false); });
    });
    if (m & 1) la ^= 1;
  }
  for (const SegGraph& sg : seg_graphs) cudaGraphExecDestroy(sg.g);
  if (st == LBM_OK && from_init) h->adj.init(ckp, lam[la].p, h->lay, h->p, dtau, h->stream);
  // results
  std::vector<double> dqh(std::max<int64_t>(nl, 1));
  std::vector<double> dt(ndom, 0.0);
  if (st == LBM_OK) {
    e = cudaMemcpyAsync(dqh.data(), dq.p, sizeof(double) * nl, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dt.data(), dtau, sizeof(double) * ndom, cudaMemcpyDeviceToHost, h->stream);
    // leave the moment cache consistent with the final state
    h->ops.refresh(h->f[h->cur].p, h->lay, h->mom[h->cur].p, h->p, h->stream);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) st = fail(LBM_ERR_CUDA, "adjoint: %s", cudaGetErrorString(e));
  }
  if (st == LBM_OK) {
    for (int64_t j = 0; j < nl; ++j) dJ_dq[h->link_order[j]] = dqh[j];
    for (int k = 0; k < ndom; ++k) dJ_dtau[k] = dt[k];
    if (seconds) {
      seconds[0] = t_fwd;
      seconds[1] = t_rec;
      seconds[2] = t_adj;
    }
  }
  cudaEventDestroy(ev[0]);
  cudaEventDestroy(ev[1]);
  cleanup();
  return st;
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
  info->device_bytes = device_bytes(h);
  info->Q = h->Q;
  info->D = h->D;
  info->precision = h->cfg.precision;
  info->real_bytes = (int32_t)h->rb;
  info->n_stored = h->lay.S;
  info->n_runs = h->n_runs;
  info->n_bodies = h->nbody;
  info->n_domains = std::max<int32_t>((int32_t)h->domains.size(), 1);
  return LBM_OK;
}

lbm_status lbm_set_tuning(lbm_handle h, const lbm_tuning* t) {
  g_msg[0] = 0;
  if (!h || !t) return fail(LBM_ERR_INVALID_ARG, "null argument");
  lbm_tuning v = *t;
  if (v.bulk_shape == -1) v.bulk_shape = h->ops.default_shape;
  if (v.bulk_shape < 0 || v.bulk_shape >= kNumBulkShapes || !((h->ops.shape_mask >> v.bulk_shape) & 1u))
    return fail(LBM_ERR_INVALID_ARG, "bulk_shape %d is not built for this stencil", t->bulk_shape);
  if (v.link_threads != 64 && v.link_threads != 128 && v.link_threads != 256)
    return fail(LBM_ERR_INVALID_ARG, "link_threads must be 64, 128 or 256");
  if (v.graph_steps < 2 || v.graph_steps > 64 || (v.graph_steps & 1))
    return fail(LBM_ERR_INVALID_ARG, "graph_steps must be even and in 2..64");
  if (v.link_seq == 0) v.link_seq = 1;
  if (v.link_seq != 1 && v.link_seq != 4) return fail(LBM_ERR_INVALID_ARG, "link_seq must be 1 or 4");
  if (v.fused != 0 && v.fused != 1) return fail(LBM_ERR_INVALID_ARG, "fused must be 0 or 1");
  if (v.bulk_shape != h->tune.bulk_shape || v.link_threads != h->tune.link_threads ||
      v.graph_steps != h->tune.graph_steps || v.link_seq != h->tune.link_seq || v.fused != h->tune.fused) {
    CUDA_TRY(cudaStreamSynchronize(h->stream));
    drop_graphs(h);
  }
  h->tune = v;
  return LBM_OK;
}

lbm_status lbm_get_tuning(lbm_handle h, lbm_tuning* t) {
  g_msg[0] = 0;
  if (!h || !t) return fail(LBM_ERR_INVALID_ARG, "null argument");
  *t = h->tune;
  return LBM_OK;
}

lbm_status lbm_autotune(lbm_handle h, int32_t steps_per_trial, lbm_tuning* best, double* ms_per_step) {
  g_msg[0] = 0;
  NvtxRange range("lbm_autotune");
  if (!h) return fail(LBM_ERR_INVALID_ARG, "null handle");
  if (steps_per_trial < 2) return fail(LBM_ERR_INVALID_ARG, "steps_per_trial must be >= 2");
  if (!h->has_state) return fail(LBM_ERR_STATE, "initialise the state first");
  if (h->profiling) return fail(LBM_ERR_STATE, "switch profiling off first");
  const size_t sb = (size_t)h->Q * h->lay.S * h->rb;
  DeviceBuf save_f, save_m, save_force;
  lbm_status st = acquire(save_f, sb);
  if (st == LBM_OK) st = acquire(save_m, h->mom[0].bytes);
  if (st == LBM_OK) st = acquire(save_force, h->force.bytes);
  auto cleanup = [&]() {
    release(save_f);
    release(save_m);
    release(save_force);
  };
  if (st != LBM_OK) {
    cleanup();
    return st;
  }
  const int cur0 = h->cur;
  const int64_t step0 = h->step;
  const bool from_init0 = h->from_init;
  const lbm_tuning tune0 = h->tune;
  auto copy = [&](void* dst, const void* src, size_t n) -> cudaError_t {
    return n ? cudaMemcpyAsync(dst, src, n, cudaMemcpyDeviceToDevice, h->stream) : cudaSuccess;
  };
  cudaError_t e = copy(save_f.p, h->f[cur0].p, sb);
  if (e == cudaSuccess) e = copy(save_m.p, h->mom[cur0].p, h->mom[cur0].bytes);
  if (e == cudaSuccess) e = copy(save_force.p, h->force.p, h->force.bytes);
  if (e != cudaSuccess) {
    cleanup();
    return fail(LBM_ERR_CUDA, "autotune: %s", cudaGetErrorString(e));
  }
  // the trials start from the saved state at an even step count, so that
  // the warm-up builds every graph the timed replays use
  auto restore = [&](int64_t step) -> cudaError_t {
    cudaError_t r = copy(h->f[cur0].p, save_f.p, sb);
    if (r == cudaSuccess) r = copy(h->mom[cur0].p, save_m.p, h->mom[cur0].bytes);
    if (r == cudaSuccess) r = copy(h->force.p, save_force.p, h->force.bytes);
    h->cur = cur0;
    h->step = step;
    h->from_init = from_init0;
    return r;
  };
  cudaEvent_t ev[2];
  CUDA_TRY(cudaEventCreate(&ev[0]));
  CUDA_TRY(cudaEventCreate(&ev[1]));
  auto trial = [&](const lbm_tuning& t, double* ms) -> lbm_status {
    lbm_status r = lbm_set_tuning(h, &t);
    if (r != LBM_OK) return r;
    double bestms = 1e300;
    for (int rep = 0; rep < 2; ++rep) {
      CUDA_TRY(restore(0));
      r = lbm_step(h, t.graph_steps + 2);
      if (r != LBM_OK) return r;
      CUDA_TRY(cudaEventRecord(ev[0], h->stream));
      r = lbm_step(h, steps_per_trial);
      if (r != LBM_OK) return r;
      CUDA_TRY(cudaEventRecord(ev[1], h->stream));
      CUDA_TRY(cudaEventSynchronize(ev[1]));
      float f_ms = 0.f;
      CUDA_TRY(cudaEventElapsedTime(&f_ms, ev[0], ev[1]));
      bestms = std::min(bestms, (double)f_ms / steps_per_trial);
    }
    *ms = bestms;
    return LBM_OK;
  };
  // split pass (link kernel, then bulk kernel) first, then the fused step
  // with the block sizes of the one-node bulk shapes
  lbm_tuning cand{h->ops.default_shape, 256, 8, 1, 0}, chosen = cand;
  double chosen_ms = 1e300;
  auto consider = [&](const lbm_tuning& t) -> lbm_status {
    double ms = 0.0;
    const lbm_status r = trial(t, &ms);
    if (r == LBM_OK && ms < chosen_ms) {
      chosen_ms = ms;
      chosen = t;
    }
    return r;
  };
  for (int sh = 0; sh < kNumBulkShapes && st == LBM_OK; ++sh) {
    if (!((h->ops.shape_mask >> sh) & 1u)) continue;
    cand.bulk_shape = sh;
    st = consider(cand);
  }
  const int link_opts[] = {64, 128};
  for (int k = 0; k < 2 && st == LBM_OK; ++k) {
    cand = chosen;
    cand.link_threads = link_opts[k];
    st = consider(cand);
  }
  if (st == LBM_OK) {
    cand = chosen;
    cand.link_seq = 4;
    st = consider(cand);
  }
  if (h->n_links > 0)
    for (int sh = 0; sh < kNumBulkShapes && st == LBM_OK; ++sh) {
      if (!((h->ops.shape_mask >> sh) & 1u) || kBulkShapes[sh].npt != 1 || kBulkShapes[sh].seq != 1) continue;
      cand = chosen;
      cand.fused = 1;
      cand.bulk_shape = sh;
      st = consider(cand);
    }
  const int graph_opts[] = {2, 32};
  for (int k = 0; k < 2 && st == LBM_OK; ++k) {
    cand = chosen;
    cand.graph_steps = graph_opts[k];
    st = consider(cand);
  }
  // put the state back and keep the fastest shapes
  if (st == LBM_OK) {
    e = restore(step0);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) st = fail(LBM_ERR_CUDA, "autotune: %s", cudaGetErrorString(e));
  } else {
    char keep[sizeof g_msg];
    memcpy(keep, g_msg, sizeof keep);
    restore(step0);
    cudaStreamSynchronize(h->stream);
    memcpy(g_msg, keep, sizeof keep);
  }
  const lbm_status st2 = lbm_set_tuning(h, st == LBM_OK ? &chosen : &tune0);
  if (st == LBM_OK) st = st2;
  if (st == LBM_OK) {
    if (best) *best = chosen;
    if (ms_per_step) *ms_per_step = chosen_ms;
  }
  cudaEventDestroy(ev[0]);
  cudaEventDestroy(ev[1]);
  cleanup();
  return st;
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
