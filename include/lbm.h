/* lbm.h -- C ABI of liblbm.so: the lattice-Boltzmann time step with the
 * velocity-interpolation bounce-back (VIBB) boundary of Jin et al.,
 * "Velocity interpolation based Bounce-Back scheme for non-slip boundary
 * condition in Lattice Boltzmann Method", arXiv:1903.01111, on NVIDIA GB300
 * (sm_103a).  Half-way and Bouzidi bounce-back are provided as the paper's
 * comparison rules.
 *
 * Conventions (all entry points):
 *  - Every call returns an lbm_status; no C++ exception or abort crosses the
 *    ABI.  On failure lbm_last_error() gives a message (thread-local).
 *  - Node index n = x + nx*(y + ny*z); node x sits at integer coordinates.
 *  - Velocity sets: D2Q9 in the order of the moment matrix M of Sec. 2:
 *    e0=(0,0) e1=(1,0) e2=(0,1) e3=(-1,0) e4=(0,-1) e5=(1,1) e6=(-1,1)
 *    e7=(-1,-1) e8=(1,-1); weights 4/9, 1/9, 1/36.  D3Q19 (not in the
 *    paper): e0=0, e1..e6 = +x,-x,+y,-y,+z,-z, e7..e18 = (1,1,0),(-1,-1,0),
 *    (1,-1,0),(-1,1,0),(1,0,1),(-1,0,-1),(1,0,-1),(-1,0,1),(0,1,1),
 *    (0,-1,-1),(0,1,-1),(0,-1,1); weights 1/3, 1/18, 1/36.
 *  - Population arrays exchanged with the caller are FP64, laid out [Q][N],
 *    and hold the post-collision populations f+_i(x, t) (the state between
 *    two steps).  Inside, the library stores FP64 or FP32 "shifted"
 *    populations f_i - w_i rho0 (LBM_FP32_SHIFTED).
 *  - Host pointers are read or written before the call returns unless said
 *    otherwise; the library never keeps caller pointers.  Device memory for
 *    the state is owned by the library.
 *  - Work is ordered on the lattice's CUDA stream (lbm_config.cuda_stream,
 *    or a stream the library creates).  Calls that return data to the host
 *    synchronise that stream.
 *  - lbm_set_geometry, lbm_step, lbm_adjoint_step (and each of its
 *    checkpoint segments) and lbm_autotune mark their host-side span with an
 *    NVTX range of the same name, for timeline profilers.
 */
#ifndef LBM_H
#define LBM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  LBM_OK = 0,
  LBM_ERR_INVALID_ARG = 1,  /* a bad argument; nothing was changed */
  LBM_ERR_STATE = 2,        /* call not valid in the handle's state */
  LBM_ERR_CUDA = 3,         /* a CUDA runtime error (message has the detail) */
  LBM_ERR_OOM = 4,          /* device or host allocation failed */
  LBM_ERR_DIVERGED = 5,     /* non-finite population or non-positive density */
  LBM_ERR_TIMEOUT = 6,      /* reserved for bounded device waits */
  LBM_ERR_UNSUPPORTED = 7   /* valid request the library does not implement */
} lbm_status;

enum { LBM_D2Q9 = 0, LBM_D3Q19 = 1 };
enum { LBM_BGK = 0, LBM_MRT = 1 };
enum { LBM_BC_DEFAULT = -1, LBM_BC_HALFWAY = 0, LBM_BC_BOUZIDI = 1, LBM_BC_VIBB = 2, LBM_BC_YU = 3 };
enum { LBM_FP64 = 0, LBM_FP32_SHIFTED = 1 };
enum { LBM_VIBB_RHO_PRINTED = 0, LBM_VIBB_RHO_LOCAL = 1 };

#define LBM_MAX_BODIES 32768

typedef struct lbm_lattice_s* lbm_handle;

/* Run configuration.
 *  stencil    LBM_D2Q9 (nz must be 1) or LBM_D3Q19.
 *  collision  LBM_BGK: f+ = f - (f - feq)/tau + F_i, feq of Sec. 2
 *             Eq. (feq) with C = 1, tau = 3 nu + 1/2 (Sec. 2).  The body
 *             force g enters by Guo forcing (velocity u = (sum f e + g/2)/rho,
 *             source (1 - 1/(2 tau)) w_i [3 (e_i - u) + 9 (e_i.u) e_i].g);
 *             the paper names a constant body force (Sec. 4.1) but no scheme.
 *             LBM_MRT (Sec. 2, Eq. mrt), D2Q9 only (D3Q19: LBM_ERR_UNSUPPORTED):
 *             relaxation of f - feq in the moment basis M with rates s = 0.3
 *             (moments 0, 3, 5), 1.5 (1, 2), 1.2 (4, 6), 1/tau (7, 8), and
 *             the Guo source projected with (1 - s_k/2) per moment.
 *  bc         default link rule for links whose own rule is LBM_BC_DEFAULT:
 *             LBM_BC_HALFWAY (bounce-back, Sec. 3), LBM_BC_BOUZIDI (Eqs.
 *             q_less, q_larger), LBM_BC_VIBB (Sec. 3.1) or LBM_BC_YU (Yu's
 *             unified interpolation, Sec. 3: the wall value
 *             q f+_i'(x_f) + (1 - q) f+_i'(x_ff) + 6 w rho0 (e_i.u_w), then
 *             f_i(x_f, t+1) = (wall value)/(1 + q) + q/(1 + q) f+_i(x_f, t),
 *             reading the unbalanced parenthesis of the second equation as
 *             closing after f_i(x_w, t+1) and f_i(x_ff, t+1) = f+_i(x_f, t)
 *             by streaming).
 *  nx,ny,nz   lattice size; N = nx*ny*nz nodes.
 *  periodic   per axis, 1 = periodic.  On a non-periodic axis every node of
 *             the two end faces must be solid (or an open column, below).
 *  inlet      D2Q9 only: column x = 0 (its non-solid nodes) is a velocity
 *             inlet by non-equilibrium extrapolation (Sec. 4.3):
 *             f+(0,y) = feq(rho(1,y), u_in(y)) + f+(1,y) - feq(rho(1,y), u(1,y)),
 *             u_in(y) = 4 inlet_umax (y - inlet_y0)(inlet_y1 - y)/(inlet_y1 - inlet_y0)^2.
 *  outlet     D2Q9 only: column x = nx-1 copies every population of column
 *             x = nx-2 (zero gradient, Sec. 4.3).
 *  tau, rho0  relaxation time (> 1/2) and reference density (the rho0 of
 *             the moving-wall term 6 w rho0 (e_i.u_w), Eqs. q_less/q_larger).
 *  g          body force per unit volume.
 *  precision  LBM_FP64 or LBM_FP32_SHIFTED.
 *  vibb_density  LBM_VIBB_RHO_PRINTED: rho_d = 2q rho_f + (1 - 2q) rho_ff for
 *             every q (Sec. 3.1, Eq. rhod; an extrapolation when q > 1/2).
 *             LBM_VIBB_RHO_LOCAL: rho_d = rho_f when q > 1/2 (the O(Ma^2)
 *             density approximation rho_s = rho_f that Sec. 3.1 quotes from
 *             the non-equilibrium extrapolation scheme).  The printed form
 *             drains mass at dead-end pore nodes of 3-D porous media and
 *             diverges there; the local form does not.
 *  cuda_stream a cudaStream_t to order all work on, or NULL for a stream the
 *             library creates and destroys. */
typedef struct {
  int32_t stencil;
  int32_t collision;
  int32_t bc;
  int32_t nx, ny, nz;
  int32_t periodic[3];
  int32_t inlet, outlet;
  double tau, rho0;
  double g[3];
  double inlet_umax, inlet_y0, inlet_y1;
  int32_t precision;
  int32_t vibb_density;
  void* cuda_stream;
} lbm_config;

/* One cut link (Sec. 3, Fig. 1): fluid node x_f = node whose neighbour
 * x_s = x_f + e_dir is solid.  dir is i' (pointing from the fluid into the
 * wall); the rule rebuilds f_i(x_f, t+1) with i = opp(i').
 *  q     |x_f - x_w| / |x_f - x_s| in (0, 1] (Sec. 3).
 *  uw    wall velocity at x_w (only the first D entries are used).
 *  bc    LBM_BC_* for this link or LBM_BC_DEFAULT.
 *  body  force accumulator 0..LBM_MAX_BODIES-1 that this link's momentum
 *        exchange adds to, or -1. */
typedef struct {
  int64_t node;
  int32_t dir;
  int16_t bc;
  int16_t body;
  double q;
  double uw[3];
} lbm_link;

/* Counters of a lattice (lbm_query). */
typedef struct {
  int64_t n_nodes, n_fluid, n_links, n_cached, step;
  int64_t device_bytes;  /* device memory the lattice holds */
  int32_t Q, D, precision, real_bytes;
  int64_t n_stored;      /* nodes with storage: fluid, open-column and ghost nodes */
  int64_t n_runs;        /* runs of consecutive fluid nodes along x */
  int32_t n_bodies;      /* force accumulators: largest link body + 1 (at least 1) */
  int32_t n_domains;     /* domains of a batch (1 without lbm_set_domains) */
} lbm_info;

/* One domain of a batch: an independent flow occupying the rows [lo, lo+n)
 * of the last axis (y for D2Q9, z for D3Q19) and the columns x < nx.  The
 * paper simulates one flow at a time; a batch packs many small ones (each
 * its own geometry, tau, body force and inlet profile) into one lattice so
 * that one launch per kernel advances them all.
 *  lo, n      rows of the domain; the domains tile the axis in order.
 *  nx         width: every node with x >= nx in these rows is solid, and the
 *             outlet column (cfg.outlet) is x = nx - 1.
 *  tau, g     relaxation time and body force of the domain (cfg.tau and cfg.g
 *             are not used when domains are set).
 *  inlet_*    inlet profile of the domain (cfg.inlet), with y counted from
 *             row lo: u_in(y) = 4 umax (y - y0)(y1 - y)/(y1 - y0)^2. */
typedef struct {
  int32_t lo, n, nx, reserved;
  double tau;
  double g[3];
  double inlet_umax, inlet_y0, inlet_y1;
} lbm_domain;

/* Launch shapes of the step (lbm_set_tuning, lbm_autotune).
 *  bulk_shape     0..7: (threads per block, nodes per thread) of the bulk
 *                 kernel = (256,1) (128,1) (512,1) (256,2) (128,2) (512,2),
 *                 then (128,1) with each thread walking 4 or 8 nodes in
 *                 sequence over the grid, the next node's addressing loaded
 *                 while the current node's pulls are in flight;
 *                 3..7 are D2Q9 only.  -1 on input: the stencil's default,
 *                 3 for D2Q9 and 1 for D3Q19 (the shape a new lattice has).
 *  link_threads   64, 128 or 256 threads per block of the link kernel.
 *  graph_steps    time steps per CUDA graph replayed by lbm_step (even,
 *                 2..64).
 *  link_seq       links per thread of the link kernel, 1 or 4 (a block
 *                 takes link_seq rounds of consecutive links, loading the
 *                 next round's record while it evaluates the current one);
 *                 0 on input means 1.
 *  fused          1 (the default): a lattice with cut links runs each step
 *                 as one kernel: a block stages its nodes' pulls in shared
 *                 memory, evaluates the link rules of its nodes into the
 *                 staged slots of the link directions and collides from
 *                 there (the link values never go through device memory);
 *                 the bulk shape then only gives its threads per block (256
 *                 for the shapes with two or sequential nodes per thread).
 *                 0: a link kernel writes each link's value into the ghost
 *                 slot of its solid neighbour and the bulk kernel pulls it
 *                 (the adjoint's recompute always takes this form).  Both
 *                 give the same populations up to rounding.
 * Shapes of the same kernel (same nodes per thread in parallel and in
 * sequence, same links per thread) give the same bits (force sums may differ
 * in the last place, as FP64 atomics are unordered); different kernels are
 * separate compilations of the same arithmetic and agree to rounding. */
typedef struct {
  int32_t bulk_shape, link_threads, graph_steps, link_seq;
  int32_t fused;
} lbm_tuning;

/* Create a lattice: validates cfg, allocates the device state (two
 * population buffers, the moment cache, the node mask, two force slots).
 * *out receives the handle.  Errors: INVALID_ARG, UNSUPPORTED, OOM, CUDA. */
lbm_status lbm_create_lattice(const lbm_config* cfg, lbm_handle* out);

/* Free a lattice and everything it owns (synchronises its stream). */
lbm_status lbm_destroy(lbm_handle h);

/* Split the lattice into n independent domains (lbm_domain); call before
 * lbm_set_geometry.  lbm_set_geometry then also checks that the first and
 * last row of every domain hold no fluid or open node (so no population
 * crosses between domains) and that nodes beyond a domain's width are
 * solid.  A periodic x axis needs every nx equal to cfg.nx.  n = 0 returns to
 * one domain run by cfg.  d: host array, copied.
 * Errors: INVALID_ARG (names the first bad domain), STATE (geometry set). */
lbm_status lbm_set_domains(lbm_handle h, const lbm_domain* d, int32_t n);

/* Node classification and cut links (Sec. 3: fluid, solid and boundary
 * nodes; missing populations are those that would stream from solid
 * nodes).  solid: N bytes on the host, nonzero = solid.  links: n_links
 * records on the host.  Everything is copied and checked: node in range and
 * fluid, dir in 1..Q-1, q in (0,1], x_s solid and inside the lattice on
 * non-periodic axes, bc and body in range, no duplicate (node, dir), and
 * every fluid node with a solid neighbour in direction i' has a link; with
 * open columns (Sec. 4.3), the nodes next to an open inlet (x = 1) and
 * before an open outlet (x = width - 2) are fluid nodes.  The second fluid
 * node x_ff = x_f - e_i' of a link falls back to x_f when it is not a fluid
 * node (narrow gaps).  Invalidates the state: call
 * lbm_init_equilibrium or lbm_set_distributions next.
 * Errors: INVALID_ARG (message names the first bad item), OOM, CUDA. */
lbm_status lbm_set_geometry(lbm_handle h, const uint8_t* solid, const lbm_link* links, int64_t n_links);

/* Initial state: f(x,0) = feq(rho(x), u(x)) (Sec. 2, Eq. feq) at every fluid
 * node, then the collision at t = 0, so that the state holds f+(x,0).
 * rho: N doubles or NULL (rho0); u: N x 3 doubles (x,y,z interleaved) or
 * NULL (rest).  Host pointers.  Resets the step counter to 0.
 * Errors: STATE (no geometry), OOM, CUDA. */
lbm_status lbm_init_equilibrium(lbm_handle h, const double* rho, const double* u);

/* Advance n >= 0 time steps, asynchronously on the lattice's stream.  Each
 * step: link rules at every cut link (half-way; Bouzidi Eqs. q_less and
 * q_larger; VIBB Sec. 3.1), open columns (Sec. 4.3), pull streaming (Eq. 1)
 * with moments and collision (Sec. 2).  Errors: STATE, CUDA. */
lbm_status lbm_step(lbm_handle h, int64_t n);

/* Macroscopic fields of the current state (Sec. 2 density and velocity
 * sums): rho = sum_i f+_i, u = (sum_i f+_i e_i - g/2)/rho, which equals the
 * velocity the last collision used.  rho: N doubles, u: D x N doubles
 * ([component][node]); both host or both device pointers (detected); solid
 * and open-column nodes get 0.  Host outputs synchronise the stream (their
 * pages are first written in parallel on the host cores, while the device
 * computes, so that a fresh allocation's page faults do not serialise the copy).
 * Errors: STATE, INVALID_ARG, OOM, CUDA. */
lbm_status lbm_moments(lbm_handle h, double* rho, double* u);

/* Force on body `body` during the last step by momentum exchange,
 * F = sum over its links of (f+_i'(x_f,t) + f_i(x_f,t+1)) e_i', summed in
 * FP64 (the paper uses the lift force in Sec. 4.3 but does not say how it
 * is computed; momentum exchange is the method of the moving-wall term it
 * cites).  F: 3 doubles on the host (z = 0 in 2-D).  Synchronises.
 * Errors: STATE, INVALID_ARG, CUDA. */
lbm_status lbm_force(lbm_handle h, int32_t body, double F[3]);

/* Forces on bodies 0..n-1 as lbm_force, in one copy: F[b*3 + a] (host);
 * bodies without links give 0.  Errors: STATE, INVALID_ARG, CUDA. */
lbm_status lbm_forces(lbm_handle h, int32_t n, double* F);

/* n >= 0 steps as lbm_step, with the force on body `body` after each of
 * them (lbm_force of that step) written to F[3*k + a], k = 0 .. n-1: a
 * monitoring loop without a host synchronisation per step.  Each step's
 * force is copied behind that step on the lattice's stream into a pinned
 * staging buffer the lattice owns (grown to at most 4096 steps x 3
 * doubles), so the device runs the steps back to back; the call waits once
 * per 4096 steps and returns when every value has landed.  Steps run one
 * launch sequence each (no multi-step graphs), so states and forces are
 * those of lbm_step(1) repeated, bit for bit.  F: 3 n doubles on the host;
 * a body without links gives zeros.
 * Errors: STATE (no state), INVALID_ARG, OOM, CUDA. */
lbm_status lbm_step_forces(lbm_handle h, int64_t n, int32_t body, double* F);

/* Copy the state out as FP64 post-collision populations f+_i(x,t), [Q][N]
 * on the host (solid and open-column nodes get 0).  Synchronises.
 * Errors: STATE, OOM, CUDA. */
lbm_status lbm_get_distributions(lbm_handle h, double* f);

/* Replace the state by caller populations f+_i(x,t), [Q][N] FP64 on the
 * host; the moment cache is recomputed from them with the lbm_moments
 * formulas.  Does not change the step counter.  Errors: STATE, OOM, CUDA. */
lbm_status lbm_set_distributions(lbm_handle h, const double* f);

/* Discrete adjoint of lbm_step, for gradients of drag and lift (the paper
 * has no gradients; this is the exact transpose of the step this library
 * computes).  Runs n_steps of lbm_step from the current state, keeping a
 * checkpoint every checkpoint_every steps, then sweeps backwards, recomputing
 * each segment from its checkpoint, and returns for the objective
 * J = dJ_dF . F_body (body >= 0; dJ_dF: 3 doubles) or
 * J = sum_b dJ_dF[3b..3b+2] . F_b (body = -1; dJ_dF: 3 x n_bodies doubles,
 * see lbm_query), F the momentum-exchange force of the last step (lbm_force):
 *   *J        J itself;
 *   dJ_dq     host, n_links doubles in the order given to lbm_set_geometry:
 *             dJ/dq of every link (explicit dependence through the link
 *             rules, summed over all steps in FP64);
 *   dJ_dtau   host, one double per domain (one without lbm_set_domains):
 *             dJ/dtau (collision and Guo forcing of every step, and of the
 *             initial collision when the state is the one lbm_init_equilibrium
 *             made);
 *   seconds   NULL or 3 doubles: forward, recompute and adjoint wall time.
 * Gradients with respect to a body's position or radius follow by the chain
 * rule with dq/d(parameter) of each link.  BGK collision only (MRT:
 * LBM_ERR_UNSUPPORTED); all link rules and open columns.  Work and the
 * state's own precision as in lbm_step (FP32 shifted storage gives FP32
 * adjoint states with FP64 time accumulation of dJ/dq and dJ/dtau).
 * Device memory: (n_steps / checkpoint_every + checkpoint_every + 2) states,
 * allocated for the call.  The lattice ends in the forward state after
 * n_steps.  Synchronises.  Errors: STATE, INVALID_ARG, UNSUPPORTED, OOM, CUDA. */
lbm_status lbm_adjoint_step(lbm_handle h, int32_t body, const double dJ_dF[3], int64_t n_steps,
                            int64_t checkpoint_every, double* J, double* dJ_dq, double* dJ_dtau, double seconds[3]);

/* Post-collision populations f+_i(x, t) of n listed nodes, FP64 unshifted,
 * written to out[k*Q + i] (host).  nodes: n host indices in [0, N).  Solid
 * and open-column nodes give 0.  Synchronises.  Used for probes and for
 * sampled checks of large lattices.  Errors: STATE, INVALID_ARG, OOM, CUDA. */
lbm_status lbm_gather(lbm_handle h, const int64_t* nodes, int64_t n, double* out);

/* Failure detection: scan the state; LBM_ERR_DIVERGED if a fluid node has
 * a non-finite population or rho <= 0 (BGK loses stability as tau -> 1/2,
 * Sec. 2).  Synchronises.  Errors: STATE, DIVERGED, CUDA. */
lbm_status lbm_check(lbm_handle h);

/* Wait for all work queued on the lattice's stream.  Errors: CUDA. */
lbm_status lbm_synchronize(lbm_handle h);

/* Fill *info with counts and sizes.  Errors: INVALID_ARG. */
lbm_status lbm_query(lbm_handle h, lbm_info* info);

/* Kernel timing for measurement.  While on, lbm_step launches the kernels
 * one by one (no CUDA graph) with a CUDA event pair around each launch on
 * the lattice's stream.  lbm_kernel_times synchronises and returns, per
 * kernel k (0 = links, 1 = open columns, 2 = bulk, or the fused step kernel
 * when the tuning's fused form runs, in which case slot 0 stays empty), the
 * number of timed launches and their summed duration in milliseconds since
 * profiling was switched on.  Errors: STATE, CUDA, OOM. */
lbm_status lbm_set_profiling(lbm_handle h, int32_t on);
lbm_status lbm_kernel_times(lbm_handle h, int64_t launches[3], double ms[3]);

/* For callers that cannot allocate device memory (code on a real-time path,
 * or a framework whose own pool owns all device memory): the
 * momentum-exchange force on `body` of the step that
 * follows a given state, computed from memory the caller owns.  No
 * counterpart in the paper: it is a packaging of lbm_force for such callers.
 *  cfg      the lattice's configuration (stencil, sizes, periodic axes,
 *           open columns, rho0, g, bc, vibb_density; precision is ignored).
 *  f_post   device, FP64 [Q][N]: post-collision populations f+(x, t) as
 *           returned by lbm_get_distributions.
 *  solid    device, N bytes (nonzero = solid); links: device, n_links
 *           lbm_link records as given to lbm_set_geometry.  The records are
 *           not validated on the host (they are device memory); a record
 *           whose direction is outside [1, Q), whose node is outside
 *           [0, N) or solid, or whose rule is unknown contributes nothing.
 *           Other malformed input (a solid neighbour that is missing, a q
 *           outside (0, 1]) gives a meaningless force, not an error.
 *  F        device, 3 doubles: receives the force of step t -> t+1, the value
 *           lbm_force(body) reports after lbm_step(1) from the same state
 *           (moments are recomputed from f+, so the two agree to rounding).
 * Covers a lattice of one domain: the per-domain tau, g, row widths and
 * inlet settings of lbm_set_domains are not read (cfg's are used for every
 * row), so the force of a batched lattice would be wrong.
 * Work is queued on cfg->cuda_stream (NULL: the legacy default stream) and
 * the call returns without synchronising.  It allocates nothing: its block
 * partial sums live in a static device array of 3 x 65,536 doubles
 * (1.5 MiB, held by every GPU that loads the library until exit), so
 * n_links is limited to LBM_NOALLOC_MAX_LINKS; larger counts return
 * LBM_ERR_INVALID_ARG.  The first call on a device looks up that array's
 * device address and keeps it for the process: it assumes the device's primary context is not reset
 * (cudaDeviceReset) afterwards.  All calls share the
 * array: calls that overlap on the GPU race; calls ordered on one stream do
 * not, and each call overwrites every entry it reads.  Deterministic: the
 * same inputs give the same bits.  Errors: INVALID_ARG, UNSUPPORTED, CUDA. */
#define LBM_NOALLOC_MAX_LINKS 16777216
lbm_status lbm_force_noalloc(const lbm_config* cfg, const double* f_post, const uint8_t* solid,
                             const lbm_link* links, int64_t n_links, int32_t body, double* F);

/* Launch shapes (lbm_tuning).  lbm_set_tuning validates and applies them
 * (from the next lbm_step); lbm_get_tuning reads the current ones.
 * Errors: INVALID_ARG. */
lbm_status lbm_set_tuning(lbm_handle h, const lbm_tuning* t);
lbm_status lbm_get_tuning(lbm_handle h, lbm_tuning* t);

/* Autotuner: times the bulk shapes (with 256-thread link blocks), then the
 * link block sizes, then 4 links per thread, then the graph lengths, each over steps_per_trial steps
 * (>= 2) from the current state after one untimed warm-up replay, and keeps
 * the fastest.  The state, the step counter and the force of the last step
 * are restored afterwards (a scratch copy of one state is allocated for the
 * call).  best: NULL or receives the chosen shapes; ms_per_step: NULL or
 * receives the chosen configuration's time per step.  Synchronises.
 * Errors: STATE, INVALID_ARG, OOM, CUDA. */
lbm_status lbm_autotune(lbm_handle h, int32_t steps_per_trial, lbm_tuning* best, double* ms_per_step);

/* Measured FP64 arithmetic rate of the current device (no counterpart in
 * the paper: a measurement aid for the FP64 kernels, which are bound by the
 * FP64 pipe).  Runs 8 independent FP64 FMA chains per thread in 8 blocks of
 * 256 threads per SM, 5 timed launches after a warm-up, on the legacy
 * default stream, and reports the best launch: *tflops = FP64 flops (an FMA
 * counts 2) per second / 1e12, *ms (NULL allowed) its duration.
 * Synchronises.  Errors: INVALID_ARG, OOM, CUDA. */
lbm_status lbm_probe_fp64(double* tflops, double* ms);

/* Message of the last failed call on this thread ("" if none). */
const char* lbm_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* LBM_H */
