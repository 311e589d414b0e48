"""Throughput of the VIBB lattice-Boltzmann step on one GB300 (or N replicas).

Workload (default): D3Q19 BGK body-force-driven flow through a periodic
random packing of overlapping spheres, 384^3 lattice, radii U[6, 14], centres
U[0, 384)^3 from seed 0, added until the node porosity is <= 0.40; tau = 0.7,
g = 1e-6 along x, VIBB on every cut link (~3.1e7 links).  A step is one full
time step: link rules + momentum-exchange force, pull streaming, moments,
collision.  The state (8.6 GB FP32 / 17.2 GB FP64) is far larger than L2, so
no L2 flush is needed between steps.

Metric: MLUPS counted over fluid nodes, FP32 shifted storage (``value``) and
FP64 (``fp64``), each with the HBM roofline fraction of its dominant kernel
(the bulk pull/collide kernel): algorithmic bytes 2*Q*s + 1 per fluid node
divided by the kernel's average CUDA-event duration inside the timed region.

--impl reference times the FP64 CPU oracle (the plain restatement of the
method that the tests check the kernels against) on a bounded sub-case of the
same recipe.

--part permeability runs the pack for --perm-steps steps (20,000 by default)
in FP32 shifted and FP64 and reports the Darcy permeability of each;
--part studies runs the link rules' accuracy studies (Poiseuille over q and
tau, Couette convergence, the Magnus lift curve) on the FP64 path.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MLUPS and % HBM roofline (FP32 vs FP64); adjoint/forward step cost ratio"
WORKLOAD = ("D3Q19 BGK body-force flow through a periodic random overlapping sphere pack: 384^3 lattice, "
            "radii U[6,14], seed 0, porosity 0.40, tau 0.7, g 1e-6, VIBB links (rho_d = rho_f for q > 1/2)")
Q3 = 19


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs, STREAM-style copy)"
    except Exception:
        return 6800.0, "fallback (6.8 TB/s, one earlier GB300 copy measurement)"


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.2)
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out = ""
        return self.summarise(out)

    @staticmethod
    def summarise(out):
        """Median SM clock under load (samples above 200 W, else all), the
        maximum clock and the throttle reasons seen under load, from the
        noheader/nounits CSV lines of FIELDS."""
        rows = []
        for line in out.splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append(dict(sm=float(parts[1]), max=float(parts[2]), power=float(parts[3]),
                                 hw=parts[5], hwt=parts[6], swt=parts[7], swp=parts[8]))
            except ValueError:
                continue
        if not rows:
            return None
        smx = max(r["max"] for r in rows)
        load = [r for r in rows if r["power"] > 200.0] or rows
        reasons = set()
        for r in load:
            for key, name in (("hw", "hw_slowdown"), ("hwt", "hw_thermal_slowdown"),
                              ("swt", "sw_thermal_slowdown"), ("swp", "sw_power_cap")):
                if r[key].lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(r["sm"] for r in load), "sm_max_mhz": smx,
                "reasons": sorted(reasons), "samples": len(rows), "samples_under_load": len(load),
                "power_w_max": max(r["power"] for r in rows)}


def _dist():
    if int(os.environ.get("WORLD_SIZE", "1")) > 1:
        import torch.distributed as dist

        if not dist.is_initialized():
            dist.init_process_group("nccl")
        return dist
    return None


def _barrier(dist, torch):
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()


def _max_over_ranks(dist, torch, v):
    """Max of a per-rank timing over all ranks (each rank runs a replica)."""
    if dist is None:
        return v
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


AUTOTUNE = True  # --tuning default: the stencil's default shapes (reproducible ncu launch lists)


BULK_SHAPE = -1  # --bulk-shape: force one bulk kernel shape (profiling a given kernel)
LINK_SEQ = 0     # --link-seq: force the link kernel's links per thread
FUSED = -1       # --fused 0/1: force the step form (link kernel + bulk kernel, or the fused kernel)


def _tune(lat, steps_per_trial):
    """The lattice's launch shapes: autotuned on its live state, the
    defaults, or the forced bulk shape / links per thread / step form (where
    the stencil has them)."""
    if BULK_SHAPE >= 0 or LINK_SEQ or FUSED >= 0:
        fused = 1 if FUSED < 0 else FUSED
        try:
            lat.set_tuning(bulk_shape=BULK_SHAPE, link_seq=LINK_SEQ or 1, fused=fused)
        except Exception:
            lat.set_tuning(bulk_shape=-1, link_seq=LINK_SEQ or 1, fused=fused)
        return lat.tuning()
    if AUTOTUNE:
        return lat.autotune(steps_per_trial)[0]
    return lat.tuning()


def _sum_over_ranks(dist, torch, v):
    """Sum of a per-rank count over all ranks."""
    if dist is None:
        return v
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(v)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def sharded_mlups(dist, torch, units_local, steps, ms_local):
    """Whole-job throughput when the ranks split one workload (no exchange):
    the units of all ranks over the slowest rank's time."""
    units = _sum_over_ranks(dist, torch, units_local)
    return units * steps / (_max_over_ranks(dist, torch, ms_local) * 1e-3) / 1e6


def replica_mlups(world, units_per_rank, steps, max_ms):
    """Whole-job throughput of `world` replicas: all units they processed
    divided by the slowest rank's time."""
    return world * units_per_rank * steps / (max_ms * 1e-3) / 1e6


def geometry(n, seed=0):
    from paper_1903_01111_gb300 import geometry as G

    return G.sphere_pack(n, porosity=0.40, rmin=6.0, rmax=14.0, seed=seed)


def run_precision(lbm, torch, geo, precision, steps, warmup, dist, peak):
    s = 8 if precision == lbm.LBM_FP64 else 4
    # a dedicated stream: torch's default stream has handle 0, which the
    # library would replace by its own stream
    stream = torch.cuda.Stream()
    lat = lbm.Lattice(geo, precision=precision, tau=0.7, g=(1e-6, 0.0, 0.0), bc=lbm.LBM_BC_VIBB,
                      stream=stream.cuda_stream, vibb_density=lbm.LBM_VIBB_RHO_LOCAL)
    info = lat.info()
    lat.init_equilibrium()
    tuning = _tune(lat, 10)
    lat.step(warmup)
    _barrier(dist, torch)
    lbm.lbm_set_profiling(lat.h, True)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    _barrier(dist, torch)
    e0.record(stream)
    lat.step(steps)
    e1.record(stream)
    _barrier(dist, torch)
    ms = e0.elapsed_time(e1)
    n_launch, kms = lbm.lbm_kernel_times(lat.h)
    lbm.lbm_set_profiling(lat.h, False)
    lat.check()
    F = lat.force(0)
    lat.close()
    ms = _max_over_ranks(dist, torch, ms)
    nf, nl, N = info.n_fluid, info.n_links, info.n_nodes
    world = dist.get_world_size() if dist is not None else 1
    mlups = replica_mlups(world, nf, steps, ms)
    fused = bool(tuning.fused) and nl > 0
    main_ms = kms[2] / max(n_launch[2], 1)
    link_ms = kms[0] / max(n_launch[0], 1)
    # algorithmic bytes per bulk launch: pulls, stores and word per fluid
    # node, and the moment-cache write of every cached node (step A4)
    bulk_bytes = nf * (2 * Q3 * s + 1) + info.n_cached * 4 * s
    link_bytes = nl * LINK_BYTES(s)
    fused_bytes = bulk_bytes + nl * FUSED_LINK_BYTES(s) + info.n_cached * 4 * s
    main_bytes = fused_bytes if fused else bulk_bytes
    # FP64 one-node bulk shapes run over the fluid-node list (k_bulk_list)
    one_node = tuning.as_dict()["bulk_nodes_per_thread"] == 1 and tuning.as_dict()["bulk_sequential_nodes"] == 1
    name = "k_fused" if fused else ("k_bulk_list" if s == 8 and one_node else "k_bulk")
    traffic = TRAFFIC_PER_FLUID_NODE_PACK_FP32.get(name) if s == 4 else None
    kernels = {name: {"launches": n_launch[2], "avg_ms": main_ms, "share": kms[2] / max(sum(kms), 1e-30),
                      "gbs": main_bytes / (main_ms * 1e-3) / 1e9, "bytes_per_launch": main_bytes}}
    if not fused:
        kernels["k_links"] = {"launches": n_launch[0], "avg_ms": link_ms, "share": kms[0] / max(sum(kms), 1e-30),
                              "gbs": link_bytes / (link_ms * 1e-3) / 1e9, "bytes_per_launch": link_bytes}
    step_bytes = fused_bytes if fused else bulk_bytes + link_bytes
    link_flops = nl * FLOPS_PER_LINK[2]  # every link of the pack is a VIBB link
    main_flops = nf * FLOPS_PER_NODE[Q3] + (link_flops if fused else 0)
    if s == 8 and not fused:
        kernels["k_links"]["roofline"] = roofline_entry(link_bytes, link_flops, link_ms, s, peak)
    return {
        "mlups": mlups, "ms_per_step": ms / steps, "n_fluid": nf, "n_links": nl, "n_nodes": N,
        "n_cached": info.n_cached, "tuning": tuning.as_dict(),
        "launches": int(sum(n_launch)), "force": F.tolist(),
        "roofline": dict(roofline_entry(main_bytes, main_flops, main_ms, s, peak), kernel=name,
                         bytes_per_launch=main_bytes, avg_launch_ms=main_ms,
                         traffic=(traffic * nf if traffic else None),
                         traffic_source=("ncu dram__bytes_read+write on a 192^3 pack, per fluid node, scaled"
                                         if traffic else None),
                         # the DRAM rate the kernel sustains on its measured traffic (not only the
                         # algorithmic bytes), as a fraction of the same peak
                         traffic_rate_frac=(traffic * nf / (main_ms * 1e-3) / 1e9 / peak if traffic else None)),
        "kernels": kernels,
        "step_gbs": step_bytes / (ms / steps * 1e-3) / 1e9,
        "step_bytes": step_bytes,
    }


# DRAM bytes (read + write) per fluid node, by kernel, on the sphere-pack
# recipe from an ncu capture of a 192^3 pack of the same recipe; traffic
# grows with the fluid node count, so a full launch moves this figure times
# its fluid nodes.  k_bulk<D3Q19, F32S, 0, 256, 1>: 575.5 MB per launch for
# 2.83M fluid nodes; k_fused<D3Q19, F32S, 0, 128>: 713.8 MB.
TRAFFIC_PER_FLUID_NODE_PACK_FP32 = {"k_bulk": 204.4, "k_fused": 253.1}


def LINK_BYTES(s):
    """Algorithmic bytes per link of the link kernel: its 16 B record, q,
    f+_i'(x_f), f+_i'(x_ff), the moment records at x_f and x_ff (4 reals
    each) and the ghost write."""
    return 16 + s + 2 * s + 2 * 4 * s + s


def FUSED_LINK_BYTES(s):
    """Algorithmic bytes per link that the fused step adds to the pull pass:
    x_ff's storage index and the metadata word (4 B each), q and
    f+_i'(x_f) (f+_i'(x_ff) is the node's own pull); the moment records
    (4 reals per cached node, read once) are added per cached node."""
    return 8 + 2 * s


# FP64 arithmetic peak: measured on the device at start-up (lbm_probe_fp64,
# independent FP64 FMA chains filling every SM, CUDA events); the figure from
# unit counts (152 SMs x 2 FP64 FMA per clock x 2 flops x 2.07 GHz = 1.26
# TFLOP/s, nominal 1.25) is kept as context.
FP64_PEAK = {"tflops": None, "source": None}
FP64_PEAK_DERIVED_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12


def measure_fp64_peak(lbm):
    tf, ms = lbm.lbm_probe_fp64()
    FP64_PEAK.update(tflops=tf, source=f"measured: lbm_probe_fp64 FP64 FMA chains, best of 5 launches ({ms:.3f} ms)",
                     derived_tflops=FP64_PEAK_DERIVED_TFLOPS)
    return tf


# Algorithmic FP64 flops of one BGK + Guo node update (FMA = 2) in the form
# the kernel evaluates, per pair of opposite directions (e.u, 4.5 (e.u)^2 -
# 1.5 u.u, A, B, omega A and omega B, the two source terms, two outputs: 20
# plus the adds of e.u) and once per node (moments, velocity, u.u, u.g, the
# rest direction, weight products): D2Q9 4 pairs -> 125, D3Q19 9 pairs -> 263.
FLOPS_PER_NODE = {9: 125, 19: 263}
# Algorithmic flops of one link rule as link_value evaluates it (a division
# counts 1) plus the momentum-exchange term (t = f+ + value, 3 FMA = 7):
# VIBB 108-112 (wall term 8, rho_d 4, the two non-equilibrium parts 2 x 20,
# n_d 7 with 2 divisions, the u*, u** weights 6-10 with 1-2 divisions, u_d
# 15, the equilibrium at d and the sum 21) -> 118 with the force term;
# Bouzidi 14-16 -> 22; half-way 9 -> 16; Yu 19 -> 26.
FLOPS_PER_LINK = {0: 16, 1: 22, 2: 118, 3: 26}


HBM_NOMINAL_GBS = 7900.0  # GB300 HBM3e specification, context for the measured copy rate


def roofline_entry(bytes_per_launch, flops_per_launch, avg_ms, s, peak_gbs):
    gbs = bytes_per_launch / (avg_ms * 1e-3) / 1e9
    if s == 8:
        tf = flops_per_launch / (avg_ms * 1e-3) / 1e12
        pk = FP64_PEAK["tflops"] or FP64_PEAK_DERIVED_TFLOPS
        return {"bound": "alu", "achieved": tf, "peak": pk, "unit": "TFLOP/s",
                "frac": tf / pk, "traffic": None, "hbm_gbs": gbs, "hbm_frac": gbs / peak_gbs,
                "peak_source": FP64_PEAK["source"] or "derived: 152 SMs x 2 FP64 FMA/clk x 2 flops x 2.07 GHz",
                "peak_derived": FP64_PEAK_DERIVED_TFLOPS}
    return {"bound": "hbm", "achieved": gbs, "peak": peak_gbs, "unit": "GB/s", "frac": gbs / peak_gbs,
            "traffic": None, "nominal_peak": HBM_NOMINAL_GBS, "frac_of_nominal": gbs / HBM_NOMINAL_GBS}


def run_sweep(lbm, torch, steps, peak, scale=1):
    """No-solid periodic lattices: D2Q9 16384 x 8192 and D3Q19 384^3 (each
    side divided by `scale`), FP32 shifted and FP64; the bulk kernel's
    roofline on each."""
    from paper_1903_01111_gb300 import geometry as G

    out = {}
    for name, stencil, shape in ((f"d2q9_{16384 // scale}x{8192 // scale}", 0, (16384 // scale, 8192 // scale, 1)),
                                 (f"d3q19_{384 // scale}^3", 1, (384 // scale,) * 3)):
        geo = G.build(stencil, shape, (1, 1, 1), [])
        Q = 9 if stencil == 0 else 19
        for prec, s in ((lbm.LBM_FP32_SHIFTED, 4), (lbm.LBM_FP64, 8)):
            stream = torch.cuda.Stream()
            lat = lbm.Lattice(geo, precision=prec, tau=0.7, g=(1e-6, 0.0, 0.0), bc=0, stream=stream.cuda_stream)
            lat.init_equilibrium()
            tuning = _tune(lat, 10)
            n = steps if s == 4 else max(10, steps // 5)
            lat.step(3)
            torch.cuda.synchronize()
            lbm.lbm_set_profiling(lat.h, True)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            lat.step(n)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            nl, kms = lbm.lbm_kernel_times(lat.h)
            lbm.lbm_set_profiling(lat.h, False)
            lat.check()
            nf = lat.info().n_fluid
            lat.close()
            bulk_ms = kms[2] / max(nl[2], 1)
            r = roofline_entry(nf * (2 * Q * s + 1), nf * FLOPS_PER_NODE[Q], bulk_ms, s, peak)
            out[f"{name}_{'fp32s' if s == 4 else 'fp64'}"] = {
                "mlups": nf * n / (ms * 1e-3) / 1e6, "ms_per_step": ms / n, "steps": n,
                "bytes_per_node": 2 * Q * s + 1, "bulk_avg_ms": bulk_ms, "roofline": r, "tuning": tuning.as_dict()}
    return out


def run_adjoint(lbm, n_steps=20000, checkpoint_every=500, fd=True, fd_all=False, fp32_repeats=5):
    """Drag gradient on the 1024 x 256 channel cylinder (radius 16.494, centre
    (256.343, 128.626), u_max 0.1, Re 40 on the mean inflow and the diameter):
    FP32-shifted forward and adjoint with FP64 sensitivity accumulation, cost
    per step of the backward sweep (recompute + adjoint) over a forward step,
    and an FP64 fourth-order central-difference check (steps 1e-3, 2e-3) of
    dJ/dR and dJ/dtau; the centre and radius keep every cut link at least
    4e-3 (in theta) away from the q = 1/2 branch switch.  fd_all: the same
    check of dJ/dc_x and dJ/dc_y (the margin holds for the centre too).  The
    FP32 adjoint is run fp32_repeats times on the same inputs: its FP32
    atomic additions land in a different order each run, and the spread of
    the gradient over the runs is reported next to its error."""
    from paper_1903_01111_gb300.autograd import CylinderSpec, branch_margin, force_only, run

    ubar = 2.0 / 3.0 * 0.1
    R = 16.494
    nu = ubar * 2 * R / 40.0
    tau = 3 * nu + 0.5
    theta = np.array([256.343, 128.626, R, tau])
    spec = CylinderSpec(kind="channel", nx=1024, ny_fluid=256, u_max=0.1, n_steps=n_steps,
                        checkpoint_every=checkpoint_every, precision=lbm.LBM_FP32_SHIFTED)
    J32, g32 = run(spec, theta)
    sec = spec.last["seconds"]
    cancel = spec.last["cancellation"]
    g32_runs = [g32] + [run(spec, theta)[1] for _ in range(max(0, fp32_repeats - 1))]
    out = {"workload": "D2Q9 1024x256 channel, cylinder R 16.494 at (256.343, 128.626), u_max 0.1, Re 40, "
                       f"tau {tau:.4f}, {n_steps} steps, checkpoints every {checkpoint_every}",
           "J_drag": J32, "grad_fp32": {"cx": g32[0], "cy": g32[1], "R": g32[2], "tau": g32[3]},
           "forward_ms_per_step": sec[0] / n_steps * 1e3,
           "backward_ms_per_step": (sec[1] + sec[2]) / n_steps * 1e3,
           "recompute_ms_per_step": sec[1] / n_steps * 1e3, "adjoint_ms_per_step": sec[2] / n_steps * 1e3,
           "ratio_backward_to_forward": (sec[1] + sec[2]) / sec[0],
           "ratio_adjoint_kernels_to_forward": sec[2] / sec[0],
           "link_sum_cancellation": {"cx": cancel[0], "cy": cancel[1], "R": cancel[2]}}
    if fd:
        spec64 = CylinderSpec(kind="channel", nx=1024, ny_fluid=256, u_max=0.1, n_steps=n_steps,
                              checkpoint_every=checkpoint_every, precision=lbm.LBM_FP64)
        J64, g64 = run(spec64, theta)
        checks = {"branch_margin": branch_margin(spec64, theta)}
        h = 1e-3

        def diff(k, step):
            tp, tm = theta.copy(), theta.copy()
            tp[k] += step
            tm[k] -= step
            return (force_only(spec64, tp) - force_only(spec64, tm)) / (2 * step)

        scale = float(np.abs(g64).max())
        for k, name in (((0, "cx"), (1, "cy"), (2, "R"), (3, "tau")) if fd_all else ((2, "R"), (3, "tau"))):
            fd_k = (4 * diff(k, h) - diff(k, 2 * h)) / 3
            errs = sorted(abs(g[k] - fd_k) / abs(fd_k) for g in g32_runs)
            vals = [g[k] for g in g32_runs]
            checks[name] = {"adjoint_fp64": g64[k], "fd_fp64": fd_k, "rel_err_fp64": abs(g64[k] - fd_k) / abs(fd_k),
                            "adjoint_fp32": g32[k], "rel_err_fp32_vs_fd": abs(g32[k] - fd_k) / abs(fd_k),
                            "err_fp32_over_max_grad": abs(g32[k] - fd_k) / scale,
                            "fp32_runs": len(g32_runs), "rel_err_fp32_min_median_max":
                                [errs[0], errs[len(errs) // 2], errs[-1]],
                            "fp32_spread_over_runs_rel": (max(vals) - min(vals)) / abs(fd_k),
                            "fp32_mean_rel_err": abs(float(np.mean(vals)) - fd_k) / abs(fd_k)}
        out["fd_check"] = checks
    return out


def run_batch(lbm, torch, peak, n_domains=256, seed=0, steps=2000, warmup=10, adjoint_steps=1024, K=32, dist=None):
    """Batched channels: n_domains D2Q9 channels (sizes U[64,512] x U[64,256]
    fluid rows, 1-8 non-overlapping cylinders with radii U[4,20], Re U[10,100]
    on the channel height, u_max 0.1, VIBB cylinders, half-way walls,
    velocity inlet and zero-gradient outlet) stacked in one lattice, FP32
    shifted storage, autotuned launch shapes, graph replays; against the same
    channels each run as its own FP64 lattice (per-domain launches on one
    stream).  Both arms run `steps` steps from the Poiseuille initial state
    and are timed over the last steps - warmup; the drag of every cylinder
    after the last step is compared.  Then the batched adjoint of the summed
    drag (every cylinder, FP32 with FP64 accumulation).  Under several ranks
    the channels are split between them (every world-th channel; no
    exchange) and the throughputs count all ranks' nodes over the slowest
    rank's time."""
    from paper_1903_01111_gb300 import batch as B

    t0 = time.perf_counter()
    specs = B.draw_channels(n_domains, seed)
    if dist is not None:
        specs = B.shard(specs, dist.get_rank(), dist.get_world_size())
    b = B.stack(specs)
    t_build = time.perf_counter() - t0
    u0 = b.initial_velocity()
    stream = torch.cuda.Stream()
    lat = lbm.batch_lattice(b, precision=lbm.LBM_FP32_SHIFTED, bc=lbm.LBM_BC_VIBB, stream=stream.cuda_stream)
    info = lat.info()
    lat.init_equilibrium(u=u0)
    tuning = _tune(lat, 20)
    lat.step(warmup)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    lat.step(steps - warmup)
    e1.record(stream)
    torch.cuda.synchronize()
    ms32 = e0.elapsed_time(e1)
    F32 = lat.forces()
    diverged = []
    try:
        lat.check()
    except lbm.LBMError:
        bad = ~np.isfinite(F32).all(axis=1)
        diverged = sorted({int(np.searchsorted(b.body0, k, side="right") - 1) for k in np.flatnonzero(bad)})
    # kernel times of a few more steps (direct launches between events)
    lbm.lbm_set_profiling(lat.h, True)
    lat.step(50)
    nlaunch, kms = lbm.lbm_kernel_times(lat.h)
    lbm.lbm_set_profiling(lat.h, False)
    lat.close()
    nf = b.n_fluid
    s = 4
    fused = bool(tuning.fused) and info.n_links > 0
    main_name = "k_fused" if fused else "k_bulk"
    main_ms = kms[2] / max(nlaunch[2], 1)
    main_bytes = nf * (2 * 9 * s + 1) + info.n_cached * 4 * s
    if fused:
        main_bytes += info.n_links * FUSED_LINK_BYTES(s) + info.n_cached * 4 * s
    mlups32 = sharded_mlups(dist, torch, nf, steps - warmup, ms32)
    # per-domain FP64 lattices on one stream
    lats = []
    for spec, geo in zip(specs, b.parts):
        one = lbm.Lattice(geo, precision=lbm.LBM_FP64, bc=lbm.LBM_BC_VIBB, tau=spec.tau, stream=stream.cuda_stream,
                          **spec.inlet())
        one.init_equilibrium(u=spec.initial_velocity(geo))
        lats.append(one)
    for one in lats:
        one.step(warmup)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    for one in lats:
        one.step(steps - warmup)
    torch.cuda.synchronize()
    s64 = time.perf_counter() - t1
    F64 = np.concatenate([one.forces(len(spec.cylinders)) for one, spec in zip(lats, specs)])
    for one in lats:
        one.close()
    mlups64 = sharded_mlups(dist, torch, nf, steps - warmup, s64 * 1e3)
    rel = np.abs(F32[:, 0] - F64[:, 0]) / np.abs(F64[:, 0])
    rel = rel[np.isfinite(rel)]
    # batched adjoint of the summed drag
    lat = lbm.batch_lattice(b, precision=lbm.LBM_FP32_SHIFTED, bc=lbm.LBM_BC_VIBB, stream=stream.cuda_stream)
    lat.set_tuning(bulk_shape=tuning.bulk_shape, link_threads=tuning.link_threads, graph_steps=tuning.graph_steps,
                   link_seq=tuning.link_seq, fused=tuning.fused)
    lat.init_equilibrium(u=u0)
    w = np.zeros((b.n_bodies, 3))
    w[:, 0] = 1.0
    J, dq, dtau, sec = lbm.lbm_adjoint_step(lat.h, -1, w, adjoint_steps, K)
    lat.close()
    return {
        "workload": f"{n_domains} D2Q9 channels (seed {seed}): nx U[64,512], fluid rows U[64,256], 1-8 cylinders "
                    "r U[4,20], Re U[10,100] on the channel height, u_max 0.1; stacked in one lattice",
        "lattice": [b.geometry.nx, b.geometry.ny], "fluid_nodes": nf, "links": int(info.n_links),
        "bodies": int(b.n_bodies), "stored_nodes": int(info.n_stored), "build_s": t_build,
        "tuning": tuning.as_dict(), "diverged_domains": diverged,
        "fp32_batched": {"value": mlups32, "unit": "MLUPS", "ms_per_step": ms32 / (steps - warmup),
                         "steps_timed": steps - warmup,
                         "roofline": dict(roofline_entry(main_bytes, nf * FLOPS_PER_NODE[9], main_ms, s, peak),
                                          kernel=main_name, bytes_per_launch=main_bytes, avg_launch_ms=main_ms),
                         "kernel_ms": {"k_links": kms[0] / max(nlaunch[0], 1), "k_open": kms[1] / max(nlaunch[1], 1),
                                       main_name: main_ms}},
        "fp64_per_domain": {"value": mlups64, "unit": "MLUPS", "ms_per_step": s64 * 1e3 / (steps - warmup),
                            "launches_per_step": 3 * n_domains},
        "speedup_fp32_batched_vs_fp64_per_domain": mlups32 / mlups64,
        "drag_fp32_batched_vs_fp64": {"after_steps": steps, "max_rel": float(rel.max()),
                                      "median_rel": float(np.median(rel)), "cylinders": int(rel.size)},
        "adjoint": {"steps": adjoint_steps, "checkpoint_every": K, "J_sum_drag": J,
                    "forward_ms_per_step": sec[0] / adjoint_steps * 1e3,
                    "backward_ms_per_step": (sec[1] + sec[2]) / adjoint_steps * 1e3,
                    "ratio_backward_to_forward": (sec[1] + sec[2]) / sec[0],
                    "dJ_dtau_range": [float(np.min(dtau)), float(np.max(dtau))]},
    }


def run_cylinder(lbm, torch, re, steps, sample_every=10, window=None):
    """Flow past the off-grid cylinder in the 2000 x 400 channel (radius 20.3
    at (400.37, 200.61), u_max 0.1, Re on the mean inflow 2/3 u_max and the
    diameter, Poiseuille start), FP32 shifted and FP64, VIBB: drag and lift
    coefficients C_D = 2 F_x / (rho0 U^2 D), C_L = 2 F_y / (rho0 U^2 D) sampled
    every `sample_every` steps; mean C_D, the lift's amplitude and the
    Strouhal number St = f D / U (FFT of C_L) over the last `window` steps."""
    from paper_1903_01111_gb300 import geometry as G

    R, u_max, H = 20.3, 0.1, 400
    ubar, D = 2.0 / 3.0 * u_max, 2 * R
    tau = 3 * ubar * D / re + 0.5
    geo = G.cylinder_channel(nx=2000, ny_fluid=H, center=(400.37, 200.61), radius=R, u_max=u_max)
    y = (np.arange(geo.N) // geo.nx) % geo.ny
    u0 = np.zeros((geo.N, 3))
    u0[:, 0] = np.where(geo.solid == 0, 4 * u_max * (y - 0.5) * (H + 0.5 - y) / H ** 2, 0.0)
    window = window or steps // 2
    m = window // sample_every
    out = {"re": re, "tau": tau, "steps": steps, "window": window}
    series = {}
    for name, prec in (("fp32s", lbm.LBM_FP32_SHIFTED), ("fp64", lbm.LBM_FP64)):
        with lbm.Lattice(geo, precision=prec, tau=tau, bc=lbm.LBM_BC_VIBB, inlet_umax=u_max, inlet_y0=0.5,
                         inlet_y1=H + 0.5) as lat:
            lat.init_equilibrium(u=u0)
            _tune(lat, 10)
            cd, cl, rho_trace = [], [], []
            n_samples = steps // sample_every
            rho_every = max(1, n_samples // 10)
            wall = 0.0
            t0 = time.perf_counter()
            for j in range(n_samples):
                lat.step(sample_every)
                F = lat.force(0)
                cd.append(2 * F[0] / (ubar ** 2 * D))
                cl.append(2 * F[1] / (ubar ** 2 * D))
                if (j + 1) % rho_every == 0:
                    # mean fluid density: the inlet/outlet pair fixes no density level
                    wall += time.perf_counter() - t0
                    rho, _ = lat.moments()
                    rho_trace.append([(j + 1) * sample_every, float(rho[rho > 0].mean())])
                    t0 = time.perf_counter()
            wall += time.perf_counter() - t0
            lat.check()
            nf = lat.info().n_fluid
        cd, cl = np.array(cd), np.array(cl)
        clw = cl[-m:] - cl[-m:].mean()
        spec = np.abs(np.fft.rfft(clw * np.hanning(m)))
        freq = np.fft.rfftfreq(m, d=sample_every)
        amp = 0.5 * (cl[-m:].max() - cl[-m:].min())
        st = freq[int(np.argmax(spec[1:]) + 1)] * D / ubar if amp > 0.05 else None  # steady wake: no shedding
        series[name] = (cd, cl)
        out[name] = {"C_D_mean": float(cd[-m:].mean()), "C_L_mean": float(cl[-m:].mean()),
                     "C_L_amplitude": float(amp), "St": (float(st) if st is not None else None),
                     "mlups_with_force_every_sample": nf * steps / wall / 1e6, "rho_mean_trace": rho_trace}
    d32, d64 = out["fp32s"], out["fp64"]
    out["fp32s_vs_fp64"] = {
        "C_D_rel": abs(d32["C_D_mean"] - d64["C_D_mean"]) / abs(d64["C_D_mean"]),
        "C_L_amplitude_rel": (abs(d32["C_L_amplitude"] - d64["C_L_amplitude"]) / d64["C_L_amplitude"]
                              if d64["C_L_amplitude"] > 0.05 else None),
        "St_rel": (abs(d32["St"] - d64["St"]) / d64["St"] if d32["St"] and d64["St"] else None),
        "max_abs_C_D_diff_over_run": float(np.abs(series["fp32s"][0] - series["fp64"][0]).max()),
        "max_abs_C_L_diff_over_run": float(np.abs(series["fp32s"][1] - series["fp64"][1]).max())}
    return out


def darcy_permeability(geo, u, nu, g):
    """Permeability of a periodic medium driven by the body-force density g
    along x, from Darcy's law: k = nu q_D / g with the superficial velocity
    q_D = (sum of u_x over the fluid nodes) / (all lattice nodes), rho0 = 1.
    u: the (D, N) velocity of lbm_moments (zero at solid nodes)."""
    return nu * float(np.sum(u[0])) / geo.N / g


def run_permeability(lbm, torch, geo, steps, tau=0.7, g=1e-6, samples=4):
    """Sphere-pack permeability after `steps` steps from rest, FP32 shifted
    and FP64 (the same VIBB step as the headline), sampled `samples` times
    along the run to show its convergence; the FP32-vs-FP64 difference is the
    precision error of the quantity the pack workload is run for."""
    nu = (tau - 0.5) / 3
    out = {"steps": steps, "tau": tau, "g": g, "nu": nu, "porosity": geo.info.get("porosity")}
    for name, prec in (("fp32s", lbm.LBM_FP32_SHIFTED), ("fp64", lbm.LBM_FP64)):
        stream = torch.cuda.Stream()
        with lbm.Lattice(geo, precision=prec, tau=tau, g=(g, 0.0, 0.0), bc=lbm.LBM_BC_VIBB,
                         stream=stream.cuda_stream, vibb_density=lbm.LBM_VIBB_RHO_LOCAL) as lat:
            lat.init_equilibrium()
            _tune(lat, 10)
            trace, wall, done = [], 0.0, 0
            for j in range(1, samples + 1):
                n = steps * j // samples - done
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                lat.step(n)
                torch.cuda.synchronize()
                wall += time.perf_counter() - t0
                done += n
                rho, u = lat.moments()
                trace.append({"step": done, "k": darcy_permeability(geo, u, nu, g),
                              "rho_mean": float(rho[rho > 0].mean())})
            lat.check()
            nf = lat.info().n_fluid
        out[name] = {"k": trace[-1]["k"], "trace": trace, "mlups": nf * steps / wall / 1e6,
                     "k_change_last_quarter": abs(trace[-1]["k"] - trace[-2]["k"]) / abs(trace[-1]["k"])
                     if samples > 1 else None}
    out["k_rel_fp32s_vs_fp64"] = abs(out["fp32s"]["k"] - out["fp64"]["k"]) / abs(out["fp64"]["k"])
    return out


def run_magnus(lbm, torch, spins=(0.0, 0.5, 1.0, 1.5, 2.0), rules=(2, 1, 3), steps=40000, sample_every=100):
    """Magnus effect (Sec. 4.3) on the GPU FP64 path: a cylinder of radius
    R = 10 spinning at omega = S U / R in a channel of width L = 400 (half-way
    walls), velocity inlet with the Poiseuille profile of centre-line speed
    U = 0.05 (non-equilibrium extrapolation), zero-gradient outlet, the field
    started from that profile.  The paper states Re = 20 with nu = 0.02,
    which gives 2 U R / nu = 50; the run keeps U and R and takes nu = 0.05
    (tau = 0.65) so that Re = 2 U R / nu = 20.  The domain is L x L with the
    cylinder at (100.37, 199.61) in fluid-row coordinates (the channel's
    centre line is y = 199.5; the paper gives no position).  Lift and drag
    coefficients C_L = F_y / (rho0 U^2 R), C_D = F_x / (rho0 U^2 R) as in
    Sec. 4.3, averaged over the last tenth of the run, per link rule.  No
    literature values are in this repository, so the curve is reported, not
    compared."""
    from paper_1903_01111_gb300 import geometry as G

    L, R, U, re = 400, 10.0, 0.05, 20.0
    nu = 2 * U * R / re
    tau = 3 * nu + 0.5
    names = {0: "halfway", 1: "bouzidi", 2: "vibb", 3: "yu"}
    out = {"L": L, "R": R, "U": U, "Re": re, "nu": nu, "tau": tau, "steps": steps, "center": [100.37, 199.61],
           "runs": []}
    for spin in spins:
        omega = spin * U / R
        geo = G.cylinder_channel(nx=L, ny_fluid=L, center=(100.37, 199.61), radius=R, u_max=U, omega=omega)
        y = (np.arange(geo.N) // geo.nx) % geo.ny
        u0 = np.zeros((geo.N, 3))
        u0[:, 0] = np.where(geo.solid == 0, 4 * U * (y - 0.5) * (L + 0.5 - y) / L ** 2, 0.0)
        row = {"S_pa": spin, "omega": omega}
        for bc in rules:
            with lbm.Lattice(geo, precision=lbm.LBM_FP64, tau=tau, bc=bc, inlet_umax=U, inlet_y0=0.5,
                             inlet_y1=L + 0.5) as lat:
                lat.init_equilibrium(u=u0)
                Fs = []
                for _ in range(steps // sample_every):
                    lat.step(sample_every)
                    Fs.append(lat.force(0))
                lat.check()
            Fs = np.array(Fs[-max(1, len(Fs) // 10):])
            row[names[bc]] = {"C_L": float(Fs[:, 1].mean() / (U * U * R)),
                              "C_D": float(Fs[:, 0].mean() / (U * U * R)),
                              "C_L_spread_last_tenth": float(np.ptp(Fs[:, 1]) / (U * U * R))}
        out["runs"].append(row)
    return out


def run_rho_d(lbm, torch, geo, steps=3000, check_every=100):
    """The printed VIBB density rule (Sec. 3.1, Eq. rhod: rho_d = 2q rho_f +
    (1 - 2q) rho_ff for every q) against the local reading (rho_d = rho_f for
    q > 1/2) on the sphere pack, in FP64 and FP32 shifted: the step at which
    lbm_check first reports a non-finite population or a non-positive
    density (None: stable over `steps`), and the mean density and its
    extremes at the end (or at the last good check)."""
    out = {"steps": steps, "check_every": check_every}
    for vd, vname in ((lbm.LBM_VIBB_RHO_PRINTED, "printed"), (lbm.LBM_VIBB_RHO_LOCAL, "local")):
        for prec, pname in ((lbm.LBM_FP64, "fp64"), (lbm.LBM_FP32_SHIFTED, "fp32s")):
            with lbm.Lattice(geo, precision=prec, tau=0.7, g=(1e-6, 0.0, 0.0), bc=lbm.LBM_BC_VIBB,
                             vibb_density=vd) as lat:
                lat.init_equilibrium()
                diverged, last = None, None
                for k in range(steps // check_every):
                    lat.step(check_every)
                    try:
                        lat.check()
                    except lbm.LBMError:
                        diverged = (k + 1) * check_every
                        break
                    if (k + 1) % max(1, steps // check_every // 5) == 0 or k + 1 == steps // check_every:
                        rho, _ = lat.moments()
                        r = rho[geo.solid == 0]
                        last = {"step": (k + 1) * check_every, "rho_mean": float(r.mean()),
                                "rho_min": float(r.min()), "rho_max": float(r.max())}
            out[f"{vname}_{pname}"] = {"diverged_at": diverged, "last_check": last}
    return out


def run_studies(lbm, torch):
    """Accuracy studies of the link rules on the GPU FP64 path (the paper's
    validation flows): plane Poiseuille flow (Sec. 4.1) between walls at
    fraction q of the first and last links, swept over q and tau, and
    cylindrical Couette flow (Sec. 4.2) over L = 20 .. 320 with the observed
    order of convergence, at a fixed wall speed (acoustic scaling: the
    Mach-number error stays) and at a wall speed falling as 1/L (diffusive
    scaling: fixed Re).  Each run goes to steady state (about 3 diffusion
    times) from rest; errors are relative L2 over the fluid nodes."""
    from paper_1903_01111_gb300 import geometry as G

    names = {0: "halfway", 1: "bouzidi", 2: "vibb", 3: "vibb_local_rho", 4: "yu"}
    rules = ((0, 0), (1, 0), (2, 0), (2, 1), (3, 0))  # (link rule, VIBB density reading)
    out = {"poiseuille": [], "couette": []}
    H, g0 = 24, 1e-6
    for tau in (0.6, 0.8, 1.2):
        nu = (tau - 0.5) / 3
        for q in (0.1, 0.3, 0.5, 0.7, 0.9):
            geo = G.channel(0, 4, H, q_lo=q, q_hi=q)
            Hw = geo.info["y_hi"] - geo.info["y_lo"]
            steps = 2 * int(16 * Hw * Hw / (nu * np.pi ** 2))
            y = np.arange(geo.ny)
            rows = slice(1, geo.ny - 1)
            ex = G.poiseuille_profile(y, geo.info["y_lo"], geo.info["y_hi"], g0, nu)[rows]
            row = {"tau": tau, "q": q, "steps": steps}
            for k, (bc, vd) in enumerate(rules):
                with lbm.Lattice(geo, precision=lbm.LBM_FP64, tau=tau, g=(g0, 0, 0), bc=bc, vibb_density=vd) as lat:
                    lat.init_equilibrium()
                    lat.step(steps)
                    _, u = lat.moments()
                ux = u[0].reshape(geo.ny, geo.nx)[rows].mean(axis=1)
                row[names[k]] = float(np.sqrt(np.sum((ux - ex) ** 2) / np.sum(ex ** 2)))
            out["poiseuille"].append(row)
    tau = 0.8
    nu = (tau - 0.5) / 3
    for scaling, L in [("acoustic", L) for L in (20, 40, 80, 160, 320)] + \
                      [("diffusive", L) for L in (20, 40, 80, 160, 320)]:
        # acoustic: wall speed omega1 r1 = 0.01 at every L (Re grows with L);
        # diffusive: wall speed 0.01 * 20 / L (Re fixed, Mach number -> 0)
        r1 = L / 4.8
        om = (0.01 if scaling == "acoustic" else 0.2 / L) / r1
        geo = G.couette(L, om)
        steps = 2 * int(11 * (geo.info["r2"] - r1) ** 2 / (nu * np.pi ** 2))
        fl = np.flatnonzero(geo.solid == 0)
        x, yy, _ = geo.coords(fl)
        dx, dy = x - geo.info["center"][0], yy - geo.info["center"][1]
        r = np.hypot(dx, dy)
        ex = G.couette_profile(r, r1, geo.info["r2"], om)
        row = {"scaling": scaling, "L": L, "steps": steps, "fluid_nodes": int(fl.size)}
        for k, (bc, vd) in enumerate(rules):
            with lbm.Lattice(geo, precision=lbm.LBM_FP64, tau=tau, bc=bc, vibb_density=vd) as lat:
                lat.init_equilibrium()
                lat.step(steps)
                _, u = lat.moments()
            ut = (-dy * u[0][fl] + dx * u[1][fl]) / r
            row[names[k]] = float(np.sqrt(np.sum((ut - ex) ** 2) / np.sum(ex ** 2)))
        out["couette"].append(row)
    for scaling in ("acoustic", "diffusive"):
        c = [row for row in out["couette"] if row["scaling"] == scaling]
        out[f"couette_order_{scaling}"] = {n: [float(np.log2(c[k][n] / c[k + 1][n])) for k in range(len(c) - 1)]
                                           for n in names.values()}
    out["magnus"] = run_magnus(lbm, torch)
    return out


def run_e2e(lbm, torch, geo, steps):
    """Same workload through the C ABI with host buffers: geometry upload,
    initialisation, the steps with every step's force read back to host
    memory (lbm_step_forces: each copy queued behind its step, no host
    synchronisation per step), and the final macroscopic fields copied to
    host memory.  `value` is the whole region; setup_s (create is outside
    it; set_geometry + init_equilibrium), the loop rate and the final
    read-back are reported apart, so the figure can be read at any step
    count.  After the region, the same loop with a host synchronisation per
    step (lbm_step(1) + lbm_force) is timed for comparison."""
    import ctypes

    solid = np.ascontiguousarray(geo.solid, np.uint8)
    links = np.ascontiguousarray(geo.links, dtype=lbm.LINK_DTYPE)
    rho = np.empty(geo.N)
    u = np.empty((3, geo.N))
    F = (ctypes.c_double * 3)()
    cfg = lbm.make_config(stencil=1, nx=geo.nx, ny=geo.ny, nz=geo.nz, periodic=geo.periodic, tau=0.7,
                          g=(1e-6, 0, 0), bc=lbm.LBM_BC_VIBB, precision=lbm.LBM_FP32_SHIFTED,
                          stream=None, vibb_density=lbm.LBM_VIBB_RHO_LOCAL)
    h = lbm.lbm_create_lattice(cfg)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    lbm.lbm_set_geometry(h, solid, links)
    lbm.lbm_init_equilibrium(h)
    ts = time.perf_counter()
    Fs = lbm.lbm_step_forces(h, steps, 0)
    tl = time.perf_counter()
    lbm.lbm_moments(h, rho, u)
    t1 = time.perf_counter()
    nsync = min(steps, 200)
    tq0 = time.perf_counter()
    for _ in range(nsync):
        lbm.lbm_step(h, 1)
        lbm._check(lbm._lib.lbm_force(h, 0, F))
    tq1 = time.perf_counter()
    info = lbm.lbm_query(h)
    tuning = lbm.lbm_get_tuning(h)
    lbm.lbm_destroy(h)
    h2d = solid.nbytes + links.nbytes
    d2h = 24 * steps + rho.nbytes + u.nbytes
    per_step_launches = 1 if tuning.fused and info.n_links else 2
    return {"value": info.n_fluid * steps / (t1 - t0) / 1e6, "unit": "MLUPS",
            "h2d_bytes_per_step": h2d / steps, "d2h_bytes_per_step": d2h / steps, "seconds": t1 - t0,
            "setup_s": ts - t0, "loop_s": tl - ts, "readback_s": t1 - tl, "steps": steps,
            "loop_mlups": info.n_fluid * steps / (tl - ts) / 1e6,
            "loop_note": "lbm_step_forces: every step's force (24 B) copied to pinned host memory behind the step",
            "last_force": Fs[-1].tolist() if steps else None,
            "loop_sync_mlups": info.n_fluid * nsync / max(tq1 - tq0, 1e-30) / 1e6,
            "loop_sync_note": f"{nsync} x (lbm_step(1) + lbm_force), a host synchronisation per step, after the region",
            "gpu_launches": steps * per_step_launches + 2}


def run_oracle(n, target_s=15.0, single_target_s=8.0):
    """The FP64 CPU oracle on an n^3 sub-case of the same recipe, on every
    host core (OpenMP over its per-node passes; the result does not depend
    on the thread count) and on one thread.  Each run's step count is set
    from a two-step timing so that it takes about target_s (all cores) or
    single_target_s (one thread) of CPU time."""
    import oracle as O

    geo = geometry(n)
    cfg = O.make_config(stencil=1, nx=n, ny=n, nz=n, periodic=(1, 1, 1), tau=0.7, g=(1e-6, 0, 0), bc=2,
                        vibb_density=1)
    nf = geo.fluid_count()
    out = {}
    for threads, target in ((os.cpu_count() or 1, target_s), (1, single_target_s)):
        used = O.set_threads(threads)
        st = O.init(cfg, geo.solid)
        O.run(cfg, geo.solid, geo.links, st, 1)
        t0 = time.perf_counter()
        O.run(cfg, geo.solid, geo.links, st, 2)
        per_step = (time.perf_counter() - t0) / 2
        steps = int(max(2, min(5000, target / max(per_step, 1e-9))))
        t0 = time.perf_counter()
        O.run(cfg, geo.solid, geo.links, st, steps)
        dt = time.perf_counter() - t0
        out[threads] = (nf * steps / dt / 1e6, used, dt, steps)
    v, used, dt, steps = out[os.cpu_count() or 1]
    v1, _, dt1, steps1 = out[1]
    return {"value": v, "unit": "MLUPS", "cores": used, "kind": "oracle",
            "sample": f"{n}^3 sub-case of the same sphere-pack recipe ({nf} fluid nodes, {len(geo.links)} links), "
                      f"{steps} steps, FP64 oracle, {used} OpenMP threads (nproc), {dt:.1f} s",
            "single_thread": {"value": v1, "unit": "MLUPS", "cores": 1, "steps": steps1, "seconds": dt1}}


def reference_arm(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    # sample sized so that the whole --steps run is about 6e8 fluid-node
    # updates (some 30 s on 16 cores at the oracle's 20 MLUPS)
    n = int(round((6e8 / (0.4 * max(args.steps, 1))) ** (1 / 3)))
    n = max(32, min(160, n))
    import oracle as O

    cores = O.set_threads(os.cpu_count() or 1)
    geo = geometry(n)
    cfg = O.make_config(stencil=1, nx=n, ny=n, nz=n, periodic=(1, 1, 1), tau=0.7, g=(1e-6, 0, 0), bc=2,
                        vibb_density=1)
    st = O.init(cfg, geo.solid)
    O.run(cfg, geo.solid, geo.links, st, args.warmup)
    t0 = time.perf_counter()
    O.run(cfg, geo.solid, geo.links, st, args.steps)
    dt = time.perf_counter() - t0
    nf = geo.fluid_count()
    v = nf * args.steps / dt / 1e6
    line = {"metric": METRIC, "value": v, "unit": "MLUPS", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": WORKLOAD, "sample": f"{n}^3 sub-case of the same recipe",
                       "fluid_nodes": nf, "links": int(len(geo.links)), "parallelism": "replicas"},
            "cpu_baseline": {"value": v, "unit": "MLUPS", "cores": cores, "kind": "oracle",
                             "sample": f"{n}^3 sub-case, {args.steps} steps, FP64 oracle, {cores} OpenMP threads"},
            "e2e": {"value": v, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=384, help="lattice side (default: the 384^3 workload)")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-sweep", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-cylinder", action="store_true")
    ap.add_argument("--cylinder-steps", type=int, default=60000)
    ap.add_argument("--sweep-steps", type=int, default=100)
    ap.add_argument("--part", default="all",
                    choices=["all", "batch", "adjoint", "sweep", "cylinder", "permeability", "studies", "rho_d"],
                    help="run one section alone (for profiling) and print its JSON")
    ap.add_argument("--batch-domains", type=int, default=256)
    ap.add_argument("--batch-steps", type=int, default=2000)
    ap.add_argument("--adjoint-steps", type=int, default=20000)
    ap.add_argument("--adjoint-fd", action="store_true", help="with --part adjoint: also the FD check")
    ap.add_argument("--sweep-scale", type=int, default=1, help="divide the sweep lattices' sides by this")
    ap.add_argument("--rho-d-steps", type=int, default=3000,
                    help="with --part rho_d: steps of each sphere-pack run (printed and local rho_d, FP64 and FP32)")
    ap.add_argument("--perm-steps", type=int, default=20000,
                    help="with --part permeability: steps of the sphere-pack run (FP32 shifted and FP64)")
    ap.add_argument("--tuning", default="auto", choices=["auto", "default"],
                    help="autotune every timed lattice (default) or keep the default launch shapes")
    ap.add_argument("--bulk-shape", type=int, default=-1,
                    help="force this bulk kernel shape where the stencil has it (profiling)")
    ap.add_argument("--link-seq", type=int, default=0, choices=[0, 1, 4],
                    help="force the link kernel's links per thread (profiling)")
    ap.add_argument("--fused", type=int, default=-1, choices=[-1, 0, 1],
                    help="force the step form: 0 link kernel + bulk kernel, 1 fused kernel (profiling)")
    args = ap.parse_args()
    global AUTOTUNE, BULK_SHAPE, LINK_SEQ, FUSED
    AUTOTUNE = args.tuning == "auto"
    BULK_SHAPE = args.bulk_shape
    LINK_SEQ = args.link_seq
    FUSED = args.fused
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        return reference_arm(args)
    if args.part != "all":
        import torch

        from paper_1903_01111_gb300 import lbm

        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        measure_fp64_peak(lbm)
        if args.part == "cylinder":
            out = [run_cylinder(lbm, torch, 20, args.cylinder_steps // 2),
                   run_cylinder(lbm, torch, 100, args.cylinder_steps)]
        elif args.part == "studies":
            out = run_studies(lbm, torch)
        elif args.part == "rho_d":
            out = run_rho_d(lbm, torch, geometry(args.n), steps=args.rho_d_steps)
        elif args.part == "permeability":
            out = run_permeability(lbm, torch, geometry(args.n), args.perm_steps)
        elif args.part == "sweep":
            out = run_sweep(lbm, torch, args.sweep_steps, _peaks()[0], scale=args.sweep_scale)
        elif args.part == "batch":
            out = run_batch(lbm, torch, _peaks()[0], n_domains=args.batch_domains, steps=args.batch_steps,
                            warmup=args.warmup, adjoint_steps=min(64, args.batch_steps), K=8)
        else:
            out = run_adjoint(lbm, n_steps=args.adjoint_steps, checkpoint_every=max(2, min(500, args.adjoint_steps)),
                              fd=args.adjoint_fd, fd_all=args.adjoint_fd)
        print(json.dumps(out), flush=True)
        return 0

    import torch

    dist = _dist()
    rank = dist.get_rank() if dist is not None else 0
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    from paper_1903_01111_gb300 import lbm

    peak, peak_src = _peaks()
    measure_fp64_peak(lbm)
    t0 = time.perf_counter()
    geo = geometry(args.n)
    t_geo = time.perf_counter() - t0
    clocks = Clocks(local)
    clocks.start()
    r32 = run_precision(lbm, torch, geo, lbm.LBM_FP32_SHIFTED, args.steps, args.warmup, dist, peak)
    ck = clocks.stop()
    r64 = None
    if not args.no_fp64:
        clocks64 = Clocks(local)
        clocks64.start()
        r64 = run_precision(lbm, torch, geo, lbm.LBM_FP64, args.steps, args.warmup, dist, peak)
        r64["clocks"] = clocks64.stop()
    e2e = None if args.no_e2e else run_e2e(lbm, torch, geo, args.steps)
    sweep = None if args.no_sweep else run_sweep(lbm, torch, args.sweep_steps, peak)
    adjoint = None if args.no_adjoint else run_adjoint(lbm, fd_all=True)
    batched = None if args.no_batch else run_batch(lbm, torch, peak, dist=dist)
    cylinder = None
    if not args.no_cylinder:
        cylinder = [run_cylinder(lbm, torch, 20, args.cylinder_steps // 2),
                    run_cylinder(lbm, torch, 100, args.cylinder_steps)]
    cpu = None
    if rank == 0 and not args.no_cpu:
        cpu = run_oracle(128)
    if rank != 0:
        return 0
    world = dist.get_world_size() if dist is not None else 1
    line = {
        "metric": METRIC, "value": r32["mlups"], "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": r32["ms_per_step"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD if args.n == 384 else WORKLOAD.replace("384^3", f"{args.n}^3"),
                   "precision": "fp32_shifted", "nodes": r32["n_nodes"], "fluid_nodes": r32["n_fluid"],
                   "links": r32["n_links"], "porosity": geo.info["porosity"], "spheres": geo.info["spheres"],
                   "l2": "inputs larger than L2 (state > 8 GB), no flush", "parallelism": "replicas",
                   "geometry_build_s": t_geo},
        "roofline": dict(r32["roofline"], peak_source=peak_src),
        "hbm_peak_source": peak_src,
        "fp64_peak": dict(FP64_PEAK),
        "kernels": r32["kernels"], "step_gbs": r32["step_gbs"], "tuning": r32["tuning"],
        "cpu_baseline": cpu, "e2e": e2e,
        "gpu_launches": r32["launches"],
        "clocks": ck,
    }
    if sweep is not None:
        line["roofline_sweep"] = sweep
    if adjoint is not None:
        line["adjoint"] = adjoint
    if batched is not None:
        line["batched"] = batched
    if cylinder is not None:
        line["cylinder"] = cylinder
    if r64 is not None:
        line["fp64"] = {"value": r64["mlups"], "unit": "MLUPS", "ms_per_step": r64["ms_per_step"],
                        "roofline": r64["roofline"], "kernels": r64["kernels"],
                        "step_gbs": r64["step_gbs"], "gpu_launches": r64["launches"], "tuning": r64["tuning"],
                        "clocks": r64["clocks"]}
    print(json.dumps(line), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
