"""Python binding of liblbm.so (C ABI in include/lbm.h).

Argument marshalling only: every step of the computation runs in the
library's CUDA kernels.  The functions keep the C names; ``Lattice`` is a
small owner object around a handle.  There is no fallback: if liblbm.so is
missing or fails to load, importing this module raises.

Arrays: host inputs are numpy arrays; ``lbm_moments`` also takes torch CUDA
tensors (device pointers) or numpy arrays (host pointers).  PyTorch is used
only for device memory and for the CUDA stream handle.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblbm.so")
if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is not built; run `python -m paper_1903_01111_gb300.build` (needs nvcc)")
_lib = ctypes.CDLL(LIB_PATH)

LBM_OK, LBM_ERR_INVALID_ARG, LBM_ERR_STATE, LBM_ERR_CUDA, LBM_ERR_OOM, LBM_ERR_DIVERGED, LBM_ERR_TIMEOUT, \
    LBM_ERR_UNSUPPORTED = range(8)
LBM_D2Q9, LBM_D3Q19 = 0, 1
LBM_BGK, LBM_MRT = 0, 1
LBM_BC_DEFAULT, LBM_BC_HALFWAY, LBM_BC_BOUZIDI, LBM_BC_VIBB, LBM_BC_YU = -1, 0, 1, 2, 3
LBM_FP64, LBM_FP32_SHIFTED = 0, 1
LBM_VIBB_RHO_PRINTED, LBM_VIBB_RHO_LOCAL = 0, 1
LBM_MAX_BODIES = 32768
STATUS_NAMES = {0: "LBM_OK", 1: "LBM_ERR_INVALID_ARG", 2: "LBM_ERR_STATE", 3: "LBM_ERR_CUDA", 4: "LBM_ERR_OOM",
                5: "LBM_ERR_DIVERGED", 6: "LBM_ERR_TIMEOUT", 7: "LBM_ERR_UNSUPPORTED"}

LINK_DTYPE = np.dtype(
    [("node", "<i8"), ("dir", "<i4"), ("bc", "<i2"), ("body", "<i2"), ("q", "<f8"), ("uw", "<f8", (3,))],
    align=True,
)
assert LINK_DTYPE.itemsize == 48


class LBMError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class lbm_config(ctypes.Structure):
    _fields_ = [
        ("stencil", ctypes.c_int32),
        ("collision", ctypes.c_int32),
        ("bc", ctypes.c_int32),
        ("nx", ctypes.c_int32),
        ("ny", ctypes.c_int32),
        ("nz", ctypes.c_int32),
        ("periodic", ctypes.c_int32 * 3),
        ("inlet", ctypes.c_int32),
        ("outlet", ctypes.c_int32),
        ("tau", ctypes.c_double),
        ("rho0", ctypes.c_double),
        ("g", ctypes.c_double * 3),
        ("inlet_umax", ctypes.c_double),
        ("inlet_y0", ctypes.c_double),
        ("inlet_y1", ctypes.c_double),
        ("precision", ctypes.c_int32),
        ("vibb_density", ctypes.c_int32),
        ("cuda_stream", ctypes.c_void_p),
    ]


class lbm_info(ctypes.Structure):
    _fields_ = [
        ("n_nodes", ctypes.c_int64),
        ("n_fluid", ctypes.c_int64),
        ("n_links", ctypes.c_int64),
        ("n_cached", ctypes.c_int64),
        ("step", ctypes.c_int64),
        ("device_bytes", ctypes.c_int64),
        ("Q", ctypes.c_int32),
        ("D", ctypes.c_int32),
        ("precision", ctypes.c_int32),
        ("real_bytes", ctypes.c_int32),
        ("n_stored", ctypes.c_int64),
        ("n_runs", ctypes.c_int64),
        ("n_bodies", ctypes.c_int32),
        ("n_domains", ctypes.c_int32),
    ]


class lbm_domain(ctypes.Structure):
    _fields_ = [
        ("lo", ctypes.c_int32),
        ("n", ctypes.c_int32),
        ("nx", ctypes.c_int32),
        ("reserved", ctypes.c_int32),
        ("tau", ctypes.c_double),
        ("g", ctypes.c_double * 3),
        ("inlet_umax", ctypes.c_double),
        ("inlet_y0", ctypes.c_double),
        ("inlet_y1", ctypes.c_double),
    ]


class lbm_tuning(ctypes.Structure):
    _fields_ = [
        ("bulk_shape", ctypes.c_int32),
        ("link_threads", ctypes.c_int32),
        ("graph_steps", ctypes.c_int32),
        ("link_seq", ctypes.c_int32),
        ("fused", ctypes.c_int32),
    ]

    def as_dict(self):
        t, npt, seq = BULK_SHAPES[self.bulk_shape]
        return {"bulk_shape": self.bulk_shape, "bulk_threads": t, "bulk_nodes_per_thread": npt,
                "bulk_sequential_nodes": seq, "link_threads": self.link_threads, "link_seq": self.link_seq,
                "graph_steps": self.graph_steps, "fused": self.fused}


# (threads per block, nodes per thread, nodes per thread in sequence) of
# bulk_shape 0..7; 3..7 are built for D2Q9 only
BULK_SHAPES = ((256, 1, 1), (128, 1, 1), (512, 1, 1), (256, 2, 1), (128, 2, 1), (512, 2, 1), (128, 1, 4), (128, 1, 8))


_H = ctypes.c_void_p
_P = ctypes.POINTER
_vp = ctypes.c_void_p
_sig = {
    "lbm_create_lattice": [_P(lbm_config), _P(_H)],
    "lbm_destroy": [_H],
    "lbm_set_geometry": [_H, _vp, _vp, ctypes.c_int64],
    "lbm_init_equilibrium": [_H, _vp, _vp],
    "lbm_step": [_H, ctypes.c_int64],
    "lbm_moments": [_H, _vp, _vp],
    "lbm_force": [_H, ctypes.c_int32, _P(ctypes.c_double)],
    "lbm_get_distributions": [_H, _vp],
    "lbm_set_distributions": [_H, _vp],
    "lbm_gather": [_H, _vp, ctypes.c_int64, _vp],
    "lbm_check": [_H],
    "lbm_synchronize": [_H],
    "lbm_query": [_H, _P(lbm_info)],
    "lbm_set_profiling": [_H, ctypes.c_int32],
    "lbm_kernel_times": [_H, _P(ctypes.c_int64), _P(ctypes.c_double)],
    "lbm_force_noalloc": [_P(lbm_config), _vp, _vp, _vp, ctypes.c_int64, ctypes.c_int32, _vp],
    "lbm_probe_fp64": [_P(ctypes.c_double), _P(ctypes.c_double)],
    "lbm_adjoint_step": [_H, ctypes.c_int32, _vp, ctypes.c_int64, ctypes.c_int64,
                         _P(ctypes.c_double), _vp, _vp, _P(ctypes.c_double)],
    "lbm_set_domains": [_H, _vp, ctypes.c_int32],
    "lbm_forces": [_H, ctypes.c_int32, _vp],
    "lbm_step_forces": [_H, ctypes.c_int64, ctypes.c_int32, _vp],
    "lbm_set_tuning": [_H, _P(lbm_tuning)],
    "lbm_get_tuning": [_H, _P(lbm_tuning)],
    "lbm_autotune": [_H, ctypes.c_int32, _P(lbm_tuning), _P(ctypes.c_double)],
}
for _name, _args in _sig.items():
    _fn = getattr(_lib, _name)
    _fn.argtypes = _args
    _fn.restype = ctypes.c_int
_lib.lbm_last_error.restype = ctypes.c_char_p
_lib.lbm_last_error.argtypes = []

EXPORTED = tuple(_sig) + ("lbm_last_error",)


def lbm_last_error() -> str:
    return _lib.lbm_last_error().decode(errors="replace")


def _check(st):
    if st != LBM_OK:
        raise LBMError(st, lbm_last_error())


def _ptr(a):
    """Pointer of a numpy array (host) or a torch tensor (host or device)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    return a.ctypes.data


def make_config(stencil=LBM_D2Q9, nx=1, ny=1, nz=1, periodic=(1, 1, 1), tau=0.8, rho0=1.0, g=(0.0, 0.0, 0.0),
                bc=LBM_BC_VIBB, collision=LBM_BGK, inlet=0, outlet=0, inlet_umax=0.0, inlet_y0=0.0, inlet_y1=0.0,
                precision=LBM_FP64, stream=None, vibb_density=LBM_VIBB_RHO_PRINTED) -> lbm_config:
    c = lbm_config()
    c.stencil, c.collision, c.bc = stencil, collision, bc
    c.nx, c.ny, c.nz = nx, ny, nz
    for a in range(3):
        c.periodic[a] = int(periodic[a])
        c.g[a] = float(g[a]) if a < len(g) else 0.0
    c.inlet, c.outlet = int(inlet), int(outlet)
    c.tau, c.rho0 = float(tau), float(rho0)
    c.inlet_umax, c.inlet_y0, c.inlet_y1 = float(inlet_umax), float(inlet_y0), float(inlet_y1)
    c.precision = precision
    c.vibb_density = vibb_density
    c.cuda_stream = stream
    return c


def lbm_create_lattice(cfg: lbm_config) -> int:
    h = _H()
    _check(_lib.lbm_create_lattice(ctypes.byref(cfg), ctypes.byref(h)))
    return h.value


def lbm_destroy(h) -> None:
    _check(_lib.lbm_destroy(h))


def lbm_set_geometry(h, solid, links) -> None:
    solid = np.ascontiguousarray(solid, np.uint8).reshape(-1)
    links = np.ascontiguousarray(links, dtype=LINK_DTYPE)
    _check(_lib.lbm_set_geometry(h, solid.ctypes.data, links.ctypes.data if links.size else None, links.size))


def lbm_init_equilibrium(h, rho=None, u=None) -> None:
    r = None if rho is None else np.ascontiguousarray(rho, np.float64).reshape(-1)
    uu = None if u is None else np.ascontiguousarray(u, np.float64).reshape(-1, 3)
    _check(_lib.lbm_init_equilibrium(h, None if r is None else r.ctypes.data, None if uu is None else uu.ctypes.data))


def lbm_step(h, n: int) -> None:
    _check(_lib.lbm_step(h, int(n)))


def lbm_moments(h, rho, u) -> None:
    """Write rho (N) and u (D x N) float64; numpy (host) or torch CUDA tensors."""
    _check(_lib.lbm_moments(h, _ptr(rho), _ptr(u)))


def lbm_force(h, body: int = 0) -> np.ndarray:
    F = (ctypes.c_double * 3)()
    _check(_lib.lbm_force(h, int(body), F))
    return np.array(F[:])


def lbm_query(h) -> lbm_info:
    info = lbm_info()
    _check(_lib.lbm_query(h, ctypes.byref(info)))
    return info


def lbm_get_distributions(h, out=None) -> np.ndarray:
    info = lbm_query(h)
    if out is None:
        out = np.empty((info.Q, info.n_nodes), np.float64)
    assert out.dtype == np.float64 and out.flags.c_contiguous and out.size == info.Q * info.n_nodes
    _check(_lib.lbm_get_distributions(h, out.ctypes.data))
    return out


def lbm_set_distributions(h, f) -> None:
    f = np.ascontiguousarray(f, np.float64)
    info = lbm_query(h)
    assert f.size == info.Q * info.n_nodes
    _check(_lib.lbm_set_distributions(h, f.ctypes.data))


def lbm_gather(h, nodes) -> np.ndarray:
    """Post-collision populations (n, Q) of the listed nodes, FP64."""
    nodes = np.ascontiguousarray(nodes, np.int64).reshape(-1)
    info = lbm_query(h)
    out = np.empty((nodes.size, info.Q), np.float64)
    _check(_lib.lbm_gather(h, nodes.ctypes.data if nodes.size else None, nodes.size, out.ctypes.data))
    return out


def lbm_adjoint_step(h, body: int, dJ_dF, n_steps: int, checkpoint_every: int):
    """Run n_steps forward with checkpoints and the adjoint sweep back.
    body >= 0: dJ_dF has 3 entries; body = -1: dJ_dF is (n_bodies, 3).
    Returns (J, dJ_dq (n_links, caller's link order), dJ_dtau, seconds[3]);
    dJ_dtau is a float for a lattice of one domain, else an array per domain."""
    info = lbm_query(h)
    w = np.ascontiguousarray(dJ_dF, np.float64).reshape(-1)
    need = 3 if body >= 0 else 3 * info.n_bodies
    if w.size != need:
        raise ValueError(f"dJ_dF needs {need} entries")
    J = ctypes.c_double(0.0)
    dtau = np.zeros(info.n_domains)
    sec = (ctypes.c_double * 3)()
    dq = np.zeros(max(info.n_links, 1))
    _check(_lib.lbm_adjoint_step(h, int(body), w.ctypes.data, int(n_steps), int(checkpoint_every), ctypes.byref(J),
                                 dq.ctypes.data, dtau.ctypes.data, sec))
    return J.value, dq[: info.n_links], (float(dtau[0]) if info.n_domains == 1 else dtau), list(sec)


def make_domains(rows):
    """ctypes array of lbm_domain from dicts with keys lo, n, nx, tau and
    optionally g, inlet_umax, inlet_y0, inlet_y1."""
    arr = (lbm_domain * len(rows))()
    for k, r in enumerate(rows):
        d = arr[k]
        d.lo, d.n, d.nx = int(r["lo"]), int(r["n"]), int(r["nx"])
        d.tau = float(r["tau"])
        g = r.get("g", (0.0, 0.0, 0.0))
        for a in range(3):
            d.g[a] = float(g[a]) if a < len(g) else 0.0
        d.inlet_umax = float(r.get("inlet_umax", 0.0))
        d.inlet_y0 = float(r.get("inlet_y0", 0.0))
        d.inlet_y1 = float(r.get("inlet_y1", 0.0))
    return arr


def lbm_set_domains(h, rows) -> None:
    arr = make_domains(rows)
    _check(_lib.lbm_set_domains(h, arr if len(rows) else None, len(rows)))


def lbm_forces(h, n: int) -> np.ndarray:
    """Forces (n, 3) on bodies 0..n-1 of the last step."""
    out = np.zeros((max(n, 1), 3))
    _check(_lib.lbm_forces(h, int(n), out.ctypes.data))
    return out[:n]


def lbm_step_forces(h, n: int, body: int = 0) -> np.ndarray:
    """n steps, and the force (n, 3) on `body` after each of them (copied
    behind each step, one synchronisation per 4096 steps)."""
    out = np.zeros((max(int(n), 1), 3))
    _check(_lib.lbm_step_forces(h, int(n), int(body), out.ctypes.data))
    return out[:int(n)]


def lbm_set_tuning(h, bulk_shape=-1, link_threads=256, graph_steps=2, link_seq=1, fused=1) -> None:
    t = lbm_tuning(int(bulk_shape), int(link_threads), int(graph_steps), int(link_seq), int(fused))
    _check(_lib.lbm_set_tuning(h, ctypes.byref(t)))


def lbm_get_tuning(h) -> lbm_tuning:
    t = lbm_tuning()
    _check(_lib.lbm_get_tuning(h, ctypes.byref(t)))
    return t


def lbm_autotune(h, steps_per_trial: int = 20):
    """Time the launch shapes on the current state (restored afterwards);
    returns (lbm_tuning chosen, ms per step)."""
    t = lbm_tuning()
    ms = ctypes.c_double(0.0)
    _check(_lib.lbm_autotune(h, int(steps_per_trial), ctypes.byref(t), ctypes.byref(ms)))
    return t, ms.value


def lbm_check(h) -> None:
    _check(_lib.lbm_check(h))


def lbm_synchronize(h) -> None:
    _check(_lib.lbm_synchronize(h))


def lbm_set_profiling(h, on: bool) -> None:
    _check(_lib.lbm_set_profiling(h, 1 if on else 0))


def lbm_kernel_times(h):
    """(launches[3], ms[3]) for kernels 0 = links, 1 = open columns, 2 = bulk."""
    n = (ctypes.c_int64 * 3)()
    ms = (ctypes.c_double * 3)()
    _check(_lib.lbm_kernel_times(h, n, ms))
    return list(n), list(ms)


def lbm_probe_fp64():
    """Measured FP64 arithmetic rate of the current device: (TFLOP/s, ms of
    the best timed launch)."""
    tf, ms = ctypes.c_double(0.0), ctypes.c_double(0.0)
    _check(_lib.lbm_probe_fp64(ctypes.byref(tf), ctypes.byref(ms)))
    return tf.value, ms.value


def _check_device_tensor(name, t, dtype, min_bytes):
    """Type, size and device of a torch tensor handed to the C library as a
    device pointer (raw integer addresses are passed through unchecked)."""
    if isinstance(t, int):
        return
    import torch

    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name}: a torch CUDA tensor or an integer device address is required")
    if not t.is_cuda or t.device.index != torch.cuda.current_device():
        raise ValueError(f"{name}: must live on the current CUDA device")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"{name}: dtype {t.dtype}, expected {dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name}: must be contiguous")
    if t.numel() * t.element_size() < min_bytes:
        raise ValueError(f"{name}: {t.numel() * t.element_size()} bytes, at least {min_bytes} needed")


def lbm_force_noalloc(cfg: lbm_config, f_post, solid, links, n_links: int, body: int, F) -> None:
    """Momentum-exchange force of the next step from caller-owned device
    memory (torch CUDA tensors or raw device addresses); allocates nothing.
    Queued on cfg.cuda_stream without synchronising.  Tensors are checked
    for dtype, size and device before the call (raw addresses are not)."""
    import torch

    Q = 9 if cfg.stencil == LBM_D2Q9 else 19
    N = int(cfg.nx) * int(cfg.ny) * int(cfg.nz)
    _check_device_tensor("f_post", f_post, torch.float64, 8 * Q * N)
    _check_device_tensor("solid", solid, None, N)
    _check_device_tensor("links", links, None, LINK_DTYPE.itemsize * int(n_links))
    _check_device_tensor("F", F, torch.float64, 24)
    _check(_lib.lbm_force_noalloc(ctypes.byref(cfg), _ptr_or_int(f_post), _ptr_or_int(solid), _ptr_or_int(links),
                                  int(n_links), int(body), _ptr_or_int(F)))


def _ptr_or_int(a):
    return a if isinstance(a, int) else _ptr(a)


LBM_NOALLOC_MAX_LINKS = 16777216

KERNEL_NAMES = ("k_links", "k_open", "k_bulk or k_fused")


class Lattice:
    """Owner of one lattice handle; mirrors the C entry points."""

    def __init__(self, geometry=None, domains=None, **cfg):
        if geometry is not None:
            cfg.setdefault("stencil", geometry.stencil)
            cfg.setdefault("nx", geometry.nx)
            cfg.setdefault("ny", geometry.ny)
            cfg.setdefault("nz", geometry.nz)
            cfg.setdefault("periodic", geometry.periodic)
            cfg.setdefault("inlet", int(geometry.open_x[0]))
            cfg.setdefault("outlet", int(geometry.open_x[1]))
        self.cfg = make_config(**cfg)
        self.h = lbm_create_lattice(self.cfg)
        if domains is not None:
            lbm_set_domains(self.h, domains)
        if geometry is not None:
            self.set_geometry(geometry.solid, geometry.links)

    def close(self):
        if self.h:
            lbm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_geometry(self, solid, links):
        lbm_set_geometry(self.h, solid, links)

    def init_equilibrium(self, rho=None, u=None):
        lbm_init_equilibrium(self.h, rho, u)

    def step(self, n=1):
        lbm_step(self.h, n)

    def step_forces(self, n, body=0):
        """n steps with the force on `body` after each one, (n, 3)."""
        return lbm_step_forces(self.h, n, body)

    def moments(self, rho=None, u=None):
        info = self.info()
        if rho is None:
            rho = np.empty(info.n_nodes)
            u = np.empty((info.D, info.n_nodes))
        lbm_moments(self.h, rho, u)
        return rho, u

    def force(self, body=0):
        return lbm_force(self.h, body)

    def forces(self, n=None):
        return lbm_forces(self.h, self.info().n_bodies if n is None else n)

    def autotune(self, steps_per_trial=20):
        return lbm_autotune(self.h, steps_per_trial)

    def set_tuning(self, **kw):
        lbm_set_tuning(self.h, **kw)

    def tuning(self):
        return lbm_get_tuning(self.h)

    def distributions(self):
        return lbm_get_distributions(self.h)

    def set_distributions(self, f):
        lbm_set_distributions(self.h, f)

    def check(self):
        lbm_check(self.h)

    def synchronize(self):
        lbm_synchronize(self.h)

    def info(self):
        return lbm_query(self.h)


def batch_lattice(batch, **cfg) -> Lattice:
    """Lattice over a stacked batch (``batch.Batch``): its domain table and
    geometry.  cfg's tau and inlet profile are placeholders (each domain has
    its own)."""
    cfg.setdefault("tau", 1.0)
    cfg.setdefault("inlet_y0", 0.0)
    cfg.setdefault("inlet_y1", 1.0)
    return Lattice(batch.geometry, domains=batch.domains, **cfg)
