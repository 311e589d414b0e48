"""FP64 CPU oracle for the VIBB lattice-Boltzmann step (arXiv:1903.01111).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py``.  The product path never imports it.

The oracle is plain C++ (``lbm_oracle.cpp``) compiled with g++; this module is
its ctypes shim.  It shares no code with the CUDA package: the only inputs both
sides read are the geometry arrays built by ``paper_1903_01111_gb300.geometry``
(mask and link list), which hold none of the method's arithmetic.

State convention (identical on both sides by definition, not by shared code):
``fp`` is the post-collision population array f+_i(x, t) laid out [Q][N] with
N = nx*ny*nz and node index x + nx*(y + ny*z); ``rho`` (N) and ``u`` (N, 3) are
the moments that the collision at time t used.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbm_oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

LINK_DTYPE = np.dtype(
    [("node", "<i8"), ("dir", "<i4"), ("bc", "<i2"), ("body", "<i2"), ("q", "<f8"), ("uw", "<f8", (3,))],
    align=True,
)
assert LINK_DTYPE.itemsize == 48


class OracleConfig(ctypes.Structure):
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
    ]


def build(force: bool = False) -> str:
    """Compile liboracle.so with g++ if it is missing or older than its source."""
    with _lock:
        if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
            tmp = _LIB + f".tmp{os.getpid()}"
            subprocess.check_call(["g++", "-O2", "-std=c++17", "-fopenmp", "-shared", "-fPIC", _SRC, "-o", tmp])
            os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        P = ctypes.POINTER
        d, i32, i64, u8 = ctypes.c_double, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint8
        lib.oracle_last_error.restype = ctypes.c_char_p
        lib.oracle_velocity_set.argtypes = [ctypes.c_int, P(i32), P(d)]
        lib.oracle_feq.argtypes = [ctypes.c_int, d, P(d), P(d)]
        lib.oracle_collide.argtypes = [P(OracleConfig), P(d), P(d), P(d), P(d)]
        lib.oracle_link_value.restype = d
        lib.oracle_link_value.argtypes = [P(OracleConfig), ctypes.c_int, ctypes.c_int, d, P(d), P(d), P(d), d, P(d),
                                          d, P(d)]
        lib.oracle_init.argtypes = [P(OracleConfig), P(u8), ctypes.c_void_p, ctypes.c_void_p, P(d), P(d), P(d)]
        lib.oracle_run.argtypes = [P(OracleConfig), P(u8), ctypes.c_void_p, i64, P(d), P(d), P(d), i64, P(d),
                                   ctypes.c_int]
        lib.oracle_moments.argtypes = [P(OracleConfig), P(u8), P(d), P(d), P(d)]
        lib.oracle_run_dual.argtypes = [P(OracleConfig), P(u8), ctypes.c_void_p, i64, P(d), P(d), ctypes.c_void_p,
                                        ctypes.c_void_p, i64, P(d), P(d), ctypes.c_int]
        lib.oracle_set_threads.argtypes = [ctypes.c_int]
        _lib = lib
    return _lib


def set_threads(n: int = 0) -> int:
    """OpenMP threads of the oracle's per-node passes (n <= 0: leave as is);
    returns the count now in use.  Results do not depend on it."""
    return int(_load().oracle_set_threads(int(n)))


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _check(rc):
    if rc != 0:
        raise RuntimeError("oracle: " + _load().oracle_last_error().decode())


def make_config(stencil=0, nx=1, ny=1, nz=1, periodic=(1, 1, 1), tau=0.8, rho0=1.0, g=(0.0, 0.0, 0.0), bc=2,
                collision=0, inlet=0, outlet=0, inlet_umax=0.0, inlet_y0=0.0, inlet_y1=0.0, vibb_density=0,
                precision=0) -> OracleConfig:
    c = OracleConfig()
    c.stencil, c.collision, c.bc = stencil, collision, bc
    c.nx, c.ny, c.nz = nx, ny, nz
    for a in range(3):
        c.periodic[a] = int(periodic[a])
        c.g[a] = float(g[a]) if a < len(g) else 0.0
    c.inlet, c.outlet = int(inlet), int(outlet)
    c.tau, c.rho0 = float(tau), float(rho0)
    c.inlet_umax, c.inlet_y0, c.inlet_y1 = float(inlet_umax), float(inlet_y0), float(inlet_y1)
    c.vibb_density = int(vibb_density)
    c.precision = int(precision)
    return c


def config_from(cfg: dict) -> OracleConfig:
    """Config from the plain dict used by the tests (keys as in make_config)."""
    return make_config(**cfg)


def nq(stencil: int) -> int:
    return 9 if stencil == 0 else 19


def velocity_set(stencil: int):
    q = nq(stencil)
    e = np.zeros((q, 3), np.int32)
    w = np.zeros(q, np.float64)
    _load().oracle_velocity_set(stencil, e.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), _dp(w))
    return e, w


def feq(stencil: int, rho: float, u) -> np.ndarray:
    out = np.zeros(nq(stencil))
    uu = np.zeros(3)
    uu[: len(u)] = u
    _load().oracle_feq(stencil, float(rho), _dp(uu), _dp(out))
    return out


def collide(cfg: OracleConfig, f):
    f = np.ascontiguousarray(f, np.float64)
    fp = np.zeros_like(f)
    rho = np.zeros(1)
    u = np.zeros(3)
    _check(_load().oracle_collide(ctypes.byref(cfg), _dp(f), _dp(fp), _dp(rho), _dp(u)))
    return fp, rho[0], u


def link_value(cfg: OracleConfig, rule, direction, q, uw, fp_f, fp_ff, rho_f, u_f, rho_ff, u_ff) -> float:
    def v3(a):
        out = np.zeros(3)
        out[: len(a)] = a
        return out

    uw, u_f, u_ff = v3(uw), v3(u_f), v3(u_ff)
    fp_f = np.ascontiguousarray(fp_f, np.float64)
    fp_ff = np.ascontiguousarray(fp_ff, np.float64)
    return _load().oracle_link_value(ctypes.byref(cfg), int(rule), int(direction), float(q), _dp(uw), _dp(fp_f),
                                     _dp(fp_ff), float(rho_f), _dp(u_f), float(rho_ff), _dp(u_ff))


class State:
    """Post-collision populations and moments at one time level."""

    def __init__(self, fp, rho, u):
        self.fp, self.rho, self.u = fp, rho, u

    def copy(self):
        return State(self.fp.copy(), self.rho.copy(), self.u.copy())


def init(cfg: OracleConfig, solid, rho=None, u=None) -> State:
    """f(x,0) = feq(rho, u) at fluid nodes, then the collision at t = 0."""
    N = cfg.nx * cfg.ny * cfg.nz
    solid = np.ascontiguousarray(solid, np.uint8).reshape(-1)
    assert solid.size == N
    fp = np.zeros(nq(cfg.stencil) * N)
    r = np.zeros(N)
    uu = np.zeros(3 * N)
    rho_p = None if rho is None else np.ascontiguousarray(rho, np.float64).reshape(-1)
    u_p = None if u is None else np.ascontiguousarray(u, np.float64).reshape(N, 3)
    _check(_load().oracle_init(ctypes.byref(cfg), solid.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)),
                               None if rho_p is None else rho_p.ctypes.data,
                               None if u_p is None else u_p.ctypes.data, _dp(fp), _dp(r), _dp(uu)))
    return State(fp.reshape(nq(cfg.stencil), N), r, uu.reshape(N, 3))


def run(cfg: OracleConfig, solid, links, state: State, nsteps: int, nbody: int = 1):
    """Advance ``state`` in place by ``nsteps``; returns the force (nbody, 3)
    of the last step (momentum exchange on every link with body >= 0)."""
    solid = np.ascontiguousarray(solid, np.uint8).reshape(-1)
    links = np.ascontiguousarray(links, dtype=LINK_DTYPE)
    force = np.zeros(max(nbody, 1) * 3)
    assert state.fp.flags.c_contiguous and state.u.flags.c_contiguous
    _check(_load().oracle_run(ctypes.byref(cfg), solid.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)),
                              links.ctypes.data if links.size else None, int(links.size), _dp(state.fp),
                              _dp(state.rho), _dp(state.u), int(nsteps), _dp(force), int(nbody)))
    return force.reshape(-1, 3)[:nbody]


def moments(cfg: OracleConfig, solid, fp):
    """rho and u of a post-collision state (see oracle_moments)."""
    N = cfg.nx * cfg.ny * cfg.nz
    solid = np.ascontiguousarray(solid, np.uint8).reshape(-1)
    fp = np.ascontiguousarray(fp, np.float64)
    r = np.zeros(N)
    uu = np.zeros(3 * N)
    _check(_load().oracle_moments(ctypes.byref(cfg), solid.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)),
                                  _dp(fp), _dp(r), _dp(uu)))
    return r, uu.reshape(N, 3)


def run_dual(cfg: OracleConfig, solid, links, dq, dtau, nsteps: int, nbody: int = 1, rho=None, u=None):
    """Forward-mode (dual number) derivatives of the force of the last of
    ``nsteps`` steps from the oracle_init state, with respect to 4 parameters:
    ``dq`` (n_links, 4) derivatives of each link's q, ``dtau`` (4,).
    Returns F (nbody, 3) and dF (nbody, 3, 4)."""
    N = cfg.nx * cfg.ny * cfg.nz
    solid = np.ascontiguousarray(solid, np.uint8).reshape(-1)
    links = np.ascontiguousarray(links, dtype=LINK_DTYPE)
    dq = np.ascontiguousarray(dq, np.float64).reshape(len(links), 4)
    dtau = np.ascontiguousarray(dtau, np.float64).reshape(4)
    F = np.zeros(nbody * 3)
    dF = np.zeros(nbody * 3 * 4)
    rho_p = None if rho is None else np.ascontiguousarray(rho, np.float64).reshape(N)
    u_p = None if u is None else np.ascontiguousarray(u, np.float64).reshape(N, 3)
    _check(_load().oracle_run_dual(ctypes.byref(cfg), solid.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)),
                                   links.ctypes.data if links.size else None, int(links.size), _dp(dq), _dp(dtau),
                                   None if rho_p is None else rho_p.ctypes.data,
                                   None if u_p is None else u_p.ctypes.data, int(nsteps), _dp(F), _dp(dF),
                                   int(nbody)))
    return F.reshape(nbody, 3), dF.reshape(nbody, 3, 4)
