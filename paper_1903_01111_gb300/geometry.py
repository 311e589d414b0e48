"""Seeded geometry and input generators: solid masks, cut-link lists with the
wall fraction q (Sec. 3 of arXiv:1903.01111: fluid, solid and boundary nodes;
q = |x_f - x_w| / |x_f - x_s|), random sphere packs and initial fields.

This module computes geometry only; it holds none of the lattice-Boltzmann
arithmetic.  Its output is the input of both the CUDA library and the CPU
oracle.  The ray-body intersections run in a small host C file
(``csrc/geometry.c``) compiled into ``libgeom.so``.

Conventions shared by the whole package (and documented in include/lbm.h):

* node index n = x + nx*(y + ny*z); node x sits at integer coordinates;
* D2Q9 directions e1=(1,0) e2=(0,1) e3=(-1,0) e4=(0,-1) e5=(1,1) e6=(-1,1)
  e7=(-1,-1) e8=(1,-1) (the order of the moment matrix M in Sec. 2);
* D3Q19 directions: rest, +-x, +-y, +-z, then (+-1,+-1,0), (+-1,0,+-1),
  (0,+-1,+-1) with opposite directions adjacent;
* a link (node, dir) has its solid neighbour at node + e_dir.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "csrc", "geometry.c")
_LIB = os.path.join(_HERE, "libgeom.so")
_lock = threading.Lock()
_lib = None

LINK_DTYPE = np.dtype(
    [("node", "<i8"), ("dir", "<i4"), ("bc", "<i2"), ("body", "<i2"), ("q", "<f8"), ("uw", "<f8", (3,))],
    align=True,
)
BODY_DTYPE = np.dtype(
    [("kind", "<i4"), ("force_id", "<i4"), ("bc", "<i4"), ("pad", "<i4"), ("c", "<f8", (3,)), ("r", "<f8"),
     ("vel", "<f8", (3,)), ("omega", "<f8", (3,))],
    align=True,
)
assert LINK_DTYPE.itemsize == 48 and BODY_DTYPE.itemsize == 96

D2Q9 = 0
D3Q19 = 1
BALL, HALFSPACE, CAVITY = 0, 1, 2


def build_lib(force: bool = False) -> str:
    with _lock:
        if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
            tmp = _LIB + f".tmp{os.getpid()}"
            subprocess.check_call(["gcc", "-O2", "-std=c11", "-fopenmp", "-shared", "-fPIC", _SRC, "-o", tmp, "-lm"])
            os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build_lib()
        lib = ctypes.CDLL(_LIB)
        vp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
        lib.geom_mask.restype = i64
        lib.geom_mask.argtypes = [i32, i32, i32, i32, vp, vp, i32, vp]
        lib.geom_pack_add.restype = i64
        lib.geom_pack_add.argtypes = [i32, i32, i32, vp, vp, vp, i64, i64, vp, ctypes.POINTER(i64)]
        lib.geom_links.restype = i64
        lib.geom_links.argtypes = [i32, i32, i32, i32, vp, vp, i32, vp, i32, i32, vp, ctypes.POINTER(i64)]
        _lib = lib
    return _lib


def ball(center, radius, vel=(0.0, 0.0, 0.0), omega=(0.0, 0.0, 0.0), force_id=0, bc=-1):
    """Closed ball |x - c| <= R (a circle in 2-D) moving rigidly with velocity
    ``vel`` and angular velocity ``omega`` about its centre."""
    b = np.zeros((), BODY_DTYPE)
    b["kind"], b["force_id"], b["bc"] = BALL, force_id, bc
    b["c"][: len(center)] = center
    b["r"] = radius
    b["vel"][: len(vel)] = vel
    b["omega"][: len(omega)] = omega
    return b


def cavity(center, radius, vel=(0.0, 0.0, 0.0), omega=(0.0, 0.0, 0.0), force_id=-1, bc=-1):
    """Solid everywhere outside the ball |x - c| < R (the outer cylinder of a
    Couette cell)."""
    b = ball(center, radius, vel, omega, force_id, bc)
    b["kind"] = CAVITY
    return b


def halfspace(normal, offset, vel=(0.0, 0.0, 0.0), force_id=-1, bc=-1):
    """Solid where n . x >= offset; ``normal`` points into the solid."""
    b = np.zeros((), BODY_DTYPE)
    n = np.zeros(3)
    n[: len(normal)] = normal
    n /= np.linalg.norm(n)
    b["kind"], b["force_id"], b["bc"] = HALFSPACE, force_id, bc
    b["c"] = n
    b["r"] = offset
    b["vel"][: len(vel)] = vel
    return b


@dataclass
class Geometry:
    stencil: int
    nx: int
    ny: int
    nz: int
    periodic: tuple
    solid: np.ndarray          # uint8 (N,), 1 = solid
    links: np.ndarray          # LINK_DTYPE (n_links,), sorted by (node, dir)
    open_x: tuple = (False, False)
    bodies: np.ndarray = None
    info: dict = field(default_factory=dict)

    @property
    def N(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def shape(self):
        return (self.nx, self.ny, self.nz)

    def fluid_count(self) -> int:
        n = int(self.N - int(self.solid.sum()))
        if self.open_x[0] or self.open_x[1]:
            s = self.solid.reshape(self.nz, self.ny, self.nx)
            if self.open_x[0]:
                n -= int((s[:, :, 0] == 0).sum())
            if self.open_x[1]:
                n -= int((s[:, :, -1] == 0).sum())
        return n

    def coords(self, node):
        node = np.asarray(node, np.int64)
        return node % self.nx, (node // self.nx) % self.ny, node // (self.nx * self.ny)


def _mask_from_bodies(stencil, shape, periodic, bodies):
    nx, ny, nz = shape
    per = np.asarray(periodic, np.int32)
    balls = bodies[bodies["kind"] != CAVITY]
    mask = np.zeros(nx * ny * nz, np.uint8)
    if balls.size:
        rc = _load().geom_mask(stencil, nx, ny, nz, per.ctypes.data, balls.ctypes.data, int(balls.size),
                               mask.ctypes.data)
        if rc < 0:
            raise MemoryError("geom_mask failed")
    for b in bodies[bodies["kind"] == CAVITY]:
        x = np.arange(nx, dtype=np.float64)[None, None, :]
        y = np.arange(ny, dtype=np.float64)[None, :, None]
        z = np.arange(nz, dtype=np.float64)[:, None, None]
        d = [x - b["c"][0], y - b["c"][1], z - b["c"][2]]
        for a, L in enumerate((nx, ny, nz)):
            if periodic[a]:
                d[a] = d[a] - L * np.floor(d[a] / L + 0.5)
        r2 = d[0] ** 2 + d[1] ** 2 + d[2] ** 2
        mask |= (r2 >= b["r"] ** 2).reshape(-1).astype(np.uint8)
    return mask


def _links(stencil, shape, periodic, bodies, mask, open_x):
    nx, ny, nz = shape
    per = np.asarray(periodic, np.int32)
    # The wall crossing of a link is searched on each ball's nearest periodic
    # image as seen from x_f; the node classes use the nearest image as seen
    # from each node.  The two agree for x_f and its neighbours when every
    # point within one lattice step of the ball lies within half a period of
    # its centre: radius below half the period minus one on each periodic
    # axis.  A larger ball would leave a solid neighbour without a crossing.
    for b in bodies[(bodies["kind"] == BALL) | (bodies["kind"] == CAVITY)]:
        for a in range(3 if stencil == D3Q19 else 2):
            if periodic[a] and not (b["r"] < shape[a] / 2.0 - 1.0):
                raise ValueError(f"ball of radius {float(b['r']):g} at {tuple(float(v) for v in b['c'])}: on the "
                                 f"periodic axis {a} (period {shape[a]}) the radius must be below "
                                 f"{shape[a] / 2.0 - 1.0:g}, half the period minus one")
    # cavities are handled by the C builder as balls with the entry root
    # replaced by the exit root; do that here in Python: split the work.
    lib = _load()
    err = ctypes.c_int64(0)
    cav = bodies[bodies["kind"] == CAVITY]
    rest = np.ascontiguousarray(bodies[bodies["kind"] != CAVITY])
    if cav.size == 0:
        n = lib.geom_links(stencil, nx, ny, nz, per.ctypes.data, rest.ctypes.data, int(rest.size), mask.ctypes.data,
                           int(open_x[0]), int(open_x[1]), None, ctypes.byref(err))
        if n < 0:
            raise ValueError(_link_error(n, err.value, shape))
        out = np.zeros(n, LINK_DTYPE)
        n2 = lib.geom_links(stencil, nx, ny, nz, per.ctypes.data, rest.ctypes.data, int(rest.size),
                            mask.ctypes.data, int(open_x[0]), int(open_x[1]), out.ctypes.data, ctypes.byref(err))
        if n2 < 0:  # the filling pass's crossing search failed
            raise ValueError(_link_error(n2, err.value, shape))
        assert n2 == n
        return out
    return _links_python(stencil, shape, periodic, bodies, mask, open_x)


def _link_error(code, node, shape):
    nx, ny, _ = shape
    xyz = (node % nx, (node // nx) % ny, node // (nx * ny))
    if code == -2:
        return f"fluid node {xyz} has a neighbour outside a non-periodic face: add a solid layer"
    if code == -3:
        return f"fluid node {xyz}: solid neighbour without a wall crossing"
    return "geometry builder out of memory"


def velocity_set(stencil):
    if stencil == D2Q9:
        e = [(0, 0, 0), (1, 0, 0), (0, 1, 0), (-1, 0, 0), (0, -1, 0), (1, 1, 0), (-1, 1, 0), (-1, -1, 0), (1, -1, 0)]
    else:
        e = [(0, 0, 0), (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1), (1, 1, 0), (-1, -1, 0),
             (1, -1, 0), (-1, 1, 0), (1, 0, 1), (-1, 0, -1), (1, 0, -1), (-1, 0, 1), (0, 1, 1), (0, -1, -1),
             (0, 1, -1), (0, -1, 1)]
    return np.array(e, np.int64)


def _entry_t(b, xf, e, shape, periodic):
    """Entry parameter t in (0, 1+eps] of xf + t e into body b, or -1."""
    d = np.asarray(xf, np.float64) - b["c"]
    for a, L in enumerate(shape):
        if periodic[a]:
            d[a] -= L * np.floor(d[a] / L + 0.5)
    if b["kind"] == HALFSPACE:
        nd = float(np.dot(b["c"], e))
        if nd <= 0:
            return -1.0
        t = (b["r"] - float(np.dot(b["c"], xf))) / nd
        return t if t > 0 else -1.0
    A = float(np.dot(e, e))
    B = float(np.dot(d, e))
    C = float(np.dot(d, d)) - b["r"] ** 2
    disc = B * B - A * C
    if disc < 0:
        return -1.0
    sq = np.sqrt(disc)
    if b["kind"] == BALL:
        t = C / (-B + sq) if B <= 0 else (-B - sq) / A
    else:  # cavity: leave the ball (larger root); C < 0 inside
        t = (-B + sq) / A if B >= 0 else C / (-B - sq)
    return t if t > 0 else -1.0


def _wall_velocity(b, xw, shape, periodic):
    uw = b["vel"].copy()
    if b["kind"] != HALFSPACE:
        r = np.asarray(xw, np.float64) - b["c"]
        for a, L in enumerate(shape):
            if periodic[a]:
                r[a] -= L * np.floor(r[a] / L + 0.5)
        uw = uw + np.cross(b["omega"], r)
    return uw


def _links_python(stencil, shape, periodic, bodies, mask, open_x):
    """Plain per-link loop (used when a cavity body is present; small cases)."""
    nx, ny, nz = shape
    E = velocity_set(stencil)
    L = np.array(shape)
    out = []
    m3 = mask.reshape(nz, ny, nx)
    for n in np.flatnonzero(mask == 0):
        xi = np.array([n % nx, (n // nx) % ny, n // (nx * ny)])
        if (open_x[0] and xi[0] == 0) or (open_x[1] and xi[0] == nx - 1):
            continue
        for d in range(1, len(E)):
            s = xi + E[d]
            oob = (s < 0) | (s >= L)
            if np.any(oob & ~np.asarray(periodic, bool)):
                if (s[0] < 0 and open_x[0]) or (s[0] >= nx and open_x[1]):
                    continue
                raise ValueError(_link_error(-2, int(n), shape))
            s = s % L
            if not m3[s[2], s[1], s[0]]:
                continue
            best, bb = 2.0, None
            for b in bodies:
                t = _entry_t(b, xi.astype(np.float64), E[d].astype(np.float64), shape, periodic)
                if 0 < t < best:
                    best, bb = t, b
            if bb is None or best > 1 + 1e-9:
                raise ValueError(_link_error(-3, int(n), shape))
            best = min(best, 1.0)
            rec = np.zeros((), LINK_DTYPE)
            rec["node"], rec["dir"], rec["bc"], rec["body"], rec["q"] = n, d, bb["bc"], bb["force_id"], best
            rec["uw"] = _wall_velocity(bb, xi + best * E[d], shape, periodic)
            out.append(rec)
    return np.array(out, LINK_DTYPE) if out else np.zeros(0, LINK_DTYPE)


def build(stencil, shape, periodic, bodies, open_x=(False, False), info=None) -> Geometry:
    """Mask and cut links for a list of bodies on an nx x ny x nz lattice."""
    nx, ny, nz = shape
    if stencil == D2Q9 and nz != 1:
        raise ValueError("D2Q9 needs nz == 1")
    bodies = np.ascontiguousarray(np.array(bodies, BODY_DTYPE).reshape(-1))
    periodic = tuple(bool(p) for p in periodic)
    mask = _mask_from_bodies(stencil, shape, periodic, bodies)
    links = _links(stencil, shape, periodic, bodies, mask, open_x)
    return Geometry(stencil, nx, ny, nz, periodic, mask, links, tuple(bool(o) for o in open_x), bodies,
                    dict(info or {}))


# --------------------------------------------------------------- workloads --

def channel(stencil, nx, ny_fluid, nz=1, q_lo=0.5, q_hi=0.5, u_lo=(0.0, 0.0, 0.0), u_hi=(0.0, 0.0, 0.0),
            bc_lo=-1, bc_hi=-1, force_lo=0, force_hi=0, open_x=(False, False)) -> Geometry:
    """Plane channel, walls normal to y.  Storage has one solid row below and
    above the ny_fluid fluid rows (rows 1..ny_fluid); the bottom wall sits at
    y = 1 - q_lo and the top wall at y = ny_fluid + q_hi, so q_lo and q_hi are
    the link fractions of the first and last fluid rows.  Periodic in x unless
    open_x, periodic in z."""
    ny = ny_fluid + 2
    bodies = [halfspace((0, -1, 0), -(1.0 - q_lo), vel=u_lo, force_id=force_lo, bc=bc_lo),
              halfspace((0, 1, 0), ny_fluid + q_hi, vel=u_hi, force_id=force_hi, bc=bc_hi)]
    per = (not (open_x[0] or open_x[1]), False, True)
    g = build(stencil, (nx, ny, nz), per, bodies, open_x=open_x,
              info=dict(kind="channel", y_lo=1.0 - q_lo, y_hi=ny_fluid + q_hi))
    return g


def poiseuille_profile(y, y_lo, y_hi, g, nu, u_top=0.0):
    """Steady plane Poiseuille velocity between walls at y_lo (fixed) and y_hi
    (moving at u_top), driven by body force g (Sec. 4.1, Eq. exact, written
    with the wall at y_lo)."""
    s = np.asarray(y, np.float64) - y_lo
    H = y_hi - y_lo
    return -g / (2 * nu) * s * s + (g * H / (2 * nu) + u_top / H) * s


def cylinder_channel(nx=2000, ny_fluid=400, center=(400.37, 200.61), radius=20.3, u_max=0.1, bc=-1,
                     omega=0.0) -> Geometry:
    """Flow past a circular cylinder in a channel: half-way walls at half a
    link below the first and above the last fluid row, velocity inlet at
    x = 0 and zero-gradient outlet at x = nx-1.  ``center`` is given in
    fluid-row coordinates (first fluid row at y = 0); storage adds one solid
    row at the bottom, so the storage centre is y + 1."""
    ny = ny_fluid + 2
    cy = center[1] + 1.0
    bodies = [halfspace((0, -1, 0), -0.5, force_id=-1, bc=0),
              halfspace((0, 1, 0), ny_fluid + 0.5, force_id=-1, bc=0),
              ball((center[0], cy, 0.0), radius, omega=(0.0, 0.0, omega), force_id=0, bc=bc)]
    g = build(D2Q9, (nx, ny, 1), (False, False, True), bodies, open_x=(True, True),
              info=dict(kind="cylinder", y_lo=0.5, y_hi=ny_fluid + 0.5, u_max=u_max, radius=radius,
                        center=(center[0], cy)))
    return g


def cylinders_channel(nx, ny_fluid, cylinders, u_max=0.1, bc=-1) -> Geometry:
    """The channel of ``cylinder_channel`` holding several cylinders:
    ``cylinders`` lists (c_x, c_y, R) in fluid-row coordinates; cylinder k
    gets force id k.  Bodies: the two walls, then the cylinders in order."""
    ny = ny_fluid + 2
    bodies = [halfspace((0, -1, 0), -0.5, force_id=-1, bc=0),
              halfspace((0, 1, 0), ny_fluid + 0.5, force_id=-1, bc=0)]
    for k, (cx, cy, r) in enumerate(cylinders):
        bodies.append(ball((cx, cy + 1.0, 0.0), r, force_id=k, bc=bc))
    return build(D2Q9, (nx, ny, 1), (False, False, True), bodies, open_x=(True, True),
                 info=dict(kind="cylinders", y_lo=0.5, y_hi=ny_fluid + 0.5, u_max=u_max,
                           cylinders=[tuple(map(float, c)) for c in cylinders]))


def couette(L, omega1, offset=(0.13, 0.27), bc=-1) -> Geometry:
    """Cylindrical Couette cell of Sec. 4.2: inner cylinder of radius L/4.8
    rotating at omega1 inside a fixed outer cylinder of radius L/2.4.  Only
    the annulus holds fluid, so the lattice is the smallest square around the
    outer cylinder plus a solid margin; the common centre sits ``offset``
    from the lattice centre so the link fractions q are generic."""
    r1, r2 = L / 4.8, L / 2.4
    n = int(np.ceil(2 * r2 + 4))
    c = (n / 2.0 + offset[0], n / 2.0 + offset[1], 0.0)
    bodies = [ball(c, r1, omega=(0, 0, omega1), force_id=0, bc=bc), cavity(c, r2, force_id=1, bc=bc)]
    return build(D2Q9, (n, n, 1), (True, True, True), bodies,
                 info=dict(kind="couette", r1=r1, r2=r2, center=c[:2], omega1=omega1))


def couette_profile(r, r1, r2, omega1):
    """Azimuthal velocity of Sec. 4.2, Eq. (exact2)."""
    r = np.asarray(r, np.float64)
    return omega1 * r1 * (r1 * r2 / (r2 ** 2 - r1 ** 2)) * (r2 / r - r / r2)


def sphere_pack(n=384, porosity=0.40, rmin=6.0, rmax=14.0, seed=0, batch=4096) -> Geometry:
    """Periodic random packing of overlapping spheres, radii U[rmin, rmax] and
    centres U[0, n)^3 drawn from ``seed``, added in sequence until the fluid
    fraction of the lattice nodes is at most ``porosity``."""
    rng = np.random.default_rng(seed)
    shape = (n, n, n)
    per = np.array([1, 1, 1], np.int32)
    N = n ** 3
    target = int(np.ceil((1.0 - porosity) * N))
    mask = np.zeros(N, np.uint8)
    solid = ctypes.c_int64(0)
    centres_all, radii_all = [], []
    lib = _load()
    while solid.value < target:
        c = np.ascontiguousarray(rng.uniform(0.0, n, size=(batch, 3)))
        r = np.ascontiguousarray(rng.uniform(rmin, rmax, size=batch))
        used = lib.geom_pack_add(n, n, n, per.ctypes.data, c.ctypes.data, r.ctypes.data, batch, target,
                                 mask.ctypes.data, ctypes.byref(solid))
        centres_all.append(c[:used])
        radii_all.append(r[:used])
    centres = np.concatenate(centres_all)
    radii = np.concatenate(radii_all)
    bodies = np.zeros(len(radii), BODY_DTYPE)
    bodies["kind"] = BALL
    bodies["force_id"] = 0
    bodies["bc"] = -1
    bodies["c"] = centres
    bodies["r"] = radii
    links = _links(D3Q19, shape, (True, True, True), bodies, mask, (False, False))
    return Geometry(D3Q19, n, n, n, (True, True, True), mask, links, (False, False), bodies,
                    dict(kind="sphere_pack", porosity=1.0 - solid.value / N, spheres=len(radii), seed=seed))


def translated(geo: Geometry, shift) -> Geometry:
    """The same geometry moved by an integer shift (sx, sy, sz) along its
    periodic axes: the mask is rolled and every link keeps its direction, q
    and wall velocity at the moved node (no ray casting, so the link data are
    bit for bit those of ``geo``)."""
    sh = [int(v) for v in shift] + [0] * (3 - len(shift))
    for a in range(3):
        if sh[a] and not geo.periodic[a]:
            raise ValueError(f"axis {a} is not periodic")
    solid = np.roll(geo.solid.reshape(geo.nz, geo.ny, geo.nx), (sh[2], sh[1], sh[0]), axis=(0, 1, 2)).reshape(-1)
    x, y, z = geo.coords(geo.links["node"])
    links = geo.links.copy()
    links["node"] = (x + sh[0]) % geo.nx + geo.nx * (((y + sh[1]) % geo.ny) + geo.ny * ((z + sh[2]) % geo.nz))
    order = np.lexsort((links["dir"], links["node"]))
    return Geometry(geo.stencil, geo.nx, geo.ny, geo.nz, geo.periodic, solid, links[order], geo.open_x, geo.bodies,
                    dict(geo.info, shift=tuple(sh)))


def ball_q_derivatives(geo: Geometry, body_index: int) -> np.ndarray:
    """Derivatives of q with respect to (c_x, c_y, c_z, R) of ball
    ``geo.bodies[body_index]`` for every link whose wall crossing lies on that
    ball (zero rows elsewhere): with d = x_w - c and x_w = x_f + q e,
    |x_f + q e - c|^2 = R^2 gives dq/dc = d / (d.e) and dq/dR = R / (d.e)."""
    b = geo.bodies[body_index]
    E = velocity_set(geo.stencil).astype(np.float64)
    out = np.zeros((len(geo.links), 4))
    x, y, z = geo.coords(geo.links["node"])
    xf = np.stack([x, y, z], 1).astype(np.float64)
    e = E[geo.links["dir"]]
    xw = xf + geo.links["q"][:, None] * e
    d = xw - b["c"]
    for a, L in enumerate(geo.shape):
        if geo.periodic[a]:
            d[:, a] -= L * np.floor(d[:, a] / L + 0.5)
    on = np.abs(np.sqrt((d * d).sum(1)) - b["r"]) < 1e-9 * max(1.0, b["r"])
    de = (d * e).sum(1)
    out[on, :3] = d[on] / de[on, None]
    out[on, 3] = b["r"] / de[on]
    return out
