"""Batches of independent D2Q9 channel flows past cylinders, packed into one
lattice (lbm_set_domains) so that one launch per kernel advances all of them.

The paper simulates one flow at a time (flow past a cylinder in a channel,
Sec. 4.3).  A batch stacks many such channels of different sizes, cylinder
layouts and Reynolds numbers along y: domain d occupies rows
[lo_d, lo_d + ny_d + 2) (its two solid wall rows included) and columns
x < nx_d; the columns beyond are solid.  Its walls keep every population
inside its rows, so the domains evolve exactly as they would alone.

This module draws the workload and maps between per-domain and stacked
indices; it holds none of the lattice-Boltzmann arithmetic.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import geometry as G


@dataclass
class DomainSpec:
    """One channel: nx x (ny_fluid + 2) nodes, cylinders (c_x, c_y, R) in
    fluid-row coordinates, peak inflow u_max and Reynolds number Re on the
    channel height and the mean inflow 2/3 u_max (tau = 3 nu + 1/2)."""

    nx: int
    ny_fluid: int
    cylinders: list
    re: float
    u_max: float = 0.1

    @property
    def nu(self) -> float:
        return (2.0 / 3.0) * self.u_max * self.ny_fluid / self.re

    @property
    def tau(self) -> float:
        return 3.0 * self.nu + 0.5

    @property
    def ny(self) -> int:
        return self.ny_fluid + 2

    def geometry(self, bc=-1) -> G.Geometry:
        return G.cylinders_channel(self.nx, self.ny_fluid, self.cylinders, u_max=self.u_max, bc=bc)

    def inlet(self) -> dict:
        """Inlet profile in the domain's own rows (walls at 1/2 and ny_fluid + 1/2)."""
        return dict(inlet_umax=self.u_max, inlet_y0=0.5, inlet_y1=self.ny_fluid + 0.5)

    def initial_velocity(self, geo: G.Geometry) -> np.ndarray:
        """Poiseuille profile of the inflow on every fluid node, (N, 3)."""
        y = (np.arange(geo.N) // geo.nx) % geo.ny
        H = self.ny_fluid
        u = np.zeros((geo.N, 3))
        u[:, 0] = np.where(geo.solid == 0, 4 * self.u_max * (y - 0.5) * (H + 0.5 - y) / H ** 2, 0.0)
        return u


def draw_channels(n_domains=256, seed=0, nx_range=(64, 512), ny_range=(64, 256), n_cyl=(1, 8), r_range=(4.0, 20.0),
                  re_range=(10.0, 100.0), u_max=0.1, gap=3.0, max_blockage=0.4, max_tries=400) -> list:
    """Seeded channel workload: sizes uniform in nx_range x ny_range (fluid
    rows), 1..8 non-overlapping cylinders per channel with radii uniform in
    r_range (capped at ny/6 and nx/4) and off-grid centres at least ``gap``
    apart and from the walls, kept clear of the inlet and outlet, Re uniform
    in re_range.  The cylinders whose x-extents overlap block at most
    ``max_blockage`` of the channel height (the flow through the remaining
    gaps speeds up by 1/(1 - blockage); a nearly closed channel would push
    the lattice Mach number past what BGK tolerates)."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n_domains):
        nx = int(rng.integers(nx_range[0], nx_range[1] + 1))
        ny = int(rng.integers(ny_range[0], ny_range[1] + 1))
        want = int(rng.integers(n_cyl[0], n_cyl[1] + 1))
        rmax = min(r_range[1], ny / 6.0, nx / 4.0)
        cyl = []
        tries = 0
        while len(cyl) < want and tries < max_tries:
            tries += 1
            r = min(float(rng.uniform(r_range[0], max(r_range[0], rmax))), rmax)
            x_lo, x_hi = r + 8.0, nx - r - 16.0
            y_lo, y_hi = r + gap, ny - 1 - r - gap
            if x_hi <= x_lo or y_hi <= y_lo:
                continue
            c = (float(rng.uniform(x_lo, x_hi)), float(rng.uniform(y_lo, y_hi)))
            if any((c[0] - a) ** 2 + (c[1] - b) ** 2 < (r + rr + gap) ** 2 for a, b, rr in cyl):
                continue
            if _max_chord(cyl + [(c[0], c[1], r)]) > max_blockage * ny:
                continue
            cyl.append((c[0], c[1], r))
        if not cyl:
            raise RuntimeError("could not place a cylinder")
        out.append(DomainSpec(nx, ny, cyl, float(rng.uniform(*re_range)), u_max))
    return out


def _max_chord(cylinders) -> float:
    """Largest total height that the cylinders cover on one vertical line."""
    xs = np.concatenate([np.linspace(a - r, a + r, 65) for a, _, r in cylinders])
    h = np.zeros_like(xs)
    for a, _, r in cylinders:
        h += 2.0 * np.sqrt(np.clip(r * r - (xs - a) ** 2, 0.0, None))
    return float(h.max())


def blockage(spec: DomainSpec) -> float:
    """Largest fraction of the channel height that the cylinders cover on
    one vertical line."""
    return _max_chord(spec.cylinders) / spec.ny_fluid


@dataclass
class Batch:
    """Stacked geometry of a list of DomainSpec and the maps back."""

    specs: list
    geometry: G.Geometry          # the stacked lattice
    domains: list                 # lbm_domain rows (dicts)
    lo: np.ndarray                # first storage row of each domain
    body0: np.ndarray             # first body id of each domain
    n_fluid: int
    parts: list = field(default_factory=list)  # per-domain geometries

    @property
    def n_bodies(self) -> int:
        return int(self.body0[-1] + len(self.specs[-1].cylinders)) if self.specs else 0

    def domain_nodes(self, d: int) -> np.ndarray:
        """Stacked node index of every node of domain d, in the domain's own
        node order (x + nx_d y)."""
        s = self.specs[d]
        y, x = np.divmod(np.arange(s.nx * s.ny), s.nx)
        return x + self.geometry.nx * (y + int(self.lo[d]))

    def domain_links(self, d: int) -> np.ndarray:
        """Indices into the stacked link list of domain d's links, in the
        domain's own link order."""
        return np.arange(self._link0[d], self._link0[d + 1])

    def initial_velocity(self) -> np.ndarray:
        u = np.zeros((self.geometry.N, 3))
        for d, (s, g) in enumerate(zip(self.specs, self.parts)):
            u[self.domain_nodes(d)] = s.initial_velocity(g)
        return u


def stack(specs, bc=-1, g=(0.0, 0.0, 0.0)) -> Batch:
    """Stack the channels along y into one lattice of width max nx_d."""
    parts = [s.geometry(bc=bc) for s in specs]
    NX = max(s.nx for s in specs)
    NY = sum(s.ny for s in specs)
    solid = np.ones(NX * NY, np.uint8)
    links = []
    lo = np.zeros(len(specs), np.int64)
    body0 = np.zeros(len(specs), np.int64)
    link0 = [0]
    rows, y0, b0, n_fluid = [], 0, 0, 0
    for d, (s, geo) in enumerate(zip(specs, parts)):
        lo[d], body0[d] = y0, b0
        m = geo.solid.reshape(s.ny, s.nx)
        solid.reshape(NY, NX)[y0:y0 + s.ny, :s.nx] = m
        lk = geo.links.copy()
        x, y = lk["node"] % s.nx, lk["node"] // s.nx
        lk["node"] = x + NX * (y + y0)
        lk["body"] = np.where(lk["body"] >= 0, lk["body"] + b0, -1)
        links.append(lk)
        link0.append(link0[-1] + len(lk))
        rows.append(dict(lo=y0, n=s.ny, nx=s.nx, tau=s.tau, g=g, **s.inlet()))
        n_fluid += geo.fluid_count()
        y0 += s.ny
        b0 += len(s.cylinders)
    geo = G.Geometry(G.D2Q9, NX, NY, 1, (False, False, True), solid,
                     np.concatenate(links) if links else np.zeros(0, G.LINK_DTYPE), (True, True), None,
                     dict(kind="channel_batch", domains=len(specs)))
    b = Batch(specs, geo, rows, lo, body0, n_fluid, parts)
    b._link0 = np.array(link0)
    return b


def shard(specs, rank: int, world: int) -> list:
    """Domains of one rank when a batch is split across ranks (no exchange
    between domains): every world-th domain, starting at rank."""
    return list(specs[rank::world])
