"""Gradients of the force on a circular cylinder with respect to its centre,
its radius and the relaxation time, through the library's discrete adjoint
(lbm_adjoint_step) behind torch.autograd.Function.

The forward pass builds the geometry for theta = (c_x, c_y, R, tau), runs the
lattice for n_steps from its initial state and returns J = w . F (the
momentum-exchange force of the last step).  The same call runs the adjoint
sweep, whose per-link dJ/dq and dJ/dtau are mapped to dJ/dtheta with the
geometric derivatives dq/d(c, R) of the links on the cylinder
(geometry.ball_q_derivatives); backward returns grad_output * dJ/dtheta.
The derivative is that of the discrete map at fixed link topology: it is exact
as long as a perturbation of theta moves no node between fluid and solid.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import torch

from . import geometry as G
from . import lbm


@dataclass
class CylinderSpec:
    """What the forward pass simulates (everything except theta)."""

    kind: str = "channel"          # "channel" (inlet/outlet, half-way walls) or "periodic"
    nx: int = 1024
    ny_fluid: int = 256
    u_max: float = 0.1             # channel: peak inflow; periodic: unused
    g: tuple = (0.0, 0.0, 0.0)     # body force
    n_steps: int = 20000
    checkpoint_every: int = 500
    bc: int = lbm.LBM_BC_VIBB
    vibb_density: int = lbm.LBM_VIBB_RHO_PRINTED
    precision: int = lbm.LBM_FP32_SHIFTED
    direction: tuple = (1.0, 0.0, 0.0)   # J = direction . F (drag: x)
    last: dict = field(default_factory=dict)  # filled by the forward pass: timings, J, gradient parts


def build_geometry(spec: CylinderSpec, cx, cy, R):
    if spec.kind == "channel":
        geo = G.cylinder_channel(nx=spec.nx, ny_fluid=spec.ny_fluid, center=(cx, cy), radius=R, u_max=spec.u_max,
                                 bc=-1)
        return geo, 2  # bodies: two walls, then the cylinder
    geo = G.build(0, (spec.nx, spec.ny_fluid, 1), (1, 1, 1), [G.ball((cx, cy, 0.0), R, force_id=0)])
    return geo, 0


def _lattice_args(spec: CylinderSpec, theta):
    cx, cy, R, tau = [float(v) for v in theta]
    geo, bi = build_geometry(spec, cx, cy, R)
    kw = dict(tau=tau, g=spec.g, bc=spec.bc, precision=spec.precision, vibb_density=spec.vibb_density)
    u0 = None
    if spec.kind == "channel":
        kw.update(inlet_umax=spec.u_max, inlet_y0=0.5, inlet_y1=spec.ny_fluid + 0.5)
        y = (np.arange(geo.N) // geo.nx) % geo.ny
        u0 = np.zeros((geo.N, 3))
        H = spec.ny_fluid
        u0[:, 0] = np.where(geo.solid == 0, 4 * spec.u_max * (y - 0.5) * (H + 0.5 - y) / H ** 2, 0.0)
    return geo, bi, kw, u0


def branch_margin(spec: CylinderSpec, theta) -> float:
    """How far theta may move (first-order estimate, in theta's units) before
    a link on the cylinder reaches q = 1/2, where the VIBB and Bouzidi rules
    switch branch and J has a kink: min over links of |q - 1/2| / max_k
    |dq/dtheta_k|.  Central differences with steps well inside this margin
    see the same smooth branch as the adjoint."""
    geo, bi = build_geometry(spec, *[float(v) for v in theta[:3]])
    d = G.ball_q_derivatives(geo, bi)[:, [0, 1, 3]]
    on = np.abs(d).sum(axis=1) > 0
    q = geo.links["q"][on]
    return float(np.min(np.abs(q - 0.5) / np.abs(d[on]).max(axis=1)))


def force_only(spec: CylinderSpec, theta) -> float:
    """J for theta without the adjoint sweep (for finite differences)."""
    geo, _, kw, u0 = _lattice_args(spec, theta)
    with lbm.Lattice(geo, **kw) as lat:
        lat.init_equilibrium(u=u0)
        lat.step(spec.n_steps)
        F = lat.force(0)
    return float(np.dot(spec.direction, F))


def run(spec: CylinderSpec, theta):
    """J and dJ/dtheta for theta = (c_x, c_y, R, tau) (numpy, FP64)."""
    geo, bi, kw, u0 = _lattice_args(spec, theta)
    with lbm.Lattice(geo, **kw) as lat:
        lat.init_equilibrium(u=u0)
        J, dJdq, dJdtau, sec = lbm.lbm_adjoint_step(lat.h, 0, spec.direction, spec.n_steps, spec.checkpoint_every)
    dq = G.ball_q_derivatives(geo, bi)
    grad = np.array([dJdq @ dq[:, 0], dJdq @ dq[:, 1], dJdq @ dq[:, 3], dJdtau])
    # sum over links of |term| / |sum of terms| for c_x, c_y, R: how much a
    # relative error of the per-link sensitivities grows in each component
    terms = dJdq[:, None] * dq[:, [0, 1, 3]]
    cancel = np.abs(terms).sum(axis=0) / np.maximum(np.abs(terms.sum(axis=0)), 1e-300)
    spec.last = dict(J=J, grad=grad, seconds=sec, n_links=len(geo.links), n_fluid=geo.fluid_count(),
                     cancellation=cancel)
    return J, grad


class CylinderForce(torch.autograd.Function):
    """J(theta) = direction . F on the cylinder after spec.n_steps steps."""

    @staticmethod
    def forward(ctx, theta: torch.Tensor, spec: CylinderSpec):
        J, grad = run(spec, theta.detach().cpu().double().numpy())
        ctx.save_for_backward(torch.as_tensor(grad, dtype=theta.dtype, device=theta.device))
        return theta.new_tensor(J)

    @staticmethod
    def backward(ctx, grad_out):
        (g,) = ctx.saved_tensors
        return grad_out * g, None


def cylinder_force(theta: torch.Tensor, spec: CylinderSpec) -> torch.Tensor:
    return CylinderForce.apply(theta, spec)
