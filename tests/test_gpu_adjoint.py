"""The GPU discrete adjoint (lbm_adjoint_step) against the oracle's
forward-mode dual-number derivatives (FP64, tight), against central finite
differences of the GPU forward map (C4-style channel, the 1e-4 target), and
its FP32-shifted version against FP64; checkpoint spacing does not change
the result."""
import numpy as np
import pytest

import oracle as O
from paper_1903_01111_gb300 import geometry as G

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1903_01111_gb300 import lbm

    return lbm


def _grad_gpu(L, geo, bi, kw, n, K=1000, direction=(1.0, 0.0, 0.0), u0=None, precision=None):
    kw = dict(kw)
    if precision is not None:
        kw["precision"] = precision
    with L.Lattice(geo, **kw) as lat:
        lat.init_equilibrium(u=u0)
        J, dq, dtau, sec = L.lbm_adjoint_step(lat.h, 0, direction, n, K)
    d = G.ball_q_derivatives(geo, bi)
    return J, np.array([dq @ d[:, 0], dq @ d[:, 1], dq @ d[:, 3], dtau]), sec


def _grad_oracle(geo, bi, kw, n, comp=0, u0=None):
    d = G.ball_q_derivatives(geo, bi)
    dq = np.zeros((len(geo.links), 4))
    dq[:, 0], dq[:, 1], dq[:, 2] = d[:, 0], d[:, 1], d[:, 3]
    cfg = O.make_config(stencil=geo.stencil, nx=geo.nx, ny=geo.ny, nz=geo.nz, periodic=geo.periodic,
                        inlet=geo.open_x[0], outlet=geo.open_x[1], **kw)
    F, dF = O.run_dual(cfg, geo.solid, geo.links, dq, [0, 0, 0, 1.0], n, u=u0)
    return F[0, comp], dF[0, comp]


def _close(a, b, rel):
    a, b = np.asarray(a), np.asarray(b)
    return np.all(np.abs(a - b) <= rel * np.abs(b) + rel * 1e-3 * np.abs(b).max())


CASES = {
    "vibb": dict(bc=2),
    "vibb_local": dict(bc=2, vibb_density=1),
    "bouzidi": dict(bc=1),
    "halfway": dict(bc=0),
    "yu": dict(bc=3),
}


@pytest.mark.parametrize("rule", list(CASES))
def test_adjoint_matches_dual_numbers_periodic_cylinder(L, rule):
    geo = G.build(0, (34, 24, 1), (1, 1, 1), [G.ball((15.37, 11.61, 0), 5.23, force_id=0)])
    kw = dict(tau=0.72, g=(2e-5, 0.0, 0.0), **CASES[rule])
    J, g, _ = _grad_gpu(L, geo, 0, kw, 60, K=17)
    Jo, go = _grad_oracle(geo, 0, kw, 60)
    assert abs(J - Jo) <= 1e-12 * abs(Jo)
    assert _close(g, go, 1e-8), (g, go)


def test_adjoint_lift_and_moving_wall(L):
    """Lift (J = F_y) of a rotating cylinder (wall velocities on the links)."""
    geo = G.build(0, (34, 24, 1), (1, 1, 1), [G.ball((15.37, 11.61, 0), 5.23, omega=(0, 0, 0.003), force_id=0)])
    kw = dict(tau=0.65, g=(2e-5, 0.0, 0.0), bc=2)
    J, g, _ = _grad_gpu(L, geo, 0, kw, 50, K=50, direction=(0.0, 1.0, 0.0))
    d = G.ball_q_derivatives(geo, 0)
    dq = np.zeros((len(geo.links), 4))
    dq[:, 0], dq[:, 1], dq[:, 2] = d[:, 0], d[:, 1], d[:, 3]
    # the oracle's u_w is held fixed, as in the adjoint (u_w is data per link)
    cfg = O.make_config(stencil=0, nx=geo.nx, ny=geo.ny, nz=1, **kw)
    F, dF = O.run_dual(cfg, geo.solid, geo.links, dq, [0, 0, 0, 1.0], 50)
    # the lift is a small difference of O(0.1) link terms summed in another order
    assert abs(J - F[0, 1]) <= 1e-12 * abs(F[0, 1]) + 1e-14
    assert _close(g, dF[0, 1], 1e-8), (g, dF[0, 1])


def test_adjoint_matches_dual_numbers_open_channel(L):
    """Inlet (non-equilibrium extrapolation), outlet (copy), half-way channel
    walls and a VIBB cylinder."""
    H, umax = 20, 0.04
    geo = G.cylinder_channel(nx=60, ny_fluid=H, center=(18.37, 10.61), radius=4.23, u_max=umax)
    y = (np.arange(geo.N) // geo.nx) % geo.ny
    u0 = np.zeros((geo.N, 3))
    u0[:, 0] = np.where(geo.solid == 0, 4 * umax * (y - 0.5) * (H + 0.5 - y) / H ** 2, 0.0)
    kw = dict(tau=0.6, bc=2, inlet_umax=umax, inlet_y0=0.5, inlet_y1=H + 0.5)
    J, g, _ = _grad_gpu(L, geo, 2, kw, 80, K=30, u0=u0)
    Jo, go = _grad_oracle(geo, 2, kw, 80, u0=u0)
    assert abs(J - Jo) <= 1e-12 * abs(Jo)
    assert _close(g, go, 1e-8), (g, go)


def test_adjoint_matches_dual_numbers_open_periodic_y(L):
    """Open inlet and outlet on a lattice periodic in y (no channel walls): the
    open columns' adjoint and its clears wrap across the y seam."""
    U = 0.03
    geo = G.build(0, (40, 16, 1), (False, True, True), [G.ball((14.37, 7.61, 0), 3.23, force_id=0)],
                  open_x=(True, True))
    u0 = np.zeros((geo.N, 3))
    u0[:, 0] = np.where(geo.solid == 0, U, 0.0)
    kw = dict(tau=0.62, bc=2, inlet_umax=U, inlet_y0=-1e7, inlet_y1=1e7)
    J, g, _ = _grad_gpu(L, geo, 0, kw, 60, K=25, u0=u0)
    Jo, go = _grad_oracle(geo, 0, kw, 60, u0=u0)
    assert abs(J - Jo) <= 1e-12 * abs(Jo)
    assert _close(g, go, 1e-8), (g, go)


def test_adjoint_matches_dual_numbers_d3q19_sphere(L):
    geo = G.build(1, (14, 12, 10), (1, 1, 1), [G.ball((7.3, 6.6, 5.2), 3.1, force_id=0)])
    kw = dict(tau=0.75, g=(1e-5, 0.0, 0.0), bc=2)
    J, g, _ = _grad_gpu(L, geo, 0, kw, 40, K=40)
    Jo, go = _grad_oracle(geo, 0, kw, 40)
    assert abs(J - Jo) <= 1e-12 * abs(Jo)
    assert _close(g, go, 1e-8), (g, go)


def test_checkpoint_spacing_does_not_change_the_gradient(L):
    geo = G.build(0, (34, 24, 1), (1, 1, 1), [G.ball((15.37, 11.61, 0), 5.23, force_id=0)])
    kw = dict(tau=0.72, g=(2e-5, 0.0, 0.0), bc=2)
    _, g1, _ = _grad_gpu(L, geo, 0, kw, 90, K=90)
    _, g2, _ = _grad_gpu(L, geo, 0, kw, 90, K=7)
    # the adjoint's link scatters are FP64 atomics: equal up to summation order
    assert np.allclose(g1, g2, rtol=1e-10, atol=1e-12 * np.abs(g1).max())


def test_fp32_adjoint_close_to_fp64(L):
    geo = G.build(0, (64, 40, 1), (1, 1, 1), [G.ball((27.37, 19.61, 0), 6.23, force_id=0)])
    kw = dict(tau=0.7, g=(1e-5, 0.0, 0.0), bc=2)
    _, g64, _ = _grad_gpu(L, geo, 0, kw, 300, K=50, precision=L.LBM_FP64)
    _, g32, _ = _grad_gpu(L, geo, 0, kw, 300, K=50, precision=L.LBM_FP32_SHIFTED)
    assert _close(g32, g64, 1e-3), (g32, g64)


def test_autograd_function_vs_central_differences(L):
    """C4-style drag on an off-grid cylinder in a channel (inlet/outlet,
    scaled down), FP64: the autograd gradient agrees with fourth-order central
    differences (steps 1e-3 and 2e-3) to 1e-4 relative.  The centre and
    radius are chosen so that no link on the cylinder reaches q = 1/2 (the
    branch switch of the VIBB rule, a kink of J) within the stencil; the same
    test through a kink fails, correctly, at the 1e-3 level."""
    import torch

    from paper_1903_01111_gb300.autograd import (CylinderSpec, branch_margin, build_geometry, cylinder_force,
                                                 force_only)

    spec = CylinderSpec(kind="channel", nx=256, ny_fluid=64, u_max=0.1, n_steps=1500, checkpoint_every=100,
                        bc=2, precision=L.LBM_FP64)
    theta0 = np.array([64.251, 32.589, 8.201, 0.62])
    h = 1e-3
    assert branch_margin(spec, theta0) > 4 * h
    th = torch.tensor(theta0, dtype=torch.float64, requires_grad=True)
    J = cylinder_force(th, spec)
    J.backward()
    g = th.grad.numpy()
    geo0, _ = build_geometry(spec, *theta0[:3])

    def diff(k, step):
        tp, tm = theta0.copy(), theta0.copy()
        tp[k] += step
        tm[k] -= step
        for t in (tp, tm):
            gt, _ = build_geometry(spec, *t[:3])
            assert np.array_equal(gt.solid, geo0.solid), "perturbation changed the node classes"
        return (force_only(spec, tp) - force_only(spec, tm)) / (2 * step)

    for k in range(4):
        fd = (4 * diff(k, h) - diff(k, 2 * h)) / 3
        assert abs(g[k] - fd) <= 1e-4 * abs(fd) + 1e-7 * np.abs(g).max(), (k, g[k], fd)
