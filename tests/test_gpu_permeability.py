"""Darcy permeability of the sphere-pack workload (the quantity its runs are
for): the formula against plane Poiseuille flow, where it has a closed form,
and FP32 shifted storage against FP64 on a small pack of the same recipe."""
import numpy as np
import pytest

from paper_1903_01111_gb300 import geometry as G

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1903_01111_gb300 import lbm

    return lbm


@pytest.fixture(scope="module")
def bench():
    import bench as B

    return B


@pytest.mark.parametrize("bc,err", [(1, 1.64e-3), (2, 2.72e-3)])
def test_permeability_of_a_plane_channel(L, bench, bc, err):
    """Between walls H apart (q = 0.3 at both) the steady body-force flow is
    the parabola of Sec. 4.1, so k = nu q_D / g has the node sum
    (1/ny) sum_y s (H - s) / 2 (s: distance from the wall; the solid rows
    count in the volume).  After 12,000 steps (two diffusion times) the FP64
    path carries the rule's own steady slip at tau = 0.8, which the oracle
    puts at +1.64e-3 (Bouzidi) and +2.72e-3 (VIBB) of the flux."""
    geo = G.channel(0, 16, 24, q_lo=0.3, q_hi=0.3)
    tau, g = 0.8, 1e-6
    nu = (tau - 0.5) / 3
    y = np.arange(geo.ny)
    fluid = (y >= 1) & (y <= geo.ny - 2)
    s = y - geo.info["y_lo"]
    H = geo.info["y_hi"] - geo.info["y_lo"]
    k_exact = float(np.sum(np.where(fluid, s * (H - s) / 2.0, 0.0))) / geo.ny
    with L.Lattice(geo, precision=L.LBM_FP64, tau=tau, g=(g, 0, 0), bc=bc) as lat:
        lat.init_equilibrium()
        lat.step(12000)
        _, u = lat.moments()
    k = bench.darcy_permeability(geo, u, nu, g)
    assert abs((k - k_exact) / k_exact - err) <= 0.02 * err, (k, k_exact)


def test_permeability_fp32_shifted_matches_fp64_on_a_small_pack(L, bench):
    """The 384^3 recipe scaled to 48^3 (radii U[3, 6]): the permeability after
    3,000 steps from rest in FP32 shifted storage is the FP64 one to 1e-4."""
    geo = G.sphere_pack(48, porosity=0.40, rmin=3.0, rmax=6.0, seed=5)
    tau, g = 0.7, 1e-6
    nu = (tau - 0.5) / 3
    ks = {}
    for prec in (L.LBM_FP64, L.LBM_FP32_SHIFTED):
        with L.Lattice(geo, precision=prec, tau=tau, g=(g, 0, 0), bc=L.LBM_BC_VIBB,
                       vibb_density=L.LBM_VIBB_RHO_LOCAL) as lat:
            lat.init_equilibrium()
            lat.step(3000)
            _, u = lat.moments()
        ks[prec] = bench.darcy_permeability(geo, u, nu, g)
    k64, k32 = ks[L.LBM_FP64], ks[L.LBM_FP32_SHIFTED]
    assert k64 > 0
    assert abs(k32 - k64) <= 1e-4 * k64, (k32, k64)
