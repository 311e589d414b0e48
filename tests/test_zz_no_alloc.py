"""lbm_force_noalloc: the momentum-exchange force from caller-owned device
memory, for callers that cannot allocate device memory (real-time code,
frameworks whose pool owns all device memory).

Checked through the C ABI against the allocating path (lbm_step(1) followed
by lbm_force on a lattice) on two calls in a row, with the same FP64
tolerance as the other force checks.  This file is collected last so that a
run stopping at the first failure has run every other test first."""
import ctypes

import numpy as np
import pytest

from paper_1903_01111_gb300 import geometry as G

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1903_01111_gb300 import lbm

    return torch, lbm


def _cases():
    cyl = G.build(0, (45, 33, 1), (1, 1, 1), [G.ball((20.37, 15.61, 0), 6.3, omega=(0, 0, 0.004), force_id=0)])
    pack = G.sphere_pack(32, porosity=0.40, rmin=3.0, rmax=6.0, seed=7)
    return [(cyl, dict(tau=0.7, g=(2e-5, 1e-5, 0), bc=2)),
            (pack, dict(tau=0.7, g=(1e-5, 0, 0), bc=2, vibb_density=1)),
            (pack, dict(tau=0.7, g=(1e-5, 0, 0), bc=1))]


@pytest.mark.parametrize("case", range(3))
def test_noalloc_force_matches_lbm_force_on_two_calls(env, case):
    torch, lbm = env
    geo, kw = _cases()[case]
    lat = lbm.Lattice(geo, precision=lbm.LBM_FP64, **kw)
    lat.init_equilibrium()
    lat.step(15)
    cfg = lbm.make_config(stencil=geo.stencil, nx=geo.nx, ny=geo.ny, nz=geo.nz, periodic=geo.periodic, **kw)
    dev = torch.device("cuda")
    solid = torch.from_numpy(np.ascontiguousarray(geo.solid, np.uint8)).to(dev)
    links = torch.from_numpy(np.ascontiguousarray(geo.links, dtype=lbm.LINK_DTYPE).view(np.uint8)).to(dev)
    F = torch.full((3,), float("nan"), dtype=torch.float64, device=dev)
    for call in range(2):
        f = torch.from_numpy(lat.distributions()).to(dev)
        torch.cuda.synchronize()
        lbm.lbm_force_noalloc(cfg, f, solid, links, len(geo.links), 0, F)
        torch.cuda.synchronize()
        got = F.cpu().numpy()
        lat.step(1)
        want = lat.force(0)
        scale = np.abs(want).max()
        assert np.all(np.isfinite(got))
        assert np.abs(got - want).max() <= 1e-10 * scale + 1e-15, (call, got, want)
        # same inputs give the same bits
        lbm.lbm_force_noalloc(cfg, f, solid, links, len(geo.links), 0, F)
        torch.cuda.synchronize()
        assert np.array_equal(F.cpu().numpy(), got)
        lat.step(3)
    lat.close()


def test_noalloc_calls_leave_free_device_memory_unchanged(env):
    """The entry point allocates nothing: after a first call on the device
    (which looks up the scratch array's address), ten more calls leave the
    device's free memory as it was."""
    torch, lbm = env
    geo, kw = _cases()[0]
    lat = lbm.Lattice(geo, precision=lbm.LBM_FP64, **kw)
    lat.init_equilibrium()
    lat.step(5)
    cfg = lbm.make_config(stencil=geo.stencil, nx=geo.nx, ny=geo.ny, nz=geo.nz, periodic=geo.periodic, **kw)
    dev = torch.device("cuda")
    f = torch.from_numpy(lat.distributions()).to(dev)
    solid = torch.from_numpy(np.ascontiguousarray(geo.solid, np.uint8)).to(dev)
    links = torch.from_numpy(np.ascontiguousarray(geo.links, dtype=lbm.LINK_DTYPE).view(np.uint8)).to(dev)
    F = torch.zeros(3, dtype=torch.float64, device=dev)
    lbm.lbm_force_noalloc(cfg, f, solid, links, len(geo.links), 0, F)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(10):
        lbm.lbm_force_noalloc(cfg, f, solid, links, len(geo.links), 0, F)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    lat.close()


def test_noalloc_rejects_link_counts_beyond_its_scratch(env):
    torch, lbm = env
    cfg = lbm.make_config(stencil=0, nx=8, ny=8, nz=1)
    st = lbm._lib.lbm_force_noalloc(ctypes.byref(cfg), 16, 16, 16, lbm.LBM_NOALLOC_MAX_LINKS + 1, 0, 16)
    assert st == lbm.LBM_ERR_INVALID_ARG
    assert "LBM_NOALLOC_MAX_LINKS" in lbm.lbm_last_error()
