"""GPU path (liblbm.so through its C ABI) against the FP64 CPU oracle.

Tolerances:
* FP64 storage: max |f_gpu - f_oracle| <= 1e-11 over fluid nodes after 200
  steps (the two sides differ only in summation order).
* FP32 shifted storage: every stored value is h = f - w rho0, so a rounding
  costs at most eps32 |h|; a step applies a few dozen roundings per value and
  errors add at most linearly over steps, so the bound used is
  tol = 4 * steps * eps32 * max|h| (max over the oracle's state), i.e. a few
  ulps of the deviation part per step.
"""
import numpy as np
import pytest

import oracle as O
from paper_1903_01111_gb300 import geometry as G

pytestmark = pytest.mark.gpu

EPS32 = float(np.finfo(np.float32).eps)


@pytest.fixture(scope="module")
def L():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1903_01111_gb300 import lbm

    return lbm


def _cfg(geo, **kw):
    base = dict(stencil=geo.stencil, nx=geo.nx, ny=geo.ny, nz=geo.nz, periodic=geo.periodic,
                inlet=int(geo.open_x[0]), outlet=int(geo.open_x[1]))
    base.update(kw)
    return base


def _run_oracle(geo, steps, nbody=1, init_u=None, **kw):
    ocfg = O.make_config(**_cfg(geo, **kw))
    st = O.init(ocfg, geo.solid, u=init_u)
    F_ref = O.run(ocfg, geo.solid, geo.links, st, steps, nbody=nbody)
    return st, F_ref


def _run_gpu(L, geo, steps, precision, nbody=1, init_u=None, fused=1, **kw):
    """The lattice through the C ABI; fused = 1: link rules inside the pull
    pass (k_fused), 0: link kernel + bulk kernel."""
    lat = L.Lattice(geo, precision=precision, **{k: v for k, v in kw.items()})
    lat.set_tuning(fused=fused)
    lat.init_equilibrium(u=init_u)
    lat.step(steps)
    f = lat.distributions()
    F = np.array([lat.force(b) for b in range(nbody)]) if steps > 0 else None
    rho, u = lat.moments()
    lat.close()
    return f, F, rho, u


def _run_both(L, geo, steps, precision, nbody=1, init_u=None, fused=1, **kw):
    st, F_ref = _run_oracle(geo, steps, nbody=nbody, init_u=init_u, **kw)
    f, F, rho, u = _run_gpu(L, geo, steps, precision, nbody=nbody, init_u=init_u, fused=fused, **kw)
    return f, F, rho, u, st, F_ref


def _fluid(geo):
    m = (geo.solid == 0).reshape(geo.nz, geo.ny, geo.nx).copy()
    if geo.open_x[0]:
        m[:, :, 0] = False
    if geo.open_x[1]:
        m[:, :, -1] = False
    return m.reshape(-1)


def _tol(L, precision, steps, st, geo):
    if precision == L.LBM_FP64:
        return 1e-11
    _, w = O.velocity_set(geo.stencil)
    fl = _fluid(geo)
    hmax = np.abs(st.fp[:, fl] - w[:, None]).max()
    return 4 * steps * EPS32 * max(hmax, 1e-6)


def _compare(L, geo, steps, precision, nbody=1, init_u=None, **kw):
    """Both step forms (link rules fused into the pull pass, and the separate
    link kernel) against the oracle, element by element."""
    st, F_ref = _run_oracle(geo, steps, nbody=nbody, init_u=init_u, **kw)
    fl = _fluid(geo)
    tol = _tol(L, precision, steps, st, geo)
    errs = []
    for fused in ((1, 0) if len(geo.links) else (1,)):
        f, F, rho, u = _run_gpu(L, geo, steps, precision, nbody=nbody, init_u=init_u, fused=fused, **kw)
        err = np.abs(f[:, fl] - st.fp[:, fl]).max()
        assert err <= tol, f"fused={fused}: max |f - oracle| = {err:.3e} > {tol:.3e}"
        assert np.all(f[:, ~fl] == 0.0)
        # moments of the state: rho, u (D x N) against the oracle's
        D = 2 + geo.stencil
        urel = 1e-12 if precision == L.LBM_FP64 else 50 * tol
        assert np.abs(rho[fl] - st.rho[fl]).max() <= urel
        assert np.abs(u[:, fl] - st.u[fl, :D].T).max() <= urel
        if F is not None and nbody:
            scale = max(np.abs(F_ref).max(), 1e-12)
            ftol = 1e-10 * scale + 1e-15 if precision == L.LBM_FP64 else 1e-4 * scale + len(geo.links) * tol
            assert np.abs(F - F_ref).max() <= ftol, (fused, F, F_ref)
        errs.append(err)
    return max(errs), tol


PRECISIONS = ["fp64", "fp32s"]


def _p(L, name):
    return L.LBM_FP64 if name == "fp64" else L.LBM_FP32_SHIFTED


# ------------------------------------------------------------------ cases --

@pytest.mark.parametrize("prec", PRECISIONS)
@pytest.mark.parametrize("bc", [0, 1, 2, 3])
def test_poiseuille_32x24(L, bc, prec):
    """Plane Poiseuille flow, 32 x 24 fluid nodes, walls at q = 0.3 from the
    first and last fluid rows, g = 1e-6, tau = 0.8, 200 steps."""
    geo = G.channel(0, 32, 24, q_lo=0.3, q_hi=0.3)
    _compare(L, geo, 200, _p(L, prec), tau=0.8, g=(1e-6, 0, 0), bc=bc)


def test_poiseuille_32x24_5000_steps(L):
    geo = G.channel(0, 32, 24, q_lo=0.3, q_hi=0.3)
    f, F, rho, u, st, F_ref = _run_both(L, geo, 5000, L.LBM_FP64, tau=0.8, g=(1e-6, 0, 0), bc=2)
    fl = _fluid(geo)
    assert np.abs(f[:, fl] - st.fp[:, fl]).max() <= 1e-11


@pytest.mark.parametrize("prec", PRECISIONS)
@pytest.mark.parametrize("bc", [0, 1, 2, 3])
def test_rotating_cylinder_ragged_lattice(L, bc, prec):
    """Off-grid rotating cylinder (moving wall velocity per link) in a
    periodic 45 x 33 lattice; the body force has two components."""
    geo = G.build(0, (45, 33, 1), (1, 1, 1), [G.ball((20.37, 15.61, 0), 6.3, omega=(0, 0, 0.004), force_id=0)])
    _compare(L, geo, 200, _p(L, prec), tau=0.7, g=(2e-5, 1e-5, 0), bc=bc)


@pytest.mark.parametrize("prec", PRECISIONS)
@pytest.mark.parametrize("bc", [0, 1, 2, 3])
def test_sphere_pack_32(L, bc, prec):
    """D3Q19 body-force flow through a periodic overlapping sphere pack
    (the 384^3 workload's recipe at 32^3 with smaller radii)."""
    geo = G.sphere_pack(32, porosity=0.40, rmin=3.0, rmax=6.0, seed=7)
    _compare(L, geo, 200, _p(L, prec), tau=0.7, g=(1e-5, 0, 0), bc=bc)


@pytest.mark.parametrize("prec", PRECISIONS)
def test_d3q19_channel_moving_walls(L, prec):
    U = (0.02, 0.0, -0.01)
    geo = G.channel(1, 12, 10, nz=7, q_lo=0.27, q_hi=0.81, u_lo=(0, 0, 0), u_hi=U)
    _compare(L, geo, 200, _p(L, prec), tau=0.9, g=(1e-5, 0, 2e-6), bc=2)


@pytest.mark.parametrize("prec", PRECISIONS)
def test_open_channel_cylinder(L, prec):
    """The channel-with-cylinder workload scaled down: half-way channel walls,
    parabolic velocity inlet, zero-gradient outlet, VIBB cylinder."""
    geo = G.cylinder_channel(nx=120, ny_fluid=30, center=(30.37, 15.61), radius=4.3)
    y = (np.arange(geo.N) // geo.nx) % geo.ny
    u0 = np.zeros((geo.N, 3))
    u0[:, 0] = np.where(geo.solid == 0, 4 * 0.05 * (y - 0.5) * (30.5 - y) / 30 ** 2, 0.0)
    _compare(L, geo, 200, _p(L, prec), nbody=1, init_u=u0, tau=0.6, bc=2, inlet_umax=0.05, inlet_y0=0.5,
             inlet_y1=30.5)


def test_narrow_gap_second_node_fallback(L):
    """Two circles 0.6 apart: links whose x_ff is solid fall back to x_f."""
    geo = G.build(0, (40, 30, 1), (1, 1, 1), [G.ball((12.2, 15.3, 0), 6.1), G.ball((25.0, 15.3, 0), 6.1)])
    for bc in (1, 2, 3):
        _compare(L, geo, 100, L.LBM_FP64, tau=0.75, g=(1e-5, 2e-6, 0), bc=bc)


@pytest.mark.parametrize("prec", PRECISIONS)
def test_no_links_periodic_box_spanning_tiles(L, prec):
    """No solid at all; 300 x 7 lattice (two 256-thread row tiles with a
    ragged tail) and random smooth initial velocity."""
    geo = G.build(0, (300, 7, 1), (1, 1, 1), [])
    rng = np.random.default_rng(3)
    u0 = np.zeros((geo.N, 3))
    u0[:, :2] = rng.uniform(-0.02, 0.02, (geo.N, 2))
    _compare(L, geo, 50, _p(L, prec), nbody=0, init_u=u0, tau=0.55, g=(1e-5, 0, 0), bc=0)


@pytest.mark.parametrize("fused", [1, 0])
def test_step_chunks_and_profiling_are_bitwise_equal(L, fused):
    """lbm_step(n) (graph replay), n x lbm_step(1) and profiled launches
    compute the same bits, in both step forms."""
    geo = G.build(0, (45, 33, 1), (1, 1, 1), [G.ball((20.37, 15.61, 0), 6.3, omega=(0, 0, 0.004))])
    outs = []
    for mode in ("graph", "single", "profiled"):
        lat = L.Lattice(geo, tau=0.7, g=(2e-5, 1e-5, 0), bc=2)
        lat.set_tuning(fused=fused, graph_steps=8)
        lat.init_equilibrium()
        if mode == "graph":
            lat.step(37)
        elif mode == "single":
            for _ in range(37):
                lat.step(1)
        else:
            L.lbm_set_profiling(lat.h, True)
            lat.step(37)
            n, ms = L.lbm_kernel_times(lat.h)
            assert n[0] == (0 if fused else 37) and n[2] == 37 and n[1] == 0 and ms[2] > 0
        outs.append((lat.distributions(), lat.force(0)))
        lat.close()
    for f, F in outs[1:]:
        assert np.array_equal(f, outs[0][0])
        # block partial sums meet in FP64 atomics, whose order may vary; the
        # lift is a sum of link terms that cancel to about 1e-3 of their
        # magnitudes, so a last-place reordering shows at ~1e-13 of it
        np.testing.assert_allclose(F, outs[0][1], rtol=1e-12, atol=1e-18)


@pytest.mark.parametrize("fused", [0, 1])
def test_step_forces_equals_step_and_force_per_step(L, fused):
    """lbm_step_forces(n) gives the state of n x lbm_step(1) bit for bit and
    the force lbm_force reports after each of those steps (the force's FP64
    block sums meet in atomics, whose order may vary: to rounding); a call
    may end in the middle of a graph-sized run of steps; n = 0 runs nothing;
    a body without links gives zeros."""
    geo = G.build(0, (45, 33, 1), (1, 1, 1), [G.ball((20.37, 15.61, 0), 6.3, omega=(0, 0, 0.004))])
    outs = []
    for mode in ("loop", "series"):
        lat = L.Lattice(geo, tau=0.7, g=(2e-5, 1e-5, 0), bc=2)
        lat.set_tuning(fused=fused, graph_steps=8)
        lat.init_equilibrium()
        if mode == "loop":
            F = []
            for _ in range(37):
                lat.step(1)
                F.append(lat.force(0))
            F = np.array(F)
        else:
            F = np.vstack([lat.step_forces(30), lat.step_forces(0), lat.step_forces(7)])
        outs.append((lat.distributions(), F))
        if mode == "series":
            assert np.array_equal(lat.step_forces(3, body=5), np.zeros((3, 3)))
        lat.close()
    assert outs[1][1].shape == (37, 3)
    assert np.array_equal(outs[1][0], outs[0][0])
    np.testing.assert_allclose(outs[1][1], outs[0][1], rtol=1e-12, atol=1e-18)


@pytest.mark.parametrize("prec", PRECISIONS)
def test_fused_and_split_steps_agree_on_a_moving_pack(L, prec):
    """The fused step and the link-kernel step on a D3Q19 pack with moving
    spheres, two bodies, every rule mixed per link and open rows absent:
    the populations agree to rounding (FP64 1e-13, FP32 the parity bound)
    and the per-body forces to their summation order."""
    geo = G.sphere_pack(28, porosity=0.5, rmin=2.5, rmax=5.0, seed=11)
    links = geo.links.copy()
    rng = np.random.default_rng(4)
    links["bc"] = rng.integers(0, 4, len(links))
    links["body"] = rng.integers(0, 2, len(links))
    links["uw"][:, 0] = 0.01 * rng.standard_normal(len(links))
    geo.links = links
    out = {}
    for fused in (1, 0):
        f, F, _, _ = _run_gpu(L, geo, 60, _p(L, prec), nbody=2, fused=fused, tau=0.7, g=(1e-5, 0, 0), bc=2)
        out[fused] = (f, F)
    _, w = O.velocity_set(1)
    h = np.abs(out[0][0] - (w[:, None] if prec == "fp32s" else 0.0)).max()
    tol = 1e-13 if prec == "fp64" else 4 * 60 * EPS32 * h
    assert np.abs(out[1][0] - out[0][0]).max() <= tol
    scale = np.abs(out[0][1]).max()
    assert np.abs(out[1][1] - out[0][1]).max() <= (1e-12 if prec == "fp64" else 1e-5) * scale


@pytest.mark.parametrize("fused", [0, 1])
def test_link_input_order_does_not_change_the_result(L, fused):
    """lbm_set_geometry puts the links in its own order: the same links given
    in a shuffled order, with two bodies (so the link kernel's body-sorted
    order differs from the fused kernel's node order), give the same
    populations bit for bit and the same per-body forces (to the order of
    their FP64 block sums)."""
    import copy

    geo = G.sphere_pack(24, porosity=0.5, rmin=2.5, rmax=4.5, seed=3)
    links = geo.links.copy()
    links["body"] = np.random.default_rng(2).integers(0, 2, len(links))
    geo.links = links
    shuffled = copy.copy(geo)
    shuffled.links = links[np.random.default_rng(1).permutation(len(links))]
    out = [_run_gpu(L, g, 25, L.LBM_FP64, nbody=2, fused=fused, tau=0.7, g=(1e-5, 0, 0), bc=2)[:2]
           for g in (geo, shuffled)]
    assert np.array_equal(out[0][0], out[1][0])
    np.testing.assert_allclose(out[1][1], out[0][1], rtol=1e-12, atol=1e-15)


def test_moments_device_pointers(L):
    import torch

    geo = G.channel(0, 32, 24, q_lo=0.3, q_hi=0.3)
    lat = L.Lattice(geo, tau=0.8, g=(1e-6, 0, 0), bc=2, stream=torch.cuda.current_stream().cuda_stream)
    lat.init_equilibrium()
    lat.step(30)
    rho_h, u_h = lat.moments()
    rho_d = torch.empty(geo.N, dtype=torch.float64, device="cuda")
    u_d = torch.empty((2, geo.N), dtype=torch.float64, device="cuda")
    L.lbm_moments(lat.h, rho_d, u_d)
    torch.cuda.synchronize()
    assert np.array_equal(rho_d.cpu().numpy(), rho_h) and np.array_equal(u_d.cpu().numpy(), u_h)
    lat.close()


@pytest.mark.parametrize("prec", PRECISIONS)
def test_set_distributions_then_step(L, prec):
    """A random post-collision state set through the ABI evolves like the
    oracle started from the same state (moments rebuilt from f+ on both
    sides)."""
    geo = G.build(0, (30, 22, 1), (1, 1, 1), [G.ball((14.2, 10.9, 0), 4.4)])
    _, w = O.velocity_set(0)
    rng = np.random.default_rng(5)
    f0 = w[:, None] * (1 + 0.01 * rng.standard_normal((9, geo.N)))
    f0[:, geo.solid == 1] = 0
    cfg = _cfg(geo, tau=0.7, g=(1e-5, 0, 0), bc=2)
    ocfg = O.make_config(**cfg)
    rho, u = O.moments(ocfg, geo.solid, f0.copy())
    st = O.State(f0.copy(), rho, u)
    O.run(ocfg, geo.solid, geo.links, st, 60)
    lat = L.Lattice(geo, precision=_p(L, prec), tau=0.7, g=(1e-5, 0, 0), bc=2)
    lat.set_distributions(f0)
    back = lat.distributions()
    fl = geo.solid == 0
    assert np.abs(back[:, fl] - f0[:, fl]).max() <= (0 if prec == "fp64" else 2 * EPS32)
    lat.step(60)
    f = lat.distributions()
    tol = 1e-11 if prec == "fp64" else 4 * 60 * EPS32 * np.abs(f0[:, fl] - w[:, None]).max() * 4
    assert np.abs(f[:, fl] - st.fp[:, fl]).max() <= tol
    lat.close()


def test_invalid_geometry_is_rejected(L):
    geo = G.channel(0, 16, 8, q_lo=0.3, q_hi=0.3)
    lat = L.Lattice(None, stencil=0, nx=geo.nx, ny=geo.ny, nz=1, periodic=geo.periodic, tau=0.8)
    bad = []
    missing = geo.links[1:]
    bad.append(missing)
    dup = np.concatenate([geo.links, geo.links[:1]])
    bad.append(dup)
    q0 = geo.links.copy()
    q0["q"][3] = 0.0
    bad.append(q0)
    to_fluid = geo.links.copy()
    to_fluid["dir"][0] = 1  # +x neighbour of a fluid node is fluid
    bad.append(to_fluid)
    for links in bad:
        with pytest.raises(L.LBMError) as ex:
            lat.set_geometry(geo.solid, links)
        assert ex.value.status == L.LBM_ERR_INVALID_ARG
    # fluid on a face of a non-periodic axis
    solid = geo.solid.copy()
    solid[:geo.nx] = 0
    with pytest.raises(L.LBMError):
        lat.set_geometry(solid, geo.links)
    with pytest.raises(L.LBMError) as ex:
        lat.step(1)
    assert ex.value.status == L.LBM_ERR_STATE
    lat.set_geometry(geo.solid, geo.links)  # the valid one still works
    lat.close()


def test_outlet_needs_a_fluid_node_before_it(L):
    """The zero-gradient outlet copies the fluid node before it (Sec. 4.3): an
    outlet row whose node at x = nx - 2 is solid (a small body touching the
    outlet column) is rejected by lbm_set_geometry."""
    geo = G.cylinder_channel(nx=40, ny_fluid=10, center=(38.0, 5.5), radius=0.6)
    s = geo.solid.reshape(geo.ny, geo.nx)
    assert s[:, geo.nx - 2].any() and not s[1:-1, geo.nx - 1].any()
    lat = L.Lattice(None, stencil=0, nx=geo.nx, ny=geo.ny, nz=1, periodic=geo.periodic, tau=0.8, inlet=1,
                    outlet=1, inlet_umax=0.05, inlet_y0=0.5, inlet_y1=10.5)
    with pytest.raises(L.LBMError) as ex:
        lat.set_geometry(geo.solid, geo.links)
    assert ex.value.status == L.LBM_ERR_INVALID_ARG and "outlet" in str(ex.value)
    lat.close()


def test_bad_configs_are_rejected(L):
    for kw in (dict(tau=0.5), dict(stencil=0, nz=2), dict(stencil=1, collision=1), dict(collision=5),
               dict(stencil=1, inlet=1, periodic=(0, 1, 1)), dict(precision=7), dict(vibb_density=3)):
        base = dict(stencil=0, nx=8, ny=8, nz=1, tau=0.8)
        base.update(kw)
        with pytest.raises(L.LBMError):
            L.Lattice(None, **base)


def test_divergence_is_reported(L):
    """Failure detection without a GPU fault: an unstable run (tau close to
    1/2, large velocity) produces non-finite values that lbm_check reports."""
    geo = G.build(0, (32, 32, 1), (1, 1, 1), [])
    u0 = np.zeros((geo.N, 3))
    x = np.arange(geo.N) % 32
    u0[:, 0] = 0.45 * np.sin(2 * np.pi * x / 32)
    lat = L.Lattice(geo, tau=0.5000001, bc=0)
    lat.init_equilibrium(u=u0)
    lat.check()
    lat.step(3000)
    with pytest.raises(L.LBMError) as ex:
        lat.check()
    assert ex.value.status == L.LBM_ERR_DIVERGED
    lat.close()


def _oracle_one_node_step(geo, e, w, opp, links_at, fp_of, x, tau, g, bc=2, vibb_density=0):
    """f+(x, t+1) from gathered f+(., t): pull, link rules (each link's own
    rule, else bc), collision."""
    cfg = O.make_config(stencil=geo.stencil, tau=tau, g=g, bc=bc, vibb_density=vibb_density)
    Q = len(w)
    f = np.empty(Q)
    nx, ny, nz = geo.shape

    def nb(n, d, s):
        c = np.array([n % nx, (n // nx) % ny, n // (nx * ny)]) + s * e[d]
        c %= np.array(geo.shape)
        return int(c[0] + nx * (c[1] + ny * c[2]))

    for i in range(Q):
        f[i] = fp_of(nb(x, i, -1))[i]
    for lk in links_at.get(x, []):
        ip = int(lk["dir"])
        i = opp[ip]
        ff = nb(x, i, 1)
        if geo.solid[ff]:
            ff = x
        vf, vff = fp_of(x), fp_of(ff)
        rf, rff = vf.sum(), vff.sum()
        uf = (vf @ e - 0.5 * np.asarray(g)) / rf
        uff = (vff @ e - 0.5 * np.asarray(g)) / rff
        rule = int(lk["bc"]) if int(lk["bc"]) >= 0 else bc
        f[i] = O.link_value(cfg, rule, ip, lk["q"], lk["uw"], vf, vff, rf, uf, rff, uff)
    fp, _, _ = O.collide(cfg, f)
    return fp


def _sampled_step_check(L, lat, geo, sample, tau, g, bc, vibb_density, shifted):
    """One step of `lat` against the one-node oracle step at `sample`, from
    the gathered state; FP64: 1e-13 absolute; FP32 shifted: 16 eps32 of the
    largest deviation |f - w rho0| (one step's roundings on the stored h)."""
    stencil = geo.stencil
    e, w = O.velocity_set(stencil)
    Q = len(w)
    opp = [int(np.flatnonzero((e == -e[i]).all(1))[0]) for i in range(Q)]
    nx, ny, _ = geo.shape
    need = set()
    for x in sample:
        c = np.array([x % nx, (x // nx) % ny, x // (nx * ny)])
        for d1 in range(Q):
            for d2 in range(Q):
                cc = (c - e[d1] + e[d2]) % np.array(geo.shape)
                need.add(int(cc[0] + nx * (cc[1] + ny * cc[2])))
    need = np.array(sorted(need))
    vals = L.lbm_gather(lat.h, need)
    table = dict(zip(need.tolist(), vals))
    sel = np.isin(geo.links["node"], sample)
    links_at = {}
    for lk in geo.links[sel]:
        links_at.setdefault(int(lk["node"]), []).append(lk)
    lat.step(1)
    got = L.lbm_gather(lat.h, sample)
    want = np.array([_oracle_one_node_step(geo, e, w, opp, links_at, lambda n: table[n], int(x), tau, g, bc,
                                           vibb_density) for x in sample])
    tol = 16 * EPS32 * np.abs(want - w[None, :]).max() if shifted else 1e-13
    err = np.abs(got - want).max(axis=1)
    assert err.max() <= tol, (sample[int(np.argmax(err))], err.max(), tol)
    return err.max(), tol


@pytest.mark.parametrize("arm", ["fp64", "fp64_split", "fp32s_bench"])
def test_full_size_sphere_pack_sampled_nodes(L, arm):
    """The 384^3 workload: after three steps from rest, f+(t+1) at sampled
    fluid nodes (150 with links, 50 anywhere) equals the oracle's pull + link
    rules + collision computed node by node from the gathered f+(t).  The
    fp32s arm is the bench's configuration: FP32 shifted storage, VIBB with
    rho_d = rho_f for q > 1/2, the fused step in 128-thread blocks; the
    fp64_split arm the split form the autotuner picks in FP64 (link kernel,
    then the bulk pass over the fluid-node list)."""
    geo = G.sphere_pack(384, seed=0)
    tau, g = 0.7, (1e-6, 0.0, 0.0)
    if arm in ("fp64", "fp64_split"):
        lat = L.Lattice(geo, tau=tau, g=g, bc=2)
        if arm == "fp64_split":
            lat.set_tuning(bulk_shape=1, link_threads=128, link_seq=1, graph_steps=8, fused=0)
        vd, shifted = 0, False
    else:
        lat = L.Lattice(geo, precision=L.LBM_FP32_SHIFTED, tau=tau, g=g, bc=2, vibb_density=L.LBM_VIBB_RHO_LOCAL)
        lat.set_tuning(bulk_shape=1, link_threads=128, link_seq=4, graph_steps=8, fused=1)
        vd, shifted = 1, True
    lat.init_equilibrium()
    lat.step(3)  # non-uniform state near the walls
    rng = np.random.default_rng(0)
    fluid = np.flatnonzero(geo.solid == 0)
    boundary = np.unique(geo.links["node"])
    sample = np.concatenate([rng.choice(boundary, 150, replace=False), rng.choice(fluid, 50, replace=False)])
    _sampled_step_check(L, lat, geo, sample, tau, g, 2, vd, shifted)
    lat.close()


@pytest.mark.parametrize("prec", PRECISIONS)
def test_full_size_cylinder_channel_sampled_nodes(L, prec):
    """The 2000 x 400 cylinder channel at Re 100 (tau 0.5812), the bench's
    cylinder run: after 50 steps from the Poiseuille start, f+(t+1) at nodes
    on the cylinder, on the walls and in the bulk (columns 2 .. nx - 3, whose
    pulls do not reach the open columns) equals the one-node oracle step
    from the gathered state."""
    R, u_max, H = 20.3, 0.1, 400
    ubar, D = 2.0 / 3.0 * u_max, 2 * R
    tau = 3 * ubar * D / 100 + 0.5
    geo = G.cylinder_channel(nx=2000, ny_fluid=H, center=(400.37, 200.61), radius=R, u_max=u_max)
    y = (np.arange(geo.N) // geo.nx) % geo.ny
    u0 = np.zeros((geo.N, 3))
    u0[:, 0] = np.where(geo.solid == 0, 4 * u_max * (y - 0.5) * (H + 0.5 - y) / H ** 2, 0.0)
    lat = L.Lattice(geo, precision=_p(L, prec), tau=tau, bc=2, inlet_umax=u_max, inlet_y0=0.5, inlet_y1=H + 0.5)
    lat.init_equilibrium(u=u0)
    lat.step(50)
    rng = np.random.default_rng(1)
    x = np.arange(geo.N) % geo.nx
    inner = (x >= 2) & (x <= geo.nx - 3)
    fluid = np.flatnonzero((geo.solid == 0) & inner)
    lk_nodes = np.unique(geo.links["node"])
    lk_nodes = lk_nodes[inner[lk_nodes]]
    on_cyl = lk_nodes[np.abs(lk_nodes % geo.nx - 400) < 30]
    on_wall = lk_nodes[np.abs(lk_nodes % geo.nx - 400) >= 30]
    sample = np.concatenate([rng.choice(on_cyl, 80, replace=False), rng.choice(on_wall, 40, replace=False),
                             rng.choice(fluid, 40, replace=False)])
    _sampled_step_check(L, lat, geo, sample, tau, (0.0, 0.0, 0.0), 2, 0, prec == "fp32s")
    lat.close()


@pytest.mark.parametrize("prec", PRECISIONS)
def test_sphere_pack_32_local_density(L, prec):
    """The LBM_VIBB_RHO_LOCAL reading (rho_d = rho_f when q > 1/2), used by
    the 384^3 porous workload."""
    geo = G.sphere_pack(32, porosity=0.40, rmin=3.0, rmax=6.0, seed=7)
    _compare(L, geo, 200, _p(L, prec), tau=0.7, g=(1e-5, 0, 0), bc=2, vibb_density=1)


@pytest.mark.parametrize("prec", PRECISIONS)
@pytest.mark.parametrize("bc", [0, 1, 2, 3])
def test_mrt_rotating_cylinder(L, bc, prec):
    """MRT collision (Sec. 2, Eq. mrt, the paper's own operator) with every
    link rule around a rotating off-grid cylinder."""
    geo = G.build(0, (45, 33, 1), (1, 1, 1), [G.ball((20.37, 15.61, 0), 6.3, omega=(0, 0, 0.004), force_id=0)])
    _compare(L, geo, 200, _p(L, prec), tau=0.62, g=(2e-5, 1e-5, 0), bc=bc, collision=1)


@pytest.mark.parametrize("prec", PRECISIONS)
def test_mrt_open_channel_cylinder(L, prec):
    geo = G.cylinder_channel(nx=120, ny_fluid=30, center=(30.37, 15.61), radius=4.3)
    y = (np.arange(geo.N) // geo.nx) % geo.ny
    u0 = np.zeros((geo.N, 3))
    u0[:, 0] = np.where(geo.solid == 0, 4 * 0.05 * (y - 0.5) * (30.5 - y) / 30 ** 2, 0.0)
    _compare(L, geo, 200, _p(L, prec), nbody=1, init_u=u0, tau=0.56, bc=2, collision=1, inlet_umax=0.05,
             inlet_y0=0.5, inlet_y1=30.5)


@pytest.mark.parametrize("bc", [0, 1, 2, 3])
def test_poiseuille_l2_error_fp32_no_worse_than_fp64(L, bc):
    """Analytic case: L2 error of the velocity against the parabolic profile
    of body-force-driven Poiseuille flow (Sec. 4.1) after 12000 steps (about
    two diffusion times), walls at q = 0.3.  The FP32-shifted run's error is
    the FP64 run's to within 1e-3 of itself."""
    geo = G.channel(0, 32, 24, q_lo=0.3, q_hi=0.3)
    tau, g = 0.8, 1e-6
    nu = (tau - 0.5) / 3
    y = np.arange(geo.ny)
    exact = G.poiseuille_profile(y, geo.info["y_lo"], geo.info["y_hi"], g, nu)
    rows = slice(1, geo.ny - 1)
    errs = {}
    for prec in (L.LBM_FP64, L.LBM_FP32_SHIFTED):
        with L.Lattice(geo, precision=prec, tau=tau, g=(g, 0, 0), bc=bc) as lat:
            lat.init_equilibrium()
            lat.step(12000)
            _, u = lat.moments()
        ux = u[0].reshape(geo.ny, geo.nx)[rows].mean(axis=1)
        errs[prec] = np.sqrt(np.sum((ux - exact[rows]) ** 2) / np.sum(exact[rows] ** 2))
    assert errs[L.LBM_FP32_SHIFTED] <= errs[L.LBM_FP64] * (1 + 1e-3), errs
    if bc != 0:
        assert errs[L.LBM_FP64] < 1e-2, errs


@pytest.mark.parametrize("prec", PRECISIONS)
@pytest.mark.parametrize("stencil", [0, 1])
def test_translated_geometry_gives_translated_state(L, prec, stencil):
    """Translation invariance on the GPU: the same geometry shifted by an
    integer vector along its periodic axes (another compacted layout, other
    runs, other seam crossings) gives the shifted populations, bit for bit."""
    if stencil == 0:
        g = G.build(0, (45, 33, 1), (1, 1, 1), [G.ball((20.37, 15.61, 0), 6.3, omega=(0, 0, 0.004), force_id=0)])
        shift = (17, 5, 0)
    else:
        g = G.sphere_pack(24, porosity=0.5, rmin=2.5, rmax=4.5, seed=3)
        shift = (7, 11, 5)
    gs = G.translated(g, shift)
    x, y, z = g.coords(np.arange(g.N))
    mp = (x + shift[0]) % g.nx + g.nx * (((y + shift[1]) % g.ny) + g.ny * ((z + shift[2]) % g.nz))
    out = []
    for geo in (g, gs):
        with L.Lattice(geo, precision=_p(L, prec), tau=0.7, g=(1e-5, 2e-6, 0), bc=2) as lat:
            lat.init_equilibrium()
            lat.step(41)
            out.append(lat.distributions())
    assert np.array_equal(out[1][:, mp], out[0])


def test_fp64_rate_probe(L):
    """lbm_probe_fp64 measures the device's FP64 FMA rate (the FP64 roofline's
    peak): a positive rate below the FP64 rate of any current GPU, from a
    launch of positive duration."""
    tflops, ms = L.lbm_probe_fp64()
    assert 0.05 < tflops < 100.0 and ms > 0.0
