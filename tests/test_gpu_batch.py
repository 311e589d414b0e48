"""Batches (lbm_set_domains): several channel flows of different sizes,
cylinder layouts and relaxation times stacked in one lattice.

* FP64 batch against the FP64 oracle run on each domain alone (1e-11 after
  150 steps), and the FP32-shifted batch within the FP32 bound of the parity
  tests;
* the batch against each domain run as its own GPU lattice: the same bits
  (the kernels do the same arithmetic; only the domain table differs);
* forces per body and the batched adjoint (J = sum over bodies of w_b . F_b,
  dJ/dtau per domain) against single-domain runs;
* launch shapes (lbm_set_tuning) change no bits, and lbm_autotune leaves the
  state as it found it.
"""
import numpy as np
import pytest

import oracle as O
from paper_1903_01111_gb300 import batch as B
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


def _small_specs(n=5, seed=3):
    return B.draw_channels(n, seed, nx_range=(28, 61), ny_range=(10, 23), n_cyl=(1, 3), r_range=(2.2, 4.6),
                           re_range=(5.0, 40.0), u_max=0.05, gap=2.0)


def _batch_lattice(L, b, precision, bc=2, **kw):
    lat = L.batch_lattice(b, precision=precision, bc=bc, **kw)
    lat.init_equilibrium(u=b.initial_velocity())
    return lat


def _single_cfg(s, geo, bc=2):
    return dict(stencil=0, nx=geo.nx, ny=geo.ny, nz=1, periodic=geo.periodic, inlet=1, outlet=1, tau=s.tau, bc=bc,
                **s.inlet())


def _fluid_mask(geo):
    m = (geo.solid == 0).reshape(geo.ny, geo.nx).copy()
    m[:, 0] = False
    m[:, -1] = False
    return m.reshape(-1)


@pytest.mark.parametrize("prec", ["fp64", "fp32s"])
def test_batch_matches_oracle_per_domain(L, prec):
    specs = _small_specs()
    b = B.stack(specs)
    steps = 150
    precision = L.LBM_FP64 if prec == "fp64" else L.LBM_FP32_SHIFTED
    lat = _batch_lattice(L, b, precision)
    lat.step(steps)
    f = lat.distributions()
    F = lat.forces()
    lat.close()
    _, w = O.velocity_set(0)
    for d, (s, geo) in enumerate(zip(specs, b.parts)):
        cfg = O.make_config(**_single_cfg(s, geo))
        u0 = s.initial_velocity(geo)
        st = O.init(cfg, geo.solid, u=u0)
        Fo = O.run(cfg, geo.solid, geo.links, st, steps, nbody=len(s.cylinders))
        fl = _fluid_mask(geo)
        fd = f[:, b.domain_nodes(d)]
        if precision == L.LBM_FP64:
            tol = 1e-11
        else:
            tol = 4 * steps * EPS32 * max(np.abs(st.fp[:, fl] - w[:, None]).max(), 1e-6)
        err = np.abs(fd[:, fl] - st.fp[:, fl]).max()
        assert err <= tol, (d, err, tol)
        Fd = F[b.body0[d]:b.body0[d] + len(s.cylinders)]
        scale = np.abs(Fo).max()
        ftol = 1e-10 * scale if precision == L.LBM_FP64 else 1e-4 * scale + len(geo.links) * tol
        assert np.abs(Fd - Fo[:len(s.cylinders)]).max() <= ftol, (d, Fd, Fo)


@pytest.mark.parametrize("prec", ["fp64", "fp32s"])
def test_batch_equals_domains_run_alone(L, prec):
    specs = _small_specs(4, seed=11)
    b = B.stack(specs)
    precision = L.LBM_FP64 if prec == "fp64" else L.LBM_FP32_SHIFTED
    lat = _batch_lattice(L, b, precision)
    lat.step(101)
    f = lat.distributions()
    F = lat.forces()
    lat.close()
    for d, (s, geo) in enumerate(zip(specs, b.parts)):
        with L.Lattice(geo, precision=precision, bc=2, tau=s.tau, **s.inlet()) as one:
            one.init_equilibrium(u=s.initial_velocity(geo))
            one.step(101)
            f1 = one.distributions()
            F1 = one.forces(len(s.cylinders))
        assert np.array_equal(f[:, b.domain_nodes(d)], f1), d
        Fd = F[b.body0[d]:b.body0[d] + len(s.cylinders)]
        # force sums run in another order (FP32 lane sums in shifted storage);
        # small components are differences of O(max |F|) link terms
        rtol = 1e-12 if precision == L.LBM_FP64 else 1e-5
        assert np.allclose(Fd, F1, rtol=rtol, atol=rtol * 10 * np.abs(F1).max()), (d, Fd, F1)


def test_batch_adjoint_equals_domains_alone(L):
    specs = _small_specs(3, seed=5)
    b = B.stack(specs)
    rng = np.random.default_rng(0)
    wts = rng.normal(size=(b.n_bodies, 3))
    wts[:, 2] = 0.0
    lat = _batch_lattice(L, b, L.LBM_FP64)
    J, dq, dtau, _ = L.lbm_adjoint_step(lat.h, -1, wts, 60, 25)
    lat.close()
    assert dtau.shape == (3,)
    Jsum = 0.0
    for d, (s, geo) in enumerate(zip(specs, b.parts)):
        wd = wts[b.body0[d]:b.body0[d] + len(s.cylinders)]
        with L.Lattice(geo, precision=L.LBM_FP64, bc=2, tau=s.tau, **s.inlet()) as one:
            one.init_equilibrium(u=s.initial_velocity(geo))
            Jd, dqd, dtd, _ = L.lbm_adjoint_step(one.h, -1, wd, 60, 25)
        Jsum += Jd
        dqb = dq[b.domain_links(d)]
        assert np.allclose(dqb, dqd, rtol=1e-9, atol=1e-12 * np.abs(dqd).max()), d
        assert abs(dtau[d] - dtd) <= 1e-9 * abs(dtd), (d, dtau[d], dtd)
    assert abs(J - Jsum) <= 1e-12 * abs(Jsum) + 1e-15


def _shapes(L, stencil):
    return [k for k, (_, npt, seq) in enumerate(L.BULK_SHAPES) if (npt == 1 and seq == 1) or stencil == 0]


@pytest.mark.parametrize("prec", ["fp64", "fp32s"])
@pytest.mark.parametrize("stencil", [0, 1])
def test_launch_shapes(L, prec, stencil):
    """Block sizes, link block sizes and graph lengths change no bits; the
    kernels with one or two nodes per thread, the sequential walk, the link
    kernel with one or four links per thread and the fused step are separate
    compilations of the same arithmetic and agree to rounding (the parity
    bound of 37 steps)."""
    precision = L.LBM_FP64 if prec == "fp64" else L.LBM_FP32_SHIFTED
    if stencil == 0:
        geo = G.build(0, (83, 41, 1), (1, 1, 1), [G.ball((30.37, 20.61, 0), 7.3, force_id=0)])
    else:
        geo = G.sphere_pack(24, porosity=0.5, rmin=2.5, rmax=4.5, seed=3)
    ref = {}
    for fused in (0, 1):
        for shape in _shapes(L, stencil):
            npt = L.BULK_SHAPES[shape][1:]
            if fused and npt != (1, 1):
                continue  # the fused kernel takes one node per thread
            for lt, gs, ls in ((256, 2, 1), (64, 8, 4), (128, 32, 4)):
                # the link kernel with 1 and 4 links per thread: two compilations
                key = (fused,) + npt + ((0 if fused else ls),)
                with L.Lattice(geo, precision=precision, bc=2, tau=0.7, g=(1e-5, 0, 0)) as lat:
                    lat.set_tuning(bulk_shape=shape, link_threads=lt, graph_steps=gs, link_seq=ls, fused=fused)
                    lat.init_equilibrium()
                    lat.step(37)
                    f = lat.distributions()
                ref.setdefault(key, f)
                assert np.array_equal(f, ref[key]), (fused, shape, lt, gs, ls)
    _, w = O.velocity_set(stencil)
    base = ref[(0, 1, 1, 1)]
    h = np.abs(base - (w[:, None] if precision == L.LBM_FP32_SHIFTED else 0.0)).max()
    tol = 1e-12 if precision == L.LBM_FP64 else 4 * 37 * EPS32 * h
    for key, f in ref.items():
        assert np.abs(f - base).max() <= tol, key


def test_autotune_restores_state_and_picks_a_valid_shape(L):
    specs = _small_specs(6, seed=2)
    b = B.stack(specs)
    lat = _batch_lattice(L, b, L.LBM_FP32_SHIFTED)
    lat.step(9)
    F0 = lat.forces()
    f0 = lat.distributions()
    t, ms = lat.autotune(10)
    assert ms > 0 and 0 <= t.bulk_shape < 8 and t.link_threads in (64, 128, 256) and t.graph_steps % 2 == 0
    assert t.link_seq in (1, 4) and t.fused in (0, 1)
    assert lat.tuning().bulk_shape == t.bulk_shape and lat.tuning().fused == t.fused
    assert lat.info().step == 9
    assert np.array_equal(lat.distributions(), f0)
    assert np.array_equal(lat.forces(), F0)
    lat.step(20)
    f1 = lat.distributions()
    lat.close()
    lat2 = _batch_lattice(L, b, L.LBM_FP32_SHIFTED)
    lat2.set_tuning(bulk_shape=t.bulk_shape, link_threads=256, graph_steps=2, link_seq=1, fused=t.fused)
    lat2.step(29)
    assert np.array_equal(lat2.distributions(), f1)
    lat2.close()


def test_set_domains_rejects_bad_tables(L):
    specs = _small_specs(2, seed=1)
    b = B.stack(specs)
    geo = b.geometry
    base = dict(stencil=0, nx=geo.nx, ny=geo.ny, nz=1, periodic=geo.periodic, inlet=1, outlet=1, tau=0.8,
                inlet_y0=0.0, inlet_y1=1.0)
    bad = [dict(b.domains[0], lo=1), dict(b.domains[0], n=2), dict(b.domains[0], nx=geo.nx + 1),
           dict(b.domains[0], tau=0.5)]
    for row in bad:
        h = L.lbm_create_lattice(L.make_config(**base))
        with pytest.raises(L.LBMError) as e:
            L.lbm_set_domains(h, [row, b.domains[1]])
        assert e.value.status == L.LBM_ERR_INVALID_ARG
        L.lbm_destroy(h)
    # rows do not cover the lattice
    h = L.lbm_create_lattice(L.make_config(**base))
    with pytest.raises(L.LBMError):
        L.lbm_set_domains(h, b.domains[:1])
    # a fluid node in a domain's boundary row
    L.lbm_set_domains(h, b.domains)
    solid = geo.solid.copy()
    solid[geo.nx * (b.domains[1]["lo"]) + 5] = 0
    with pytest.raises(L.LBMError) as e:
        L.lbm_set_geometry(h, solid, geo.links)
    assert e.value.status == L.LBM_ERR_INVALID_ARG
    # domains after the geometry
    L.lbm_set_geometry(h, geo.solid, geo.links)
    with pytest.raises(L.LBMError) as e:
        L.lbm_set_domains(h, b.domains)
    assert e.value.status == L.LBM_ERR_STATE
    L.lbm_destroy(h)


def _slab(nx, ny, nzf, q_lo, q_hi, sphere):
    """D3Q19 slab channel: walls normal to z at q_lo below the first and q_hi
    above the last of nzf fluid layers (one solid layer each side), periodic
    in x and y, one sphere (force id 0)."""
    bodies = [G.halfspace((0, 0, -1), -(1.0 - q_lo), force_id=-1),
              G.halfspace((0, 0, 1), nzf + q_hi, force_id=-1),
              G.ball(sphere[:3], sphere[3], force_id=0)]
    return G.build(1, (nx, ny, nzf + 2), (True, True, False), bodies)


@pytest.mark.parametrize("prec", ["fp64", "fp32s"])
def test_d3q19_domains_stacked_along_z_equal_domains_alone(L, prec):
    """D3Q19 domains stack along z (the last axis): two slab channels with
    their own tau and body force, each equal bit for bit to the same slab run
    as a lattice of its own."""
    precision = L.LBM_FP64 if prec == "fp64" else L.LBM_FP32_SHIFTED
    parts = [(_slab(14, 12, 9, 0.3, 0.6, (6.3, 5.7, 5.2, 2.6)), 0.7, (1e-5, 0.0, 0.0)),
             (_slab(14, 12, 13, 0.45, 0.8, (8.1, 6.4, 7.3, 3.4)), 0.9, (0.0, 2e-5, 0.0))]
    nx, ny = 14, 12
    nz = sum(g.nz for g, _, _ in parts)
    solid = np.ones(nx * ny * nz, np.uint8)
    links, rows, z0, b0 = [], [], 0, 0
    for g, tau, gv in parts:
        solid[nx * ny * z0:nx * ny * (z0 + g.nz)] = g.solid
        lk = g.links.copy()
        lk["node"] += nx * ny * z0
        lk["body"] = np.where(lk["body"] >= 0, lk["body"] + b0, -1)
        links.append(lk)
        rows.append(dict(lo=z0, n=g.nz, nx=nx, tau=tau, g=gv))
        z0 += g.nz
        b0 += 1
    links = np.concatenate(links)
    with L.Lattice(None, domains=rows, stencil=1, nx=nx, ny=ny, nz=nz, periodic=(1, 1, 0), tau=1.0, bc=2,
                   precision=precision) as lat:
        lat.set_geometry(solid, links)
        lat.init_equilibrium()
        lat.step(61)
        f = lat.distributions()
        F = lat.forces()
        assert lat.info().n_domains == 2
    z0 = 0
    for d, (g, tau, gv) in enumerate(parts):
        with L.Lattice(g, precision=precision, tau=tau, g=gv, bc=2) as one:
            one.init_equilibrium()
            one.step(61)
            f1 = one.distributions()
            F1 = one.force(0)
        sl = slice(nx * ny * z0, nx * ny * (z0 + g.nz))
        assert np.array_equal(f[:, sl], f1), d
        # the sums run in another order; small components are differences of
        # O(max |F|) link terms
        rtol = 1e-12 if precision == L.LBM_FP64 else 1e-5
        assert np.allclose(F[d], F1, rtol=rtol, atol=rtol * 10 * np.abs(F1).max()), (d, F[d], F1)
        z0 += g.nz
