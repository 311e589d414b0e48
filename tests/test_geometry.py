"""The geometry builder (input generator shared by the CUDA path and the
oracle): every cut link is present exactly once, and each q is the first wall
crossing along the link (Sec. 3: q = |x_f - x_w| / |x_f - x_s|), checked by
sampling the solid indicator along the link and bisecting it."""
import numpy as np
import pytest

from paper_1903_01111_gb300 import geometry as G


def _inside_any(bodies, x, shape, periodic):
    x = np.asarray(x, float)
    kind = bodies["kind"]
    hs = kind == G.HALFSPACE
    if hs.any() and np.any(bodies["c"][hs] @ x >= bodies["r"][hs]):
        return True
    d = x[None, :] - bodies["c"]
    for a, L in enumerate(shape):
        if periodic[a]:
            d[:, a] -= L * np.floor(d[:, a] / L + 0.5)
    r2 = (d * d).sum(1)
    rr = bodies["r"] ** 2
    return bool(np.any((kind == G.BALL) & (r2 <= rr)) or np.any((kind == G.CAVITY) & (r2 >= rr)))


def _check(geo, sample=400, seed=0):
    E = G.velocity_set(geo.stencil)
    shape = geo.shape
    L = np.array(shape)
    nx, ny, nz = shape
    solid = geo.solid.reshape(nz, ny, nx)
    # completeness: every (fluid node, dir) with a solid neighbour has one link
    keys = set(zip(geo.links["node"].tolist(), geo.links["dir"].tolist()))
    assert len(keys) == len(geo.links)
    fluid = np.flatnonzero(geo.solid == 0)
    x, y, z = geo.coords(fluid)
    open_lo, open_hi = geo.open_x
    expected = 0
    for d in range(1, len(E)):
        s = np.stack([x + E[d][0], y + E[d][1], z + E[d][2]], 1)
        ok = np.ones(len(fluid), bool)
        if open_lo:
            ok &= x != 0
        if open_hi:
            ok &= x != nx - 1
        for a in range(3):
            if not geo.periodic[a]:
                ok &= (s[:, a] >= 0) & (s[:, a] < L[a])
        s = s % L
        hit = ok & (solid[s[:, 2], s[:, 1], s[:, 0]] == 1)
        expected += int(hit.sum())
        for n in fluid[hit][:50]:
            assert (int(n), d) in keys
    assert expected == len(geo.links)
    # q: first crossing along the link
    rng = np.random.default_rng(seed)
    idx = rng.choice(len(geo.links), size=min(sample, len(geo.links)), replace=False)
    for k in idx:
        lk = geo.links[k]
        xf = np.array(geo.coords(lk["node"]), float).reshape(3)
        e = E[lk["dir"]].astype(float)
        q = lk["q"]
        assert 0 < q <= 1
        ts = np.linspace(0, q, 64)[:-1]
        assert not any(_inside_any(geo.bodies, xf + t * e, shape, geo.periodic) for t in ts)
        lo, hi = 0.0, min(1.0, q + 1e-6)
        assert _inside_any(geo.bodies, xf + hi * e, shape, geo.periodic)
        for _ in range(60):
            mid = 0.5 * (lo + hi)
            if _inside_any(geo.bodies, xf + mid * e, shape, geo.periodic):
                hi = mid
            else:
                lo = mid
        assert abs(hi - q) < 1e-9


def test_channel_links():
    g = G.channel(0, 8, 6, q_lo=0.3, q_hi=0.8)
    _check(g)
    assert np.allclose(g.links["q"][g.links["dir"] == 4], 0.3)  # straight down
    assert np.allclose(g.links["q"][g.links["dir"] == 2], 0.8)  # straight up
    g3 = G.channel(1, 6, 5, nz=4, q_lo=0.45, q_hi=0.1)
    _check(g3)


def test_cylinder_links():
    g = G.build(0, (40, 30, 1), (1, 1, 1), [G.ball((17.3, 14.6, 0), 6.4)])
    _check(g)


def test_rotating_ball_wall_velocity():
    om = 0.013
    c = np.array([17.3, 14.6, 0.0])
    g = G.build(0, (40, 30, 1), (1, 1, 1), [G.ball(c, 6.4, omega=(0, 0, om))])
    E = G.velocity_set(0)
    for lk in g.links:
        xf = np.array(g.coords(lk["node"]), float).reshape(3)
        r = xf + lk["q"] * E[lk["dir"]] - c
        assert abs(np.linalg.norm(lk["uw"]) - om * 6.4) < 1e-12
        assert abs(float(lk["uw"] @ r)) < 1e-12


def test_couette_cavity_links():
    g = G.couette(20, 0.002)
    _check(g)


def test_sphere_pack_links_and_porosity():
    g = G.sphere_pack(40, porosity=0.4, rmin=3, rmax=6, seed=3)
    assert 0.39 < g.info["porosity"] <= 0.40
    _check(g, sample=300)


def test_sphere_pack_is_seeded():
    a = G.sphere_pack(24, porosity=0.5, rmin=2, rmax=4, seed=5)
    b = G.sphere_pack(24, porosity=0.5, rmin=2, rmax=4, seed=5)
    assert np.array_equal(a.solid, b.solid) and np.array_equal(a.links, b.links)


def test_open_channel_has_no_links_on_open_columns():
    g = G.channel(0, 12, 5, open_x=(True, True), bc_lo=0, bc_hi=0)
    x, _, _ = g.coords(g.links["node"])
    assert x.min() >= 1 and x.max() <= 10
    _check(g)


def test_nonperiodic_face_without_solid_layer_is_rejected():
    with pytest.raises(ValueError):
        G.build(0, (8, 6, 1), (1, 0, 1), [])


def test_ball_wider_than_half_a_period_is_rejected():
    """On a periodic axis the link builder sees each ball through its nearest
    image from x_f; a ball whose radius reaches half the period minus one
    could leave a solid neighbour without a wall crossing, so it is rejected
    with the limit in the message (a sphere-pack cube smaller than its
    largest sphere allows, here 16^3 for radii up to 14, is the usual way to
    meet it); just below the limit the build succeeds."""
    with pytest.raises(ValueError, match="half the period minus one"):
        G.sphere_pack(16, porosity=0.40, rmin=6.0, rmax=14.0, seed=0)
    with pytest.raises(ValueError, match="half the period minus one"):
        G.build(0, (20, 30, 1), (1, 1, 1), [G.ball((10.3, 15.2, 0), 9.0)])
    g = G.build(0, (20, 30, 1), (1, 1, 1), [G.ball((10.3, 15.2, 0), 8.9)])
    assert len(g.links) > 0
    # a non-periodic axis imposes no such limit
    walls = [G.halfspace((0, -1), -0.5), G.halfspace((0, 1), 18.5)]  # solid at y <= 0.5 and y >= 18.5
    g = G.build(0, (40, 20, 1), (1, 0, 1), [G.ball((20.3, 10.2, 0), 8.0)] + walls)
    assert len(g.links) > 0
