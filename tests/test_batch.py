"""Host side of batches: the seeded channel workload and the stacking maps
(no GPU)."""
import numpy as np

from paper_1903_01111_gb300 import batch as B


def test_draw_is_seeded_and_within_ranges():
    a = B.draw_channels(40, seed=4)
    b = B.draw_channels(40, seed=4)
    assert [(s.nx, s.ny_fluid, s.cylinders, s.re) for s in a] == [(s.nx, s.ny_fluid, s.cylinders, s.re) for s in b]
    for s in a:
        assert 64 <= s.nx <= 512 and 64 <= s.ny_fluid <= 256 and 10 <= s.re <= 100
        assert 1 <= len(s.cylinders) <= 8
        assert s.tau > 0.5
        assert B.blockage(s) <= 0.4 + 1e-12
        for i, (x, y, r) in enumerate(s.cylinders):
            assert 4.0 <= r <= min(20.0, s.ny_fluid / 6) + 1e-12
            assert r + 8 <= x <= s.nx - r - 16
            assert y - r >= 3.0 - 1e-9 and y + r <= s.ny_fluid - 1 - 3.0 + 1e-9
            for (x2, y2, r2) in s.cylinders[i + 1:]:
                assert np.hypot(x - x2, y - y2) >= r + r2 + 3.0 - 1e-9


def test_reynolds_number_sets_tau():
    s = B.DomainSpec(100, 64, [(30.2, 31.7, 5.1)], re=40.0, u_max=0.1)
    nu = (2 / 3) * 0.1 * 64 / 40.0
    assert abs(s.tau - (3 * nu + 0.5)) < 1e-15


def test_stack_places_every_domain_block():
    specs = B.draw_channels(7, seed=9, nx_range=(30, 70), ny_range=(12, 30), n_cyl=(1, 3), r_range=(2.0, 5.0))
    b = B.stack(specs)
    g = b.geometry
    assert g.nx == max(s.nx for s in specs) and g.ny == sum(s.ny for s in specs)
    covered = np.zeros(g.N, bool)
    for d, (s, part) in enumerate(zip(specs, b.parts)):
        nodes = b.domain_nodes(d)
        assert np.array_equal(g.solid[nodes], part.solid)
        covered[nodes] = True
        lk = g.links[b.domain_links(d)]
        assert np.array_equal(lk["node"], nodes[part.links["node"]])
        assert np.array_equal(lk["q"], part.links["q"]) and np.array_equal(lk["dir"], part.links["dir"])
        body = part.links["body"]
        assert np.array_equal(lk["body"], np.where(body >= 0, body + b.body0[d], -1))
        row = b.domains[d]
        assert row["lo"] == b.lo[d] and row["n"] == s.ny and row["nx"] == s.nx and row["tau"] == s.tau
        # the first and last row of every domain are solid (its walls)
        m = g.solid.reshape(g.ny, g.nx)
        assert m[b.lo[d]].all() and m[b.lo[d] + s.ny - 1].all()
    assert np.all(g.solid[~covered] == 1)
    assert b.n_fluid == sum(p.fluid_count() for p in b.parts)
    assert b.n_bodies == sum(len(s.cylinders) for s in specs)


def test_shards_cover_every_domain_once():
    specs = B.draw_channels(13, seed=1)
    got = []
    for r in range(4):
        got += B.shard(specs, r, 4)
    assert sorted(id(s) for s in got) == sorted(id(s) for s in specs)
