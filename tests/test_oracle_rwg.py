"""Pins of the oracle's RWG functions and box grouping (Sec. II.A, ref. [20])."""
import math

import numpy as np

from oracle import farfield, groups, rwg
from paper_2103_05822_gb300.inputs import icosphere


def test_rwg_count_on_closed_sphere():
    for nu in (1, 3, 5):
        v, f = icosphere(1.0, nu)
        r = rwg.build_rwg(v, f)
        assert r.n == 30 * nu * nu
        assert np.all(r.tri[:, 0] < r.tri[:, 1])
        assert np.all(r.edge[:, 0] < r.edge[:, 1])
        # ascending edge order
        key = r.edge[:, 0] * (len(v) + 1) + r.edge[:, 1]
        assert np.all(np.diff(key) > 0)
        # free vertices are the third vertex of each triangle
        for s in range(2):
            t = f[r.tri[:, s]]
            assert np.all((t == r.free[:, s:s + 1]).any(axis=1))
            assert np.all(r.free[:, s] != r.edge[:, 0]) and np.all(r.free[:, s] != r.edge[:, 1])


def test_open_mesh_boundary_edges_carry_no_rwg():
    v = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [1, 1, 0]], float)
    f = np.array([[0, 1, 2], [1, 3, 2]])
    r = rwg.build_rwg(v, f)
    assert r.n == 1 and tuple(r.edge[0]) == (1, 2)
    assert tuple(r.free[0]) == (0, 3)


def test_normal_component_is_one_across_edge():
    """RWG property: the component normal to the common edge is 1 on both sides."""
    v, f = icosphere(1.0, 3)
    r = rwg.build_rwg(v, f)
    for n in range(0, r.n, 7):
        a, b = v[r.edge[n, 0]], v[r.edge[n, 1]]
        mid = 0.5 * (a + b)
        e = (b - a) / np.linalg.norm(b - a)
        for side in range(2):
            p = v[r.free[n, side]]
            m = (mid - p) - np.dot(mid - p, e) * e  # in-plane normal to the edge, away from p
            m /= np.linalg.norm(m)
            val = rwg.evaluate(v, r, n, side, mid)
            expect = 1.0 if side == 0 else -1.0
            assert abs(np.dot(val, m) - expect) < 1e-12


def test_static_moment_closed_form():
    """k -> 0: int b_n dr = l (c_minus - c_plus), c the triangle centroids."""
    v, f = icosphere(1.0, 3)
    r = rwg.build_rwg(v, f)
    ids = np.arange(r.n)
    pts, amp = farfield.rwg_quadrature(v, r, ids, order=3)
    got = amp.sum(axis=1)
    cp = v[f[r.tri[:, 0]]].mean(axis=1)
    cm = v[f[r.tri[:, 1]]].mean(axis=1)
    expect = r.length[:, None] * (cm - cp)
    assert np.allclose(got, expect, atol=1e-14, rtol=0)
    # divergence integrates to zero over the support: (l/A+) A+ - (l/A-) A- = 0
    for n in range(5):
        assert abs(rwg.divergence(r, n, 0) * r.area[n, 0] + rwg.divergence(r, n, 1) * r.area[n, 1]) < 1e-13


def test_groups_partition_and_order():
    v, f = icosphere(2.0, 6)
    r = rwg.build_rwg(v, f)
    mp = rwg.midpoints(v, r)
    g = groups.make_groups(mp, 0.5)
    allids = np.sort(np.concatenate(g.members))
    assert np.array_equal(allids, np.arange(r.n))
    lin = g.box_index[:, 0] + g.K[0] * (g.box_index[:, 1] + g.K[1] * g.box_index[:, 2])
    assert np.all(np.diff(lin) > 0)
    for gi, ids in enumerate(g.members):
        assert np.all(np.diff(ids) > 0)
        d = np.abs(mp[ids] - g.centre[gi])
        assert np.all(d <= 0.5 * g.box + 1e-12)
    assert g.K == tuple(max(1, math.ceil(e / 0.5)) for e in (mp.max(0) - mp.min(0)))
