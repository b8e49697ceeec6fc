"""Pins for the oracle's mesh topology and geometry (Sec. 3.1, Eq. cs1_discr).

Closed forms on the unjittered equilateral lattice, properties of the
circumcentre and of closed polygons on jittered meshes, and a brute-force
side pairing."""
import math

import numpy as np
import pytest

import oracle
import synth

S3 = math.sqrt(3.0)


def test_topology_matches_brute_force_pairing():
    m = synth.lattice(7, seed=3)
    nbr = oracle.topology(m.tri)
    nt = m.nt
    for e in range(nt):
        for j in range(3):
            side = {int(m.tri[e, (j + 1) % 3]), int(m.tri[e, (j + 2) % 3])}
            others = [f for f in range(nt) if f != e and side <= set(int(v) for v in m.tri[f])]
            assert len(others) <= 1
            assert nbr[e, j] == (others[0] if others else -1)


def test_topology_rejects_a_side_shared_by_three_cells():
    tri = np.array([[0, 1, 2], [1, 0, 3], [0, 1, 4]], dtype=np.int32)
    with pytest.raises(oracle.OracleError) as ei:
        oracle.topology(tri)
    assert ei.value.code == oracle.ERR_NONMANIFOLD


def test_equilateral_lattice_closed_forms():
    n = 9
    m = synth.lattice(n, jitter=0.0)
    g = oracle.geometry(m.xy, m.tri)
    np.testing.assert_allclose(g.area, S3 / 4, rtol=1e-14)
    np.testing.assert_allclose(g.length, 1.0, rtol=1e-14)
    inner = g.nbr >= 0
    # circumcentre distance across a side: twice the inradius 1/(2 sqrt 3)
    np.testing.assert_allclose(g.dist[inner], 1 / S3, rtol=1e-13)
    # boundary: circumcentre to side = inradius
    np.testing.assert_allclose(g.dist[~inner], 1 / (2 * S3), rtol=1e-13)
    # circumcentre of an equilateral triangle is its centroid
    np.testing.assert_allclose(g.cc, synth.cell_centroids(m), atol=1e-13)
    # normals of up triangles point at -90, 30, 150 degrees (some order)
    ang = np.degrees(np.arctan2(g.normal[..., 1], g.normal[..., 0]))
    up = np.sort(np.round(ang[0::2]), axis=1)
    down = np.sort(np.round(ang[1::2]), axis=1)
    assert np.all(up == np.array([-90.0, 30.0, 150.0]))
    assert np.all(down == np.array([-150.0, -30.0, 90.0]))


def test_right_triangle_hand_values():
    xy = np.array([[0.0, 0.0], [2.0, 0.0], [0.0, 2.0]])
    tri = np.array([[0, 1, 2]], dtype=np.int32)
    g = oracle.geometry(xy, tri)
    assert g.area[0] == pytest.approx(2.0)
    np.testing.assert_allclose(g.cc[0], [1.0, 1.0], atol=1e-15)
    # side 0 joins (2,0)-(0,2): length 2 sqrt 2, outward normal (1,1)/sqrt2,
    # and the circumcentre lies on it (right angle): delta = 0
    assert g.length[0, 0] == pytest.approx(2 * math.sqrt(2))
    np.testing.assert_allclose(g.normal[0, 0], [1 / math.sqrt(2), 1 / math.sqrt(2)])
    assert abs(g.dist[0, 0]) < 1e-15
    # side 1 joins (0,2)-(0,0): normal (-1, 0), delta = 1
    np.testing.assert_allclose(g.normal[0, 1], [-1.0, 0.0], atol=1e-15)
    assert g.dist[0, 1] == pytest.approx(1.0)
    # side 2 joins (0,0)-(2,0): normal (0, -1), delta = 1
    np.testing.assert_allclose(g.normal[0, 2], [0.0, -1.0], atol=1e-15)
    assert g.dist[0, 2] == pytest.approx(1.0)


def test_clockwise_triangle_is_rejected():
    xy = np.array([[0.0, 0.0], [0.0, 1.0], [1.0, 0.0]])
    with pytest.raises(oracle.OracleError) as ei:
        oracle.geometry(xy, np.array([[0, 1, 2]], dtype=np.int32))
    assert ei.value.code == oracle.ERR_ORIENTATION


@pytest.mark.parametrize("seed,defects", [(0, False), (5, False), (2, True)])
def test_jittered_mesh_geometric_identities(seed, defects):
    n = 20
    m = synth.defect_lattice(n, seed=seed) if defects else synth.lattice(n, seed=seed)
    g = oracle.geometry(m.xy, m.tri)
    p = m.xy[m.tri]                                   # [nt, 3, 2]
    r = np.linalg.norm(p - g.cc[:, None, :], axis=2)  # circumradius thrice
    np.testing.assert_allclose(r[:, 1], r[:, 0], rtol=1e-12)
    np.testing.assert_allclose(r[:, 2], r[:, 0], rtol=1e-12)
    # a closed polygon: sum_j l_j n_j = 0
    s = (g.length[..., None] * g.normal).sum(axis=1)
    assert np.abs(s).max() < 1e-13
    # outward: the normal points from the centroid toward the side midpoint
    mid = 0.5 * (p[:, [1, 2, 0], :] + p[:, [2, 0, 1], :])
    cen = p.mean(axis=1)
    assert np.all(((mid - cen[:, None, :]) * g.normal).sum(axis=2) > 0)
    # area is conserved (boundary vertices are fixed): (n-1)^2 sqrt3 / 2
    assert g.area.sum() == pytest.approx((n - 1) ** 2 * S3 / 2, rel=1e-13)
    # Delaunay: d_{e,ep} > 0 equals |c_ep - c_e| and is symmetric
    e, j = np.nonzero(g.nbr >= 0)
    ep = g.nbr[e, j]
    dcc = np.linalg.norm(g.cc[ep] - g.cc[e], axis=1)
    assert np.all(g.dist[e, j] > 0)
    np.testing.assert_allclose(g.dist[e, j], dcc, rtol=1e-9)
    back = np.array([list(g.nbr[b]).index(a) for a, b in zip(e, ep)])
    np.testing.assert_allclose(g.dist[ep, back], g.dist[e, j], rtol=1e-13)
    np.testing.assert_allclose(g.normal[ep, back], -g.normal[e, j], atol=1e-15)
