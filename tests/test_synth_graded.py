"""The graded unstructured Delaunay mesh generator (the stand-in for the
paper's refined transition-layer meshes): a valid counter-clockwise disk
triangulation that is Delaunay (checked by brute force against every
circumcircle, independent of the triangulation library), graded (cell areas
spanning the refinement levels), not two-colourable (so IC(0) takes the
greedy multicolour path), and numbered for locality along a Morton curve."""
import collections

import numpy as np
import pytest

import oracle
import synth

pytest.importorskip("scipy")


def _circumcircles(xy, tri):
    a, b, c = xy[tri[:, 0]], xy[tri[:, 1]], xy[tri[:, 2]]
    bx, by = b[:, 0] - a[:, 0], b[:, 1] - a[:, 1]
    cx, cy = c[:, 0] - a[:, 0], c[:, 1] - a[:, 1]
    d = 2.0 * (bx * cy - by * cx)
    ux = (cy * (bx * bx + by * by) - by * (cx * cx + cy * cy)) / d
    uy = (bx * (cx * cx + cy * cy) - cx * (bx * bx + by * by)) / d
    centre = a + np.stack([ux, uy], axis=1)
    return centre, ux * ux + uy * uy


def test_graded_mesh_is_a_delaunay_disk_triangulation():
    m = synth.graded_mesh(9, seed=3)
    xy, tri = m.xy, m.tri
    # counter-clockwise, every vertex used
    a, b, c = xy[tri[:, 0]], xy[tri[:, 1]], xy[tri[:, 2]]
    cross = (b[:, 0] - a[:, 0]) * (c[:, 1] - a[:, 1]) - (b[:, 1] - a[:, 1]) * (c[:, 0] - a[:, 0])
    assert np.all(cross > 0)
    assert np.unique(tri).size == m.nv
    # a disk: V - E + F = 1, and each side shared by at most two cells
    nbr = oracle.topology(tri)
    n_bnd = int((nbr < 0).sum())
    n_sides = (3 * m.nt + n_bnd) // 2
    assert m.nv - n_sides + m.nt == 1
    # empty circumcircles, brute force over all vertices
    centre, r2 = _circumcircles(xy, tri)
    for e in range(m.nt):
        d2 = ((xy - centre[e]) ** 2).sum(axis=1)
        inside = d2 < r2[e] * (1.0 - 1e-9)
        inside[tri[e]] = False
        assert not inside.any(), e


@pytest.mark.parametrize("n,seed", [(6, 0), (24, 1), (64, 2)])
def test_graded_problem_assembles_as_an_m_matrix(n, seed):
    p = synth.graded_problem(n, seed=seed)
    A = oracle.assemble_problem(p)      # raises on d <= 0 (interior or Dirichlet)
    offdiag = A.val[A.col != np.repeat(np.arange(A.n), np.diff(A.rowptr))]
    assert np.all(offdiag <= 0.0)
    assert p.mesh.dirichlet.size >= n - 1


def test_graded_mesh_is_refined_and_not_two_colourable():
    m = synth.graded_mesh(24, seed=1, levels=2)
    area = synth.triangle_areas(m)
    assert area.max() / area.min() > 8.0     # two halvings of the spacing
    nbr = oracle.topology(m.tri)
    colour = -np.ones(m.nt, dtype=int)
    odd_cycle = False
    for s in range(m.nt):
        if colour[s] >= 0:
            continue
        colour[s] = 0
        queue = collections.deque([s])
        while queue and not odd_cycle:
            e = queue.popleft()
            for f in nbr[e]:
                if f < 0:
                    continue
                if colour[f] < 0:
                    colour[f] = 1 - colour[e]
                    queue.append(f)
                elif colour[f] == colour[e]:
                    odd_cycle = True
    assert odd_cycle


def test_morton_numbering_shortens_neighbour_distances():
    spans = {}
    for order in ("morton", "none"):
        m = synth.graded_mesh(40, seed=2, order=order)
        nbr = oracle.topology(m.tri)
        e, j = np.nonzero(nbr >= 0)
        spans[order] = np.mean(np.abs(nbr[e, j] - e))
    # the triangulation's own numbering is local at the median but has a long
    # tail of far neighbours; the Morton numbering removes most of it
    assert spans["morton"] * 10 < spans["none"]
