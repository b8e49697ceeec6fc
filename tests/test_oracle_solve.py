"""Pins for the oracle's solvers: dense brute force, IC(0) special cases,
agreement between preconditioners, and the discretisation's convergence
order under refinement (Eq. error, Eq. conv_order)."""
import math

import numpy as np
import pytest

import oracle
import synth


def test_dense_cholesky_matches_library_solve():
    rng = np.random.default_rng(0)
    M = rng.standard_normal((40, 40))
    A = M @ M.T + 40 * np.eye(40)
    b = rng.standard_normal(40)
    x = oracle.dense_cholesky_solve(A, b)
    np.testing.assert_allclose(x, np.linalg.solve(A, b), rtol=1e-12)


def test_dense_cholesky_rejects_indefinite():
    with pytest.raises(oracle.OracleError):
        oracle.dense_cholesky_solve(np.array([[1.0, 2.0], [2.0, 1.0]]), np.ones(2))


@pytest.mark.parametrize("maker", [lambda: synth.centred_block_problem(16, seed=0),
                                   lambda: synth.channel_block_problem(16, seed=1)])
def test_pcg_matches_dense_cholesky_on_tiny_mesh(maker):
    p = maker()
    A = oracle.assemble_problem(p)
    b = synth.rhs(p.mesh, 123)
    xd = oracle.dense_cholesky_solve(A.dense(), b)
    for pc, perm in [(oracle.PC_JACOBI, None), (oracle.PC_IC0, None),
                     (oracle.PC_IC0, oracle.red_black_order(A.n)), (oracle.PC_NONE, None)]:
        x, st = oracle.pcg(A, b, rtol=1e-14, precond=pc, perm=perm, raise_on_error=False)
        assert st.status in (oracle.OK, oracle.ERR_NOT_CONVERGED)
        assert np.linalg.norm(x - xd) / np.linalg.norm(xd) < 1e-11, (pc, perm is not None)


def _strip_mesh(k):
    """One row strip of 2(k-1) triangles: the cell graph is a path."""
    m = synth.lattice(k, jitter=0.0)
    return m.xy[: 2 * k], m.tri[: 2 * (k - 1)]


def test_ic0_is_exact_cholesky_on_a_path_graph():
    """With no fill (a path in natural order) IC(0) is the exact factor, so
    PCG converges in a single iteration."""
    xy, tri = _strip_mesh(30)
    nt = tri.shape[0]
    nbr = oracle.topology(tri)
    assert np.all((nbr >= 0).sum(axis=1) <= 2)
    # Dirichlet at the rightmost boundary side
    last = nt - 1
    bside = [last * 3 + j for j in range(3) if nbr[last, j] < 0]
    eps = np.linspace(0.4, 1.0, xy.shape[0])
    A = oracle.assemble(xy, tri, np.array(bside[:1], np.int32), eps,
                        synth.iso_kinv(synth.kozeny_carman_kinv(eps)))
    b = np.random.default_rng(1).standard_normal(nt)
    x, st = oracle.pcg(A, b, rtol=1e-12, precond=oracle.PC_IC0)
    assert st.iters == 1
    np.testing.assert_allclose(x, np.linalg.solve(A.dense(), b), rtol=1e-10)


def test_red_black_ic0_first_step_matches_closed_form():
    """On the two-coloured lattice IC(0) in red/black order has L = A's
    pattern with black pivots d'_i = a_ii - sum_red a_ij^2 / a_jj.  The first
    PCG iterate from x0 = 0 is x1 = (b.z / z.Az) z with z = M^-1 b."""
    p = synth.channel_block_problem(12, seed=2)
    A = oracle.assemble_problem(p)
    D = A.dense()
    n = A.n
    red = np.arange(0, n, 2)
    blk = np.arange(1, n, 2)
    assert np.all(D[np.ix_(red, red)] == np.diag(np.diag(D)[red]))   # bipartite
    b = synth.rhs(p.mesh, 7)
    dr = np.diag(D)[red]
    E = D[np.ix_(red, blk)]
    dpb = np.diag(D)[blk] - (E * E / dr[:, None]).sum(axis=0)
    # M = (Dt + L) Dt^-1 (Dt + U): forward then backward block sweeps
    wr = b[red] / dr
    wb = (b[blk] - E.T @ wr) / dpb
    zb = wb
    zr = wr - (E @ zb) / dr
    z = np.empty(n)
    z[red] = zr
    z[blk] = zb
    x1_want = (b @ z) / (z @ D @ z) * z
    x1, st = oracle.pcg(A, b, rtol=0.0, maxit=1, precond=oracle.PC_IC0,
                        perm=oracle.red_black_order(n), raise_on_error=False)
    assert st.iters == 1
    np.testing.assert_allclose(x1, x1_want, rtol=1e-11)


def test_jacobi_first_step_matches_closed_form():
    p = synth.centred_block_problem(12, seed=3)
    A = oracle.assemble_problem(p)
    D = A.dense()
    b = synth.rhs(p.mesh, 8)
    z = b / np.diag(D)
    x1_want = (b @ z) / (z @ D @ z) * z
    x1, _ = oracle.pcg(A, b, rtol=0.0, maxit=1, precond=oracle.PC_JACOBI,
                       raise_on_error=False)
    np.testing.assert_allclose(x1, x1_want, rtol=1e-12)


def test_preconditioners_reach_the_same_solution():
    p = synth.channel_block_problem(40, seed=5)
    A = oracle.assemble_problem(p)
    b = synth.rhs(p.mesh, 9)
    xs = []
    for pc, perm in [(oracle.PC_JACOBI, None), (oracle.PC_IC0, None),
                     (oracle.PC_IC0, oracle.red_black_order(A.n))]:
        x, st = oracle.pcg(A, b, rtol=1e-13, precond=pc, perm=perm, raise_on_error=False)
        assert st.rel_res < 1e-12
        xs.append(x)
    for x in xs[1:]:
        assert np.linalg.norm(x - xs[0]) / np.linalg.norm(xs[0]) < 1e-9


def test_warm_start_and_zero_rhs():
    p = synth.centred_block_problem(12)
    A = oracle.assemble_problem(p)
    b = synth.rhs(p.mesh, 1)
    x, st = oracle.pcg(A, b, rtol=1e-12)
    x2, st2 = oracle.pcg(A, b, x0=x, rtol=1e-10)
    assert st2.iters == 0
    np.testing.assert_array_equal(x2, x)
    z, stz = oracle.pcg(A, np.zeros(A.n), x0=np.ones(A.n), rtol=1e-10)
    assert np.all(z == 0) and stz.iters == 0


def test_max_iter_reports_not_converged():
    p = synth.centred_block_problem(16)
    A = oracle.assemble_problem(p)
    x, st = oracle.pcg(A, synth.rhs(p.mesh, 1), rtol=1e-12, maxit=3, raise_on_error=False)
    assert st.status == oracle.ERR_NOT_CONVERGED and st.iters == 3


def _manufactured_error(n, jitter):
    """-div(Xi grad eta) = f on [0,1] x [0, sqrt3/2], Xi = dt I (clear fluid),
    eta = sin(pi x) sin(pi y) + x y, Dirichlet data on every boundary side.
    Returns (h, area-weighted L2 error at circumcentres) as in Eq. error."""
    m = synth.lattice(n, seed=n, jitter=jitter)
    s = 1.0 / (n - 1)
    xy = m.xy * s
    nbr = oracle.topology(m.tri)
    e, j = np.nonzero(nbr < 0)
    bsides = (e * 3 + j).astype(np.int32)
    eps = np.ones(m.nv)
    kinv = np.zeros((m.nv, 3))
    A = oracle.assemble(xy, m.tri, bsides, eps, kinv)
    T, sigma, isd, _ = oracle.side_coefficients(xy, m.tri, bsides, eps, kinv,
                                                oracle.PER_VERTEX, oracle.CP2, synth.NU,
                                                synth.DT)
    g = oracle.geometry(xy, m.tri)
    ex = lambda x, y: np.sin(math.pi * x) * np.sin(math.pi * y) + x * y
    lap = lambda x, y: -2 * math.pi ** 2 * np.sin(math.pi * x) * np.sin(math.pi * y)
    # f = -dt * lap(eta), integrated per cell with the 3 edge-midpoint rule
    p = xy[m.tri]
    mids = 0.5 * (p[:, [1, 2, 0], :] + p[:, [2, 0, 1], :])
    f = -synth.DT * lap(mids[..., 0], mids[..., 1]).mean(axis=1) * g.area
    # Dirichlet sides carry eta(midpoint) with coefficient T
    f += (T * isd * ex(mids[..., 0], mids[..., 1])).sum(axis=1)
    x, st = oracle.pcg(A, f, rtol=1e-13, precond=oracle.PC_IC0, raise_on_error=False)
    err = x - ex(g.cc[:, 0], g.cc[:, 1])
    return s, math.sqrt(np.sum(g.area * err ** 2))


@pytest.mark.parametrize("jitter", [0.0, 0.05])
def test_convergence_order_under_refinement(jitter):
    """r_c of Eq. conv_order between successive halvings of h is >= 1.5
    (second order on these near-uniform Delaunay meshes)."""
    res = [_manufactured_error(n, jitter) for n in (9, 17, 33, 65)]
    rates = [math.log(res[i][1] / res[i + 1][1]) / math.log(res[i][0] / res[i + 1][0])
             for i in range(len(res) - 1)]
    assert res[-1][1] < res[0][1] / 20
    assert min(rates[1:]) > 1.5, rates
