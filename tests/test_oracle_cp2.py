"""Pins of the oracle's CP2 step (Sec. 3.2.3, App. A, App. C) against facts the
paper and the mathematics fix, not against the oracle itself:

* Eq. flux_k_+_2/3: a uniform velocity gives its exact side flux; the mean
  flux is antisymmetric across a side; hand-computed area weights on a
  two-triangle mesh.
* Eq. Cs2_6 / App. C (co-normal tangential flux): zero for an isotropic
  tensor; together with the TPFA part it is the exact flux l (Xi g).n of a
  linear eta under a uniform anisotropic tensor (this fixes the co-normal
  components, their signs and the distances); antisymmetric across a side.
* Eq. RT0: a uniform flux field reproduces its velocity exactly.
* Eq. grad_PSI: along an eigenvector of Kinv the update is the closed-form
  eigenvalue of Mbar.
* The whole step: mass balance per cell (Eq. Cs2_5), flux continuity, a
  uniform channel flow passes unchanged, and with an isotropic tensor the
  second solve returns the first (no tangential correction).
"""
import math

import numpy as np
import pytest

import oracle
import synth


def _jp(nbr, e, ep):
    return int(np.nonzero(nbr[ep] == e)[0][0])


def _uniform_problem(n, seed=0, beta=20.0, alpha_deg=30.0, eps0=0.4, field_loc=oracle.PER_VERTEX):
    mesh = synth.lattice(n, seed)
    nf = mesh.xy.shape[0] if field_loc == oracle.PER_VERTEX else mesh.tri.shape[0]
    eps = np.full(nf, eps0)
    kinv = synth.aniso_kinv(np.full(nf, 2.0e4), beta, math.radians(alpha_deg))
    return synth.Problem(mesh, eps, kinv, field_loc)


def _coeffs(p):
    m = p.mesh
    return oracle.side_coefficients(m.xy, m.tri, m.dirichlet, p.eps, p.kinv, p.field_loc,
                                    oracle.CP2, p.nu, p.dt)


def _fields(p):
    return (p.eps, p.kinv, p.field_loc, p.nu, p.dt)


# ------------------------------------------------------------- mean flux

def test_mean_flux_of_uniform_velocity_is_exact():
    p = synth.channel_block_problem(10, seed=3)
    m = p.mesh
    T, _, isd, nbr = _coeffs(p)
    g = oracle.geometry(m.xy, m.tri)
    U = np.array([0.7, -0.3])
    nt = m.tri.shape[0]
    u = np.repeat(U[:, None], nt, axis=1)
    fbar = oracle.cp2_mean_flux(m.xy, m.tri, nbr, isd, u)
    exact = g.length * (g.normal @ U)
    open_side = (nbr >= 0) | (isd != 0)
    np.testing.assert_allclose(fbar[open_side], exact[open_side], rtol=0, atol=1e-14)
    assert np.all(fbar[~open_side] == 0.0)


def test_mean_flux_is_antisymmetric_across_a_side():
    p = synth.channel_block_problem(10, seed=4)
    m = p.mesh
    _, _, isd, nbr = _coeffs(p)
    rng = np.random.default_rng(11)
    u = rng.normal(size=(2, m.tri.shape[0]))
    fbar = oracle.cp2_mean_flux(m.xy, m.tri, nbr, isd, u)
    for e, j in zip(*np.nonzero(nbr >= 0)):
        ep = nbr[e, j]
        assert fbar[e, j] == pytest.approx(-fbar[ep, _jp(nbr, e, ep)], abs=1e-14)


def test_mean_flux_area_weights_by_hand():
    # e = (0,0),(1,0),(0,1): area 1/2; ep = (1,0),(2,2),(0,1): area 3/2.
    # Shared side (1,0)-(0,1) is local side 0 of e: n = (1,1)/sqrt2, l = sqrt2.
    xy = np.array([[0, 0], [1, 0], [0, 1], [2, 2]], dtype=float)
    tri = np.array([[0, 1, 2], [1, 3, 2]], dtype=np.int32)
    nbr = oracle.topology(tri)
    assert nbr[0, 0] == 1
    isd = np.zeros((2, 3), dtype=np.int32)
    # only e moves, with u.n = 1/sqrt2: flux sqrt2 * 1/sqrt2 weighted by A_ep/(A_e+A_ep) = 3/4
    f = oracle.cp2_mean_flux(xy, tri, nbr, isd, np.array([[1.0, 0.0], [0.0, 0.0]]))
    assert f[0, 0] == pytest.approx(0.75, abs=1e-15)
    # only ep moves, (0,2).n = sqrt2 into e: weighted by A_e/(A_e+A_ep) = 1/4, flux -> +0.5 out of e
    f = oracle.cp2_mean_flux(xy, tri, nbr, isd, np.array([[0.0, 0.0], [0.0, 2.0]]))
    assert f[0, 0] == pytest.approx(0.5, abs=1e-15)
    assert f[1, _jp(nbr, 0, 1)] == pytest.approx(-0.5, abs=1e-15)
    # no-flux boundary sides carry nothing
    assert np.all(f[nbr < 0] == 0.0)


# ------------------------------------------------------- tangential flux

def test_tangential_flux_vanishes_for_isotropic_tensor():
    p = synth.centred_block_problem(12, seed=1)
    m = p.mesh
    T, _, isd, nbr = _coeffs(p)
    eta = synth.normal_noise(m.tri.shape[0], 5)
    tau = oracle.cp2_tangential_flux(m.xy, m.tri, nbr, isd, *_fields(p), eta)
    scale = np.abs(T).max() * np.abs(eta).max()
    assert np.abs(tau).max() <= 1e-13 * scale


def _availability(nbr, isd):
    """est[e, j, k]: one-sided estimate k (0: from e, 1: from ep) exists --
    neither of that cell's other two sides is a no-flux side."""
    nt = nbr.shape[0]
    usable = (nbr >= 0) | (isd != 0)
    est = np.zeros((nt, 3, 2), dtype=bool)
    for e in range(nt):
        for j in range(3):
            est[e, j, 0] = usable[e, (j + 1) % 3] and usable[e, (j + 2) % 3]
            ep = nbr[e, j]
            if ep >= 0:
                jp = _jp(nbr, e, ep)
                est[e, j, 1] = usable[ep, (jp + 1) % 3] and usable[ep, (jp + 2) % 3]
    return est


def _touches_boundary(nbr, e, j):
    """Side j of e or any other side of e or ep lies on the boundary."""
    if np.any(nbr[e] < 0):
        return True
    ep = nbr[e, j]
    return bool(np.any(nbr[ep] < 0))


@pytest.mark.parametrize("field_loc", [oracle.PER_VERTEX, oracle.PER_CELL])
def test_flux_of_linear_eta_is_exact_under_uniform_anisotropic_tensor(field_loc):
    """Phi_j = -T_j (eta_e - eta_ep) + tau_j equals l_j (Xi g).n_j for
    eta = a + g.x sampled at circumcentres, on every side away from the
    boundary (the two one-sided co-normal estimates are each exact)."""
    p = _uniform_problem(12, seed=2, field_loc=field_loc)
    m = p.mesh
    T, _, isd, nbr = _coeffs(p)
    g = oracle.geometry(m.xy, m.tri)
    Xi = oracle.xi(p.eps[:1], p.kinv[:1], p.nu, p.dt)[0]
    Xm = np.array([[Xi[0], Xi[1]], [Xi[1], Xi[2]]])
    assert abs(Xm[0, 1]) > 0.1 * Xm[0, 0]          # genuinely anisotropic
    grad = np.array([0.8, -1.3])
    eta = 0.4 + g.cc @ grad
    tau = oracle.cp2_tangential_flux(m.xy, m.tri, nbr, isd, *_fields(p), eta)
    checked = 0
    for e in range(m.tri.shape[0]):
        for j in range(3):
            ep = nbr[e, j]
            if ep < 0 or _touches_boundary(nbr, e, j):
                continue
            phi = -T[e, j] * (eta[e] - eta[ep]) + tau[e, j]
            exact = g.length[e, j] * (Xm @ grad) @ g.normal[e, j]
            assert phi == pytest.approx(exact, rel=1e-11, abs=1e-13 * np.abs(Xm).max())
            checked += 1
    assert checked > 100


def test_flux_of_linear_eta_is_exact_next_to_dirichlet_sides():
    """eta = g_x (x - x_D) vanishes at every Dirichlet midpoint (x_D = n - 3/4
    on the zigzag right edge), so every one-sided estimate that crosses a
    Dirichlet side is exact too; every side with at least one estimate
    carries the exact flux."""
    n = 12
    p = _uniform_problem(n, seed=6)
    m = p.mesh
    T, _, isd, nbr = _coeffs(p)
    g = oracle.geometry(m.xy, m.tri)
    mid_x = {round(0.5 * (m.xy[m.tri[s // 3, (s % 3 + 1) % 3], 0] +
                          m.xy[m.tri[s // 3, (s % 3 + 2) % 3], 0]), 12) for s in m.dirichlet}
    assert mid_x == {n - 0.75}
    Xi = oracle.xi(p.eps[:1], p.kinv[:1], p.nu, p.dt)[0]
    Xm = np.array([[Xi[0], Xi[1]], [Xi[1], Xi[2]]])
    grad = np.array([1.7, 0.0])
    eta = (g.cc[:, 0] - (n - 0.75)) * grad[0]
    tau = oracle.cp2_tangential_flux(m.xy, m.tri, nbr, isd, *_fields(p), eta)
    est = _availability(nbr, isd)
    checked_dir = 0
    for e in range(m.tri.shape[0]):
        for j in range(3):
            ep = nbr[e, j]
            if ep < 0 and not isd[e, j]:
                assert tau[e, j] == 0.0
                continue
            if not est[e, j].any():
                continue
            eta_ep = eta[ep] if ep >= 0 else 0.0
            phi = -T[e, j] * (eta[e] - eta_ep) + tau[e, j]
            exact = g.length[e, j] * (Xm @ grad) @ g.normal[e, j]
            assert phi == pytest.approx(exact, rel=1e-10, abs=1e-12 * np.abs(Xm).max())
            checked_dir += ep < 0
    assert checked_dir >= n - 3


def test_tangential_flux_is_antisymmetric_across_a_side():
    p = synth.channel_block_problem(12, seed=8)
    m = p.mesh
    T, _, isd, nbr = _coeffs(p)
    eta = synth.normal_noise(m.tri.shape[0], 9)
    tau = oracle.cp2_tangential_flux(m.xy, m.tri, nbr, isd, *_fields(p), eta)
    scale = np.abs(tau).max()
    assert scale > 0
    for e, j in zip(*np.nonzero(nbr >= 0)):
        ep = nbr[e, j]
        assert tau[e, j] == pytest.approx(-tau[ep, _jp(nbr, e, ep)], abs=1e-13 * scale)


# --------------------------------------------------------- RT0, grad Psi

def _all_dirichlet(nbr):
    return (nbr < 0).astype(np.int32)


def test_rt0_cell_velocity_of_uniform_fluxes_is_exact():
    p = _uniform_problem(9, seed=3)
    m = p.mesh
    nt = m.tri.shape[0]
    nbr = oracle.topology(m.tri)
    isd = _all_dirichlet(nbr)
    g = oracle.geometry(m.xy, m.tri)
    U = np.array([-0.25, 1.5])
    fbar = g.length * (g.normal @ U)
    zero3 = np.zeros((nt, 3))
    u23 = np.repeat(U[:, None], nt, axis=1)
    gk = synth.normal_noise(2 * nt, 4).reshape(2, nt)
    Q, u_next, g_next = oracle.cp2_update(m.xy, m.tri, nbr, isd, *_fields(p), fbar, zero3, zero3,
                                          np.zeros(nt), u23, gk)
    np.testing.assert_allclose(u_next, u23, rtol=0, atol=1e-13)
    np.testing.assert_allclose(g_next, gk, rtol=0, atol=1e-10 * np.abs(gk).max() + 1e-9)


@pytest.mark.parametrize("field_loc", [oracle.PER_VERTEX, oracle.PER_CELL])
def test_grad_psi_update_along_an_eigenvector_of_kinv(field_loc):
    """Kinv = R diag(beta/k, 1/k) R^T: along the first column of R, Mbar acts
    as (1 + nu eps (beta/k) dt)/dt; along the second as (1 + nu eps/k dt)/dt."""
    beta, alpha, kinv_k = 20.0, math.radians(30.0), 2.0e4
    p = _uniform_problem(7, seed=5, beta=beta, field_loc=field_loc)
    m = p.mesh
    nt = m.tri.shape[0]
    nbr = oracle.topology(m.tri)
    isd = _all_dirichlet(nbr)
    zero3 = np.zeros((nt, 3))
    v1 = np.array([math.cos(alpha), math.sin(alpha)])
    v2 = np.array([-math.sin(alpha), math.cos(alpha)])
    for v, lam in ((v1, beta * kinv_k), (v2, kinv_k)):
        # u_next = 0 (no flux anywhere); u23 = -0.01 v  ->  g_next - g_k = Mbar (0.01 v)
        u23 = np.repeat((-0.01 * v)[:, None], nt, axis=1)
        gk = np.zeros((2, nt))
        _, u_next, g_next = oracle.cp2_update(m.xy, m.tri, nbr, isd, *_fields(p), zero3, zero3,
                                              zero3, np.zeros(nt), u23, gk)
        assert np.all(u_next == 0.0)
        mu = (1.0 + p.nu * 0.4 * lam * p.dt) / p.dt
        np.testing.assert_allclose(g_next, np.repeat((0.01 * mu * v)[:, None], nt, axis=1),
                                   rtol=1e-12, atol=1e-14 * mu)


# -------------------------------------------------------------- the step

def test_step_conserves_mass_and_keeps_fluxes_continuous():
    p = synth.channel_block_problem(12, seed=2)
    m = p.mesh
    nt = m.tri.shape[0]
    rng = np.random.default_rng(21)
    u23 = rng.normal(size=(2, nt)) * 0.1 + np.array([[0.05], [0.0]])
    gk = rng.normal(size=(2, nt))
    r = oracle.cp2_step(p, u23, gk)
    nbr = oracle.topology(m.tri)
    scale = np.abs(r.Q).max()
    # Eq. Cs2_5: no net flux out of any cell at the end of the step
    assert np.abs(r.Q.sum(axis=1)).max() <= 1e-12 * scale
    # the mean flux alone does not balance (the reason for the step)
    assert np.abs(r.fbar.sum(axis=1)).max() > 1e-3 * scale
    for e, j in zip(*np.nonzero(nbr >= 0)):
        ep = nbr[e, j]
        assert r.Q[e, j] == pytest.approx(-r.Q[ep, _jp(nbr, e, ep)], abs=1e-12 * scale)
    # the tensor is anisotropic, so the second solve moves eta
    assert np.abs(r.eta - r.eta_tilde).max() > 1e-3 * np.abs(r.eta).max()


def test_step_passes_a_uniform_channel_flow_unchanged():
    """Walls top and bottom (no flux), Dirichlet at both ends: a uniform
    velocity along the channel is already divergence free, so eta = 0 and
    the velocity and eps grad Psi stay as they are."""
    n = 11
    p = _uniform_problem(n, seed=7)
    m = p.mesh
    j, i = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    ends = ((i == 0) | (i == n - 1)).ravel()
    m.dirichlet = synth.sides_on_vertex_set(m.tri, ends)
    nt = m.tri.shape[0]
    U = np.array([0.3, 0.0])
    u23 = np.repeat(U[:, None], nt, axis=1)
    gk = synth.normal_noise(2 * nt, 1).reshape(2, nt)
    r = oracle.cp2_step(p, u23, gk)
    T, _, _, _ = _coeffs(p)
    assert np.abs(r.eta).max() <= 1e-12 * 0.3 / np.abs(T).max() * 10
    np.testing.assert_allclose(r.u_next, u23, rtol=0, atol=1e-12)
    np.testing.assert_allclose(r.g_next, gk, rtol=0, atol=1e-8)


def test_step_with_isotropic_tensor_needs_no_correction():
    p = synth.centred_block_problem(12, seed=3)
    m = p.mesh
    nt = m.tri.shape[0]
    rng = np.random.default_rng(5)
    u23 = rng.normal(size=(2, nt))
    r = oracle.cp2_step(p, u23, np.zeros((2, nt)))
    np.testing.assert_allclose(r.eta, r.eta_tilde, rtol=0, atol=1e-11 * np.abs(r.eta).max())
    assert np.abs(r.Q.sum(axis=1)).max() <= 1e-12 * np.abs(r.Q).max()
