"""Pins of the oracle's CP1 step (Sec. 3.2.2, Eq. cs1_sys2, Eq. CS1_sys_coeff,
App. B) against facts the paper and the mathematics fix:

* the mass terms Mbar_kk A_e equal the diagonal mass of the assembled CP1
  matrices, and along an eigenvector of Kinv the 2x2 mass block acts as its
  closed-form eigenvalue;
* nu L is the off-diagonal part of the assembled CP1 matrix as an operator
  (symmetric, zero on constants without Dirichlet sides);
* without coupling (isotropic Kinv) the step is a backward-Euler viscous
  update of the predictor increment: w = du_breve + du_tilde solves
  (Mbar A + nu L) w = Mbar A du_breve -- this fixes the sign of the
  right-hand side -- and the outer iteration stops after one sweep;
* with coupling, the outer iteration run to convergence is the solution of
  the full 2 nt x 2 nt coupled system, solved here by brute force.
"""
import math

import numpy as np
import pytest

import oracle
import synth


def _problem(n, seed, beta=20.0, alpha_deg=30.0, field_loc=synth.PER_VERTEX, iso=False):
    mesh = synth.lattice(n, seed)
    nf = mesh.nv if field_loc == synth.PER_VERTEX else mesh.nt
    rng = np.random.default_rng(seed)
    eps = rng.uniform(0.4, 1.0, nf)
    kinv_s = synth.kozeny_carman_kinv(eps) * 1e-3
    kinv = synth.iso_kinv(kinv_s) if iso else synth.aniso_kinv(kinv_s, beta,
                                                               math.radians(alpha_deg))
    # no-slip walls: every boundary side holds a zero increment
    nbr = oracle.topology(mesh.tri)
    e, j = np.nonzero(nbr < 0)
    mesh.dirichlet = (e * 3 + j).astype(np.int32)
    return synth.Problem(mesh, eps, kinv, field_loc)


def _args(p):
    return (p.eps, p.kinv, p.field_loc, p.nu, p.dt)


def test_mass_diagonal_equals_the_assembled_cp1_mass():
    p = _problem(9, 1)
    m = p.mesh
    mass = oracle.cp1_mass(m.xy, m.tri, *_args(p))
    for kind, col in ((oracle.CP1_X, 0), (oracle.CP1_Y, 2)):
        _, sigma, _, _ = oracle.side_coefficients(m.xy, m.tri, m.dirichlet, p.eps, p.kinv,
                                                  p.field_loc, kind, p.nu, p.dt)
        np.testing.assert_allclose(mass[:, col], sigma, rtol=1e-14)


@pytest.mark.parametrize("field_loc", [synth.PER_VERTEX, synth.PER_CELL])
def test_mass_block_along_eigenvectors_of_kinv(field_loc):
    beta, alpha, k = 20.0, math.radians(30.0), 3.0e3
    mesh = synth.lattice(6, 2)
    nf = mesh.nv if field_loc == synth.PER_VERTEX else mesh.nt
    eps = np.full(nf, 0.5)
    kinv = synth.aniso_kinv(np.full(nf, k), beta, alpha)
    p = synth.Problem(mesh, eps, kinv, field_loc)
    mass = oracle.cp1_mass(mesh.xy, mesh.tri, *_args(p))
    area = synth.triangle_areas(mesh)
    v1 = np.array([math.cos(alpha), math.sin(alpha)])
    v2 = np.array([-math.sin(alpha), math.cos(alpha)])
    for v, lam in ((v1, beta * k), (v2, k)):
        mu = (1.0 + p.nu * 0.5 * lam * p.dt) / p.dt
        got = np.stack([mass[:, 0] * v[0] + mass[:, 1] * v[1],
                        mass[:, 1] * v[0] + mass[:, 2] * v[1]], axis=1)
        np.testing.assert_allclose(got, mu * area[:, None] * v[None, :], rtol=1e-12)


def test_laplacian_is_the_off_diagonal_part_of_the_cp1_matrix():
    p = _problem(10, 3)
    m = p.mesh
    A = oracle.assemble(m.xy, m.tri, m.dirichlet, *_args(p)[:3], oracle.CP1_X, p.nu, p.dt)
    T, sigma, isd, nbr = oracle.side_coefficients(m.xy, m.tri, m.dirichlet, *_args(p)[:3],
                                                  oracle.CP1_X, p.nu, p.dt)
    u = synth.normal_noise(m.nt, 4)
    w = synth.normal_noise(m.nt, 5)
    Lu = oracle.cp1_laplacian(T, nbr, isd, u)
    # A u - sigma u cancels the mass term, so compare on the scale of sigma u
    np.testing.assert_allclose(Lu, A.matvec(u) - sigma * u, rtol=0,
                               atol=1e-14 * np.abs(sigma * u).max())
    Lw = oracle.cp1_laplacian(T, nbr, isd, w)
    assert abs(Lu @ w - u @ Lw) <= 1e-12 * abs(Lu @ w)
    # constants are in the kernel once the Dirichlet sides are gone
    none = np.zeros_like(isd)
    assert np.abs(oracle.cp1_laplacian(T, nbr, none, np.full(m.nt, 3.0))).max() <= 1e-12


def test_uncoupled_step_is_a_backward_euler_viscous_update():
    p = _problem(11, 4, iso=True)
    m = p.mesh
    du_b = synth.cell_vector_field(m, 6, scale=0.1)
    r = oracle.cp1_step(p, du_b, toll=1e-4)
    assert r.outer == 1 and r.err == 0.0
    mass = oracle.cp1_mass(m.xy, m.tri, *_args(p))
    assert np.all(mass[:, 1] == 0.0)
    for k, kind, col in ((0, oracle.CP1_X, 0), (1, oracle.CP1_Y, 2)):
        A = oracle.assemble(m.xy, m.tri, m.dirichlet, *_args(p)[:3], kind, p.nu, p.dt)
        w = oracle.dense_cholesky_solve(A.dense(), mass[:, col] * du_b[k])
        np.testing.assert_allclose(du_b[k] + r.du[k], w, rtol=0,
                                   atol=1e-12 * np.abs(w).max())
    # the viscous update smooths: the total increment is smaller in the energy norm
    for k in range(2):
        assert np.linalg.norm(du_b[k] + r.du[k]) < np.linalg.norm(du_b[k])


def test_converged_outer_iteration_solves_the_coupled_system():
    p = _problem(8, 5, beta=10.0)
    m = p.mesh
    nt = m.nt
    du_b = synth.cell_vector_field(m, 7, scale=0.1)
    r = oracle.cp1_step(p, du_b, toll=1e-14, criterion="max", max_outer=5000)
    assert r.err <= 1e-14
    Ax = oracle.assemble(m.xy, m.tri, m.dirichlet, *_args(p)[:3], oracle.CP1_X, p.nu, p.dt)
    Ay = oracle.assemble(m.xy, m.tri, m.dirichlet, *_args(p)[:3], oracle.CP1_Y, p.nu, p.dt)
    mass = oracle.cp1_mass(m.xy, m.tri, *_args(p))
    T, _, isd, nbr = oracle.side_coefficients(m.xy, m.tri, m.dirichlet, *_args(p)[:3],
                                              oracle.CP1_X, p.nu, p.dt)
    # (Mbar A + nu L) [u; v] = -nu L du_breve, with the full 2x2 mass block per cell
    K = np.zeros((2 * nt, 2 * nt))
    K[:nt, :nt] = Ax.dense()
    K[nt:, nt:] = Ay.dense()
    K[np.arange(nt), nt + np.arange(nt)] = mass[:, 1]
    K[nt + np.arange(nt), np.arange(nt)] = mass[:, 1]
    rhs = -np.concatenate([oracle.cp1_laplacian(T, nbr, isd, du_b[0]),
                           oracle.cp1_laplacian(T, nbr, isd, du_b[1])])
    want = np.linalg.solve(K, rhs)
    np.testing.assert_allclose(r.du.ravel(), want, rtol=0, atol=1e-10 * np.abs(want).max())
    # the paper's stopping rule (min of the two changes, toll 1e-4) stops earlier
    r4 = oracle.cp1_step(p, du_b, toll=1e-4)
    assert 1 <= r4.outer <= r.outer and r4.err <= 1e-4


def test_outer_sweeps_grow_with_the_anisotropy_and_stay_at_the_papers_count_when_weak():
    """App. B reports 3-4 outer sweeps (toll 1e-4 to 1e-3).  The outer
    iteration is block Jacobi between the x and y systems, coupled only by
    Mbar_12 A_e, which vanishes for an isotropic tensor and grows with the
    principal ratio beta: one sweep when isotropic, at most 4 for beta <= 2,
    and more as beta grows (the channel workload's beta = 100 needs tens)."""
    import dataclasses
    sweeps = {}
    for beta in (1.0, 2.0, 10.0, 100.0):
        p = synth.channel_block_problem(24, seed=2, beta=beta)
        m = p.mesh
        nbr = oracle.topology(m.tri)
        e, j = np.nonzero(nbr < 0)
        p = dataclasses.replace(p, mesh=dataclasses.replace(m, dirichlet=(e * 3 + j).astype(np.int32)))
        du_b = synth.cell_vector_field(m, 5, mean=(0.05, 0.01), scale=0.02)
        sweeps[beta] = oracle.cp1_step(p, du_b, toll=1e-4).outer
    assert sweeps[1.0] == 1
    assert 2 <= sweeps[2.0] <= 4
    assert sweeps[2.0] < sweeps[10.0] < sweeps[100.0]
