"""Pins for the oracle's side tensor and matrix assembly
(Eq. Cs2_4, Eq. CS2_sys_coeff, Eq. CS1_sys_coeff)."""
import math

import numpy as np
import pytest

import oracle
import synth

S3 = math.sqrt(3.0)
NU, DT = synth.NU, synth.DT


# ------------------------------------------------------------------ Xi

def test_xi_clear_fluid_is_eps_dt_identity():
    eps = np.array([1.0, 0.7])
    x = oracle.xi(eps, np.zeros((2, 3)), NU, DT)
    np.testing.assert_allclose(x, [[DT, 0, DT], [0.7 * DT, 0, 0.7 * DT]], rtol=1e-15)


def test_xi_isotropic_closed_form():
    eps, k = 0.4, 1.0125e9
    x = oracle.xi([eps], [[k, 0.0, k]], NU, DT)[0]
    want = eps * DT / (1.0 + NU * eps * DT * k)
    np.testing.assert_allclose(x, [want, 0.0, want], rtol=1e-13)


@pytest.mark.parametrize("alpha_deg,beta", [(30.0, 100.0), (-45.0, 100.0), (10.0, 3.0)])
def test_xi_anisotropic_eigenpairs(alpha_deg, beta):
    """Xi shares the principal axes of K^-1 with eigenvalues eps dt / (1 + c mu_i)."""
    eps, kinv = 0.4, 2.0e8
    a = math.radians(alpha_deg)
    comp = synth.aniso_kinv(np.array([kinv]), beta, a)
    X = oracle.xi([eps], comp, NU, DT)[0]
    Xm = np.array([[X[0], X[1]], [X[1], X[2]]])
    c = NU * eps * DT
    v1 = np.array([math.cos(a), math.sin(a)])
    v2 = np.array([-math.sin(a), math.cos(a)])
    np.testing.assert_allclose(Xm @ v1, eps * DT / (1 + c * beta * kinv) * v1, rtol=1e-12,
                               atol=1e-20)
    np.testing.assert_allclose(Xm @ v2, eps * DT / (1 + c * kinv) * v2, rtol=1e-12, atol=1e-20)


# ------------------------------------------------------------------ matrix

def _dirichlet_rows(m):
    rows = np.zeros(m.nt, dtype=bool)
    rows[m.dirichlet // 3] = True
    return rows


@pytest.mark.parametrize("maker", [lambda: synth.centred_block_problem(24, seed=2),
                                   lambda: synth.channel_block_problem(24, seed=4)])
def test_cp2_matrix_is_a_symmetric_m_matrix(maker):
    p = maker()
    A = oracle.assemble_problem(p)
    D = A.dense()
    assert np.array_equal(D, D.T)
    d = np.diag(D)
    off = D - np.diag(d)
    assert np.all(d > 0)
    assert np.all(off <= 0)
    rs = D.sum(axis=1)
    drow = _dirichlet_rows(p.mesh)
    scale = np.abs(D).max()
    assert np.all(np.abs(rs[~drow]) <= 1e-12 * scale)     # pure no-flux rows
    assert np.all(rs[drow] > 0)                            # Dirichlet rows dominate
    assert np.linalg.eigvalsh(D).min() > 0


def test_cp1_matrix_rows_are_strictly_dominant_by_the_mass_term():
    p = synth.centred_block_problem(16, seed=1)
    for kind in (oracle.CP1_X, oracle.CP1_Y):
        A = oracle.assemble_problem(p, kind)
        T, sigma, isd, nbr = oracle.side_coefficients(p.mesh.xy, p.mesh.tri, p.mesh.dirichlet,
                                                      p.eps, p.kinv, p.field_loc, kind, p.nu,
                                                      p.dt)
        D = A.dense()
        assert np.array_equal(D, D.T)
        rs = D.sum(axis=1)
        dir_part = (T * isd).sum(axis=1)
        np.testing.assert_allclose(rs, sigma + dir_part, rtol=1e-12)
        assert np.all(sigma > 0)
        # sigma = Mbar_kk A_e >= A_e / dt, equality in clear fluid
        g = oracle.geometry(p.mesh.xy, p.mesh.tri)
        assert np.all(sigma >= g.area / p.dt * (1 - 1e-14))


@pytest.mark.parametrize("field_loc", [oracle.PER_VERTEX, oracle.PER_CELL])
def test_cp1_mass_term_closed_form_for_uniform_fields(field_loc):
    """Uniform eps and Kinv on the unjittered lattice: every cell's CP1 mass
    term is Mbar_kk A_e = (1 + nu eps Kinv_kk dt)/dt * sqrt3/4 (the mean of
    identical nodal values is that value), and T = nu l/d = nu sqrt3."""
    m = synth.lattice(8, jitter=0.0)
    nf = m.nv if field_loc == oracle.PER_VERTEX else m.nt
    eps0, kxx, kxy, kyy = 0.4, 3.0e7, 1.0e6, 5.0e6
    eps = np.full(nf, eps0)
    kinv = np.tile([kxx, kxy, kyy], (nf, 1))
    for kind, kk in ((oracle.CP1_X, kxx), (oracle.CP1_Y, kyy)):
        T, sigma, isd, nbr = oracle.side_coefficients(m.xy, m.tri, m.dirichlet, eps, kinv,
                                                      field_loc, kind, NU, DT)
        want = (1.0 + NU * eps0 * kk * DT) / DT * S3 / 4
        np.testing.assert_allclose(sigma, want, rtol=1e-13)
        np.testing.assert_allclose(T[nbr >= 0], NU * S3, rtol=1e-13)


def test_uniform_isotropic_lattice_transmissibility_closed_form():
    """Unjittered lattice, clear fluid: Xi = dt I, so every interior side has
    T = l d_n / d = 1 * dt / (1/sqrt3) and a Dirichlet side l dt / (1/(2 sqrt3))."""
    n = 10
    m = synth.lattice(n, jitter=0.0)
    eps = np.ones(m.nv)
    kinv = np.zeros((m.nv, 3))
    A = oracle.assemble(m.xy, m.tri, m.dirichlet, eps, kinv)
    D = A.dense()
    off = D[np.nonzero(D - np.diag(np.diag(D)))]
    np.testing.assert_allclose(off, -S3 * DT, rtol=1e-13)
    drow = _dirichlet_rows(m)
    np.testing.assert_allclose(D.sum(axis=1)[drow], 2 * S3 * DT, rtol=1e-12)


def test_anisotropic_lattice_transmissibility_hand_values():
    """Uniform rotated K^-1 on the unjittered lattice: a side with normal angle
    phi gets T = sqrt3 (mu1 cos^2(phi-a) + mu2 sin^2(phi-a))."""
    n, beta, a = 8, 100.0, math.radians(30.0)
    eps0, kinv0 = 0.4, 1.0e8
    m = synth.lattice(n, jitter=0.0)
    eps = np.full(m.nv, eps0)
    kinv = synth.aniso_kinv(np.full(m.nv, kinv0), beta, a)
    T, sigma, isd, nbr = oracle.side_coefficients(m.xy, m.tri, m.dirichlet, eps, kinv,
                                                  oracle.PER_VERTEX, oracle.CP2, NU, DT)
    c = NU * eps0 * DT
    mu1 = eps0 * DT / (1 + c * beta * kinv0)
    mu2 = eps0 * DT / (1 + c * kinv0)
    g = oracle.geometry(m.xy, m.tri)
    phi = np.arctan2(g.normal[..., 1], g.normal[..., 0])
    want = S3 * (mu1 * np.cos(phi - a) ** 2 + mu2 * np.sin(phi - a) ** 2)
    inner = nbr >= 0
    np.testing.assert_allclose(T[inner], want[inner], rtol=1e-12)
    # the side whose normal is the principal axis (30 deg) sees mu1 only
    on_axis = inner & (np.abs(np.degrees(phi) - 30.0) < 1e-9)
    assert on_axis.any()
    np.testing.assert_allclose(T[on_axis], S3 * mu1, rtol=1e-12)


def test_quadratic_form_equals_side_energy():
    """x^T A x = sum_sides T (x_e - x_ep)^2 + sum_Dirichlet T x_e^2 + sum sigma x^2."""
    p = synth.channel_block_problem(14, seed=9)
    for kind in (oracle.CP2, oracle.CP1_X):
        A = oracle.assemble_problem(p, kind)
        T, sigma, isd, nbr = oracle.side_coefficients(p.mesh.xy, p.mesh.tri, p.mesh.dirichlet,
                                                      p.eps, p.kinv, p.field_loc, kind, p.nu,
                                                      p.dt)
        x = np.random.default_rng(0).standard_normal(A.n)
        e, j = np.nonzero(nbr >= 0)
        energy = 0.5 * np.sum(T[e, j] * (x[e] - x[nbr[e, j]]) ** 2)   # each side twice
        e2, j2 = np.nonzero(isd)
        energy += np.sum(T[e2, j2] * x[e2] ** 2) + np.sum(sigma * x * x)
        assert x @ A.matvec(x) == pytest.approx(energy, rel=1e-12)


def test_linear_field_is_flux_free_for_uniform_isotropic_xi():
    """Two-point fluxes are exact for a linear field at circumcentres when
    Xi = xi I (K-orthogonal): interior no-flux rows of A eta_lin vanish."""
    m = synth.lattice(18, seed=11)
    g = oracle.geometry(m.xy, m.tri)
    A = oracle.assemble(m.xy, m.tri, m.dirichlet, np.ones(m.nv), np.zeros((m.nv, 3)))
    eta = 0.3 + 1.7 * g.cc[:, 0] - 0.9 * g.cc[:, 1]
    r = A.matvec(eta)
    interior = np.all(g.nbr >= 0, axis=1)
    assert interior.sum() > 100
    assert np.abs(r[interior]).max() < 1e-12 * np.abs(eta).max()
    # with a varying scalar Xi the row equals minus the side-averaged flux
    eps = np.linspace(0.3, 1.0, m.nv)
    A2 = oracle.assemble(m.xy, m.tri, m.dirichlet, eps, np.zeros((m.nv, 3)))
    xi_side = 0.5 * DT * (eps[m.tri[:, [1, 2, 0]]] + eps[m.tri[:, [2, 0, 1]]])
    flux = g.length * xi_side * (g.normal @ np.array([1.7, -0.9]))
    r2 = A2.matvec(eta)
    np.testing.assert_allclose(r2[interior], -flux[interior].sum(axis=1), rtol=1e-9,
                               atol=1e-13)


def test_singular_and_non_delaunay_inputs_are_rejected():
    m = synth.lattice(6, seed=0)
    with pytest.raises(oracle.OracleError) as ei:
        oracle.assemble(m.xy, m.tri, np.zeros(0, np.int32), np.ones(m.nv), np.zeros((m.nv, 3)))
    assert ei.value.code == oracle.ERR_SINGULAR
    # push one interior vertex far enough to break the Delaunay property
    xy = m.xy.copy()
    v = 2 * 6 + 2
    xy[v] += [0.0, 0.6]
    with pytest.raises(oracle.OracleError) as ei:
        oracle.assemble(xy, m.tri, m.dirichlet, np.ones(m.nv), np.zeros((m.nv, 3)))
    assert ei.value.code in (oracle.ERR_NONDELAUNAY, oracle.ERR_ORIENTATION)
