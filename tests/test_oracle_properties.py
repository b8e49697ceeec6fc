"""Properties of the oracle's corrector steps on random small meshes
(hypothesis): whatever the lattice size, jitter seed, field location,
anisotropy and velocity field,
* the CP2 step leaves no net flux in any cell (Eq. Cs2_5) and its side
  fluxes are antisymmetric across every interior side;
* the CP1 step run to convergence solves the coupled 2 nt x 2 nt system
  (Eq. cs1_sys2 with the mass block) -- checked through its residual."""
import math

import numpy as np
import pytest

import oracle
import synth

hyp = pytest.importorskip("hypothesis")
st = pytest.importorskip("hypothesis.strategies")


def _problem(n, seed, per_cell, beta, alpha_deg, walls):
    mesh = synth.lattice(n, seed)
    if walls:
        nbr = oracle.topology(mesh.tri)
        e, j = np.nonzero(nbr < 0)
        mesh.dirichlet = (e * 3 + j).astype(np.int32)
    nf = mesh.nt if per_cell else mesh.nv
    rng = np.random.default_rng(seed)
    eps = rng.uniform(0.35, 1.0, nf)
    kinv = synth.aniso_kinv(synth.kozeny_carman_kinv(eps) * 1e-3, beta, math.radians(alpha_deg))
    return synth.Problem(mesh, eps, kinv, synth.PER_CELL if per_cell else synth.PER_VERTEX)


@hyp.settings(max_examples=100, deadline=None)
@hyp.given(n=st.integers(2, 9), seed=st.integers(0, 10_000), per_cell=st.booleans(),
           beta=st.floats(1.0, 200.0), alpha=st.floats(-90.0, 90.0),
           mean=st.floats(-0.1, 0.1))
def test_cp2_step_conserves_mass_and_keeps_fluxes_continuous(n, seed, per_cell, beta, alpha,
                                                              mean):
    p = _problem(n, seed, per_cell, beta, alpha, walls=False)
    m = p.mesh
    u23 = synth.cell_vector_field(m, seed, mean=(mean, 0.0), scale=0.02)
    gk = synth.cell_vector_field(m, seed + 1, scale=1e-3)
    r = oracle.cp2_step(p, u23, gk, dense=True)
    scale = max(np.abs(r.fbar).max(), np.abs(r.Q).max(), 1e-300)
    assert np.abs(r.Q.sum(axis=1)).max() <= 1e-10 * scale
    nbr = oracle.topology(m.tri)
    e, j = np.nonzero(nbr >= 0)
    if e.size:
        ep = nbr[e, j]
        jp = np.argmax(nbr[ep] == e[:, None], axis=1)
        assert np.abs(r.Q[e, j] + r.Q[ep, jp]).max() <= 1e-12 * scale
    assert np.all(np.isfinite(r.u_next)) and np.all(np.isfinite(r.g_next))


@hyp.settings(max_examples=60, deadline=None)
@hyp.given(n=st.integers(2, 7), seed=st.integers(0, 10_000), per_cell=st.booleans(),
           beta=st.floats(1.0, 30.0), alpha=st.floats(-90.0, 90.0))
def test_cp1_step_converges_to_the_coupled_solution(n, seed, per_cell, beta, alpha):
    p = _problem(n, seed, per_cell, beta, alpha, walls=True)
    m = p.mesh
    nt = m.nt
    du_b = synth.cell_vector_field(m, seed, scale=0.05)
    r = oracle.cp1_step(p, du_b, toll=1e-13, criterion="max", max_outer=20000, dense=True)
    f = (p.eps, p.kinv, p.field_loc)
    Ax = oracle.assemble(m.xy, m.tri, m.dirichlet, *f, oracle.CP1_X, p.nu, p.dt)
    Ay = oracle.assemble(m.xy, m.tri, m.dirichlet, *f, oracle.CP1_Y, p.nu, p.dt)
    mass = oracle.cp1_mass(m.xy, m.tri, *f, p.nu, p.dt)
    T, _, isd, nbr = oracle.side_coefficients(m.xy, m.tri, m.dirichlet, *f, oracle.CP1_X,
                                              p.nu, p.dt)
    lap = [-oracle.cp1_laplacian(T, nbr, isd, du_b[k]) for k in range(2)]
    u, v = r.du
    res_x = Ax.matvec(u) + mass[:, 1] * v - lap[0]
    res_y = Ay.matvec(v) + mass[:, 1] * u - lap[1]
    scale = max(np.abs(Ax.matvec(u)).max(), np.abs(Ay.matvec(v)).max(), np.abs(lap[0]).max(),
                np.abs(lap[1]).max(), 1e-300)
    assert r.err <= 1e-13
    assert max(np.abs(res_x).max(), np.abs(res_y).max()) <= 1e-9 * scale, nt
