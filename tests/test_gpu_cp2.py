"""The CP2 step (cps_cp2_setup / cps_cp2_step, Sec. 3.2.3) against the
oracle's step, element by element: both solutions eta~ and eta, the outward
side fluxes, the RT0 cell velocity and the eps grad(Psi) update.  Vertex and
cell fields, isotropic and anisotropic tensors, a mesh with bisected sides,
the log-permeability form, FP64 and mixed precision, one and two cells, and
the benchmark's 2,093,058-cell workload (there the oracle's own step kernels
are evaluated on the GPU's eta~ and eta, and the solves are checked through
their true residuals with the oracle's matrix)."""
import dataclasses

import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

cps = pytest.importorskip("paper_2309_03543_gb300")


@pytest.fixture(scope="module")
def ctx(cuda_device):
    c = cps.Context(0)
    yield c
    c.close()


def _uniform_cell_aniso(n, seed):
    mesh = synth.lattice(n, seed)
    eps = np.full(mesh.nt, 0.5)
    kinv = synth.aniso_kinv(np.full(mesh.nt, 1.5e4), 50.0, np.radians(-20.0))
    return synth.Problem(mesh, eps, kinv, synth.PER_CELL)


def _tiny(mesh):
    eps = np.linspace(0.4, 1.0, mesh.nv)
    kinv = synth.aniso_kinv(synth.kozeny_carman_kinv(eps), 30.0, np.radians(40.0))
    return synth.Problem(mesh, eps, kinv, synth.PER_VERTEX)


def _cases():
    two = synth.lattice(2, seed=0)
    one = dataclasses.replace(two, tri=np.ascontiguousarray(two.tri[1:]),
                              dirichlet=np.array([0], dtype=np.int32))
    lp, theta = synth.log_permeability_problem(21, seed=4)
    return {
        "channel_aniso_n24": (synth.channel_block_problem(24, seed=1), None),
        "channel_aniso_n45": (synth.channel_block_problem(45, seed=2), None),
        "centred_iso_n20": (synth.centred_block_problem(20, seed=2), None),
        "cell_aniso_n17": (_uniform_cell_aniso(17, 3), None),
        "defect_n16": (synth.defect_problem(16, seed=3), None),
        "logk_n21": (lp, theta),
        "one_cell": (_tiny(one), None),
        "two_cells": (_tiny(two), None),
        "lattice3": (_tiny(synth.lattice(3, seed=5)), None),
    }


CASES = _cases()


def _gpu_step(ctx, p, theta, u23, gk, rtol, precision):
    m = p.mesh
    if theta is not None:
        field_loc, kinv = cps.PER_CELL_LOGK, theta
    else:
        field_loc, kinv = p.field_loc, p.kinv
    s = ctx.assemble(m.xy, m.tri, m.dirichlet, p.eps, kinv, field_loc, cps.KIND_CP2, p.nu, p.dt)
    s.cp2_setup(m.xy, m.tri, p.eps, kinv)
    out = s.cp2_step(u23, gk, rtol=rtol, precision=precision)
    res = {k: v.cpu().numpy() for k, v in out.items() if isinstance(v, torch.Tensor)}
    res["stats"] = out["stats"]
    s.free()
    return res


def _rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def _check_against_oracle(r, o, tol, u23):
    """Relative L2 error of each output within tol, and every element within
    tol times the larger of the output's and its inputs' magnitude (a flux
    or velocity that cancels to ~0 is compared on the scale of the fluxes
    and velocities it is made of)."""
    assert _rel(r["eta_tilde"], o.eta_tilde) <= tol
    assert _rel(r["eta"], o.eta) <= tol
    fscale = np.abs(o.fbar).max()
    uscale = np.abs(u23).max()
    for got, want, floor in ((r["flux"], o.Q.T, fscale), (r["u_next"], o.u_next, uscale),
                             (r["g_next"], o.g_next, 0.0)):
        scale = max(np.abs(want).max(), floor)
        assert np.linalg.norm(got - want) <= tol * max(np.linalg.norm(want), floor)
        np.testing.assert_allclose(got, want, rtol=0, atol=tol * scale)


def _check_invariants(r, nbr, tol, fscale):
    Q = r["flux"].T
    scale = max(np.abs(Q).max(), fscale)
    # Eq. Cs2_5: the new velocity leaves no cell with net flux
    assert np.abs(Q.sum(axis=1)).max() <= tol * max(scale, 1e-300)
    e, j = np.nonzero(nbr >= 0)
    if e.size:
        ep = nbr[e, j]
        jp = np.argmax(nbr[ep] == e[:, None], axis=1)
        assert np.abs(Q[e, j] + Q[ep, jp]).max() <= 1e-12 * max(scale, 1e-300)


@pytest.mark.parametrize("name", sorted(CASES))
def test_cp2_step_matches_oracle_fp64(ctx, name):
    p, theta = CASES[name]
    m = p.mesh
    u23 = synth.cell_vector_field(m, 11, mean=(0.05, 0.01), scale=0.02)
    gk = synth.cell_vector_field(m, 12, scale=1e-3)
    o = oracle.cp2_step(p, u23, gk, rtol=1e-13)
    r = _gpu_step(ctx, p, theta, u23, gk, 1e-12, cps.FP64)
    _check_against_oracle(r, o, 1e-9, u23)
    _check_invariants(r, oracle.topology(m.tri), 1e-10, np.abs(o.fbar).max())


@pytest.mark.parametrize("name", ["channel_aniso_n45", "defect_n16", "two_cells"])
def test_cp2_step_matches_oracle_mixed(ctx, name):
    p, theta = CASES[name]
    m = p.mesh
    u23 = synth.cell_vector_field(m, 21, mean=(0.05, 0.0), scale=0.02)
    gk = synth.cell_vector_field(m, 22, scale=1e-3)
    o = oracle.cp2_step(p, u23, gk, rtol=1e-13)
    r = _gpu_step(ctx, p, theta, u23, gk, 1e-12, cps.MIXED)
    _check_against_oracle(r, o, 1e-8, u23)


def test_cp2_step_of_a_divergence_free_uniform_flow(ctx):
    """Dirichlet at both ends, walls top and bottom: the uniform flow passes."""
    n = 30
    p = _uniform_cell_aniso(n, 6)
    m = p.mesh
    j, i = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    m.dirichlet = synth.sides_on_vertex_set(m.tri, ((i == 0) | (i == n - 1)).ravel())
    u23 = np.repeat(np.array([[0.3], [0.0]]), m.nt, axis=1)
    gk = synth.cell_vector_field(m, 3)
    r = _gpu_step(ctx, p, None, u23, gk, 1e-12, cps.FP64)
    np.testing.assert_allclose(r["u_next"], u23, rtol=0, atol=1e-12)
    np.testing.assert_allclose(r["g_next"], gk, rtol=0, atol=1e-9)


def test_cp2_entry_points_reject_bad_use(ctx):
    p = CASES["channel_aniso_n24"][0]
    m = p.mesh
    s = ctx.assemble(m.xy, m.tri, m.dirichlet, p.eps, p.kinv, p.field_loc, cps.KIND_CP2, p.nu,
                     p.dt)
    u = np.zeros((2, m.nt))
    out = s.cp2_step(u, u, check=False)          # no set-up yet
    assert out["status"] == cps._cps.ERR_ARG
    s.free()
    s1 = ctx.assemble(m.xy, m.tri, m.dirichlet, p.eps, p.kinv, p.field_loc, cps.KIND_CP1_X,
                      p.nu, p.dt)
    with pytest.raises(cps.CpsError):
        s1.cp2_setup(m.xy, m.tri, p.eps, p.kinv)  # not a CP2 system
    s1.free()


def test_cp2_step_full_size_workload(ctx):
    """2,093,058 cells (channel block, anisotropic K, the benchmark's seeds):
    the solves through their true residuals with the oracle's matrix, and the
    step's fluxes, velocity and eps grad(Psi) against the oracle's step
    kernels evaluated on the GPU's eta~ and eta, on every cell."""
    p = synth.channel_block_problem(1024, seed=0)
    m = p.mesh
    u23 = synth.cell_vector_field(m, 11, mean=(0.05, 0.01), scale=0.02)
    gk = synth.cell_vector_field(m, 12, scale=1e-3)
    rtol = 1e-10
    r = _gpu_step(ctx, p, None, u23, gk, rtol, cps.FP64)
    A = oracle.assemble_problem(p)
    T, _, isd, nbr = oracle.side_coefficients(m.xy, m.tri, m.dirichlet, p.eps, p.kinv,
                                              p.field_loc, oracle.CP2, p.nu, p.dt)
    args = (m.xy, m.tri, nbr, isd)
    fields = (p.eps, p.kinv, p.field_loc, p.nu, p.dt)
    fbar = oracle.cp2_mean_flux(*args, u23)
    b1 = fbar.sum(axis=1)
    assert np.linalg.norm(b1 - A.matvec(r["eta_tilde"])) <= 2 * rtol * np.linalg.norm(b1)
    tau = oracle.cp2_tangential_flux(*args, *fields, r["eta_tilde"])
    b2 = b1 + tau.sum(axis=1)
    assert np.linalg.norm(b2 - A.matvec(r["eta"])) <= 2 * rtol * np.linalg.norm(b2)
    Q, u_next, g_next = oracle.cp2_update(*args, *fields, fbar, T, tau, r["eta"], u23, gk)
    # coefficients at this size carry ~u L/h relative rounding (coordinates up
    # to 1023 across sides of length ~1), as the full-size assembly test states
    tol = 64 * np.finfo(float).eps * 1023
    for got, want in ((r["flux"], Q.T), (r["u_next"], u_next), (r["g_next"], g_next)):
        np.testing.assert_allclose(got, want, rtol=0, atol=tol * np.abs(want).max())
    _check_invariants(r, nbr, 10 * rtol, np.abs(fbar).max())
