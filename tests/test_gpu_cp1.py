"""The CP1 step (cps_cp1_setup / cps_cp1_step, Sec. 3.2.2, App. B) against the
oracle's step: the increments of both components after the outer iteration,
the number of outer sweeps, vertex and cell fields, isotropic (uncoupled) and
anisotropic tensors, a mesh with bisected sides, the log-permeability form,
FP64 and mixed precision, one and two cells; and at 2,093,058 cells the sweep
equations themselves through true residuals with the oracle's matrices."""
import dataclasses
import math

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


def _walls(mesh):
    """No-slip: every boundary side holds a zero increment."""
    nbr = oracle.topology(mesh.tri)
    e, j = np.nonzero(nbr < 0)
    return dataclasses.replace(mesh, dirichlet=(e * 3 + j).astype(np.int32))


def _aniso(n, seed, field_loc, beta=20.0):
    mesh = _walls(synth.lattice(n, seed))
    nf = mesh.nv if field_loc == synth.PER_VERTEX else mesh.nt
    rng = np.random.default_rng(seed)
    eps = rng.uniform(0.4, 1.0, nf)
    kinv = synth.aniso_kinv(synth.kozeny_carman_kinv(eps) * 1e-3, beta, math.radians(30.0))
    return synth.Problem(mesh, eps, kinv, field_loc)


def _with_walls(p):
    return dataclasses.replace(p, mesh=_walls(p.mesh))


def _cases():
    two = synth.lattice(2, seed=0)
    one = dataclasses.replace(two, tri=np.ascontiguousarray(two.tri[1:]))
    lp, theta = synth.log_permeability_problem(15, seed=4)
    return {
        "vertex_aniso_n20": (_aniso(20, 1, synth.PER_VERTEX), None),
        "cell_aniso_n17": (_aniso(17, 2, synth.PER_CELL), None),
        "channel_aniso_n33": (_with_walls(synth.channel_block_problem(33, seed=3)), None),
        "centred_iso_n18": (_with_walls(synth.centred_block_problem(18, seed=4)), None),
        "defect_n12": (synth.defect_problem(12, seed=3), None),   # obtuse cells at the walls
        "logk_n15": (_with_walls(lp), theta),
        "one_cell": (synth.Problem(_walls(one), np.array([0.5, 0.6, 0.7, 0.8]),
                                   synth.aniso_kinv(np.full(4, 50.0), 5.0, 0.3),
                                   synth.PER_VERTEX), None),
        "two_cells": (_aniso(2, 0, synth.PER_VERTEX), None),
    }


CASES = _cases()


def _systems(ctx, p, theta):
    m = p.mesh
    fl, kinv = (cps.PER_CELL_LOGK, theta) if theta is not None else (p.field_loc, p.kinv)
    sx = ctx.assemble(m.xy, m.tri, m.dirichlet, p.eps, kinv, fl, cps.KIND_CP1_X, p.nu, p.dt)
    sy = ctx.assemble(m.xy, m.tri, m.dirichlet, p.eps, kinv, fl, cps.KIND_CP1_Y, p.nu, p.dt)
    cps.cp1_setup(sx, sy, m.xy, m.tri, p.eps, kinv)
    return sx, sy


def _rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


@pytest.mark.parametrize("path", ["one_launch", "host"])
@pytest.mark.parametrize("name", sorted(CASES))
def test_cp1_step_matches_oracle_fp64(ctx, name, path):
    """Both ways of running the step: the whole outer iteration in one launch
    (the default) and the host-driven sweeps of single solves."""
    p, theta = CASES[name]
    du_b = synth.cell_vector_field(p.mesh, 9, mean=(0.01, -0.02), scale=0.05)
    o = oracle.cp1_step(p, du_b, toll=1e-4, rtol=1e-13)
    sx, sy = _systems(ctx, p, theta)
    cps.set_cp1_path(sx, cps.CP1_ONE_LAUNCH if path == "one_launch" else cps.CP1_HOST)
    du, st = cps.cp1_step(sx, sy, du_b, toll=1e-4, rtol=1e-12)
    assert st["outer"] == o.outer
    assert st["err"] <= 1e-4
    assert _rel(du.cpu().numpy(), o.du) <= 1e-9
    sx.free()
    sy.free()


@pytest.mark.parametrize("beta", [1.0, 1.5, 2.0])
def test_cp1_weak_anisotropy_takes_the_papers_sweep_count(ctx, beta):
    """App. B's 3-4 outer sweeps: an isotropic tensor needs one sweep (no
    coupling), a weakly anisotropic one (beta <= 2) at most four, the same
    count as the oracle's, with the same increments."""
    p = _with_walls(synth.channel_block_problem(40, seed=2, beta=beta))
    du_b = synth.cell_vector_field(p.mesh, 5, mean=(0.05, 0.01), scale=0.02)
    o = oracle.cp1_step(p, du_b, toll=1e-4, rtol=1e-13)
    sx, sy = _systems(ctx, p, None)
    du, st = cps.cp1_step(sx, sy, du_b, toll=1e-4, rtol=1e-12)
    assert st["outer"] == o.outer
    assert st["outer"] == 1 if beta == 1.0 else 2 <= st["outer"] <= 4
    assert _rel(du.cpu().numpy(), o.du) <= 1e-9
    sx.free()
    sy.free()


@pytest.mark.parametrize("path", ["one_launch", "host"])
@pytest.mark.parametrize("name", ["vertex_aniso_n20", "defect_n12", "two_cells"])
def test_cp1_step_matches_oracle_mixed(ctx, name, path):
    p, theta = CASES[name]
    du_b = synth.cell_vector_field(p.mesh, 19, scale=0.05)
    o = oracle.cp1_step(p, du_b, toll=1e-4, rtol=1e-13)
    sx, sy = _systems(ctx, p, theta)
    cps.set_cp1_path(sx, cps.CP1_ONE_LAUNCH if path == "one_launch" else cps.CP1_HOST)
    du, st = cps.cp1_step(sx, sy, du_b, toll=1e-4, rtol=1e-12, precision=cps.MIXED)
    assert st["outer"] == o.outer
    assert _rel(du.cpu().numpy(), o.du) <= 1e-8
    sx.free()
    sy.free()


def test_cp1_entry_points_reject_bad_use(ctx):
    p, _ = CASES["vertex_aniso_n20"]
    m = p.mesh
    sx = ctx.assemble(m.xy, m.tri, m.dirichlet, p.eps, p.kinv, p.field_loc, cps.KIND_CP1_X,
                      p.nu, p.dt)
    s2 = ctx.assemble(m.xy, m.tri, m.dirichlet, p.eps, p.kinv, p.field_loc, cps.KIND_CP2,
                      p.nu, p.dt)
    with pytest.raises(cps.CpsError):
        cps.cp1_setup(sx, s2, m.xy, m.tri, p.eps, p.kinv)        # partner is not CP1_Y
    with pytest.raises(cps.CpsError):
        cps.set_cp1_path(sx, cps.CP1_HOST)                        # no set-up
    _, st = cps.cp1_step(sx, s2, np.zeros((2, m.nt)), check=False)  # no set-up
    assert st["status"] == cps._cps.ERR_ARG
    sx.free()
    s2.free()


def test_cp1_sweeps_full_size(ctx):
    """2,093,058 cells, anisotropic channel block with no-slip walls: the
    uncoupled sweep solves (Mbar_kk A + nu L) du_k = -nu L du_breve_k, and one
    coupled sweep solves it with -Mbar_12 A du_other of the sweep before, each
    through its true residual with the oracle's matrices."""
    p = _with_walls(synth.channel_block_problem(1024, seed=0))
    m = p.mesh
    du_b = synth.cell_vector_field(m, 9, mean=(0.01, -0.02), scale=0.05)
    rtol = 1e-10
    sx, sy = _systems(ctx, p, None)
    du0, st0 = cps.cp1_step(sx, sy, du_b, toll=1e-4, max_outer=0, rtol=rtol)
    du0 = du0.cpu().numpy()
    du1, st1 = cps.cp1_step(sx, sy, du_b, toll=0.0, max_outer=1, rtol=rtol, check=False)
    du1 = du1.cpu().numpy()
    assert st0["outer"] == 0 and st1["outer"] == 1
    f = (p.eps, p.kinv, p.field_loc)
    T, _, isd, nbr = oracle.side_coefficients(m.xy, m.tri, m.dirichlet, *f, oracle.CP1_X,
                                              p.nu, p.dt)
    mass = oracle.cp1_mass(m.xy, m.tri, *f, p.nu, p.dt)
    for k, kind in ((0, oracle.CP1_X), (1, oracle.CP1_Y)):
        A = oracle.assemble(m.xy, m.tri, m.dirichlet, *f, kind, p.nu, p.dt)
        lap = -oracle.cp1_laplacian(T, nbr, isd, du_b[k])
        assert np.linalg.norm(A.matvec(du0[k]) - lap) <= 2 * rtol * np.linalg.norm(lap)
        b1 = lap - mass[:, 1] * du0[1 - k]
        assert np.linalg.norm(A.matvec(du1[k]) - b1) <= 2 * rtol * np.linalg.norm(b1)
    sx.free()
    sy.free()
