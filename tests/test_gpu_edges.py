"""Degenerate and tiny systems through every solver path: one cell, two
cells, and the 3 x 3 lattice (8 cells), against the oracle's dense Cholesky
solve.  Every way of running the FP64 Jacobi loop (tuned, streaming, one
cluster, persistent), IC(0), the reduced system where the cells are
two-coloured, mixed precision, and the batched call over all three."""
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


def _problem(mesh):
    eps = np.linspace(0.4, 1.0, mesh.nv)
    return synth.Problem(mesh, eps, synth.iso_kinv(synth.kozeny_carman_kinv(eps)),
                         synth.PER_VERTEX)


def _cases():
    two = synth.lattice(2, seed=0)          # 2 cells, Dirichlet side on cell 1
    one = dataclasses.replace(two, tri=np.ascontiguousarray(two.tri[1:]),
                              dirichlet=np.array([0], dtype=np.int32))
    return {"one_cell": _problem(one), "two_cells": _problem(two),
            "lattice3": _problem(synth.lattice(3, seed=1))}


CASES = _cases()


def _assemble(ctx, p):
    m = p.mesh
    return ctx.assemble(m.xy, m.tri, m.dirichlet, p.eps, p.kinv, p.field_loc, cps.KIND_CP2,
                        p.nu, p.dt)


def _err(x, xo):
    return np.linalg.norm(x.cpu().numpy() - xo) / np.linalg.norm(xo)


@pytest.mark.parametrize("name", sorted(CASES))
def test_tiny_systems_every_path(ctx, name):
    p = CASES[name]
    A = oracle.assemble_problem(p)
    b = synth.rhs(p.mesh, 3)
    xo = oracle.dense_cholesky_solve(A.dense(), b)
    s = _assemble(ctx, p)
    bt = torch.as_tensor(b, device="cuda")
    paths = [cps.PATH_AUTO, cps.PATH_STREAM, cps.PATH_STREAM_1RED, cps.PATH_CLUSTER,
             cps.PATH_CLUSTER_1RED, cps.PATH_CLUSTER_PIPE, cps.PATH_CLUSTER_SSTEP2,
             cps.PATH_CLUSTER_SSTEP3, cps.PATH_PERSISTENT, cps.PATH_PERSISTENT_1RED]
    for path in paths:
        s.set_solver_path(path)
        x, st = s.solve(bt, rtol=1e-12)
        assert _err(x, xo) < 1e-9, (path, _err(x, xo))
    s.set_solver_path(cps.PATH_AUTO)
    x, st = s.solve(bt, rtol=1e-12, precision=cps.MIXED)
    assert _err(x, xo) < 1e-8
    s.set_precond(cps.PC_IC0)
    x, st = s.solve(bt, rtol=1e-12)
    assert _err(x, xo) < 1e-9
    if p.mesh.nt > 1:                         # these lattices are two-coloured
        s.set_precond(cps.PC_REDUCED)
        for path in (cps.PATH_STREAM, cps.PATH_PERSISTENT, cps.PATH_PERSISTENT_1RED):
            s.set_solver_path(path)
            x, st = s.solve(bt, rtol=1e-12)
            assert _err(x, xo) < 1e-9, ("reduced", path)
    s.free()


def test_tiny_systems_batched(ctx):
    systems, bs, ref = [], [], []
    for name in sorted(CASES):
        p = CASES[name]
        A = oracle.assemble_problem(p)
        b = synth.rhs(p.mesh, 5)
        ref.append(oracle.dense_cholesky_solve(A.dense(), b))
        systems.append(_assemble(ctx, p))
        bs.append(torch.as_tensor(b, device="cuda"))
    for prec, tol in ((cps.FP64, 1e-9), (cps.MIXED, 1e-8)):
        xs = [torch.zeros_like(b) for b in bs]
        cps.solve_batch(systems, bs, xs, rtol=1e-12, precision=prec)
        for x, xo in zip(xs, ref):
            assert _err(x, xo) < tol
    for s in systems:
        s.free()
