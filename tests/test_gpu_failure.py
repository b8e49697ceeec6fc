"""Failure detection on the GPU without a GPU fault.

The persistent solves synchronise their blocks with software grid barriers,
and the one-launch ensemble and CP1 step synchronise teams of blocks; every
wait there is bounded.  A test hook makes the next such launch wait for one
arrival that never comes: the waits must run out (about a second), the call
must report CPS_ERR_TIMEOUT, and the context must stay usable for the next
call."""
import time

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


@pytest.mark.parametrize("precond", ["jacobi", "jacobi_single_reduction", "ic0_single_reduction",
                                     "reduced", "reduced_single_reduction"])
def test_stalled_grid_barrier_times_out_and_recovers(ctx, precond):
    p = synth.channel_block_problem(64, seed=5)
    m = p.mesh
    s = ctx.assemble(m.xy, m.tri, m.dirichlet, p.eps, p.kinv, p.field_loc, cps.KIND_CP2,
                     p.nu, p.dt)
    if precond.startswith("reduced"):
        s.set_precond(cps.PC_REDUCED)
    if precond == "ic0_single_reduction":
        s.set_precond(cps.PC_IC0)
    s.set_solver_path(cps.PATH_PERSISTENT_1RED if precond.endswith("single_reduction")
                      else cps.PATH_PERSISTENT)
    b = synth.rhs(m, 3)
    bt = torch.as_tensor(b, device="cuda")
    assert ctx.lib.cps_test_inject(s.handle, 1) == 0
    t0 = time.time()
    with pytest.raises(cps.CpsError) as ei:
        s.solve(bt, rtol=1e-10)
    assert ei.value.code == cps._cps.ERR_TIMEOUT
    assert time.time() - t0 < 60
    # the hook is one-shot and the context survives: the next solve is right
    x, st = s.solve(bt, rtol=1e-10)
    A = oracle.assemble_problem(p)
    r = b - A.matvec(x.cpu().numpy())
    assert np.linalg.norm(r) / np.linalg.norm(b) <= 1e-10 * 1.01
    assert ctx.lib.cps_test_inject(s.handle, 7) == cps._cps.ERR_ARG
    s.free()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_stalled_team_wait_in_the_batch_times_out_and_recovers(ctx, precision):
    """The 30k- and 9k-cell members are solved by teams of blocks: their waits
    stall and run out; the small members, solved by single blocks, finish."""
    prec = cps.FP64 if precision == "fp64" else cps.MIXED
    ctx.set_batch_path(cps.BATCH_ONE_LAUNCH)
    sizes = [30000, 600, 9000, 2500]
    probs = [synth.ensemble_member_problem(nt, seed=70 + i) for i, nt in enumerate(sizes)]
    systems = [ctx.assemble(p.mesh.xy, p.mesh.tri, p.mesh.dirichlet, p.eps, p.kinv, p.field_loc,
                            cps.KIND_CP2, p.nu, p.dt) for p in probs]
    bs = [torch.as_tensor(synth.rhs(p.mesh, 80 + i), device="cuda") for i, p in enumerate(probs)]
    xs = [torch.zeros_like(b) for b in bs]
    assert ctx.lib.cps_test_inject(systems[0].handle, 1) == 0
    t0 = time.time()
    st = cps.solve_batch(systems, bs, xs, rtol=1e-10, precision=prec, check=False)
    assert time.time() - t0 < 60
    assert st[0].status == cps._cps.ERR_TIMEOUT and st[2].status == cps._cps.ERR_TIMEOUT
    assert st[1].status == 0 and st[3].status == 0
    # one-shot, and the context survives: every member is right next time
    for x in xs:
        x.zero_()
    st = cps.solve_batch(systems, bs, xs, rtol=1e-10, precision=prec)
    for p, b, x in zip(probs, bs, xs):
        A = oracle.assemble_problem(p)
        bn = b.cpu().numpy()
        r = bn - A.matvec(x.cpu().numpy())
        assert np.linalg.norm(r) / np.linalg.norm(bn) <= 1e-10 * 1.01
    for s in systems:
        s.free()


def test_stalled_team_wait_in_the_cp1_step_times_out_and_recovers(ctx):
    import dataclasses
    p = synth.channel_block_problem(24, seed=6)
    m = p.mesh
    nbr = oracle.topology(m.tri)
    e, j = np.nonzero(nbr < 0)
    m = dataclasses.replace(m, dirichlet=(e * 3 + j).astype(np.int32))
    p = dataclasses.replace(p, mesh=m)
    sx = ctx.assemble(m.xy, m.tri, m.dirichlet, p.eps, p.kinv, p.field_loc, cps.KIND_CP1_X,
                      p.nu, p.dt)
    sy = ctx.assemble(m.xy, m.tri, m.dirichlet, p.eps, p.kinv, p.field_loc, cps.KIND_CP1_Y,
                      p.nu, p.dt)
    cps.cp1_setup(sx, sy, m.xy, m.tri, p.eps, p.kinv)
    du_b = synth.cell_vector_field(m, 9, mean=(0.01, -0.02), scale=0.05)
    assert ctx.lib.cps_test_inject(sx.handle, 1) == 0
    t0 = time.time()
    _, st = cps.cp1_step(sx, sy, du_b, toll=1e-4, rtol=1e-12, check=False)
    assert st["status"] == cps._cps.ERR_TIMEOUT
    assert time.time() - t0 < 60
    o = oracle.cp1_step(p, du_b, toll=1e-4, rtol=1e-13)
    du, st = cps.cp1_step(sx, sy, du_b, toll=1e-4, rtol=1e-12)
    assert st["outer"] == o.outer
    d = du.cpu().numpy()
    assert np.linalg.norm(d - o.du) / np.linalg.norm(o.du) <= 1e-9
    sx.free()
    sy.free()
