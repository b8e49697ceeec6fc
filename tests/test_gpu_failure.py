"""Failure detection on the GPU without a GPU fault.

The persistent solves synchronise their blocks with software grid barriers;
every wait there is bounded.  A test hook makes the next persistent launch
wait for one arrival that never comes: the waits must run out (about a
second), the solve must report CPS_ERR_TIMEOUT, and the context must stay
usable for the next solve."""
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
                                     "reduced"])
def test_stalled_grid_barrier_times_out_and_recovers(ctx, precond):
    p = synth.channel_block_problem(64, seed=5)
    m = p.mesh
    s = ctx.assemble(m.xy, m.tri, m.dirichlet, p.eps, p.kinv, p.field_loc, cps.KIND_CP2,
                     p.nu, p.dt)
    if precond == "reduced":
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
