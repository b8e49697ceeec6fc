"""The benchmark workload at full size: the channel-block lattice of
1024 x 1024 vertices (2,093,058 cells, anisotropic K), with the benchmark's
seeds.  Every matrix entry is compared with the oracle's assembly, the SpMV
with the oracle's on every row, and the FP64 Jacobi solve -- in the launch
configuration the benchmark times (autotuned) -- is checked through its true
residual with the oracle's matrix (an oracle solve at this size would take
minutes; the residual bound holds at any size)."""
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


@pytest.fixture(scope="module")
def workload():
    p = synth.channel_block_problem(1024, seed=0)
    return p, synth.rhs(p.mesh, seed=1), oracle.assemble_problem(p)


def _entries(rows, cols, vals):
    """(row, col) pairs in order with duplicates summed."""
    order = np.lexsort((cols, rows))
    rows, cols, vals = rows[order], cols[order], vals[order]
    start = np.flatnonzero(np.r_[True, (rows[1:] != rows[:-1]) | (cols[1:] != cols[:-1])])
    return rows[start], cols[start], np.add.reduceat(vals, start)


def test_full_size_assembly_spmv_and_solve(ctx, workload):
    p, b, A = workload
    m = p.mesh
    nt = m.nt
    assert nt == 2_093_058
    s = ctx.assemble(m.xy, m.tri, m.dirichlet, p.eps, p.kinv, p.field_loc, cps.KIND_CP2,
                     p.nu, p.dt)
    # every entry of the assembled matrix
    diag, col, val = (t.cpu().numpy() for t in s.export_matrix())
    rows3 = np.tile(np.arange(nt), 3)
    col3, val3 = col.ravel().astype(np.int64), val.ravel()
    live = col3 != rows3
    assert np.all(val3[~live] == 0.0)
    g = _entries(np.r_[np.arange(nt), rows3[live]], np.r_[np.arange(nt), col3[live]],
                 np.r_[diag, val3[live]])
    orows = np.repeat(np.arange(nt), np.diff(A.rowptr))
    w = _entries(orows, A.col.astype(np.int64), A.val)
    assert np.array_equal(g[0], w[0]) and np.array_equal(g[1], w[1])
    # The circumcentre distance d_{e,ep} is a difference of coordinates of
    # magnitude up to L = 1023 across sides of length ~1, so both sides carry
    # a rounding of about u L / h relative in every coefficient (summation
    # orders differ); the bound allows 64 u L / h.
    tri_xy = m.xy[m.tri]
    h = np.min(np.linalg.norm(tri_xy - np.roll(tri_xy, 1, axis=1), axis=2))
    tol = 64 * np.finfo(np.float64).eps * np.abs(m.xy).max() / h
    assert np.all(w[2] != 0.0)
    err = np.abs(g[2] - w[2]) / np.abs(w[2])
    assert err.max() <= tol, (err.max(), tol)
    # the SpMV on every row, against |A| |x| row by row
    x = np.random.default_rng(7).standard_normal(nt)
    y = s.matvec(x).cpu().numpy()
    yo = A.matvec(x)
    absA = oracle.CSR(A.rowptr, A.col, np.abs(A.val))
    e2 = np.abs(y - yo) / absA.matvec(np.abs(x))
    assert e2.max() <= tol, (e2.max(), tol)
    # the solve as the benchmark runs it
    bt = torch.as_tensor(b, device="cuda")
    xs, st = s.solve(bt, rtol=1e-10)
    r = b - A.matvec(xs.cpu().numpy())
    rel = np.linalg.norm(r) / np.linalg.norm(b)
    assert rel <= 1e-10 * 1.01
    assert abs(rel - st.rel_res) <= 0.01 * rel
    s.free()
