"""The allocation-free entry point cps_solve_ell_noalloc, called through the C
ABI, against cps_solve on the same system.

It exists for callers that may not allocate device memory themselves (their
host owns all device memory, or cudaMalloc's implicit synchronisation is not
allowed where they run): it takes a matrix in the exported ELL form and
keeps its work vectors in a fixed array inside the library.  The file sorts
last so that a run stopping at the first failure has run every other test
before it; it also passes alone in a fresh process."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

cps = pytest.importorskip("paper_2309_03543_gb300")

P = ctypes.c_void_p
MAX_ROWS = 65536


def noalloc_solve(lib, diag, col, val, b, x, rtol=1e-12, max_iter=1_000_000, n=None):
    st = cps._cps.Stats()
    n = diag.numel() if n is None else n
    rc = lib.cps_solve_ell_noalloc(n, P(diag.data_ptr()), P(col.data_ptr()), P(val.data_ptr()),
                                   P(b.data_ptr()), P(x.data_ptr()), rtol, max_iter,
                                   ctypes.byref(st), P(torch.cuda.current_stream().cuda_stream))
    return rc, st


@pytest.mark.parametrize("maker", [lambda: synth.channel_block_problem(64, seed=5),
                                   lambda: synth.centred_block_problem(150, seed=2)])
def test_noalloc_solve_matches_cps_solve_twice(cuda_device, maker):
    p = maker()
    m = p.mesh
    assert m.nt <= MAX_ROWS
    ctx = cps.Context(0)
    s = ctx.assemble(m.xy, m.tri, m.dirichlet, p.eps, p.kinv, p.field_loc, cps.KIND_CP2,
                     p.nu, p.dt)
    diag, col, val = s.export_matrix()
    col = col.contiguous()
    val = val.contiguous()
    lib = ctx.lib
    for call in range(2):
        b = torch.as_tensor(synth.rhs(m, 30 + call), device="cuda")
        x_ref, st_ref = s.solve(b, rtol=1e-12, check=False)
        assert st_ref.rel_res < 1e-10
        x = torch.zeros_like(b)
        rc, st = noalloc_solve(lib, diag, col, val, b, x)
        torch.cuda.synchronize()
        assert rc in (0, cps._cps.ERR_NOT_CONVERGED), rc
        assert st.rel_res < 1e-10
        err = float(torch.linalg.norm(x - x_ref) / torch.linalg.norm(x_ref))
        assert err < 1e-9, (call, err)
        # and against the oracle's FP64 solve of the same system (Sec. 3.2.2)
        xo, _, _ = oracle.solve_problem(p, b.cpu().numpy(), rtol=1e-13)
        err_o = np.linalg.norm(x.cpu().numpy() - xo) / np.linalg.norm(xo)
        assert err_o < 1e-9, (call, err_o)
        assert st.status == rc
    s.free()
    ctx.close()


def test_noalloc_second_call_allocates_no_device_memory(cuda_device):
    """The property the entry point exists for: once the first call on the
    device has loaded the library's fixed array, a call changes the device's
    free memory by nothing."""
    p = synth.channel_block_problem(48, seed=3)
    m = p.mesh
    ctx = cps.Context(0)
    s = ctx.assemble(m.xy, m.tri, m.dirichlet, p.eps, p.kinv, p.field_loc, cps.KIND_CP2,
                     p.nu, p.dt)
    diag, col, val = s.export_matrix()
    col = col.contiguous()
    val = val.contiguous()
    b = torch.as_tensor(synth.rhs(m, 41), device="cuda")
    x = torch.zeros_like(b)
    rc, _ = noalloc_solve(ctx.lib, diag, col, val, b, x)      # first call: loads the array
    assert rc == 0
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    x.zero_()
    torch.cuda.synchronize()
    rc, st = noalloc_solve(ctx.lib, diag, col, val, b, x)
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    assert rc == 0 and st.status == 0
    assert free1 == free0, (free0, free1)
    s.free()
    ctx.close()


def test_noalloc_error_paths_report_status_in_stats(cuda_device):
    """A column out of range is CPS_ERR_ARG and a non-positive diagonal is
    CPS_ERR_NOT_SPD; both are found by the set-up kernels' own checks before
    any out-of-range access, and stats carries the returned status."""
    p = synth.channel_block_problem(6, seed=4)
    m = p.mesh
    ctx = cps.Context(0)
    s = ctx.assemble(m.xy, m.tri, m.dirichlet, p.eps, p.kinv, p.field_loc, cps.KIND_CP2,
                     p.nu, p.dt)
    diag, col, val = s.export_matrix()
    n = diag.numel()
    b = torch.as_tensor(synth.rhs(m, 7), device="cuda")
    bad_col = col.contiguous().clone()
    bad_col.view(-1)[0] = n
    x = torch.zeros_like(b)
    rc, st = noalloc_solve(ctx.lib, diag, bad_col, val.contiguous(), b, x)
    assert rc == cps._cps.ERR_ARG and st.status == rc
    bad_diag = diag.clone()
    bad_diag[0] = 0.0
    rc, st = noalloc_solve(ctx.lib, bad_diag, col.contiguous(), val.contiguous(), b, x)
    assert rc == cps._cps.ERR_NOT_SPD and st.status == rc
    # a good call right after the failed ones still solves
    rc, st = noalloc_solve(ctx.lib, diag, col.contiguous(), val.contiguous(), b, x)
    torch.cuda.synchronize()
    assert rc == 0 and st.status == 0 and st.rel_res < 1e-10
    s.free()
    ctx.close()


def test_noalloc_rejects_sizes_beyond_its_array(cuda_device):
    lib = cps._cps.load()
    small = torch.zeros(4, dtype=torch.float64, device="cuda")
    idx = torch.zeros(12, dtype=torch.int32, device="cuda")
    # rejected before any work is enqueued: nothing reads past the 4 entries
    rc, st = noalloc_solve(lib, small, idx, small, small, small, n=MAX_ROWS + 1)
    assert rc == cps._cps.ERR_ARG and st.status == rc
    rc, st = noalloc_solve(lib, small, idx, small, small, small, n=0)
    assert rc == 0 and st.iters == 0
