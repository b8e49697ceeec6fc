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
    s.free()
    ctx.close()


def test_noalloc_rejects_sizes_beyond_its_array(cuda_device):
    lib = cps._cps.load()
    small = torch.zeros(4, dtype=torch.float64, device="cuda")
    idx = torch.zeros(12, dtype=torch.int32, device="cuda")
    # rejected before any work is enqueued: nothing reads past the 4 entries
    rc, _ = noalloc_solve(lib, small, idx, small, small, small, n=MAX_ROWS + 1)
    assert rc == cps._cps.ERR_ARG
    rc, st = noalloc_solve(lib, small, idx, small, small, small, n=0)
    assert rc == 0 and st.iters == 0
