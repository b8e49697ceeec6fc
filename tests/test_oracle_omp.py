"""The multi-threaded timing variant of the oracle's Jacobi-PCG (the
benchmark's CPU baseline) against the single-threaded oracle: the same
iterates up to the summation order of the inner products."""
import numpy as np
import pytest

import oracle
import synth


@pytest.mark.parametrize("maker", [lambda: synth.channel_block_problem(40, seed=5),
                                   lambda: synth.centred_block_problem(33, seed=2)])
def test_omp_pcg_matches_single_thread_oracle(maker):
    p = maker()
    b = synth.rhs(p.mesh, 11)
    A = oracle.assemble_problem(p)
    x1, s1 = oracle.pcg(A, b, rtol=1e-11)
    x2, s2 = oracle.pcg_jacobi_omp(A, b, rtol=1e-11)
    assert s2.status == oracle.OK
    assert abs(s1.iters - s2.iters) <= 2
    assert s2.rel_res <= 1.01e-11
    assert np.linalg.norm(x1 - x2) / np.linalg.norm(x1) < 1e-10
    # a warm start from the solution takes no iteration
    _, s3 = oracle.pcg_jacobi_omp(A, b, x0=x1, rtol=1e-10)
    assert s3.iters == 0


def test_omp_pcg_bounded_sample_runs_exactly_maxit():
    p = synth.channel_block_problem(24, seed=1)
    b = synth.rhs(p.mesh, 2)
    A = oracle.assemble_problem(p)
    _, st = oracle.pcg_jacobi_omp(A, b, rtol=0.0, maxit=37)
    assert st.iters == 37 and st.status == oracle.ERR_NOT_CONVERGED
    _, s1 = oracle.pcg(A, b, rtol=0.0, maxit=37, raise_on_error=False)
    assert abs(st.rel_res - s1.rel_res) <= 1e-9 * s1.rel_res
    assert oracle.omp_threads() >= 1


def test_omp_pcg_zero_rhs_and_bad_diagonal():
    p = synth.channel_block_problem(8, seed=1)
    A = oracle.assemble_problem(p)
    x, st = oracle.pcg_jacobi_omp(A, np.zeros(A.n), rtol=1e-10)
    assert st.status == oracle.OK and np.all(x == 0.0) and st.iters == 0
    bad = oracle.CSR(A.rowptr.copy(), A.col.copy(), A.val.copy())
    for k in range(bad.rowptr[0], bad.rowptr[1]):
        if bad.col[k] == 0:
            bad.val[k] = -1.0
    _, st = oracle.pcg_jacobi_omp(bad, np.ones(A.n), rtol=1e-10)
    assert st.status == oracle.ERR_NOT_SPD
