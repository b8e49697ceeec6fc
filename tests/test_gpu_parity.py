"""CUDA path vs the CPU oracle, through the C ABI, element by element.

Assembly: the exported ELL matrix against the oracle's CSR (FP64, 1e-13
relative per entry).  Solves: relative L2 error of x against the oracle's
solution at rtol 1e-13 -- 1e-9 for FP64 and 1e-8 for mixed precision.
Sizes span several thread blocks and a ragged tail."""
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


def assemble(ctx, p, kind=cps.KIND_CP2):
    m = p.mesh
    return ctx.assemble(m.xy, m.tri, m.dirichlet, p.eps, p.kinv, p.field_loc, kind, p.nu, p.dt)


def problems():
    yield "block37", synth.centred_block_problem(37, seed=3)
    yield "channel64", synth.channel_block_problem(64, seed=5)
    yield "logperm29", synth.log_permeability_problem(29, seed=2)[0]
    yield "ensemble", synth.ensemble_member_problem(3000, seed=11)
    yield "defect20", synth.defect_problem(20, seed=3)


PROBLEMS = dict(problems())


def csr_rows(A):
    rows = []
    for i in range(A.n):
        d = {}
        for k in range(A.rowptr[i], A.rowptr[i + 1]):
            d[int(A.col[k])] = d.get(int(A.col[k]), 0.0) + A.val[k]
        rows.append(d)
    return rows


def ell_rows(diag, col, val):
    diag = diag.cpu().numpy()
    col = col.cpu().numpy()
    val = val.cpu().numpy()
    rows = []
    for e in range(diag.shape[0]):
        d = {e: diag[e]}
        for j in range(3):
            if col[j, e] != e:
                d[int(col[j, e])] = d.get(int(col[j, e]), 0.0) + val[j, e]
            else:
                assert val[j, e] == 0.0
        rows.append(d)
    return rows


@pytest.mark.parametrize("name", sorted(PROBLEMS))
@pytest.mark.parametrize("kind", [cps.KIND_CP2, cps.KIND_CP1_X, cps.KIND_CP1_Y])
def test_assembly_matches_oracle(ctx, name, kind):
    p = PROBLEMS[name]
    s = assemble(ctx, p, kind)
    A = oracle.assemble_problem(p, kind)
    got = ell_rows(*s.export_matrix())
    want = csr_rows(A)
    scale = np.abs(A.val).max()
    for e, (g, w) in enumerate(zip(got, want)):
        assert g.keys() == w.keys(), e
        for c in w:
            assert abs(g[c] - w[c]) <= 1e-13 * max(abs(w[c]), 1e-300) + 1e-15 * scale, (e, c)
    info = s.info()
    assert info["is_mmatrix"] and info["nt"] == p.mesh.nt
    g = oracle.geometry(p.mesh.xy, p.mesh.tri)
    assert info["n_interior_sides"] == int((g.nbr >= 0).sum()) // 2
    s.free()


@pytest.mark.parametrize("name", sorted(PROBLEMS))
@pytest.mark.parametrize("precond", [cps.PC_JACOBI, cps.PC_IC0])
@pytest.mark.parametrize("precision,tol", [(cps.FP64, 1e-9), (cps.MIXED, 1e-8)])
def test_solve_matches_oracle(ctx, name, precond, precision, tol):
    """Relative L2 error against the oracle's solution at rtol 1e-13.  The
    GPU solves to rtol 1e-12; where FP64 cannot reach that true residual on
    an ill-conditioned system the call reports CPS_ERR_NOT_CONVERGED with the
    residual it reached, which must still be below 1e-10."""
    p = PROBLEMS[name]
    s = assemble(ctx, p)
    s.set_precond(precond)
    b = synth.rhs(p.mesh, 17)
    xo, sto, A = oracle.solve_problem(p, b, rtol=1e-13)
    x, st = s.solve(torch.as_tensor(b, device="cuda"), rtol=1e-12, precision=precision,
                    check=False)
    assert st.status in (0, cps._cps.ERR_NOT_CONVERGED)
    assert st.rel_res < (1e-12 if st.status == 0 else 1e-10)
    x = x.cpu().numpy()
    err = np.linalg.norm(x - xo) / np.linalg.norm(xo)
    assert err < tol, err
    # the GPU's own residual claim, checked with the oracle's matrix
    r = b - A.matvec(x)
    assert np.linalg.norm(r) / np.linalg.norm(b) < 2 * max(st.rel_res, 1e-13)
    s.free()


def test_ic0_needs_fewer_iterations_than_jacobi(ctx):
    p = PROBLEMS["channel64"]
    s = assemble(ctx, p)
    b = torch.as_tensor(synth.rhs(p.mesh, 3), device="cuda")
    _, sj = s.solve(b, rtol=1e-10)
    s.set_precond(cps.PC_IC0)
    _, si = s.solve(b, rtol=1e-10)
    A = oracle.assemble_problem(p)
    _, so = oracle.pcg(A, b.cpu().numpy(), rtol=1e-10, precond=oracle.PC_IC0,
                       perm=oracle.red_black_order(A.n))
    assert si.iters < 0.75 * sj.iters
    # same ordering (red/black on the lattice) as the oracle's coloured IC(0)
    assert abs(si.iters - so.iters) <= max(8, 0.05 * so.iters)
    s.free()


def test_two_solves_one_matrix_warm_start(ctx):
    """CP2 solves twice per step on one matrix (Eq. Cs2_7); the second can
    start from the first solution."""
    p = PROBLEMS["channel64"]
    s = assemble(ctx, p)
    b1 = synth.rhs(p.mesh, 1)
    b2 = b1 + 1e-3 * synth.rhs(p.mesh, 2)
    x1, st1 = s.solve(torch.as_tensor(b1, device="cuda"), rtol=1e-11)
    x2 = x1.clone()
    _, st2 = s.solve(torch.as_tensor(b2, device="cuda"), x=x2, rtol=1e-11)
    assert st2.iters < st1.iters
    xo, _, _ = oracle.solve_problem(p, b2, rtol=1e-13)
    assert np.linalg.norm(x2.cpu().numpy() - xo) / np.linalg.norm(xo) < 1e-8
    # solving again from the solution needs no iteration
    _, st3 = s.solve(torch.as_tensor(b2, device="cuda"), x=x2.clone(), rtol=1e-6)
    assert st3.iters == 0
    s.free()


def test_zero_rhs_and_max_iter(ctx):
    p = PROBLEMS["block37"]
    s = assemble(ctx, p)
    x = torch.ones(p.mesh.nt, dtype=torch.float64, device="cuda")
    _, st = s.solve(torch.zeros_like(x), x=x)
    assert st.iters == 0 and torch.all(x == 0)
    b = torch.as_tensor(synth.rhs(p.mesh, 1), device="cuda")
    with pytest.raises(cps.CpsError) as ei:
        s.solve(b, rtol=1e-12, max_iter=5)
    assert ei.value.code == cps._cps.ERR_NOT_CONVERGED
    x, st = s.solve(b, rtol=1e-12, max_iter=5, check=False)
    assert st.iters == 5 and st.status == cps._cps.ERR_NOT_CONVERGED
    s.free()


def test_host_buffers_round_trip(ctx):
    p = PROBLEMS["block37"]
    s = assemble(ctx, p)
    b = synth.rhs(p.mesh, 4)
    x, st = s.solve(torch.as_tensor(b), rtol=1e-12)     # CPU tensor in, CPU tensor out
    assert x.device.type == "cpu"
    xo, _, _ = oracle.solve_problem(p, b, rtol=1e-13)
    assert np.linalg.norm(x.numpy() - xo) / np.linalg.norm(xo) < 1e-9
    s.free()


def test_matvec_matches_oracle(ctx):
    p = PROBLEMS["channel64"]
    s = assemble(ctx, p)
    A = oracle.assemble_problem(p)
    v = np.random.default_rng(3).standard_normal(p.mesh.nt)
    y = s.matvec(torch.as_tensor(v, device="cuda")).cpu().numpy()
    np.testing.assert_allclose(y, A.matvec(v), rtol=1e-12, atol=1e-14 * np.abs(A.val).max())
    s.free()


def test_invalid_meshes_are_rejected(ctx):
    m = synth.lattice(8, seed=0)
    one = np.ones(m.nv)
    zero = np.zeros((m.nv, 3))
    E = cps._cps
    with pytest.raises(cps.CpsError) as ei:        # CP2 without Dirichlet sides
        ctx.assemble(m.xy, m.tri, np.zeros(0, np.int32), one, zero)
    assert ei.value.code == E.ERR_SINGULAR
    with pytest.raises(cps.CpsError) as ei:        # clockwise triangle
        tri = m.tri.copy()
        tri[5] = tri[5][[0, 2, 1]]
        ctx.assemble(m.xy, tri, m.dirichlet, one, zero)
    assert ei.value.code in (E.ERR_ORIENTATION, E.ERR_NONMANIFOLD, E.ERR_NONDELAUNAY)
    with pytest.raises(cps.CpsError) as ei:        # non-Delaunay vertex move
        xy = m.xy.copy()
        xy[2 * 8 + 2] += [0.0, 0.6]
        ctx.assemble(xy, m.tri, m.dirichlet, one, zero)
    assert ei.value.code in (E.ERR_NONDELAUNAY, E.ERR_ORIENTATION)
    with pytest.raises(cps.CpsError) as ei:        # a side of three triangles
        tri = np.concatenate([m.tri, m.tri[:1, [1, 0, 2]]])
        ctx.assemble(m.xy, tri, m.dirichlet, one, zero)
    assert ei.value.code in (E.ERR_NONMANIFOLD, E.ERR_ORIENTATION)
    with pytest.raises(cps.CpsError) as ei:        # vertex id out of range
        tri = m.tri.copy()
        tri[0, 0] = m.nv + 5
        ctx.assemble(m.xy, tri, m.dirichlet, one, zero)
    assert ei.value.code == E.ERR_ARG
    with pytest.raises(cps.CpsError) as ei:        # Dirichlet side that is interior
        ctx.assemble(m.xy, m.tri, np.array([3 * 40 + 0], np.int32), one, zero)
    assert ei.value.code == E.ERR_ARG
    with pytest.raises(cps.CpsError) as ei:        # zero porosity
        ctx.assemble(m.xy, m.tri, m.dirichlet, np.zeros(m.nv), zero)
    assert ei.value.code == E.ERR_ARG
    # the context still works after every rejection
    s = ctx.assemble(m.xy, m.tri, m.dirichlet, one, zero)
    s.free()


def test_adjoint_matches_oracle(ctx):
    p, theta = synth.log_permeability_problem(24, seed=4)
    s = assemble(ctx, p)
    b = synth.rhs(p.mesh, 5)
    x, _ = s.solve(torch.as_tensor(b, device="cuda"), rtol=1e-12)
    target = 0.5 * torch.as_tensor(synth.rhs(p.mesh, 6), device="cuda") * 1e3
    g = 2 * (x - target)
    nt = p.mesh.nt
    dT = torch.zeros(3, nt, dtype=torch.float64, device="cuda")
    dth = torch.zeros(nt, dtype=torch.float64, device="cuda")
    lam, st = s.adjoint(x, g, dT=dT, dtheta=dth, rtol=1e-12)
    A = oracle.assemble_problem(p)
    lam_o, _ = oracle.pcg(A, g.cpu().numpy(), rtol=1e-13, raise_on_error=False)
    assert np.linalg.norm(lam.cpu().numpy() - lam_o) / np.linalg.norm(lam_o) < 1e-9
    T, sigma, isd, nbr = oracle.side_coefficients(p.mesh.xy, p.mesh.tri, p.mesh.dirichlet,
                                                  p.eps, p.kinv, p.field_loc, oracle.CP2, p.nu,
                                                  p.dt)
    dT_o = oracle.side_gradient(nbr, isd, lam_o, x.cpu().numpy())
    np.testing.assert_allclose(dT.cpu().numpy().T, dT_o, rtol=1e-7,
                               atol=1e-9 * np.abs(dT_o).max())
    dth_o = oracle.theta_gradient(p.mesh.xy, p.mesh.tri, nbr, isd, p.eps, theta, p.nu, p.dt, dT_o)
    np.testing.assert_allclose(dth.cpu().numpy(), dth_o, rtol=1e-7,
                               atol=1e-9 * np.abs(dth_o).max())
    s.free()


def test_autotuned_solves_on_a_large_system(ctx):
    """Above 131072 cells the first solve of each precision autotunes the
    iteration kernels; the tuned solves must still be right.  Checked with
    the oracle's matrix (true residual) and its Jacobi-PCG iterate count."""
    p = synth.channel_block_problem(300, seed=8)
    assert p.mesh.nt >= 1 << 17
    s = assemble(ctx, p)
    A = oracle.assemble_problem(p)
    b = synth.rhs(p.mesh, 2)
    bt = torch.as_tensor(b, device="cuda")
    for prec in (cps.FP64, cps.MIXED):
        x, st = s.solve(bt, rtol=1e-10, precision=prec)
        tu = s.tuning(prec)
        nk = 3 if prec == cps.FP64 else 2
        assert all(u in (1, 2, 4) for u in tu["unroll"][:nk])
        assert all(0 < g <= 4096 for g in tu["grid"][:nk])
        assert all(b in ((256, 1024) if prec == cps.FP64 else (256,)) for b in tu["block"][:nk])
        r = b - A.matvec(x.cpu().numpy())
        assert np.linalg.norm(r) / np.linalg.norm(b) <= 1e-10 * 1.01
    s.set_precond(cps.PC_IC0)
    x, st = s.solve(bt, rtol=1e-10)
    r = b - A.matvec(x.cpu().numpy())
    assert np.linalg.norm(r) / np.linalg.norm(b) <= 1e-10 * 1.01
    s.free()


@pytest.mark.parametrize("batch_path", ["one_launch", "graph"])
def test_batched_solve_matches_oracle_per_system(ctx, batch_path):
    """Uneven ensemble solved together (in one launch whose blocks take whole
    systems, or one launch per phase with per-system convergence masks):
    every member against its own oracle solve; a zero RHS member returns
    zeros; the result equals the loop of single solves."""
    ctx.set_batch_path(cps.BATCH_ONE_LAUNCH if batch_path == "one_launch" else cps.BATCH_GRAPH)
    sizes = [600, 2500, 9000, 1200, 30000]
    probs = [synth.ensemble_member_problem(nt, seed=40 + i) for i, nt in enumerate(sizes)]
    systems = [assemble(ctx, p) for p in probs]
    bs = [torch.as_tensor(synth.rhs(p.mesh, 90 + i), device="cuda") for i, p in enumerate(probs)]
    bs[3] = torch.zeros_like(bs[3])
    xs = [torch.zeros_like(b) for b in bs]
    stats = cps.solve_batch(systems, bs, xs, rtol=1e-12, check=False)
    xos = {}
    for i, (p, b, x, st) in enumerate(zip(probs, bs, xs, stats)):
        if i == 3:
            assert torch.all(x == 0) and st.iters == 0
            continue
        assert st.status in (0, cps._cps.ERR_NOT_CONVERGED) and st.rel_res < 1e-10
        xo, _, _ = oracle.solve_problem(p, b.cpu().numpy(), rtol=1e-13)
        xos[i] = xo
        err = np.linalg.norm(x.cpu().numpy() - xo) / np.linalg.norm(xo)
        assert err < 1e-9, (i, err)
        # a single solve may take another recurrence (the tuner's single-
        # reduction cluster path): the same iterates in exact arithmetic, but
        # at rtol 1e-12, near the FP64 floor, the counts drift a few percent
        x1, st1 = systems[i].solve(b, rtol=1e-12, check=False)
        assert abs(st1.iters - st.iters) <= max(8, 0.05 * st1.iters)
    # a second batched call on the same handles (state reuse) in mixed mode:
    # every member against its own oracle solve at the mixed tolerance (the
    # members' solves run concurrently, so a fault between them would show)
    for rtol in (1e-10, 1e-12):
        xs2 = [torch.zeros_like(b) for b in bs]
        stats2 = cps.solve_batch(systems, bs, xs2, rtol=rtol, precision=cps.MIXED, check=False)
        for i, (x, st) in enumerate(zip(xs2, stats2)):
            if i == 3:
                assert torch.all(x == 0) and st.iters == 0
                continue
            assert st.status in (0, cps._cps.ERR_NOT_CONVERGED)
            assert st.rel_res <= (rtol if st.status == 0 else 1e-10)
            if rtol == 1e-12:
                err = np.linalg.norm(x.cpu().numpy() - xos[i]) / np.linalg.norm(xos[i])
                assert err < 1e-8, (i, err)
    for s in systems:
        s.free()
    ctx.set_batch_path(cps.BATCH_ONE_LAUNCH)


@pytest.mark.parametrize("path", ["textbook", "single_reduction", "pipelined", "s_step2",
                                  "s_step3"])
@pytest.mark.parametrize("name", ["block37", "channel64", "defect20"])
def test_cluster_path_matches_oracle(ctx, name, path):
    """The one-launch cluster solve (system held in the cluster's shared
    memory, neighbours read through distributed shared memory), with the
    textbook, the single-reduction, the pipelined and the s-step (s = 2, 3)
    recurrences, against the oracle, and against the streaming path on the
    same system (same iterates in exact arithmetic, so nearly the same
    iteration count; at rtol 1e-12, near the FP64 floor, the pipelined and
    s-step recurrences may drift and restart)."""
    cluster = {"textbook": cps.PATH_CLUSTER, "single_reduction": cps.PATH_CLUSTER_1RED,
               "pipelined": cps.PATH_CLUSTER_PIPE, "s_step2": cps.PATH_CLUSTER_SSTEP2,
               "s_step3": cps.PATH_CLUSTER_SSTEP3}[path]
    p = PROBLEMS[name]
    s = assemble(ctx, p)
    b = synth.rhs(p.mesh, 23)
    bt = torch.as_tensor(b, device="cuda")
    s.set_solver_path(cluster)
    x, st = s.solve(bt, rtol=1e-12, check=False)
    assert st.status in (0, cps._cps.ERR_NOT_CONVERGED) and st.rel_res < 1e-10
    xo, _, _ = oracle.solve_problem(p, b, rtol=1e-13)
    err = np.linalg.norm(x.cpu().numpy() - xo) / np.linalg.norm(xo)
    assert err < 1e-9, err
    s.set_solver_path(cps.PATH_STREAM)
    x2, st2 = s.solve(bt, rtol=1e-12, check=False)
    if path in ("pipelined", "s_step2", "s_step3"):
        # these recurrences lose accuracy sooner: at 1e-12 the run may
        # restart from the true residual, but stays within twice the count
        assert st.iters <= 2 * st2.iters + 8
    else:
        assert abs(st2.iters - st.iters) <= max(8, 0.02 * st.iters)
    # warm start and zero right-hand side on the cluster path
    s.set_solver_path(cluster)
    x3 = x.clone()
    _, st3 = s.solve(bt, x=x3, rtol=1e-8)
    assert st3.iters == 0
    z = torch.ones_like(bt)
    _, st4 = s.solve(torch.zeros_like(bt), x=z)
    assert torch.all(z == 0)
    s.set_solver_path(cps.PATH_AUTO)
    x5, st5 = s.solve(bt, rtol=1e-10)
    assert st5.rel_res <= 1e-10
    s.free()


def test_cluster_path_rejects_oversized_systems(ctx):
    p = synth.channel_block_problem(300, seed=1)
    s = assemble(ctx, p)
    for path in (cps.PATH_CLUSTER, cps.PATH_CLUSTER_1RED, cps.PATH_CLUSTER_PIPE,
                 cps.PATH_CLUSTER_SSTEP2, cps.PATH_CLUSTER_SSTEP3):
        with pytest.raises(cps.CpsError):
            s.set_solver_path(path)
    s.free()


@pytest.mark.parametrize("name", ["block37", "channel64", "logperm29", "ensemble"])
def test_reduced_system_solve_matches_oracle(ctx, name):
    """Two-coloured lattices: exact elimination of one colour, CG on the Schur
    complement of the other; the full solution against the oracle."""
    p = PROBLEMS[name]
    s = assemble(ctx, p)
    s.set_precond(cps.PC_REDUCED)
    b = synth.rhs(p.mesh, 29)
    x, st = s.solve(torch.as_tensor(b, device="cuda"), rtol=1e-12, check=False)
    assert st.status in (0, cps._cps.ERR_NOT_CONVERGED) and st.rel_res < 1e-10
    xo, sto, A = oracle.solve_problem(p, b, rtol=1e-13)
    err = np.linalg.norm(x.cpu().numpy() - xo) / np.linalg.norm(xo)
    assert err < 1e-9, err
    r = b - A.matvec(x.cpu().numpy())
    assert np.linalg.norm(r) / np.linalg.norm(b) < 2 * max(st.rel_res, 1e-13)
    # fewer iterations than Jacobi on the full system
    s.set_precond(cps.PC_JACOBI)
    _, sj = s.solve(torch.as_tensor(b, device="cuda"), rtol=1e-10)
    s.set_precond(cps.PC_REDUCED)
    _, sr = s.solve(torch.as_tensor(b, device="cuda"), rtol=1e-10)
    assert sr.iters < 0.75 * sj.iters
    # warm start from the solution: nothing to do
    _, sw = s.solve(torch.as_tensor(b, device="cuda"), x=x.clone(), rtol=1e-8)
    assert sw.iters == 0
    with pytest.raises(cps.CpsError):
        s.solve(torch.as_tensor(b, device="cuda"), precision=cps.MIXED)
    s.free()


def test_reduced_system_needs_two_colours(ctx):
    p = PROBLEMS["defect20"]
    s = assemble(ctx, p)
    with pytest.raises(cps.CpsError) as ei:
        s.set_precond(cps.PC_REDUCED)
    assert ei.value.code == cps._cps.ERR_ARG
    s.set_precond(cps.PC_IC0)            # the same ordering serves IC(0)
    _, st = s.solve(torch.as_tensor(synth.rhs(p.mesh, 1), device="cuda"), rtol=1e-10)
    assert st.rel_res <= 1e-10
    s.free()


@pytest.mark.parametrize("name", ["block37", "channel64", "defect20", "channel300"])
def test_persistent_path_matches_oracle(ctx, name):
    """One cooperative launch runs the whole Jacobi-PCG solve, iterations
    separated by software grid barriers: against the oracle, and the iterate
    count against the streaming path on the same system."""
    p = PROBLEMS[name] if name in PROBLEMS else synth.channel_block_problem(300, seed=8)
    s = assemble(ctx, p)
    b = synth.rhs(p.mesh, 31)
    bt = torch.as_tensor(b, device="cuda")
    s.set_solver_path(cps.PATH_PERSISTENT)
    x, st = s.solve(bt, rtol=1e-12, check=False)
    assert st.status in (0, cps._cps.ERR_NOT_CONVERGED) and st.rel_res < 1e-10
    assert s.tuning()["persistent"]
    xo, sto, A = oracle.solve_problem(p, b, rtol=1e-13)
    err = np.linalg.norm(x.cpu().numpy() - xo) / np.linalg.norm(xo)
    assert err < 1e-9, err
    r = b - A.matvec(x.cpu().numpy())
    assert np.linalg.norm(r) / np.linalg.norm(b) < 2 * max(st.rel_res, 1e-13)
    s.set_solver_path(cps.PATH_STREAM)
    _, st2 = s.solve(bt, rtol=1e-12, check=False)
    assert abs(st2.iters - st.iters) <= max(8, 0.02 * st.iters)
    s.set_solver_path(cps.PATH_PERSISTENT)
    # warm start from the solution, zero right-hand side, iteration cap
    _, st3 = s.solve(bt, x=x.clone(), rtol=1e-8)
    assert st3.iters == 0
    z = torch.ones_like(bt)
    s.solve(torch.zeros_like(bt), x=z)
    assert torch.all(z == 0)
    _, st4 = s.solve(bt, rtol=1e-14, max_iter=5, check=False)
    assert st4.status == cps._cps.ERR_NOT_CONVERGED and st4.iters == 5
    s.free()


@pytest.mark.parametrize("path", ["textbook", "single_reduction", "single_reduction_l2"])
@pytest.mark.parametrize("name", ["block37", "channel64", "channel300"])
def test_persistent_reduced_system_matches_oracle(ctx, name, path):
    """The reduced (black-cell Schur complement) CG in one persistent launch,
    with the textbook and with the single-reduction (Chronopoulos-Gear)
    recurrences (the latter also with its five vectors in persisting L2):
    against the oracle, and the iteration count against the streaming loop
    (the same iterates in exact arithmetic)."""
    p = PROBLEMS[name] if name in PROBLEMS else synth.channel_block_problem(300, seed=8)
    s = assemble(ctx, p)
    s.set_precond(cps.PC_REDUCED)
    pin = {"textbook": cps.PATH_PERSISTENT, "single_reduction": cps.PATH_PERSISTENT_1RED,
           "single_reduction_l2": cps.PATH_PERSISTENT_1RED_L2}[path]
    try:
        s.set_solver_path(pin)
    except cps.CpsError:
        assert path == "single_reduction_l2"      # the set-aside cannot hold five vectors
        pytest.skip("persisting L2 set-aside too small for five vectors")
    b = synth.rhs(p.mesh, 37)
    bt = torch.as_tensor(b, device="cuda")
    x, st = s.solve(bt, rtol=1e-12, check=False)
    assert st.status in (0, cps._cps.ERR_NOT_CONVERGED) and st.rel_res < 1e-10
    tu = s.tuning()
    assert tu["reduced_persistent"]
    assert tu["reduced_single_reduction"] == (path != "textbook")
    assert tu["reduced_l2_window"] == ("vectors5" if path == "single_reduction_l2" else "none")
    xo, _, A = oracle.solve_problem(p, b, rtol=1e-13)
    err = np.linalg.norm(x.cpu().numpy() - xo) / np.linalg.norm(xo)
    assert err < 1e-9, err
    s.set_solver_path(cps.PATH_STREAM)
    x2, st2 = s.solve(bt, rtol=1e-12, check=False)
    if path == "textbook":
        assert abs(st2.iters - st.iters) <= max(8, 0.02 * st.iters)
    else:
        # the single-reduction recurrences drift sooner near the FP64 floor
        # and may restart from the true residual once more
        assert abs(st2.iters - st.iters) <= 8 + 0.08 * st2.iters
    assert torch.allclose(x, x2, rtol=1e-9, atol=1e-12 * float(x.abs().max()))
    s.free()


def test_path_autotuner_reports_every_candidate(ctx):
    """On a system above the tuning threshold the first Jacobi solve times
    streaming, streaming with the matrix or the vectors in persisting L2
    (where they fit) and the persistent launches, textbook and
    single-reduction, and keeps the fastest; the first reduced-system solve
    times streaming against persistent."""
    p = synth.channel_block_problem(300, seed=8)
    s = assemble(ctx, p)
    b = torch.as_tensor(synth.rhs(p.mesh, 4), device="cuda")
    _, st = s.solve(b, rtol=1e-10)
    tu = s.tuning()
    pr = tu["probe_us_per_iter"]
    assert pr["stream"] > 0 and pr["persistent"] > 0 and pr["cluster"] == 0
    assert pr["stream_1red"] > 0
    assert pr["persistent_1red"] > 0
    chosen = [k for k in ("stream", "stream_l2_matrix", "stream_l2_vectors", "persistent",
                          "persistent_l2_vectors", "stream_1red", "stream_1red_l2_vectors",
                          "persistent_1red", "persistent_1red_l2_vectors")
              if pr[k] > 0]
    best = min(chosen, key=lambda k: pr[k])
    assert tu["persistent"] == best.startswith("persistent")
    assert tu["persistent_single_reduction"] == best.startswith("persistent_1red")
    assert tu["stream_single_reduction"] == best.startswith("stream_1red")
    want = {"stream_l2_matrix": ("matrix",), "stream_l2_vectors": ("vectors",),
            "persistent_l2_vectors": ("vectors",),
            "stream_1red_l2_vectors": ("vectors", "vectors5"),
            "persistent_1red_l2_vectors": ("vectors5",)}.get(best, ("none",))
    assert tu["l2_window"] in want
    s.set_precond(cps.PC_REDUCED)
    _, st = s.solve(b, rtol=1e-10)
    tu = s.tuning()
    pr = tu["probe_us_per_iter"]
    assert pr["reduced_stream"] > 0 and pr["reduced_persistent"] > 0
    assert pr["reduced_persistent_1red"] > 0
    red = [k for k in ("reduced_stream", "reduced_persistent", "reduced_stream_l2_vectors",
                       "reduced_persistent_l2_vectors", "reduced_persistent_1red",
                       "reduced_persistent_1red_l2_vectors") if pr[k] > 0]
    best = min(red, key=lambda k: pr[k])
    assert tu["reduced_persistent"] == best.startswith("reduced_persistent")
    assert tu["reduced_single_reduction"] == best.startswith("reduced_persistent_1red")
    want = {"reduced_stream_l2_vectors": "vectors", "reduced_persistent_l2_vectors": "vectors",
            "reduced_persistent_1red_l2_vectors": "vectors5"}.get(best, "none")
    assert tu["reduced_l2_window"] == want
    s.free()


@pytest.mark.parametrize("name", ["channel64", "defect20", "ensemble", "channel300"])
def test_stream_single_reduction_matches_oracle(ctx, name):
    """The single-reduction (Chronopoulos-Gear) FP64 Jacobi loop -- streaming
    and in one persistent launch, each without and with its vectors in
    persisting L2 -- against the oracle; the same iterates as the textbook
    loop in exact arithmetic, so nearly the same iteration count.  channel300
    (178k cells, several hundred rows per persistent block, a ragged last
    block) runs with tuned launch shapes."""
    p = PROBLEMS[name] if name in PROBLEMS else synth.channel_block_problem(300, seed=8)
    s = assemble(ctx, p)
    b = synth.rhs(p.mesh, 31)
    bt = torch.as_tensor(b, device="cuda")
    xo, _, A = oracle.solve_problem(p, b, rtol=1e-13)
    s.set_solver_path(cps.PATH_STREAM)
    _, st0 = s.solve(bt, rtol=1e-12, check=False)
    for path in (cps.PATH_STREAM_1RED, cps.PATH_STREAM_1RED_L2, cps.PATH_PERSISTENT_1RED,
                 cps.PATH_PERSISTENT_1RED_L2):
        try:
            s.set_solver_path(path)
        except cps.CpsError:
            # no persisting set-aside for the vectors here
            assert path in (cps.PATH_STREAM_1RED_L2, cps.PATH_PERSISTENT_1RED_L2)
            continue
        x, st = s.solve(bt, rtol=1e-12, check=False)
        assert st.status in (0, cps._cps.ERR_NOT_CONVERGED) and st.rel_res < 1e-10
        err = np.linalg.norm(x.cpu().numpy() - xo) / np.linalg.norm(xo)
        assert err < 1e-9, (path, err)
        # s = A p and w = A r are carried by recurrence, so near the FP64
        # floor (rtol 1e-12 here) the recursive residual drifts from the true
        # one sooner than in the textbook loop and the solve may restart from
        # the true residual once or twice: a few percent more iterations
        assert abs(st.iters - st0.iters) <= max(8, 0.08 * st0.iters), (path, st.iters, st0.iters)
        tu = s.tuning()
        persistent = path in (cps.PATH_PERSISTENT_1RED, cps.PATH_PERSISTENT_1RED_L2)
        assert tu["stream_single_reduction"] == (not persistent)
        assert tu["persistent_single_reduction"] == persistent
        # the GPU's own residual claim, checked with the oracle's matrix
        r = b - A.matvec(x.cpu().numpy())
        assert np.linalg.norm(r) / np.linalg.norm(b) < 2 * max(st.rel_res, 1e-13)
        # warm start from the solution, and a zero right-hand side
        x2 = x.clone()
        _, st2 = s.solve(bt, x=x2, rtol=1e-8)
        assert st2.iters == 0
        z = torch.ones_like(bt)
        s.solve(torch.zeros_like(bt), x=z)
        assert torch.all(z == 0)
    s.free()


@pytest.mark.parametrize("name", ["block37", "channel64", "logperm29", "ensemble", "defect20",
                                  "channel300"])
def test_persistent_ic0_matches_oracle(ctx, name):
    """IC(0) in the colour order as one persistent launch of the single-
    reduction recurrences (black forward and red backward sweeps read from
    the scaled matrix), without and with its vectors in persisting L2,
    against the oracle's solution and against the streaming IC(0) loop (the
    same preconditioned iterates in exact arithmetic).  On a graph that
    needs more than two colours the pin falls back to the streaming
    kernels."""
    p = PROBLEMS[name] if name in PROBLEMS else synth.channel_block_problem(300, seed=8)
    s = assemble(ctx, p)
    s.set_precond(cps.PC_IC0)
    b = synth.rhs(p.mesh, 37)
    bt = torch.as_tensor(b, device="cuda")
    xo, _, A = oracle.solve_problem(p, b, rtol=1e-13)
    s.set_solver_path(cps.PATH_STREAM)
    x0, st0 = s.solve(bt, rtol=1e-12, max_iter=100_000, check=False)
    assert not s.tuning()["ic0_persistent"]
    for path in (cps.PATH_PERSISTENT_1RED, cps.PATH_PERSISTENT_1RED_L2):
        s.set_solver_path(path)
        x, st = s.solve(bt, rtol=1e-12, max_iter=100_000, check=False)
        assert st.status in (0, cps._cps.ERR_NOT_CONVERGED) and st.rel_res < 1e-10
        err = np.linalg.norm(x.cpu().numpy() - xo) / np.linalg.norm(xo)
        assert err < 1e-9, (path, err)
        assert abs(st.iters - st0.iters) <= max(8, 0.08 * st0.iters), (path, st.iters, st0.iters)
        r = b - A.matvec(x.cpu().numpy())
        assert np.linalg.norm(r) / np.linalg.norm(b) < 2 * max(st.rel_res, 1e-13)
        persistent = s.tuning()["ic0_persistent"]
        if name != "defect20":                  # the lattices are two-coloured
            assert persistent
    # warm start from the solution; a zero right-hand side
    s.set_solver_path(cps.PATH_PERSISTENT_1RED)
    x2 = x.clone()
    _, st2 = s.solve(bt, x=x2, rtol=1e-8)
    assert st2.iters == 0
    z = torch.ones_like(bt)
    s.solve(torch.zeros_like(bt), x=z)
    assert torch.all(z == 0)
    # the tuner times both ways on a fresh pin
    s.set_solver_path(cps.PATH_AUTO)
    x3, st3 = s.solve(bt, rtol=1e-12, max_iter=100_000, check=False)
    assert np.linalg.norm(x3.cpu().numpy() - xo) / np.linalg.norm(xo) < 1e-9
    pr = s.tuning()["probe_us_per_iter"]
    assert (pr["ic0_stream"] > 0) == (name != "defect20")   # probed on two colours only
    s.free()


def test_pinned_shapes_and_stream_l2_path(ctx):
    """Launch shapes pinned instead of tuned, and the streaming path with
    r, p, q in persisting L2, on a system above the tuning threshold: the
    solve still matches the oracle's matrix, and the tuning report echoes
    the pin.  Out-of-range shapes are rejected."""
    p = synth.channel_block_problem(300, seed=8)
    s = assemble(ctx, p)
    A = oracle.assemble_problem(p)
    b = synth.rhs(p.mesh, 5)
    bt = torch.as_tensor(b, device="cuda")
    s.set_kernel_shapes(cps.FP64, [4, 1, 2], [608, 152, 152], [256, 1024, 1024])
    try:                                        # persistent with r, p, q in L2, pinned
        s.set_solver_path(cps.PATH_PERSISTENT_L2)
        pinned = True
    except cps.CpsError:
        pinned = False                          # no persisting set-aside on this GPU
    if pinned:
        xp, _ = s.solve(bt, rtol=1e-10)
        rp_ = b - A.matvec(xp.cpu().numpy())
        assert np.linalg.norm(rp_) / np.linalg.norm(b) <= 1e-10 * 1.01
        assert s.tuning()["persistent"] and s.tuning()["l2_window"] == "vectors"
    try:
        s.set_solver_path(cps.PATH_STREAM_L2)
        window = True
    except cps.CpsError:
        s.set_solver_path(cps.PATH_STREAM)      # no persisting set-aside on this GPU
        window = False
    x, st = s.solve(bt, rtol=1e-10)
    r = b - A.matvec(x.cpu().numpy())
    assert np.linalg.norm(r) / np.linalg.norm(b) <= 1e-10 * 1.01
    tu = s.tuning()
    assert tu["unroll"] == [4, 1, 2] and tu["grid"] == [608, 152, 152]
    assert tu["block"] == [256, 1024, 1024]
    assert tu["l2_window"] == ("vectors" if window else "none")
    for bad in (([3, 1, 2], [608, 152, 152], [256, 256, 256]),
                ([4, 1, 2], [0, 152, 152], [256, 256, 256]),
                ([4, 1, 2], [608, 152, 152], [512, 256, 256])):
        with pytest.raises(cps.CpsError):
            s.set_kernel_shapes(cps.FP64, *bad)
    with pytest.raises(cps.CpsError):
        s.set_kernel_shapes(cps.MIXED, [2, 2, 2], [608, 608, 608], [1024, 256, 256])
    s.free()
