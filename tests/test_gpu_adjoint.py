"""Differentiable corrector solves on the GPU against the oracle: one solve
(torch autograd, adjoint backward) and a chained, checkpointed sequence of
solves, checked against the oracle's dense-solve gradient."""
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


def _oracle_parts(p, theta):
    kinv = synth.iso_kinv(np.exp(-theta))
    A = oracle.assemble(p.mesh.xy, p.mesh.tri, p.mesh.dirichlet, p.eps, kinv, oracle.PER_CELL,
                        oracle.CP2, p.nu, p.dt)
    T, sigma, isd, nbr = oracle.side_coefficients(p.mesh.xy, p.mesh.tri, p.mesh.dirichlet,
                                                  p.eps, kinv, oracle.PER_CELL, oracle.CP2,
                                                  p.nu, p.dt)
    return A.dense(), nbr, isd


def test_log_permeability_assembly_matches_oracle(ctx):
    p, theta = synth.log_permeability_problem(20, seed=5)
    m = p.mesh
    s = ctx.assemble(m.xy, m.tri, m.dirichlet, p.eps, theta, cps.PER_CELL_LOGK, cps.KIND_CP2,
                     p.nu, p.dt)
    D, _, _ = _oracle_parts(p, theta)
    diag, col, val = s.export_matrix()
    diag = diag.cpu().numpy()
    np.testing.assert_allclose(diag, np.diag(D), rtol=1e-13)
    col = col.cpu().numpy()
    val = val.cpu().numpy()
    for j in range(3):
        e = np.nonzero(col[j] != np.arange(m.nt))[0]
        np.testing.assert_allclose(val[j, e], D[e, col[j, e]], rtol=1e-13)
    s.free()


def test_corrector_solve_gradient_matches_oracle(ctx):
    p, theta_np = synth.log_permeability_problem(16, seed=1)
    m = p.mesh
    model = cps.LogPermeabilityCorrector(ctx, m.xy, m.tri, m.dirichlet, p.eps, p.nu, p.dt,
                                         rtol=1e-12)
    theta = torch.tensor(theta_np, device="cuda", requires_grad=True)
    b = torch.tensor(synth.rhs(m, 3), device="cuda", requires_grad=True)
    target = torch.tensor(synth.rhs(m, 4), device="cuda") * 1e3
    x = model.solve(theta, b)
    loss = ((x - target) ** 2).sum()
    loss.backward()
    D, nbr, isd = _oracle_parts(p, theta_np)
    xo = oracle.dense_cholesky_solve(D, b.detach().cpu().numpy())
    assert np.linalg.norm(x.detach().cpu().numpy() - xo) / np.linalg.norm(xo) < 1e-10
    lam = oracle.dense_cholesky_solve(D, 2 * (xo - target.cpu().numpy()))
    dT = oracle.side_gradient(nbr, isd, lam, xo)
    dth = oracle.theta_gradient(m.xy, m.tri, nbr, isd, p.eps, theta_np, p.nu, p.dt, dT)
    np.testing.assert_allclose(theta.grad.cpu().numpy(), dth, rtol=1e-7,
                               atol=1e-9 * np.abs(dth).max())
    np.testing.assert_allclose(b.grad.cpu().numpy(), lam, rtol=1e-7, atol=1e-9 * np.abs(lam).max())
    model.free()


def test_chained_checkpointed_gradient_matches_oracle(ctx):
    """b_t = rhs_t + 0.1 x_{t-1}, loss = sum_t |x_t - x*_t|^2, checkpoint
    every 2 of 5 steps: equal to the un-checkpointed gradient (deterministic
    kernels) and to the oracle's dense chained adjoint."""
    p, theta_np = synth.log_permeability_problem(16, seed=2)
    m = p.mesh
    steps = 5
    area = synth.triangle_areas(m)
    rhs = [torch.tensor(area * synth.normal_noise(m.nt, 100 + t), device="cuda")
           for t in range(steps)]
    targets = [0.3 * r * 1e3 for r in rhs]
    model = cps.LogPermeabilityCorrector(ctx, m.xy, m.tri, m.dirichlet, p.eps, p.nu, p.dt,
                                         rtol=1e-12)
    grads = []
    for every in (2, 0):
        theta = torch.tensor(theta_np, device="cuda", requires_grad=True)
        xs = cps.chained_solve(model, theta, rhs, coupling=0.1, checkpoint_every=every)
        loss = sum(((x - t) ** 2).sum() for x, t in zip(xs, targets))
        loss.backward()
        grads.append(theta.grad.cpu().numpy())
    np.testing.assert_array_equal(grads[0], grads[1])
    D, nbr, isd = _oracle_parts(p, theta_np)
    xo, xp = [], np.zeros(m.nt)
    for t in range(steps):
        xp = oracle.dense_cholesky_solve(D, rhs[t].cpu().numpy() + 0.1 * xp)
        xo.append(xp)
    dT = np.zeros((m.nt, 3))
    lam_next = np.zeros(m.nt)
    for t in reversed(range(steps)):
        lam = oracle.dense_cholesky_solve(D, 2 * (xo[t] - targets[t].cpu().numpy())
                                          + 0.1 * lam_next)
        dT += oracle.side_gradient(nbr, isd, lam, xo[t])
        lam_next = lam
    dth = oracle.theta_gradient(m.xy, m.tri, nbr, isd, p.eps, theta_np, p.nu, p.dt, dT)
    np.testing.assert_allclose(grads[0], dth, rtol=1e-7, atol=1e-9 * np.abs(dth).max())
    model.free()
