"""Pins for the oracle's adjoint: gradients of a loss through one and through
chained corrector solves, against central finite differences of the oracle's
own dense solves.  The step is h = 1e-4 in theta: the losses here are of order
1e10, so with h = 1e-6 the FP64 rounding of the two losses (about 1e-6
absolute) already shows at the 1e-5 level, while the O(h^2) truncation at
1e-4 stays below 1e-8 relative."""
import numpy as np
import pytest

import oracle
import synth


def _setup(n=8, seed=0):
    p, theta = synth.log_permeability_problem(n, seed=seed)
    return p, theta


def _solve_dense(p, theta, b):
    kinv = synth.iso_kinv(np.exp(-theta))
    A = oracle.assemble(p.mesh.xy, p.mesh.tri, p.mesh.dirichlet, p.eps, kinv, oracle.PER_CELL,
                        oracle.CP2, p.nu, p.dt)
    return oracle.dense_cholesky_solve(A.dense(), b), A


def _grad_one_solve(p, theta, b, target):
    x, A = _solve_dense(p, theta, b)
    g = 2 * (x - target)
    lam = oracle.dense_cholesky_solve(A.dense(), g)
    kinv = synth.iso_kinv(np.exp(-theta))
    T, sigma, isd, nbr = oracle.side_coefficients(p.mesh.xy, p.mesh.tri, p.mesh.dirichlet,
                                                  p.eps, kinv, oracle.PER_CELL, oracle.CP2,
                                                  p.nu, p.dt)
    dT = oracle.side_gradient(nbr, isd, lam, x)
    dth = oracle.theta_gradient(p.mesh.xy, p.mesh.tri, nbr, isd, p.eps, theta, p.nu, p.dt, dT)
    return x, lam, dth


def test_single_solve_theta_gradient_matches_central_differences():
    p, theta = _setup(8, 1)
    b = synth.rhs(p.mesh, 3)
    target = 0.5 * _solve_dense(p, theta + 0.3, b)[0]
    loss = lambda th: float(np.sum((_solve_dense(p, th, b)[0] - target) ** 2))
    _, _, dth = _grad_one_solve(p, theta, b, target)
    h = 1e-4
    rng = np.random.default_rng(0)
    for c in rng.choice(p.mesh.nt, 12, replace=False):
        e = np.zeros_like(theta)
        e[c] = h
        fd = (loss(theta + e) - loss(theta - e)) / (2 * h)
        assert dth[c] == pytest.approx(fd, rel=1e-6, abs=1e-9 * abs(dth).max())


def test_rhs_gradient_is_the_adjoint_state():
    p, theta = _setup(6, 2)
    b = synth.rhs(p.mesh, 4)
    target = np.zeros(p.mesh.nt)
    x, lam, _ = _grad_one_solve(p, theta, b, target)
    h = 1e-6
    loss = lambda bb: float(np.sum((_solve_dense(p, theta, bb)[0] - target) ** 2))
    for c in (0, 5, p.mesh.nt - 1):
        e = np.zeros_like(b)
        e[c] = h
        fd = (loss(b + e) - loss(b - e)) / (2 * h)
        assert lam[c] == pytest.approx(fd, rel=1e-6, abs=1e-12)


def test_chained_solves_gradient_matches_central_differences():
    """x_t = A^-1 (b_t + 0.1 x_{t-1}), L = sum_t |x_t - x*_t|^2.  Backward:
    lambda_t = A^-1 (2 (x_t - x*_t) + 0.1 lambda_{t+1}),
    dL/dtheta = sum_t chain(-(lambda_t,e - lambda_t,ep)(x_t,e - x_t,ep))."""
    p, theta = _setup(6, 3)
    steps = 5
    nt = p.mesh.nt
    area = synth.triangle_areas(p.mesh)
    noise = [area * synth.normal_noise(nt, 100 + t) for t in range(steps)]
    targets = [0.3 * noise[t] / area.mean() * 1e-3 for t in range(steps)]

    def forward(th):
        xs, xp = [], np.zeros(nt)
        for t in range(steps):
            xp, _ = _solve_dense(p, th, noise[t] + 0.1 * xp)
            xs.append(xp)
        return xs

    def loss(th):
        return float(sum(np.sum((x - y) ** 2) for x, y in zip(forward(th), targets)))

    xs = forward(theta)
    _, A = _solve_dense(p, theta, noise[0])
    kinv = synth.iso_kinv(np.exp(-theta))
    T, sigma, isd, nbr = oracle.side_coefficients(p.mesh.xy, p.mesh.tri, p.mesh.dirichlet,
                                                  p.eps, kinv, oracle.PER_CELL, oracle.CP2,
                                                  p.nu, p.dt)
    dT = np.zeros((nt, 3))
    lam_next = np.zeros(nt)
    for t in reversed(range(steps)):
        lam = oracle.dense_cholesky_solve(A.dense(), 2 * (xs[t] - targets[t]) + 0.1 * lam_next)
        dT += oracle.side_gradient(nbr, isd, lam, xs[t])
        lam_next = lam
    dth = oracle.theta_gradient(p.mesh.xy, p.mesh.tri, nbr, isd, p.eps, theta, p.nu, p.dt, dT)
    h = 1e-4
    for c in np.random.default_rng(1).choice(nt, 8, replace=False):
        e = np.zeros_like(theta)
        e[c] = h
        fd = (loss(theta + e) - loss(theta - e)) / (2 * h)
        assert dth[c] == pytest.approx(fd, rel=1e-6, abs=1e-9 * abs(dth).max())
