"""Pins of the oracle's implicit gradient of the refined pose (NEXT-4): the
pose that minimises the robust objective of eq. (3)-(4) over held pairs
(x_i, y_i), and the gradient of a loss of that pose with respect to the points
through the implicit function theorem at the optimum.

Pinned by: the gradient and the exact Hessian against central differences of
E(Exp(xi) T) (the Exp of the C oracle, Rodrigues); the optimum of a very large
mu (plain least squares) against Kabsch; the implicit gradient against central
differences of re-optimised poses, for the robust kernel and, at large mu,
through Kabsch's closed form; and translation equivariance (moving every x, or
every y, by the same vector moves the pose by a known amount, so the summed
gradients are fixed).
"""
import numpy as np
import pytest
from scipy.spatial.transform import Rotation

import oracle


def _problem(n=300, seed=0, outliers=30):
    rng = np.random.default_rng(seed)
    X = rng.uniform(-1, 1, (n, 3))
    R = Rotation.from_rotvec([0.1, -0.2, 0.3]).as_matrix()
    t = np.array([0.2, 0.1, -0.3])
    Y = X @ R.T + t + rng.normal(0, 0.02, (n, 3))
    Y[:outliers] += rng.normal(0, 0.3, (outliers, 3))
    T = np.eye(4)
    T[:3, :3], T[:3, 3] = R, t
    return X, Y, T


def _xi(Tn, T):
    D = Tn @ np.linalg.inv(T)
    return np.concatenate([Rotation.from_matrix(D[:3, :3]).as_rotvec(), D[:3, 3]])


def _E(X, Y, T, mu):
    r = X @ T[:3, :3].T + T[:3, 3] - Y
    s = (r * r).sum(1)
    return float((mu * s / (mu + s)).sum())


def test_gradient_and_hessian_against_differences():
    X, Y, T = _problem(80, seed=1)
    mu = 0.05 ** 2
    T = oracle.apply_xi(np.array([0.01, -0.02, 0.015, 0.01, 0.02, -0.01]), T)  # away from the optimum
    E, g, H = oracle.pose_grad_hess(X, Y, T, mu)
    assert abs(E - _E(X, Y, T, mu)) <= 1e-12 * E
    h = 1e-5
    f = lambda xi: _E(X, Y, oracle.apply_xi(xi, T), mu)
    for a in range(6):
        ea = np.zeros(6)
        ea[a] = h
        assert abs((f(ea) - f(-ea)) / (2 * h) - g[a]) <= 1e-6 * np.abs(g).max()
        for b in range(6):
            eb = np.zeros(6)
            eb[b] = h
            fd = (f(ea + eb) - f(ea - eb) - f(-ea + eb) + f(-ea - eb)) / (4 * h * h)
            assert abs(fd - H[a, b]) <= 1e-4 * np.abs(H).max(), (a, b, fd, H[a, b])
    assert np.allclose(H, H.T, rtol=0, atol=1e-12 * np.abs(H).max())


def test_least_squares_optimum_is_kabsch():
    X, Y, T0 = _problem(200, seed=2, outliers=0)
    T, gn = oracle.pose_optimum(X, Y, T0, mu=1e12)
    R, t = oracle.kabsch(X, Y)
    assert gn < 1e-6
    assert np.abs(T[:3, :3] - R).max() < 1e-9 and np.abs(T[:3, 3] - t).max() < 1e-9


@pytest.mark.parametrize("mu, outliers", [(0.05 ** 2, 30), (1e12, 0)])
def test_implicit_gradient_against_reoptimised_poses(mu, outliers):
    X, Y, T0 = _problem(300, seed=0, outliers=outliers)
    T, gn = oracle.pose_optimum(X, Y, T0, mu)
    assert gn < 1e-9 * max(1.0, np.abs(oracle.pose_grad_hess(X, Y, T, mu)[2]).max())
    grads = [oracle.pose_implicit_grad(X, Y, T, mu, np.eye(6)[j]) for j in range(6)]
    h = 1e-6
    for k, c in ((5, 0), (40, 2), (100, 1)):
        for which in (0, 1):
            A, B = [X.copy(), Y.copy()], [X.copy(), Y.copy()]
            A[which][k, c] += h
            B[which][k, c] -= h
            if mu > 1e6:  # plain least squares: through Kabsch's closed form
                def opt(P, Q):
                    R, t = oracle.kabsch(P, Q)
                    M = np.eye(4)
                    M[:3, :3], M[:3, 3] = R, t
                    return M
                Ta, Tb = opt(*A), opt(*B)
            else:
                Ta, Tb = oracle.pose_optimum(A[0], A[1], T, mu)[0], oracle.pose_optimum(B[0], B[1], T, mu)[0]
            fd = (_xi(Ta, T) - _xi(Tb, T)) / (2 * h)
            an = np.array([grads[j][which][k, c] for j in range(6)])
            assert np.abs(fd - an).max() <= 1e-6 * max(np.abs(fd).max(), 1e-3), (k, c, which, fd, an)


def test_implicit_gradient_translation_equivariance():
    X, Y, T0 = _problem(200, seed=3)
    mu = 0.05 ** 2
    T, _ = oracle.pose_optimum(X, Y, T0, mu)
    rng = np.random.default_rng(4)
    dL = rng.normal(size=6)
    dX, dY = oracle.pose_implicit_grad(X, Y, T, mu, dL)
    # every x moved by d: the pose becomes [R | t - R d]; every y by d: [R | t + d]
    assert np.allclose(dX.sum(0), -T[:3, :3].T @ dL[3:], rtol=0, atol=1e-9 * np.abs(dL).max())
    assert np.allclose(dY.sum(0), dL[3:], rtol=0, atol=1e-9 * np.abs(dL).max())
