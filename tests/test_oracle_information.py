"""Pins of the oracle's information matrix (loop verification, eq. (5)-(6)):
Lambda = sum over the correspondences K of G_p^T G_p, G_p = [-[p]_x | I].

Each check comes from the mathematics rather than from the oracle's own
formula: the quadratic form xi^T Lambda xi equals sum |w x p + v|^2 over K
(G_p xi written with cross products), it is the first-order expansion of the
alignment error sum |T(xi) p - p|^2 of eq. (4) for a small motion xi (the
approximation eq. (6) makes), its trace is sum (2 |p|^2 + 3), its translation
block is |K| I, its rotation-translation blocks vanish for a point set
symmetric about the origin, and |K| is the consensus inlier count of the same
pose (a separate oracle routine), with the grid search equal to brute force.
"""
import numpy as np
import pytest

import oracle
from synth import make_pair

EPS = 0.05


@pytest.fixture(scope="module")
def pair0():
    return make_pair(0, 0)


def _moved_inliers(P, Q, T, eps, brute=False):
    X = P @ T[:3, :3].T + T[:3, 3]
    nn, _ = oracle.nn_within(Q, X, eps, brute=brute)
    return X[nn >= 0]


def test_information_quadratic_form_is_sum_of_cross_products(pair0):
    info, n, _, _ = oracle.information(pair0.P, pair0.Q, pair0.T, EPS)
    X = _moved_inliers(pair0.P, pair0.Q, pair0.T, EPS)
    assert n == len(X) > 1000
    rng = np.random.default_rng(3)
    for _ in range(5):
        xi = rng.normal(size=6)
        w, v = xi[:3], xi[3:]
        direct = float((np.linalg.norm(np.cross(w, X) + v, axis=1) ** 2).sum())
        assert abs(xi @ info @ xi - direct) <= 1e-10 * direct


def test_information_approximates_the_alignment_error(pair0):
    """For a small motion xi, sum |T(xi) p - p|^2 over K -> xi^T Lambda xi."""
    info, _, _, _ = oracle.information(pair0.P, pair0.Q, pair0.T, EPS)
    X = _moved_inliers(pair0.P, pair0.Q, pair0.T, EPS)
    rng = np.random.default_rng(4)
    for scale in (1e-4, 1e-5):
        xi = rng.normal(size=6) * scale
        Txi = oracle.apply_xi(xi, np.eye(4))
        f = float((np.linalg.norm(X @ Txi[:3, :3].T + Txi[:3, 3] - X, axis=1) ** 2).sum())
        q = float(xi @ info @ xi)
        assert abs(f / q - 1.0) < 50 * scale, (scale, f, q)


def test_information_invariants(pair0):
    info, n, _, _ = oracle.information(pair0.P, pair0.Q, pair0.T, EPS)
    X = _moved_inliers(pair0.P, pair0.Q, pair0.T, EPS)
    assert np.allclose(info, info.T, rtol=0, atol=1e-9)
    assert np.allclose(info[3:, 3:], n * np.eye(3))
    assert abs(np.trace(info) - float((2 * (X * X).sum(1) + 3).sum())) <= 1e-9 * np.trace(info)
    assert np.linalg.eigvalsh(info).min() > 0  # a 3D scene constrains all six directions
    # the consensus routine counts the same correspondences
    cnt, _, _ = oracle.consensus(pair0.P, pair0.Q, pair0.T[None, :3, :3], pair0.T[None, :3, 3], EPS)
    assert cnt[0] == n
    # a search band past eps changes what is reported as ambiguous, not K
    info_b, n_b, namb, _ = oracle.information(pair0.P, pair0.Q, pair0.T, EPS, band=2e-3)
    assert n_b == n and namb > 0 and np.array_equal(info_b, info)


def test_information_symmetric_set_has_no_coupling():
    rng = np.random.default_rng(5)
    H = rng.uniform(-1, 1, (200, 3))
    P = np.concatenate([H, -H])
    info, n, _, _ = oracle.information(P, P, np.eye(4), EPS)
    assert n == 400
    assert np.abs(info[:3, 3:]).max() < 1e-12 and np.abs(info[3:, :3]).max() < 1e-12
    assert np.allclose(info[:3, :3], (P * P).sum() * np.eye(3) - P.T @ P)


def test_information_grid_equals_brute_force():
    p = make_pair(0, 1, n_p=600, n_q=600)
    info, n, _, _ = oracle.information(p.P, p.Q, p.T, EPS)
    X = _moved_inliers(p.P, p.Q, p.T, EPS, brute=True)
    assert n == len(X)
    xi = np.arange(1.0, 7.0)
    direct = float((np.linalg.norm(np.cross(xi[:3], X) + xi[3:], axis=1) ** 2).sum())
    assert abs(xi @ info @ xi - direct) <= 1e-10 * direct
