"""Gradient of the refined pose with respect to the points (implicit
differentiation of the robust alignment of eq. (3)-(4) at its optimum, with the
pose perturbation of eq. (5)), through lsr_pose_implicit_grad and the
RefinedPose autograd Function, against the FP64 oracle.

The oracle side holds the same pairs: the nearest Q point of T p within eps,
found in FP64 by a k-d tree over the same float32 coordinates. Points whose
pair an FP32 search may decide differently (distance within 1e-6 m of eps, or
a runner-up within 1e-6 m of the nearest) are counted; where there are none,
the GPU's gradient, Hessian, lambda and point gradients must equal the
oracle's up to FP64 summation order and the FP32 rounding of the outputs.
Then the gradient is checked against central differences of re-optimised
poses (oracle.pose_optimum on the held pairs) for a few coordinates.

The library takes mu as a float32, so the oracle is given that same value.
"""
import numpy as np
import pytest

import oracle
from synth import make_pair

gpu = pytest.mark.gpu
EPS = 0.0375


@pytest.fixture(scope="module")
def lsr():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1801_01572_gb300 as m
    return m


def held_pairs(P, Q, T, eps):
    """FP64 nearest Q point of every moved P point within eps; the count of
    points whose pair an FP32 search may decide the other way."""
    spatial = pytest.importorskip("scipy.spatial")
    P64, Q64 = P.astype(np.float64), Q.astype(np.float64)
    Z = P64 @ T[:3, :3].T + T[:3, 3]
    d, j = spatial.cKDTree(Q64).query(Z, k=2)
    held = d[:, 0] < eps
    amb = (np.abs(d[:, 0] - eps) < 1e-6) | (held & (d[:, 1] - d[:, 0] < 1e-6))
    return held, j[:, 0], int(amb.sum())


def dl_dxi(G, T):
    """dL/dxi of the left perturbation for a loss with gradient G = dL/dT."""
    M = G[:3, :3] @ T[:3, :3].T + np.outer(G[:3, 3], T[:3, 3])
    return np.r_[M[2, 1] - M[1, 2], M[0, 2] - M[2, 0], M[1, 0] - M[0, 1], G[:3, 3]]


@pytest.mark.parametrize("case", ["objects5k", "room50k"])
@gpu
def test_implicit_gradient_matches_oracle(lsr, case):
    """At the oracle's refined pose (given to both sides), where no held pair
    lies in the FP32 band on these seeded pairs."""
    fp = make_pair(0, 0) if case == "objects5k" else make_pair(4, 3)
    T, _ = oracle.refine_gnc(fp.P, fp.Q, fp.T, EPS, 1.0, levels=3, iters=50)
    with lsr.Context(0) as ctx:
        rng = np.random.default_rng(7)
        G = np.zeros((4, 4))
        G[:3, :] = rng.normal(size=(3, 4))
        dP, dQ, g, H, lam, n = ctx.pose_implicit_grad(fp.P, fp.Q, T, G, EPS, EPS * EPS)
    held, nn, namb = held_pairs(fp.P, fp.Q, T, EPS)
    assert namb == 0 and n == held.sum()
    X, Y = fp.P[held].astype(np.float64), fp.Q[nn[held]].astype(np.float64)
    mu = float(np.float32(EPS * EPS))
    _, g_ref, H_ref = oracle.pose_grad_hess(X, Y, T, mu)
    hs = np.abs(H_ref).max()
    assert np.abs(H - H_ref).max() <= 1e-9 * hs
    assert np.abs(g - g_ref).max() <= 1e-9 * hs * 1e-2 + 1e-9 * np.abs(g_ref).max()
    lam_ref = np.linalg.solve(H_ref, dl_dxi(G, T))
    assert np.allclose(lam, lam_ref, rtol=1e-7, atol=1e-9 * np.abs(lam_ref).max())
    dX, dY = oracle.pose_implicit_grad(X, Y, T, mu, dl_dxi(G, T))
    refP = np.zeros_like(dP, dtype=np.float64)
    refP[held] = dX
    refQ = np.zeros_like(dQ, dtype=np.float64)
    np.add.at(refQ, nn[held], dY)
    sp, sq = np.abs(refP).max(), np.abs(refQ).max()
    assert np.abs(dP - refP).max() <= 2e-6 * sp
    assert np.abs(dQ - refQ).max() <= 2e-6 * sq
    assert np.all(dP[~held] == 0)


@gpu
def test_implicit_gradient_against_reoptimised_poses(lsr):
    """Central differences of L(T*(points)) with T* re-optimised on the held
    pairs by the oracle's Newton iteration (h = 2e-4 m on float32 points)."""
    fp = make_pair(0, 0)
    with lsr.Context(0) as ctx:
        T, _ = ctx.stage_refine(fp.P, fp.Q, fp.T, EPS, 1.0, 3, 50)
        held, nn, namb = held_pairs(fp.P, fp.Q, T, EPS)
        if namb:
            pytest.skip("pairs within the FP32 band")
        mu = float(np.float32(EPS * EPS))
        X, Y = fp.P[held].astype(np.float64), fp.Q[nn[held]].astype(np.float64)
        T0, _ = oracle.pose_optimum(X, Y, T, mu)
        rng = np.random.default_rng(11)
        G = np.zeros((4, 4))
        G[:3, :] = rng.normal(size=(3, 4))
        dP, dQ, _, _, _, _ = ctx.pose_implicit_grad(fp.P, fp.Q, T0, G, EPS, mu)
    L = lambda Tx: float((G * Tx).sum())  # noqa: E731
    idx_held = np.nonzero(held)[0]
    h = 2e-4
    for i in rng.choice(idx_held, 4, replace=False):
        k = int(np.nonzero(idx_held == i)[0][0])
        for c in range(3):
            Xp, Xm = X.copy(), X.copy()
            Xp[k, c] += h
            Xm[k, c] -= h
            Tp, _ = oracle.pose_optimum(Xp, Y, T0, mu)
            Tm, _ = oracle.pose_optimum(Xm, Y, T0, mu)
            fd = (L(Tp) - L(Tm)) / (2 * h)
            assert abs(dP[i, c] - fd) <= 2e-3 * np.abs(dP).max() + 1e-3 * abs(fd), (i, c, dP[i, c], fd)
    for j in rng.choice(np.unique(nn[held]), 3, replace=False):
        rows = np.nonzero(nn[held] == j)[0]
        for c in range(3):
            Yp, Ym = Y.copy(), Y.copy()
            Yp[rows, c] += h
            Ym[rows, c] -= h
            Tp, _ = oracle.pose_optimum(X, Yp, T0, mu)
            Tm, _ = oracle.pose_optimum(X, Ym, T0, mu)
            fd = (L(Tp) - L(Tm)) / (2 * h)
            assert abs(dQ[j, c] - fd) <= 2e-3 * np.abs(dQ).max() + 1e-3 * abs(fd), (j, c, dQ[j, c], fd)


@gpu
def test_refined_pose_autograd_function(lsr):
    import torch
    fp = make_pair(0, 1)
    P = torch.from_numpy(fp.P).cuda().requires_grad_()
    Q = torch.from_numpy(fp.Q).cuda().requires_grad_()
    T0 = torch.tensor(fp.T, dtype=torch.float64)
    with lsr.Context(0) as ctx:
        T = lsr.RefinedPose.apply(P, Q, T0, EPS, 1.0, 3, 50, ctx)
        T_ref, _ = ctx.stage_refine(fp.P, fp.Q, fp.T, EPS, 1.0, 3, 50)
        assert np.array_equal(T.detach().cpu().numpy(), T_ref)
        W = torch.randn(4, 4, dtype=torch.float64, generator=torch.Generator().manual_seed(3))
        (W * T.cpu()).sum().backward()
        dP, dQ, _, _, _, n = ctx.pose_implicit_grad(fp.P, fp.Q, T_ref, W.numpy(), EPS, EPS * EPS)
    assert n > 1000
    assert np.allclose(P.grad.cpu().numpy(), dP, rtol=1e-5, atol=1e-6 * np.abs(dP).max())
    assert np.allclose(Q.grad.cpu().numpy(), dQ, rtol=1e-5, atol=1e-6 * np.abs(dQ).max())


@gpu
def test_implicit_gradient_degenerate_inputs(lsr):
    fp = make_pair(0, 0, n_p=500, n_q=500)
    far = np.eye(4)
    far[:3, 3] = 100.0  # no pair within eps: H = 0 is singular
    with lsr.Context(0) as ctx:
        with pytest.raises(lsr.LsrError) as e:
            ctx.pose_implicit_grad(fp.P, fp.Q, far, np.eye(4), EPS)
        assert e.value.code == lsr.LSR_E_ARG
        bad = np.eye(4)
        bad[0, 0] = np.nan
        with pytest.raises(lsr.LsrError) as e:
            ctx.pose_implicit_grad(fp.P, fp.Q, bad, np.eye(4), EPS)
        assert e.value.code == lsr.LSR_E_ARG
        # host outputs and device outputs agree
        import torch
        T, _ = ctx.stage_refine(fp.P, fp.Q, fp.T, EPS, 1.0, 3, 50)
        a = ctx.pose_implicit_grad(fp.P, fp.Q, T, np.eye(4), EPS)
        dP = torch.empty((500, 3), dtype=torch.float32, device="cuda")
        dQ = torch.empty((500, 3), dtype=torch.float32, device="cuda")
        ctx.pose_implicit_grad(torch.from_numpy(fp.P).cuda(), torch.from_numpy(fp.Q).cuda(), T, np.eye(4), EPS,
                               None, dP, dQ)
        assert np.array_equal(a[0], dP.cpu().numpy())
        assert np.allclose(a[1], dQ.cpu().numpy(), rtol=1e-6, atol=1e-7 * np.abs(a[1]).max())
