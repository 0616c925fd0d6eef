"""The differentiable robust alignment objective at the config-4 size: 32
pairs of 50,000-point room clouds in one batched forward and one backward
through RobustAlignBatch (a torch.autograd.Function over lsr_objective_fwd /
lsr_objective_bwd), the nearest neighbours recomputed in the backward.

Gradients with respect to the se(3) 6-vector are checked against FP64 central
finite differences (h = 1e-6) and against the oracle's analytic gradient, at
relative tolerance 1e-4. The objective is piecewise smooth: with 50,000 points
some nearest neighbours switch within +-h of any pose, so the finite
differences are taken of the objective with the correspondences of the base
pose held (the function the analytic gradient differentiates), evaluated in
FP64 from the oracle's neighbours and pose update; every component must agree
at relative 1e-4 (plus 1e-6 of the largest component, for components near
zero, plus the terms of the few points whose pair an FP32 search may form
differently: each such pair moves the sum by its own term). Point gradients are checked against the oracle's and against FP64
central differences of the held objective in the point coordinates (a seeded
1% of them), excluding only the points whose nearest neighbour an FP32 search
may pick differently: a runner-up within 1e-6 m of the nearest, or a distance
within 1e-6 m of eps (and, for Q, the rows those points touch).
"""
import numpy as np
import pytest

import oracle
from synth import make_pair

gpu = pytest.mark.gpu
EPS = 0.0375
MU = EPS * EPS


@pytest.fixture(scope="module")
def run4():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1801_01572_gb300 as lsr
    pairs = [make_pair(4, i) for i in range(32)]
    rng = np.random.default_rng(44)
    xis = np.concatenate([rng.normal(0, 2e-3, (32, 3)), rng.normal(0, 3e-3, (32, 3))], axis=1)
    T0s = np.stack([p.T for p in pairs])
    clouds = []
    for p in pairs:
        clouds.append(torch.tensor(p.P, device="cuda", requires_grad=True))
        clouds.append(torch.tensor(p.Q, device="cuda", requires_grad=True))
    xt = torch.tensor(xis, dtype=torch.float64, requires_grad=True)
    with lsr.Context(0) as ctx:
        E = lsr.RobustAlignBatch.apply(xt, torch.tensor(T0s), EPS, MU, ctx, *clouds)
        E.sum().backward()
        torch.cuda.synchronize()
    return dict(pairs=pairs, xis=xis, T0s=T0s, E=E.detach().cpu().numpy(), dxi=xt.grad.numpy(),
                dP=[c.grad.cpu().numpy() for c in clouds[0::2]], dQ=[c.grad.cpu().numpy() for c in clouds[1::2]])


def held_objective(P, Q, nn, xi, T0):
    """E with the correspondences nn held: sum rho~(|T(xi) p_i - q_nn(i)|^2)."""
    T = oracle.apply_xi(xi, T0)
    m = nn >= 0
    r = P[m] @ T[:3, :3].T + T[:3, 3] - Q[nn[m]]
    s = (r * r).sum(1)
    return float((MU * s / (MU + s) - MU * EPS ** 2 / (MU + EPS ** 2)).sum())


@gpu
@pytest.mark.parametrize("i", [0, 11, 31])
def test_config4_objective_and_pose_gradient(run4, i):
    p, xi, T0 = run4["pairs"][i], run4["xis"][i], run4["T0s"][i]
    P, Q = p.P.astype(np.float64), p.Q.astype(np.float64)
    E_ref, dP_ref, dQ_ref, dxi_ref, nn = oracle.objective(P, Q, xi, T0, EPS, MU)
    assert (nn >= 0).sum() > 0.3 * len(P)
    assert abs(run4["E"][i] - E_ref) <= 1e-5 * abs(E_ref)
    g = run4["dxi"][i]
    scale = np.abs(dxi_ref).max()
    # the pairs an FP32 search may form differently each move dxi by their own
    # term (or their term with the runner-up neighbour): that is added to the bound
    slack = ambiguous_dxi(P, Q, xi, T0)
    assert np.all(np.abs(g - dxi_ref) <= 1e-4 * np.abs(dxi_ref) + 1e-6 * scale + slack), (g, dxi_ref, slack)
    h = 1e-6
    for k in range(6):
        e = np.zeros(6)
        e[k] = h
        fd = (held_objective(P, Q, nn, xi + e, T0) - held_objective(P, Q, nn, xi - e, T0)) / (2 * h)
        assert abs(g[k] - fd) <= 1e-4 * abs(fd) + 1e-6 * scale + slack[k], (k, g[k], fd)
    assert abs(held_objective(P, Q, nn, xi, T0) - E_ref) <= 1e-9 * abs(E_ref)


def ambiguous_dxi(P, Q, xi, T0):
    """Per component, the sum over the FP32-ambiguous points of the absolute
    dxi terms they contribute with their nearest and with their runner-up
    neighbour (oracle, FP64)."""
    spatial = pytest.importorskip("scipy.spatial")
    T = oracle.apply_xi(xi, T0)
    Z = P @ T[:3, :3].T + T[:3, 3]
    d, j = spatial.cKDTree(Q).query(Z, k=2)
    amb = np.nonzero((np.abs(d[:, 0] - EPS) < 1e-6) | ((d[:, 0] < EPS + 1e-6) & (d[:, 1] - d[:, 0] < 1e-6)))[0]
    slack = np.zeros(6)
    for a in amb:
        for q in j[a]:
            _, _, _, dx, _ = oracle.objective(P[a:a + 1], Q[q:q + 1], xi, T0, EPS, MU)
            slack += np.abs(dx)
    return slack


def ambiguous_points(P, Q, xi, T0):
    """Points of P whose FP32 nearest neighbour within eps may differ from the
    FP64 one (runner-up within 1e-6 m of the nearest, or the nearest within
    1e-6 m of eps), and the Q rows either candidate of such a point touches."""
    spatial = pytest.importorskip("scipy.spatial")
    T = oracle.apply_xi(xi, T0)
    Z = P @ T[:3, :3].T + T[:3, 3]
    d, j = spatial.cKDTree(Q).query(Z, k=2)
    amb = (np.abs(d[:, 0] - EPS) < 1e-6) | ((d[:, 0] < EPS + 1e-6) & (d[:, 1] - d[:, 0] < 1e-6))
    rows = np.zeros(len(Q), bool)
    rows[j[amb].reshape(-1)] = True
    return amb, rows


def term_objective(p, q, T):
    """One pair's term of the objective in FP64."""
    r = T[:3, :3] @ p + T[:3, 3] - q
    s = float(r @ r)
    return MU * s / (MU + s) - MU * EPS ** 2 / (MU + EPS ** 2)


@gpu
@pytest.mark.parametrize("i", [0, 11, 31])
def test_config4_point_gradients(run4, i):
    p, xi, T0 = run4["pairs"][i], run4["xis"][i], run4["T0s"][i]
    P, Q = p.P.astype(np.float64), p.Q.astype(np.float64)
    _, dP_ref, dQ_ref, _, nn = oracle.objective(P, Q, xi, T0, EPS, MU)
    ambP, ambQ = ambiguous_points(P, Q, xi, T0)
    assert ambP.mean() < 1e-3
    for got, ref, skip in ((run4["dP"][i], dP_ref, ambP), (run4["dQ"][i], dQ_ref, ambQ)):
        big = np.abs(ref).max()
        err = np.abs(got - ref).max(1)
        ok = err <= 1e-4 * np.abs(ref).max(1) + 1e-6 * big
        assert np.all(ok | skip), (np.nonzero(~(ok | skip))[0][:10], (~ok & ~skip).sum())
    # points with no neighbour within eps have no gradient on either side
    far = nn < 0
    assert np.all(run4["dP"][i][far] == 0)
    # FP64 central differences of the held objective in a seeded 1% of the coordinates
    T = oracle.apply_xi(xi, T0)
    rng = np.random.default_rng(100 + i)
    h = 1e-6
    held = np.nonzero((nn >= 0) & ~ambP)[0]
    for a in rng.choice(held, min(len(held), 3 * len(P) // 100), replace=False):
        c = int(rng.integers(3))
        e = np.zeros(3)
        e[c] = h
        fd = (term_objective(P[a] + e, Q[nn[a]], T) - term_objective(P[a] - e, Q[nn[a]], T)) / (2 * h)
        assert abs(run4["dP"][i][a, c] - fd) <= 1e-4 * abs(fd) + 1e-6 * np.abs(dP_ref).max(), (a, c)
    rowsQ = np.unique(nn[held])
    rowsQ = rowsQ[~ambQ[rowsQ]]
    for b in rng.choice(rowsQ, min(len(rowsQ), 3 * len(Q) // 100), replace=False):
        c = int(rng.integers(3))
        e = np.zeros(3)
        e[c] = h
        users = np.nonzero(nn == b)[0]
        fd = sum((term_objective(P[a], Q[b] + e, T) - term_objective(P[a], Q[b] - e, T)) / (2 * h) for a in users)
        assert abs(run4["dQ"][i][b, c] - fd) <= 1e-4 * abs(fd) + 1e-6 * np.abs(dQ_ref).max(), (b, c)
