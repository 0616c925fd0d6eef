"""Pins of the FP64 oracle against things other than itself: brute force on tiny
inputs, closed forms, invariants, special cases that reduce to a library
routine, and an independent library implementation of the RNG. Each test is
chosen so that a plausible slip in the oracle (a dropped term, a wrong sign or
index, a transposed operand, a flipped comparison) fails it. CPU only."""
import numpy as np
import pytest
from scipy.optimize import minimize_scalar
from scipy.spatial.distance import cdist
from scipy.spatial.transform import Rotation

from synth import make_pair, pose_error, random_pose


# ------------------------------------------------------------------ RNG
def test_philox_matches_numpy_philox(orc):
    """Philox-4x64-10 (Salmon et al., SC'11) against numpy's implementation; numpy
    increments its counter before each block, so counter c there is c+1 here."""
    rng = np.random.default_rng(7)
    for _ in range(50):
        ctr = rng.integers(0, 2**63, 4, dtype=np.uint64)
        ctr[0] = ctr[0] | np.uint64(1)  # avoid the borrow in ctr - 1
        key = rng.integers(0, 2**63, 2, dtype=np.uint64)
        ref = np.random.Philox(counter=[int(ctr[0]) - 1, *[int(c) for c in ctr[1:]]],
                               key=[int(k) for k in key]).random_raw(4)
        assert np.array_equal(orc.philox4x64_10(ctr, key), np.asarray(ref, np.uint64))


def test_sample_indices_definition_and_uniformity(orc):
    """index = floor(x * N / 2^64) of the 4 Philox words of counter (h,0,0,0), key
    (seed, pair); and a chi-square check of uniformity over 1e6 draws."""
    seed, pair, n = 1234, 5, 97
    idx = orc.sample_indices(seed, pair, 0, 250_000, n)
    for h in (0, 1, 77, 249_999):
        words = np.random.Philox(counter=[h - 1 if h else 2**64 - 1, 0 if h else 2**64 - 1,
                                          0 if h else 2**64 - 1, 0 if h else 2**64 - 1],
                                 key=[seed, pair]).random_raw(4)
        expect = [(int(w) * n) >> 64 for w in words]
        assert list(idx[h]) == expect
    counts = np.bincount(idx.ravel(), minlength=n)
    exp = idx.size / n
    chi2 = ((counts - exp) ** 2 / exp).sum()
    assert chi2 < 96 + 5 * np.sqrt(2 * 96)  # dof 96, far tail


# ------------------------------------------------------------------ neighbours
@pytest.mark.parametrize("r", [0.03, 0.1, 0.25])
def test_radius_grid_equals_brute(orc, r):
    rng = np.random.default_rng(1)
    P = rng.uniform(-0.5, 0.5, (1500, 3))
    P[100:120] = P[0]  # duplicates
    X = np.concatenate([P[:300], rng.uniform(-1, 1, (200, 3))])
    assert np.array_equal(orc.radius_count_grid(P, X, r), orc.radius_count_brute(P, X, r))


def test_nn_within_grid_equals_brute(orc):
    rng = np.random.default_rng(2)
    Q = rng.uniform(0, 1, (2000, 3))
    X = rng.uniform(-0.1, 1.1, (1000, 3))
    for r in (0.02, 0.05):
        a, da = orc.nn_within(Q, X, r)
        b, db = orc.nn_within(Q, X, r, brute=True)
        assert np.array_equal(a, b)
        assert np.allclose(da[a >= 0], db[b >= 0], rtol=0, atol=0)
        # definition: nothing closer than the returned one, nothing within r when -1
        D = cdist(X, Q)
        assert np.all(D[a < 0].min(axis=1) >= r)
        assert np.allclose(np.sqrt(da[a >= 0]), D[a >= 0].min(axis=1))


# ------------------------------------------------------------------ eigen / normals
def test_eig3_matches_library(orc):
    rng = np.random.default_rng(3)
    for _ in range(200):
        M = rng.standard_normal((3, 3))
        A = M @ M.T * rng.uniform(1e-6, 10)
        w, V = orc.eig3(A)
        wl = np.linalg.eigvalsh(A)
        assert np.allclose(w, wl, rtol=1e-12, atol=1e-14 * np.abs(wl).max())
        assert np.allclose(V @ np.diag(w) @ V.T, A, atol=1e-12 * np.abs(A).max())
        assert np.allclose(V.T @ V, np.eye(3), atol=1e-12)


def test_normals_plane_exact_and_oriented(orc):
    rng = np.random.default_rng(4)
    R = Rotation.random(random_state=5).as_matrix()
    uv = rng.uniform(-0.3, 0.3, (3000, 2))
    P = np.c_[uv, np.zeros(len(uv))] @ R.T + [0.2, -0.1, 0.4]
    vp = R @ [0, 0, 2.0] + [0.2, -0.1, 0.4]
    N, curv, cnt, _ = orc.normals(P, vp, 0.05)
    n_true = R[:, 2]
    ok = cnt >= 3
    assert ok.mean() > 0.99
    assert np.abs(N[ok] - n_true).max() < 1e-9  # oriented toward vp (+z side of the plane)
    assert np.all(curv[ok] < 1e-12)
    assert np.array_equal(cnt, orc.radius_count_brute(P, P, 0.05))
    # flipping the viewpoint flips the orientation
    N2, _, _, _ = orc.normals(P, 2 * P.mean(0) - vp, 0.05)
    assert np.abs(N2[ok] + n_true).max() < 1e-9


def test_normals_sphere_symmetric_cap_is_radial(orc):
    """A neighbourhood symmetric about the radial axis has the radial axis as its
    smallest principal direction (exactly, by symmetry)."""
    Rs = 0.4
    pts = [[0, 0, Rs]]
    for pol in np.linspace(0.02, 0.12, 6):
        for az in np.arange(12) * (2 * np.pi / 12):
            pts.append([Rs * np.sin(pol) * np.cos(az), Rs * np.sin(pol) * np.sin(az), Rs * np.cos(pol)])
    G = Rotation.random(random_state=6).as_matrix()
    P = np.array(pts) @ G.T + [1.0, 2.0, 3.0]
    N, curv, cnt, _ = orc.normals(P, [1.0, 2.0, 3.0], 0.06, qidx=[0])
    radial = -G[:, 2]  # oriented toward the centre (viewpoint)
    assert cnt[0] == len(P)
    assert np.abs(N[0] - radial).max() < 1e-12
    assert curv[0] > 0


def test_normals_rigid_equivariance_and_invalid(orc):
    fp = make_pair(0)
    P = fp.P.astype(np.float64)[:1500]
    T = random_pose(np.random.default_rng(8))
    vp = np.array([0.3, -2.0, 1.0])
    N1, c1, k1, d1 = orc.normals(P, vp, 0.05)
    PT = P @ T[:3, :3].T + T[:3, 3]
    N2, c2, k2, _ = orc.normals(PT, T[:3, :3] @ vp + T[:3, 3], 0.05)
    assert np.array_equal(k1, k2)
    good = (k1 >= 3) & (d1[:, 0] > 1e-6) & (d1[:, 1] > 1e-6)
    assert np.abs(N1[good] @ T[:3, :3].T - N2[good]).max() < 1e-9
    bad = k1 < 3
    assert np.all(N1[bad] == 0) and np.all(c1[bad] == -1)


def test_normal_neighbourhood_median_size_config0(orc):
    fp = make_pair(0)
    _, _, k, _ = orc.normals(fp.P, fp.vpP, 0.05)
    assert np.median(k) >= 8


# ------------------------------------------------------------------ pair features / FPFH
def test_pair_features_closed_form(orc):
    """Source normal tilted by b toward the joining line, target normal tilted by g
    about it: (alpha, phi, theta) = (sin g, sin b, b)."""
    for b, g in [(0.3, 0.0), (0.3, 0.4), (-0.7, 0.2), (1.1, -0.5)]:
        ns = [np.sin(b), 0, np.cos(b)]
        nt = [0, np.sin(g), np.cos(g)]
        if abs(np.sin(b)) <= abs(0.0):
            continue
        ok, f = orc.pair_features([0, 0, 0], ns, [0.1, 0, 0], nt)
        assert ok
        assert np.allclose(f, [np.sin(g), np.sin(b), b], atol=1e-14)
        # the source rule makes the features independent of argument order
        ok2, f2 = orc.pair_features([0.1, 0, 0], nt, [0, 0, 0], ns)
        assert ok2 and np.allclose(f, f2, atol=1e-14)


def test_pair_features_degenerate_frame_skipped(orc):
    ok, _ = orc.pair_features([0, 0, 0], [1, 0, 0], [0.1, 0, 0], [1, 0, 0])
    assert not ok


def test_spfh_fpfh_plane_one_hot(orc):
    """Noiseless plane: alpha = phi = theta = 0 for every pair, so each
    sub-histogram is one-hot at bin floor(0.5 * 11) = 5."""
    rng = np.random.default_rng(9)
    uv = rng.uniform(-0.5, 0.5, (3000, 2))
    R = Rotation.random(random_state=10).as_matrix()
    P = np.c_[uv, np.zeros(len(uv))] @ R.T
    N = np.tile(R[:, 2], (len(P), 1))
    S, k, _ = orc.spfh(P, N, 0.125)
    F = orc.fpfh(P, N, S, 0.125)
    onehot = np.zeros(33)
    onehot[[5, 16, 27]] = 1
    assert np.all(k > 0)
    assert np.abs(S - onehot).max() < 1e-12
    assert np.abs(F - onehot).max() < 1e-12


def test_spfh_counts_and_fpfh_weights_tiny(orc):
    """Three points worked by hand. p0 at the origin (normal +z); p1 at (0.1,0,0)
    with normal tilted by b = 0.3 about y toward p0's line; p2 at (0,0.05,0) with
    normal +z. Features: (p0,p2): all zero -> bins (5,5,5); (p0,p1): source p1
    (|n1.e| = sin b > 0), giving (alpha, phi, theta) = (0, sin b, b); FPFH(p0) = SPFH(p0) + (1/2)(SPFH(p1)/0.1 + SPFH(p2)/0.05),
    renormalised per sub-histogram."""
    b = 0.3
    P = np.array([[0, 0, 0], [0.1, 0, 0], [0, 0.05, 0]], float)
    N = np.array([[0, 0, 1], [-np.sin(b), 0, np.cos(b)], [0, 0, 1]], float)

    def bins(f):
        x = [(f[0] + 1) / 2 * 11, (f[1] + 1) / 2 * 11, (f[2] + np.pi) / (2 * np.pi) * 11]
        return [int(np.clip(np.floor(v), 0, 10)) + 11 * q for q, v in enumerate(x)]

    def onehot(bs):
        h = np.zeros(33)
        h[bs] = 1
        return h

    ok01, f01 = orc.pair_features(P[0], N[0], P[1], N[1])
    ok02, f02 = orc.pair_features(P[0], N[0], P[2], N[2])
    ok12, f12 = orc.pair_features(P[1], N[1], P[2], N[2])
    # (p0, p1): source p1, e = (-1,0,0), u = n1 = (-sin b, 0, cos b), v = (0,-1,0),
    # w = u x v = (cos b, 0, sin b); target normal +z: alpha = 0, phi = u.e = sin b,
    # theta = atan2(w.nt, u.nt) = atan2(sin b, cos b) = b.
    assert ok01 and np.allclose(f01, [0.0, np.sin(b), b], atol=1e-14)
    assert ok02 and np.allclose(f02, [0, 0, 0], atol=1e-14)
    S, k, _ = orc.spfh(P, N, 0.2)
    assert list(k) == [2, 2, 2]
    S0 = (onehot(bins(f01)) + onehot(bins(f02))) / 2
    S1 = (onehot(bins(f01)) + onehot(bins(f12))) / 2
    S2 = (onehot(bins(f02)) + onehot(bins(f12))) / 2
    assert np.allclose(S, [S0, S1, S2], atol=1e-15)
    F = orc.fpfh(P, N, S, 0.2)
    raw = S0 + 0.5 * (S1 / 0.1 + S2 / 0.05)
    expect = raw / np.repeat(raw.reshape(3, 11).sum(1), 11)
    assert np.allclose(F[0], expect, atol=1e-14)


def test_fpfh_rigid_invariance(orc):
    fp = make_pair(0)
    P = fp.P.astype(np.float64)
    N, _, _, _ = orc.normals(P, fp.vpP, 0.05)
    S, _, _ = orc.spfh(P, N, 0.125)
    F = orc.fpfh(P, N, S, 0.125)
    T = random_pose(np.random.default_rng(11))
    PT = P @ T[:3, :3].T + T[:3, 3]
    N2, _, _, _ = orc.normals(PT, T[:3, :3] @ fp.vpP + T[:3, 3], 0.05)
    S2, _, _ = orc.spfh(PT, N2, 0.125)
    F2 = orc.fpfh(PT, N2, S2, 0.125)
    assert np.abs(F - F2).max() < 1e-9
    sums = F.reshape(-1, 3, 11).sum(-1)
    valid = np.abs(N).sum(1) > 0
    assert np.allclose(sums[valid & (np.abs(F).sum(1) > 0)], 1.0)


# ------------------------------------------------------------------ matching
def test_match_equals_library_argmin(orc):
    rng = np.random.default_rng(12)
    A = rng.uniform(size=(300, 33))
    B = rng.uniform(size=(500, 33))
    B[7] = B[3]  # exact tie: smallest index wins
    A[0] = B[3]
    nn, d1, d2 = orc.match(A, B)
    D = cdist(A, B, "sqeuclidean")
    assert np.array_equal(nn, D.argmin(1))
    assert nn[0] == 3
    srt = np.sort(D, axis=1)
    assert np.allclose(d1, srt[:, 0]) and np.allclose(d2, srt[:, 1])


# ------------------------------------------------------------------ pre-rejection
def _pair_for_hyp(scale):
    rng = np.random.default_rng(13)
    P = rng.uniform(-1, 1, (400, 3))
    R = Rotation.random(random_state=14).as_matrix()
    Q = scale * P @ R.T + [0.5, 0, 0]
    return P, Q, np.arange(400)


@pytest.mark.parametrize("scale,survive", [(1.0, True), (1.04, True), (0.96, True), (1.2, False), (0.8, False)])
def test_prerejection_tau_direction(orc, scale, survive):
    """Exact correspondences under a similarity of scale s: every edge ratio is s,
    so hypotheses survive iff tau <= s <= 1/tau (tau = 0.9)."""
    P, Q, nn = _pair_for_hyp(scale)
    v = np.ones(400, np.uint8)
    flag = orc.hypotheses(P, Q, nn, v, v, 20000, 3, 0, 0.9)
    idx = orc.sample_indices(3, 0, 0, 20000, 400)
    distinct = np.array([len(set(r)) == 4 for r in idx])
    if survive:
        assert np.all(flag[distinct] == 1) and np.all(flag[~distinct] == 0)
    else:
        assert np.all(flag == 0)


def test_prerejection_invalid_and_cyclic_edges(orc):
    P, Q, nn = _pair_for_hyp(1.0)
    v = np.ones(400, np.uint8)
    vq = v.copy()
    vq[:200] = 0
    flag = orc.hypotheses(P, Q, nn, v, vq, 20000, 3, 0, 0.9)
    idx = orc.sample_indices(3, 0, 0, 20000, 400)
    assert np.all(flag[(idx < 200).any(1)] == 0)
    # a distortion on the closing edge (3 -> 0) alone must reject: move Q so only
    # the pair of points 0 and the last sample of one hypothesis disagrees
    h = int(np.nonzero(flag == 1)[0][0])
    i = idx[h]
    Q2 = Q.copy()
    Q2[i[0]] = Q[i[0]] + 0.0  # unchanged baseline
    base = orc.hypotheses(P, Q2, nn, v, vq, h + 1, 3, 0, 0.9)[h]
    assert base == 1
    # stretch p3-p0 only: move q0 far along (q0 - q3) while keeping |q0 - q1| ratio
    # (pick the direction orthogonal to q1 - q0 within the plane of q0, q1, q3)
    e01 = Q[i[1]] - Q[i[0]]
    e30 = Q[i[0]] - Q[i[3]]
    d = e30 - e01 * (e30 @ e01) / (e01 @ e01)
    d /= np.linalg.norm(d)
    Q3 = Q.copy()
    Q3[i[0]] = Q[i[0]] + 0.6 * np.linalg.norm(e30) * d
    ratio01 = np.linalg.norm(Q3[i[1]] - Q3[i[0]]) / np.linalg.norm(P[i[1]] - P[i[0]])
    ratio30 = np.linalg.norm(Q3[i[0]] - Q3[i[3]]) / np.linalg.norm(P[i[0]] - P[i[3]])
    assert ratio30 > 1 / 0.9 and 0.9 < ratio01 < 1 / 0.9 + 0.5
    assert orc.hypotheses(P, Q3, nn, v, vq, h + 1, 3, 0, 0.9)[h] == 0


# ------------------------------------------------------------------ rigid transform
def test_kabsch_noiseless_and_reflection(orc):
    rng = np.random.default_rng(15)
    for _ in range(100):
        T = random_pose(rng)
        p = rng.uniform(-1, 1, (4, 3))
        q = p @ T[:3, :3].T + T[:3, 3]
        R, t = orc.kabsch(p, q)
        assert np.abs(R - T[:3, :3]).max() < 1e-12 and np.abs(t - T[:3, 3]).max() < 1e-12
    # mirrored target: the best proper rotation, det +1
    p = rng.uniform(-1, 1, (4, 3))
    q = p * [1, 1, -1]
    R, _ = orc.kabsch(p, q)
    assert abs(np.linalg.det(R) - 1) < 1e-12


def _horn(p, q):
    """Horn (1987) closed form: the optimal unit quaternion is the top eigenvector
    of the 4x4 matrix built from the cross-covariance."""
    pc, qc = p - p.mean(0), q - q.mean(0)
    S = pc.T @ qc
    Sxx, Sxy, Sxz, Syx, Syy, Syz, Szx, Szy, Szz = S.ravel()
    N = np.array([[Sxx + Syy + Szz, Syz - Szy, Szx - Sxz, Sxy - Syx],
                  [Syz - Szy, Sxx - Syy - Szz, Sxy + Syx, Szx + Sxz],
                  [Szx - Sxz, Sxy + Syx, -Sxx + Syy - Szz, Syz + Szy],
                  [Sxy - Syx, Szx + Sxz, Syz + Szy, -Sxx - Syy + Szz]])
    w, V = np.linalg.eigh(N)
    q0, qx, qy, qz = V[:, -1]
    R = Rotation.from_quat([qx, qy, qz, q0]).as_matrix()
    return R, q.mean(0) - R @ p.mean(0)


def test_kabsch_equals_horn_noisy(orc):
    rng = np.random.default_rng(16)
    for _ in range(100):
        T = random_pose(rng)
        p = rng.uniform(-1, 1, (4, 3))
        q = p @ T[:3, :3].T + T[:3, 3] + rng.normal(0, 0.05, (4, 3))
        R, t = orc.kabsch(p, q)
        Rh, th = _horn(p, q)
        assert np.abs(R - Rh).max() < 1e-9 and np.abs(t - th).max() < 1e-9


# ------------------------------------------------------------------ consensus
def test_consensus_equals_brute(orc):
    rng = np.random.default_rng(17)
    P = rng.uniform(-0.5, 0.5, (800, 3))
    Q = rng.uniform(-0.5, 0.5, (900, 3))
    Rs, ts = [], []
    for _ in range(5):
        T = random_pose(rng, 0.2)
        Rs.append(T[:3, :3])
        ts.append(T[:3, 3])
    cnt, sd, _ = orc.consensus(P, Q, np.array(Rs), np.array(ts), 0.04)
    for h in range(5):
        X = P @ Rs[h].T + ts[h]
        dmin = cdist(X, Q).min(1)
        inl = dmin < 0.04
        assert cnt[h] == inl.sum()
        assert np.isclose(sd[h], (dmin[inl] ** 2).sum(), rtol=1e-12)


# ------------------------------------------------------------------ robust refinement / objective
def test_line_process_closed_form():
    """Eliminating l from l r^2 + mu (sqrt(l) - 1)^2 gives l* = (mu/(mu + r^2))^2
    and the Geman-McClure cost mu r^2 / (mu + r^2) (eq. (3)-(4))."""
    mu = 0.0375 ** 2
    for r2 in [0.0, 1e-5, 1e-4, 1e-3, 0.05]:
        f = lambda l: l * r2 + mu * (np.sqrt(l) - 1) ** 2  # noqa: E731
        res = minimize_scalar(f, bounds=(0, 1), method="bounded", options=dict(xatol=1e-12))
        lstar = (mu / (mu + r2)) ** 2
        assert abs(res.x - lstar) < 1e-6
        assert abs(f(lstar) - mu * r2 / (mu + r2)) < 1e-15


def test_exp_so3_matches_library(orc):
    rng = np.random.default_rng(18)
    for s in (1e-9, 1e-4, 0.5, 3.0):
        w = rng.standard_normal(3)
        w = w / np.linalg.norm(w) * s
        assert np.abs(orc.exp_so3(w) - Rotation.from_rotvec(w).as_matrix()).max() < 1e-13


def test_refine_recovers_noiseless_pose(orc):
    fp = make_pair(0)
    P = fp.P.astype(np.float64)
    Q = P @ fp.T[:3, :3].T + fp.T[:3, 3]
    Tp = np.eye(4)
    Tp[:3, :3] = Rotation.from_rotvec([0.01, -0.005, 0.008]).as_matrix()
    Tp[:3, 3] = [0.004, -0.003, 0.002]
    T0 = Tp @ fp.T
    T, it = orc.refine(P, Q, T0, 0.0375, 0.0375 ** 2, iters=100)
    ang, tr = pose_error(T, fp.T)
    assert ang < 1e-7 and tr < 1e-9


def test_objective_gradient_finite_differences(orc):
    """Analytic dE/dP, dE/dQ, dE/dxi against FP64 central differences (h = 1e-6)
    on a case where no correspondence changes within the step."""
    fp = make_pair(0)
    P = fp.P.astype(np.float64)[:600]
    Q = fp.Q.astype(np.float64)
    eps, mu = 0.0375, 0.0375 ** 2
    xi = np.array([0.002, -0.001, 0.0015, 0.001, 0.002, -0.001])
    T0 = fp.T.copy()
    E, dP, dQ, dxi, nn = orc.objective(P, Q, xi, T0, eps, mu)
    assert (nn >= 0).sum() > 100
    h = 1e-6
    for k in range(6):
        e = np.zeros(6)
        e[k] = h
        Ep, *_, nnp = orc.objective(P, Q, xi + e, T0, eps, mu, grad=False)
        Em, *_, nnm = orc.objective(P, Q, xi - e, T0, eps, mu, grad=False)
        assert np.array_equal(nnp, nn) and np.array_equal(nnm, nn)
        fd = (Ep - Em) / (2 * h)
        assert abs(fd - dxi[k]) <= 1e-4 * max(1.0, np.abs(dxi).max())
    rng = np.random.default_rng(19)
    for i in rng.choice(np.nonzero(nn >= 0)[0], 10, replace=False):
        for a in range(3):
            Pp, Pm = P.copy(), P.copy()
            Pp[i, a] += h
            Pm[i, a] -= h
            fd = (orc.objective(Pp, Q, xi, T0, eps, mu, grad=False)[0]
                  - orc.objective(Pm, Q, xi, T0, eps, mu, grad=False)[0]) / (2 * h)
            assert abs(fd - dP[i, a]) <= 1e-4 * max(1e-3, abs(dP[i, a]))
        j = nn[i]
        for a in range(3):
            Qp, Qm = Q.copy(), Q.copy()
            Qp[j, a] += h
            Qm[j, a] -= h
            fd = (orc.objective(P, Qp, xi, T0, eps, mu, grad=False)[0]
                  - orc.objective(P, Qm, xi, T0, eps, mu, grad=False)[0]) / (2 * h)
            assert abs(fd - dQ[j, a]) <= 1e-4 * max(1e-3, abs(dQ[j, a]))


def test_objective_gradient_zero_at_noiseless_optimum(orc):
    fp = make_pair(0)
    P = fp.P.astype(np.float64)
    Q = P @ fp.T[:3, :3].T + fp.T[:3, 3]
    E, dP, dQ, dxi, nn = orc.objective(P, Q, np.zeros(6), fp.T, 0.0375, 0.0375 ** 2)
    assert np.abs(dxi).max() < 1e-12 and np.abs(dP).max() < 1e-12
    assert E < 0  # every point sits at r = 0, rho~ = -rho(eps^2)


# ------------------------------------------------------------------ end to end
@pytest.mark.slow
def test_register_config0_recovers_ground_truth(orc):
    """Algorithm 1 + refinement on the 5,000-point objects pair: within the
    noise-level sanity bound of 0.5 deg / 5 mm of the generator's pose."""
    fp = make_pair(0)
    r = orc.register(fp.P, fp.Q, fp.vpP, fp.vpQ, seed=fp.seed)
    assert r["status"] == 0
    ang, tr = pose_error(r["T"], fp.T)
    assert ang < 0.5 and tr < 0.005
    assert r["inliers"] > 0.5 * len(fp.P)


def test_prerejection_edges_are_the_cyclic_sides(orc):
    """A unit square mapped to a 60-degree rhombus keeps all four side lengths and
    changes both diagonals (sqrt 2 -> sqrt 3 and 1). With exact correspondences a
    hypothesis survives iff its sample order walks the sides, i.e. its cyclic
    order is a rotation or a reversal of (0, 1, 2, 3)."""
    P = np.array([[0, 0, 0], [1, 0, 0], [1, 1, 0], [0, 1, 0]], float)
    h3 = np.sqrt(3) / 2
    Q = np.array([[0, 0, 0], [1, 0, 0], [1.5, h3, 0], [0.5, h3, 0]], float)
    v = np.ones(4, np.uint8)
    H = 4000
    flag = orc.hypotheses(P, Q, np.arange(4), v, v, H, 21, 2, 0.9)
    idx = orc.sample_indices(21, 2, 0, H, 4)
    sides = {(0, 1), (1, 2), (2, 3), (0, 3)}
    n_ok = 0
    for h in range(H):
        i = list(idx[h])
        if len(set(i)) < 4:
            assert flag[h] == 0
            continue
        walk = all(tuple(sorted((i[k], i[(k + 1) % 4]))) in sides for k in range(4))
        assert flag[h] == (1 if walk else 0), (h, i)
        n_ok += walk
    assert n_ok > 0


# ------------------------------------------------------------------ graduated refinement
def test_gnc_stride_definition(orc):
    assert [orc.gnc_stride(5000, l, 4) for l in range(4)] == [1, 1, 1, 1]
    assert [orc.gnc_stride(150_000, l, 4) for l in range(4)] == [36, 16, 4, 1]
    assert [orc.gnc_stride(10 ** 6, l, 4) for l in range(4)] == [64, 16, 4, 1]
    assert orc.gnc_stride(10 ** 6, 0, 1) == 1


def test_gnc_one_level_is_plain_refinement(orc):
    fp = make_pair(0)
    T0 = fp.T.copy()
    T0[:3, 3] += [0.01, -0.005, 0.004]
    a, _ = orc.refine(fp.P, fp.Q, T0, 0.0375, 0.0375 ** 2, iters=50)
    b, _ = orc.refine_gnc(fp.P, fp.Q, T0, 0.0375, 1.0, levels=1, iters=50)
    assert np.array_equal(a, b)


def test_gnc_result_independent_of_start(orc):
    """Starts up to ~1 deg / 2 cm apart (the spread of near-best hypotheses)
    reach the same pose, which single-level refinement does not guarantee."""
    fp = make_pair(0, 0, n_p=3000, n_q=3000)
    rng = np.random.default_rng(20)
    outs = []
    for _ in range(4):
        d = np.eye(4)
        d[:3, :3] = Rotation.from_rotvec(rng.normal(0, 0.01, 3)).as_matrix()
        d[:3, 3] = rng.normal(0, 0.01, 3)
        T, _ = orc.refine_gnc(fp.P, fp.Q, d @ fp.T, 0.0375, 1.0, levels=3, iters=100, tol=1e-12)
        outs.append(T)
    for T in outs[1:]:
        ang, tr = pose_error(T, outs[0])
        assert ang < 1e-6 and tr < 1e-8
    ang, tr = pose_error(outs[0], fp.T)
    assert ang < 0.5 and tr < 0.005


def test_gnc_recovers_noiseless_pose(orc):
    fp = make_pair(0)
    P = fp.P.astype(np.float64)
    Q = P @ fp.T[:3, :3].T + fp.T[:3, 3]
    d = np.eye(4)
    d[:3, :3] = Rotation.from_rotvec([0.02, 0.01, -0.015]).as_matrix()
    d[:3, 3] = [0.02, -0.01, 0.01]
    T, _ = orc.refine_gnc(P, Q, d @ fp.T, 0.0375, 1.0, levels=3, iters=100)
    ang, tr = pose_error(T, fp.T)
    assert ang < 1e-7 and tr < 1e-9
