"""Pins of the oracle's consensus variants: the single-cell lookup of eq. (1)
as the consensus search, and the per-inlier normal check (the other reading of
Sec. IV's normal check in hypothesis testing).

Single cell: never more inliers than the exact search; all of them when every
moved point sits in the cell of its partner (a lattice of cell centres and
offsets inside the cell); none for a point moved across a face from its only
partner.

Per-inlier normals: with equal normals it is the plain consensus; flipped
normals give none; normals carried by the rotation keep every inlier while a
tilt past the threshold drops them; and a pure-Python loop over every pair
(brute force) gives the same counts and sums on a small random case."""
import numpy as np

import oracle
from synth import make_pair


def test_single_cell_consensus_bounds_and_lattice():
    p = make_pair(0, 0)
    R, t = p.T[:3, :3], p.T[:3, 3]
    eps = 0.0375
    c1, s1 = oracle.consensus_single_cell(p.P, p.Q, R[None], t[None], eps)
    ce, se, _ = oracle.consensus(p.P, p.Q, R[None], t[None], eps)
    assert 0.3 * ce[0] < c1[0] <= ce[0]
    h = eps
    g = np.stack(np.meshgrid(np.arange(4), np.arange(4), np.arange(2), indexing="ij"), -1).reshape(-1, 3)
    Q = (g + 0.5) * h  # even counts: the centroid is a lattice corner, so these are cell centres
    c = Q.mean(axis=0)
    assert np.allclose(np.mod((Q - c) / h, 1.0), 0.5)  # every point at the centre of its own cell
    rng = np.random.default_rng(4)
    P = Q + rng.uniform(-0.3, 0.3, Q.shape) * h
    cnt, sd = oracle.consensus_single_cell(P, Q, np.eye(3)[None], np.zeros((1, 3)), eps)
    assert cnt[0] == len(Q) and np.isclose(sd[0], ((P - Q) ** 2).sum())
    # one point moved 0.6 cells along x: now in the neighbour's cell, nearest to
    # that neighbour at 0.4 cells (the exact search would find its own partner too)
    P2 = Q.copy()
    P2[0, 0] += 0.6 * h
    cnt2, _ = oracle.consensus_single_cell(P2, Q, np.eye(3)[None], np.zeros((1, 3)), eps)
    assert cnt2[0] == len(Q)
    P3 = Q.copy()
    P3[-1, 0] += 0.6 * h  # the last lattice row: the cell beyond is empty, so it is missed
    cnt3, _ = oracle.consensus_single_cell(P3, Q, np.eye(3)[None], np.zeros((1, 3)), eps)
    ce3, _, _ = oracle.consensus(P3, Q, np.eye(3)[None], np.zeros((1, 3)), eps)
    assert cnt3[0] == len(Q) - 1 and ce3[0] == len(Q)


def _rot_x(a):
    c, s = np.cos(a), np.sin(a)
    return np.array([[1, 0, 0], [0, c, -s], [0, s, c]])


def test_normals_consensus_reduces_and_rotates():
    rng = np.random.default_rng(5)
    P = np.c_[rng.uniform(0, 1, (400, 2)), np.zeros(400)]
    R = _rot_x(np.pi / 2)
    t = np.array([0.2, -0.1, 0.3])
    Q = P @ R.T + t + rng.normal(0, 0.002, (400, 3))
    n = np.tile([0.0, 0.0, 1.0], (400, 1))
    eps, cs = 0.0375, np.cos(np.deg2rad(30))
    plain, sd_plain, _ = oracle.consensus(P, Q, R[None], t[None], eps)
    # normals carried by the rotation: every inlier kept
    c1, s1, _ = oracle.consensus_normals(P, n, Q, n @ R.T, R[None], t[None], eps, cs)
    assert c1[0] == plain[0] > 350 and np.isclose(s1[0], sd_plain[0])
    # the same normals on both sides do not agree after a 90 degree rotation
    c2, _, _ = oracle.consensus_normals(P, n, Q, n, R[None], t[None], eps, cs)
    assert c2[0] == 0
    # flipped target normals: none
    c3, _, _ = oracle.consensus_normals(P, n, Q, -(n @ R.T), R[None], t[None], eps, cs)
    assert c3[0] == 0
    # target normals tilted by 20 degrees keep everything, by 40 degrees nothing
    for deg, want in ((20, plain[0]), (40, 0)):
        nq = n @ R.T @ _rot_x(np.deg2rad(deg)).T
        c4, _, _ = oracle.consensus_normals(P, n, Q, nq, R[None], t[None], eps, cs)
        assert c4[0] == want
    # invalid (zero) normals never count
    nz = n.copy()
    nz[:10] = 0
    c5, _, _ = oracle.consensus_normals(P, nz, Q, n @ R.T, R[None], t[None], eps, cs)
    assert c5[0] == plain[0] - np.sum(((P[:10] @ R.T + t)[:, None] - Q[None]) ** 2 < eps * eps, axis=2).any(1).sum()


def test_normals_consensus_brute_force():
    rng = np.random.default_rng(9)
    P = rng.uniform(0, 0.3, (120, 3))
    Q = rng.uniform(0, 0.3, (150, 3))
    NP = rng.normal(size=(120, 3))
    NP /= np.linalg.norm(NP, axis=1, keepdims=True)
    NQ = rng.normal(size=(150, 3))
    NQ /= np.linalg.norm(NQ, axis=1, keepdims=True)
    Rs = np.stack([_rot_x(a) for a in (0.0, 0.3, -1.1)])
    ts = rng.normal(0, 0.01, (3, 3))
    eps, cs = 0.05, 0.2
    cnt, sd, _ = oracle.consensus_normals(P, NP, Q, NQ, Rs, ts, eps, cs)
    for k in range(3):
        c, s = 0, 0.0
        for i in range(len(P)):
            x = Rs[k] @ P[i] + ts[k]
            best, bj = None, -1
            for j in range(len(Q)):
                d = float(((x - Q[j]) ** 2).sum())
                if best is None or d < best:
                    best, bj = d, j
            if best < eps * eps and float((Rs[k] @ NP[i]) @ NQ[bj]) >= cs:
                c += 1
                s += best
        assert cnt[k] == c and np.isclose(sd[k], s, rtol=1e-12, atol=0)
