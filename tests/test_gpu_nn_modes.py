"""The nearest-neighbour modes and the consensus variants against the FP64
oracle: the exact search and the single-cell O(1) lookup of eq. (1)
(lsr_stage_nn), the consensus with either search and with the per-inlier
normal check (lsr_stage_consensus_modes, the kernels the registration runs in
those modes), and whole registrations in those modes.

Decisions an FP32 evaluation may take the other way are found on the oracle
side and excluded: a distance within 1e-6 m of the radius, a runner-up within
1e-6 m of the nearest, a point within 1e-5 cells of a face of the
single-cell lattice (or a cell next to such a point), a cosine within 1e-5 of
the threshold."""
import numpy as np
import pytest

import oracle
from synth import make_pair, pose_error, random_pose

gpu = pytest.mark.gpu
EPS = 0.0375


@pytest.fixture(scope="module")
def ctx():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1801_01572_gb300 as lsr
    c = lsr.Context(0)
    yield c
    c.close()


def _moved(fp, T=None):
    T = fp.T if T is None else T
    return (fp.P.astype(np.float64) @ T[:3, :3].T + T[:3, 3]).astype(np.float32)


def _second_nn(Q, X):
    spatial = pytest.importorskip("scipy.spatial")
    d, j = spatial.cKDTree(Q.astype(np.float64)).query(X.astype(np.float64), k=2)
    return d, j


def _cell_ambiguous(Q, X, cell):
    """Queries whose single-cell result an FP32 lattice may change: the query
    near a face, or its cell holding (or facing) a Q point near a face."""
    Q64, X64 = Q.astype(np.float64), X.astype(np.float64)
    c = Q64.mean(axis=0)
    fq = (Q64 - c) / cell
    kq = np.floor(fq).astype(np.int64)
    band = 1e-5
    bad = set()
    frac = fq - kq
    for i in np.nonzero(np.any((frac < band) | (frac > 1 - band), axis=1))[0]:
        bad.add(tuple(kq[i]))
        for a in range(3):
            if frac[i, a] < band:
                k = kq[i].copy()
                k[a] -= 1
                bad.add(tuple(k))
            if frac[i, a] > 1 - band:
                k = kq[i].copy()
                k[a] += 1
                bad.add(tuple(k))
    fx = (X64 - c) / cell
    kx = np.floor(fx).astype(np.int64)
    fr = fx - kx
    amb = np.any((fr < band) | (fr > 1 - band), axis=1)
    amb |= np.array([tuple(k) in bad for k in kx])
    return amb


@gpu
@pytest.mark.parametrize("config,n", [(0, None), (1, 40000)])
def test_exact_nn_matches_oracle(ctx, config, n):
    fp = make_pair(config, 0, n_p=n, n_q=n) if n else make_pair(config, 0)
    X = _moved(fp)
    nn, d2 = ctx.stage_nn(fp.Q, X, EPS)
    ref, rd2 = oracle.nn_within(fp.Q, X, EPS)
    d, j = _second_nn(fp.Q, X)
    amb = (np.abs(d[:, 0] - EPS) < 1e-6) | (d[:, 1] - d[:, 0] < 1e-6)
    sure = ~amb
    assert sure.mean() > 0.99
    assert np.array_equal(nn[sure], ref[sure])
    has = sure & (ref >= 0)
    assert np.allclose(d2[has], rd2[has], rtol=1e-5, atol=1e-9)
    assert np.all(np.isinf(d2[sure & (ref < 0)]))


@gpu
@pytest.mark.parametrize("config,n", [(0, None), (1, 40000)])
def test_single_cell_nn_matches_oracle(ctx, config, n):
    import paper_1801_01572_gb300 as lsr
    fp = make_pair(config, 0, n_p=n, n_q=n) if n else make_pair(config, 0)
    X = _moved(fp)
    nn, d2 = ctx.stage_nn(fp.Q, X, EPS, lsr.NN_SINGLE_CELL)
    ref, rd2 = oracle.nn_single_cell(fp.Q, X, EPS)
    amb = _cell_ambiguous(fp.Q, X, EPS)
    # ties between two candidates of the cell
    same = (ref >= 0) & (nn >= 0) & (nn != ref)
    if same.any():
        dd = ((fp.Q[nn[same]].astype(np.float64) - X[same]) ** 2).sum(1)
        amb[np.nonzero(same)[0][np.abs(dd - rd2[same]) < 1e-9]] = True
    sure = ~amb
    assert sure.mean() > 0.95
    assert np.array_equal(nn[sure], ref[sure])
    has = sure & (ref >= 0)
    assert np.allclose(d2[has], rd2[has], rtol=1e-5, atol=1e-9)
    # the single cell only ever loses neighbours: never closer than the exact
    # search (the two kernels may round the same distance one unit apart)
    ex, exd2 = ctx.stage_nn(fp.Q, X, 10 * EPS)
    found = nn >= 0
    assert np.all(d2[found] >= exd2[found] * (1 - 1e-6))


def _poses(fp, rng, n):
    Rt = []
    for k in range(n):
        T = fp.T if k % 4 == 0 else random_pose(rng, 0.02) @ fp.T
        Rt.append(np.concatenate([T[:3, :3], T[:3, 3:]], axis=1).reshape(12))
    return np.asarray(Rt, np.float32)


@gpu
def test_consensus_modes_match_oracle(ctx):
    import paper_1801_01572_gb300 as lsr
    fp = make_pair(0, 0)
    rng = np.random.default_rng(12)
    Rt = _poses(fp, rng, 12)
    Rs = Rt.reshape(-1, 3, 4)[:, :, :3].astype(np.float64)
    ts = Rt.reshape(-1, 3, 4)[:, :, 3].astype(np.float64)
    # exact, no normals: the plain consensus
    c0, s0 = ctx.stage_consensus_modes(fp.P, fp.Q, Rt, EPS)
    r0, rs0, a0 = oracle.consensus(fp.P, fp.Q, Rs, ts, EPS, band=1e-6)
    assert np.all(np.abs(c0 - r0) <= a0)
    assert np.allclose(s0, rs0, rtol=1e-4)
    cw, _ = ctx.stage_consensus(fp.P, fp.Q, Rt, EPS)
    assert np.array_equal(cw, c0)
    # single cell
    c1, s1 = ctx.stage_consensus_modes(fp.P, fp.Q, Rt, EPS, lsr.NN_SINGLE_CELL)
    r1, rs1 = oracle.consensus_single_cell(fp.P, fp.Q, Rs, ts, EPS)
    for k in range(len(Rt)):
        X = (fp.P.astype(np.float64) @ Rs[k].T + ts[k]).astype(np.float32)
        amb = _cell_ambiguous(fp.Q, X, EPS).sum()
        assert abs(int(c1[k]) - int(r1[k])) <= amb, (k, c1[k], r1[k], amb)
    assert np.all(c1 <= c0)
    # per-inlier normals (oracle normals of the same clouds, cast to FP32)
    NP = oracle.normals(fp.P, fp.vpP, 0.05)[0].astype(np.float32)
    NQ = oracle.normals(fp.Q, fp.vpQ, 0.05)[0].astype(np.float32)
    cs = float(np.cos(np.deg2rad(30)))
    c2, s2 = ctx.stage_consensus_modes(fp.P, fp.Q, Rt, EPS, lsr.NN_EXACT, lsr.NORMALS_INLIERS, NP, NQ, cs)
    r2, rs2, a2 = oracle.consensus_normals(fp.P, NP, fp.Q, NQ, Rs, ts, EPS, cs, band=1e-5)
    for k in range(len(Rt)):
        X = fp.P.astype(np.float64) @ Rs[k].T + ts[k]
        d, _ = _second_nn(fp.Q, X)
        ties = int(((d[:, 0] < EPS + 1e-6) & (d[:, 1] - d[:, 0] < 1e-6)).sum())
        assert abs(int(c2[k]) - int(r2[k])) <= a2[k] + ties, (k, c2[k], r2[k], a2[k], ties)
    assert np.all(c2 <= c0) and c2[0] > 0.5 * c0[0]
    # both variants at once: never more than either
    c3, _ = ctx.stage_consensus_modes(fp.P, fp.Q, Rt, EPS, lsr.NN_SINGLE_CELL, lsr.NORMALS_INLIERS, NP, NQ, cs)
    assert np.all(c3 <= c1) and np.all(c3 <= c2)


@gpu
@pytest.mark.parametrize("mode", ["single_cell", "inlier_normals"])
def test_registration_in_variant_modes(mode):
    """Registration with a variant consensus selects a hypothesis in the basin
    of the same optimum: the exact refinement then lands on the exact mode's
    pose (and the oracle's) within 0.05 deg / 0.5 mm."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1801_01572_gb300 as lsr
    fp = make_pair(0, 0)
    kw = {"nn_mode": lsr.NN_SINGLE_CELL} if mode == "single_cell" else {"normal_mode": lsr.NORMALS_INLIERS}
    with lsr.Context(0) as base, lsr.Context(0, **kw) as var:
        a = base.register_pair(fp.P, fp.Q, fp.vpP, fp.vpQ)
        b = var.register_pair(fp.P, fp.Q, fp.vpP, fp.vpQ)
    assert a.status == b.status == lsr.STATUS_ALIGNED
    ang, tr = pose_error(b.T, a.T)
    assert ang < 0.05 and tr < 5e-4, (ang, tr)
    if mode == "single_cell":
        assert b.hyp_inliers <= a.hyp_inliers and b.survivors == a.survivors and b.n_normal_ok == a.n_normal_ok
    else:
        assert b.n_normal_ok == b.survivors  # no sampled-pair check in this mode
