"""GPU vs FP64 oracle, stage by stage and end to end, through the C ABI.

Stage isolation: every GPU stage gets the oracle's output of the previous stage
cast to FP32, and the oracle recomputes the stage from the same FP32 values in
FP64, so each comparison sees only that stage's arithmetic. Decisions the FP32
path may legitimately take either way (a neighbour at the radius, a feature at
a bin edge, a pre-rejection ratio at tau, a point at eps) are counted by the
oracle and excluded or bounded; everything else must match exactly (indices,
counts, survivor ids) or within the stated tolerance (values).
"""
import numpy as np
import pytest

import oracle
from synth import make_pair, pose_error

gpu = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1801_01572_gb300 as lsr
    c = lsr.Context(0)
    yield c
    c.close()


@pytest.fixture(scope="module")
def pair0():
    return make_pair(0, 0)


def _f32(a):
    return np.asarray(a, np.float64).astype(np.float32)


def _oracle_features(P, vp):
    """Oracle normals -> SPFH -> FPFH on FP32-cast inputs at every stage."""
    P32 = _f32(P)
    N, curv, cnt, diag = oracle.normals(P32, vp, 0.05)
    N32 = _f32(N)
    S, k, nclose = oracle.spfh(P32, N32, 0.125)
    S32 = _f32(S)
    F = oracle.fpfh(P32, N32, S32, 0.125)
    return dict(P=P32, N=N, N32=N32, cnt=cnt, diag=diag, S=S, S32=S32, k=k, nclose=nclose, F=F, F32=_f32(F))


@pytest.fixture(scope="module")
def feats0(pair0):
    return _oracle_features(pair0.P, pair0.vpP), _oracle_features(pair0.Q, pair0.vpQ)


# ------------------------------------------------------------------ normals
@gpu
@pytest.mark.parametrize("which", ["P", "Q"])
def test_normals_parity(ctx, pair0, feats0, which):
    f = feats0[0] if which == "P" else feats0[1]
    vp = pair0.vpP if which == "P" else pair0.vpQ
    N, cnt, curv = ctx.stage_normals(f["P"], vp, 0.05)
    near_r = f["diag"][:, 2] > 0
    assert np.array_equal(cnt[~near_r], f["cnt"][~near_r])
    valid = (f["cnt"] >= 3) & ~near_r
    gap, orient = f["diag"][:, 0], f["diag"][:, 1]
    good = valid & (gap > 1e-3) & (orient > 1e-3)
    assert good.mean() > 0.9
    err = np.linalg.norm(N[good] - f["N"][good], axis=1)
    tol = 2e-5 + 2e-6 / gap[good]
    assert np.all(err <= tol), (err.max(), np.argmax(err - tol))
    inval = f["cnt"] < 3
    assert np.all(N[inval & ~near_r] == 0) and np.all(curv[inval & ~near_r] == -1)


# ------------------------------------------------------------------ SPFH / FPFH
@gpu
@pytest.mark.parametrize("which", [0, 1])
def test_spfh_parity(ctx, feats0, which):
    f = feats0[which]
    S, k = ctx.stage_spfh(f["P"], f["N32"], 0.125)
    clean = f["nclose"] == 0
    assert clean.mean() > 0.5
    assert np.array_equal(k[clean], f["k"][clean])
    assert np.abs(S[clean] - f["S"][clean]).max() < 1e-6
    # borderline pairs: each can move 1/k between bins of each sub-histogram
    kk = np.maximum(f["k"] - f["nclose"], 1)
    l1 = np.abs(S - f["S"]).sum(1)
    assert np.all(l1 <= 6.0 * f["nclose"] / kk + 1e-5)


@gpu
@pytest.mark.parametrize("which", [0, 1])
def test_fpfh_parity(ctx, feats0, which):
    f = feats0[which]
    F = ctx.stage_fpfh(f["P"], f["N32"], f["S32"], 0.125)
    err = np.abs(F - f["F"]).max(1)
    assert np.quantile(err, 0.999) < 1e-5
    assert err.max() < 2e-3


# ------------------------------------------------------------------ matching
@gpu
def test_match_parity_fp32(ctx, feats0):
    fP, fQ = feats0
    A, B = fP["F32"].astype(np.float64), fQ["F32"].astype(np.float64)
    nn_ref, d1, d2 = oracle.match(A, B)
    nn, dg, _ = ctx.stage_match(fP["F32"], fQ["F32"])
    sure = (d2 - d1) > 1e-5
    assert sure.mean() > 0.5
    assert np.array_equal(nn[sure], nn_ref[sure])
    # elsewhere the GPU's choice is a near-tie of the true minimum
    D = ((A[~sure] - B[nn[~sure]]) ** 2).sum(1)
    assert np.all(D - d1[~sure] <= 1e-5)
    assert np.allclose(dg, d1, atol=2e-6, rtol=1e-5)


# ------------------------------------------------------------------ hypotheses
@gpu
def test_hypotheses_parity(ctx, pair0, feats0):
    fP, fQ = feats0
    nn_ref, _, _ = oracle.match(fP["F32"].astype(np.float64), fQ["F32"].astype(np.float64))
    vP = (np.abs(fP["N"]).sum(1) > 0).astype(np.uint8)
    vQ = (np.abs(fQ["N"]).sum(1) > 0).astype(np.uint8)
    H = 1_000_000
    flag = oracle.hypotheses(fP["P"], fQ["P"], nn_ref, vP, vQ, H, pair0.seed, 0, 0.9)
    surv, ns = ctx.stage_hypotheses(fP["P"], fQ["P"], nn_ref.astype(np.int32), vP, vQ, H, pair0.seed, 0, 0.9)
    assert ns == len(surv) and np.all(np.diff(surv) > 0)
    sure = set(np.nonzero(flag == 1)[0].tolist())
    amb = set(np.nonzero(flag == 2)[0].tolist())
    got = set(surv.tolist())
    assert sure <= got and got <= sure | amb
    assert len(sure) > 100


# ------------------------------------------------------------------ rigid fit / consensus
@gpu
def test_rigid4_parity(ctx):
    rng = np.random.default_rng(3)
    from synth import random_pose
    ps, qs, Rr, tr = [], [], [], []
    for _ in range(2000):
        T = random_pose(rng)
        p = rng.uniform(-1.5, 1.5, (4, 3))
        q = p @ T[:3, :3].T + T[:3, 3] + rng.normal(0, 0.01, (4, 3))
        p32, q32 = _f32(p), _f32(q)
        R, t = oracle.kabsch(p32, q32)
        ps.append(p32.ravel())
        qs.append(q32.ravel())
        Rr.append(R)
        tr.append(t)
    Rt = ctx.stage_rigid4(np.array(ps), np.array(qs))
    R = Rt[:, [0, 1, 2, 4, 5, 6, 8, 9, 10]].reshape(-1, 3, 3)
    t = Rt[:, [3, 7, 11]]
    assert np.abs(R - np.array(Rr)).max() < 5e-4
    assert np.quantile(np.abs(R - np.array(Rr)).max((1, 2)), 0.99) < 2e-5
    assert np.abs(t - np.array(tr)).max() < 2e-3


@gpu
def test_consensus_parity(ctx, pair0):
    rng = np.random.default_rng(4)
    P, Q = pair0.P, pair0.Q
    Rs, ts = [], []
    for k in range(64):
        # poses around the ground truth (many inliers) and random ones (few)
        from synth import random_pose
        if k % 2 == 0:
            dT = random_pose(rng, 0.01)
            ang = 0.02 * rng.standard_normal(3)
            from scipy.spatial.transform import Rotation
            dT[:3, :3] = Rotation.from_rotvec(ang).as_matrix()
            T = dT @ pair0.T
        else:
            T = random_pose(rng)
        Rs.append(_f32(T[:3, :3]))
        ts.append(_f32(T[:3, 3]))
    Rs, ts = np.array(Rs), np.array(ts)
    cnt_ref, sd_ref, amb = oracle.consensus(P, Q, Rs.astype(np.float64), ts.astype(np.float64), 0.0375, band=1e-5)
    Rt = np.concatenate([Rs, ts[:, :, None]], axis=2).reshape(-1, 12)
    cnt, sd = ctx.stage_consensus(P, Q, Rt, 0.0375)
    assert np.all(np.abs(cnt - cnt_ref) <= amb)
    assert np.all(np.abs(sd - sd_ref) <= 1e-5 * sd_ref + amb * 0.0375 ** 2 + 1e-9)
    assert cnt_ref.max() > 0.5 * len(P)


@gpu
@pytest.mark.parametrize("config,n", [(0, None), (1, 60000)])
def test_consensus_classified_counts_equal_exact(ctx, config, n):
    """Inlier counts through the voxel classification (lsr_stage_consensus)
    equal, bit for bit, those of the exact eps-grid kernel (the allocation-free
    entry point) for poses near the truth, perturbed, and random."""
    import ctypes as C
    import torch
    import paper_1801_01572_gb300 as lsr
    from synth import random_pose
    fp = make_pair(config, 3, n_p=n, n_q=n)
    rng = np.random.default_rng(17 + config)
    Rt = []
    from scipy.spatial.transform import Rotation
    for k in range(400):
        if k % 4 < 2:  # near the truth (within ~0.3 deg / 2 mm), or perturbed (~3 deg / 2 cm)
            s_r, s_t = (0.005, 0.002) if k % 4 == 0 else (0.05, 0.02)
            dT = np.eye(4)
            dT[:3, :3] = Rotation.from_rotvec(rng.normal(0, s_r, 3)).as_matrix()
            dT[:3, 3] = rng.normal(0, s_t, 3)
            T = dT @ fp.T
        else:
            T = random_pose(rng)
            T[:3, 3] = fp.T[:3, 3] + rng.normal(0, 0.3, 3)
        Rt.append(np.concatenate([T[:3, :3], T[:3, 3:]], axis=1).reshape(12))
    Rt = np.asarray(Rt, np.float32)
    cnt, sd = ctx.stage_consensus(fp.P, fp.Q, Rt, 0.0375)
    nh = len(Rt)
    P, Q, R = (torch.from_numpy(a).cuda() for a in (fp.P, fp.Q, Rt))
    ref = torch.zeros(nh, dtype=torch.int32, device="cuda")
    rsd = torch.zeros(nh, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    rc = lsr.lib().lsr_consensus_static(C.c_void_p(P.data_ptr()), len(fp.P), C.c_void_p(Q.data_ptr()), len(fp.Q),
                                        C.c_void_p(R.data_ptr()), nh, C.c_float(0.0375), C.c_void_p(ref.data_ptr()),
                                        C.c_void_p(rsd.data_ptr()), None)
    assert rc == lsr.LSR_OK
    ref = ref.cpu().numpy()
    assert np.array_equal(cnt, ref)
    assert np.allclose(sd, rsd.cpu().numpy(), rtol=1e-9, atol=1e-12)
    assert ref.max() > len(fp.P) // 3 and (ref < len(fp.P) // 10).sum() > 100


# ------------------------------------------------------------------ refinement
@gpu
def test_refine_parity(ctx, pair0):
    from scipy.spatial.transform import Rotation
    dT = np.eye(4)
    dT[:3, :3] = Rotation.from_rotvec([0.02, -0.01, 0.015]).as_matrix()
    dT[:3, 3] = [0.01, -0.008, 0.005]
    T0 = dT @ pair0.T
    eps = 0.0375
    for levels in (1, 4):
        T_ref, _ = oracle.refine_gnc(pair0.P, pair0.Q, T0, eps, 1.0, levels=levels, iters=50)
        T, it = ctx.stage_refine(pair0.P, pair0.Q, T0, eps, 1.0, levels, 50)
        ang, tr = pose_error(T, T_ref)
        assert ang < 0.05 and tr < 5e-4, (levels, ang, tr)
        assert it > 0


# ------------------------------------------------------------------ end to end
@gpu
def test_register_config0_matches_oracle(ctx, pair0):
    r = ctx.register_pair(pair0.P, pair0.Q, pair0.vpP, pair0.vpQ)
    ref = oracle.register(pair0.P, pair0.Q, pair0.vpP, pair0.vpQ, seed=0)
    assert r.status == 0 and ref["status"] == 0
    a_gt, t_gt = pose_error(r.T, pair0.T)
    assert a_gt < 0.5 and t_gt < 5e-3
    ang, tr = pose_error(r.T, ref["T"])
    assert ang < 0.05 and tr < 5e-4, (ang, tr)
    assert abs(r.survivors - ref["survivors"]) <= 0.01 * ref["survivors"]


@gpu
def test_register_host_and_device_inputs_agree(ctx, pair0):
    import torch
    a = ctx.register_pair(pair0.P, pair0.Q, pair0.vpP, pair0.vpQ)
    b = ctx.register_pair(torch.from_numpy(pair0.P).cuda(), torch.from_numpy(pair0.Q).cuda(), pair0.vpP, pair0.vpQ)
    assert np.array_equal(a.T, b.T) and a.inliers == b.inliers and a.best_h == b.best_h


@gpu
def test_register_is_deterministic(ctx, pair0):
    a = ctx.register_pair(pair0.P, pair0.Q, pair0.vpP, pair0.vpQ)
    b = ctx.register_pair(pair0.P, pair0.Q, pair0.vpP, pair0.vpQ)
    assert np.array_equal(a.T, b.T) and a.survivors == b.survivors and a.best_h == b.best_h


@gpu
def test_batch_equals_single_pairs(ctx):
    pairs = [make_pair(0, i, n_p=1500 + 700 * i, n_q=2500 - 400 * i) for i in range(3)]
    ctx.set_params(n_hypotheses=300_000, seed=77, pair_id=5)
    try:
        batch = ctx.register_batch([p.P for p in pairs], [p.Q for p in pairs],
                                   [np.r_[p.vpP, p.vpQ] for p in pairs])
        for i, p in enumerate(pairs):
            ctx.set_params(pair_id=5 + i)
            s = ctx.register_pair(p.P, p.Q, p.vpP, p.vpQ)
            assert np.array_equal(s.T, batch[i].T) and s.best_h == batch[i].best_h
    finally:
        import paper_1801_01572_gb300 as lsr
        ctx.set_params(lsr.default_params())


# ------------------------------------------------------------------ edge cases
@gpu
def test_edge_cases(ctx, pair0):
    import paper_1801_01572_gb300 as lsr
    with pytest.raises(lsr.LsrError) as e:
        ctx.register_pair(pair0.P[:3], pair0.Q)
    assert e.value.code == lsr.LSR_E_ARG
    P = pair0.P.copy()
    P[10, 1] = np.nan
    with pytest.raises(lsr.LsrError) as e:
        ctx.register_pair(P, pair0.Q)
    assert e.value.code == lsr.LSR_E_ARG
    # the context stays usable after argument errors
    r = ctx.register_pair(pair0.P[:4], pair0.Q[:4])
    assert r.status == lsr.STATUS_NO_ALIGNMENT and np.array_equal(r.T, np.eye(4))
    # all points identical: no valid normal, nothing sampled
    same = np.zeros((500, 3), np.float32)
    r = ctx.register_pair(same, same)
    assert r.status == lsr.STATUS_NO_ALIGNMENT and r.survivors == 0
    # ragged sizes and a far-away outlier (forces a wrapped grid)
    Q = np.concatenate([pair0.Q, np.array([[1e4, -3e4, 2e4]], np.float32)])
    r = ctx.register_pair(pair0.P[:3333], Q, pair0.vpP, pair0.vpQ)
    assert r.status == lsr.STATUS_ALIGNED
    a, t = pose_error(r.T, pair0.T)
    assert a < 0.5 and t < 5e-3
