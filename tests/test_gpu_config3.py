"""Full-size checks of the BF16 tensor-core matching workload: 200,000-point
room pairs (config 3), descriptor matching on the tensor cores with FP32
accumulation and the FP32 re-rank of the top 8 candidates.

The certified matcher must give exactly the FP32 path's correspondences (index
and distance, every query), hence the oracle's indices wherever the oracle's
distance gap exceeds 1e-5 (checked on sampled queries, which the oracle
matches by brute force one by one), and the registration through it must give
the FP32 path's pose bit for bit, which agrees with the FP64 oracle's
refinement fixed point within 0.05 deg / 0.5 mm (see test_gpu_config1.py for
why the fixed point is the oracle comparison at this size).
"""
import numpy as np
import pytest

import oracle
from synth import make_pair, pose_error

gpu = pytest.mark.gpu


@pytest.fixture(scope="module")
def lsr_mod():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1801_01572_gb300 as lsr
    return lsr


@pytest.fixture(scope="module")
def pair3():
    return make_pair(3, 0)


@gpu
def test_config3_bf16_matching_equals_fp32_and_oracle(lsr_mod, pair3):
    ctx = lsr_mod.Context(0)
    try:
        F = []
        for X, vp in ((pair3.P, pair3.vpP), (pair3.Q, pair3.vpQ)):
            N, _, _ = ctx.stage_normals(X, vp, 0.05)
            S, _ = ctx.stage_spfh(X, N, 0.125)
            F.append(ctx.stage_fpfh(X, N, S, 0.125))
        nn32, d32, _ = ctx.stage_match(F[0], F[1], precision=lsr_mod.MATCH_FP32)
        nn16, d16, fb = ctx.stage_match(F[0], F[1], precision=lsr_mod.MATCH_BF16)
    finally:
        ctx.close()
    assert np.array_equal(nn16, nn32)
    assert np.array_equal(d16.view(np.uint32), d32.view(np.uint32))
    assert fb < 0.1 * len(pair3.P), fb
    q = np.sort(np.random.default_rng(3).choice(len(pair3.P), 300, replace=False))
    nr, d1, d2 = oracle.match(F[0].astype(np.float64), F[1].astype(np.float64), qidx=q)
    sure = (d2 - d1) > 1e-5
    assert sure.mean() > 0.3
    assert np.array_equal(nn16[q][sure], nr[sure])


@gpu
def test_config3_register_bf16_equals_fp32_and_oracle_fixed_point(lsr_mod, pair3):
    res = {}
    for prec in (lsr_mod.MATCH_FP32, lsr_mod.MATCH_BF16):
        with lsr_mod.Context(0, match_precision=prec) as ctx:
            res[prec] = ctx.register_pair(pair3.P, pair3.Q, pair3.vpP, pair3.vpQ)
    r32, r16 = res[lsr_mod.MATCH_FP32], res[lsr_mod.MATCH_BF16]
    assert r16.status == 0
    assert np.array_equal(r16.T, r32.T) and r16.inliers == r32.inliers
    T_ref, _ = oracle.refine_gnc(pair3.P, pair3.Q, pair3.T, 0.0375, 1.0, levels=3, iters=50)
    ang, tr = pose_error(r16.T, T_ref)
    assert ang < 0.05 and tr < 5e-4, (ang, tr)
