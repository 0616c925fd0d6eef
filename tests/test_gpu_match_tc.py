"""BF16 tensor-core feature matching (Algorithm 1, feature pre-matching).

The contraction is checked against the exact (float64) product of the same
BF16 operands, rebuilt here from the matcher's definition (centring, rounding,
hi/lo split): its accumulation error must stay inside the bound the matcher's
certificate assumes, and its distances inside the certificate's whole error
budget. The certified matcher must return exactly the FP32 path's indices and
distances (and so the oracle's indices wherever the oracle's distance gap
exceeds 1e-5), including ties, near-duplicate clusters that force the exact
fallback, and ragged tile edges, in both operand layouts.
"""
import numpy as np
import pytest

import oracle
from synth import make_pair

gpu = pytest.mark.gpu
D = 33


@pytest.fixture(scope="module")
def ctx():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1801_01572_gb300 as lsr
    c = lsr.Context(0)
    yield c
    c.close()


def bf16(x):
    """Round float32 to the nearest BF16 (ties to even), returned as float64."""
    u = np.ascontiguousarray(x, np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def fpfh_like(n, rng):
    """Descriptors shaped like FPFH: three non-negative 11-bin sub-histograms,
    each summing to 1, peaked on a few bins."""
    g = rng.gamma(0.35, 1.0, size=(n, 3, 11))
    g /= g.sum(2, keepdims=True)
    return g.reshape(n, D).astype(np.float32)


@pytest.fixture(scope="module")
def real_feats():
    """Oracle FPFH of both clouds of the 5,000-point object pair."""
    p = make_pair(0, 0)
    out = []
    for X, vp in ((p.P, p.vpP), (p.Q, p.vpQ)):
        X32 = X.astype(np.float32)
        N, _, _, _ = oracle.normals(X32, vp, 0.05)
        N32 = N.astype(np.float32)
        S, _, _ = oracle.spfh(X32, N32, 0.125)
        F = oracle.fpfh(X32, N32, S.astype(np.float32), 0.125)
        out.append(F.astype(np.float32))
    return out


def center_like_device(B):
    """The matcher's centre, with the device's sampling and FP32 summation order
    (8 row groups summed sequentially, then the groups in order)."""
    n = len(B)
    step = n // 2048 if n > 2048 else 1
    m = (n + step - 1) // step
    rows = B[::step][:m].astype(np.float32)
    part = np.zeros((8, D), np.float32)
    for g in range(8):
        for i in range(g, m, 8):
            part[g] = part[g] + rows[i]
    tot = np.zeros(D, np.float32)
    for g in range(8):
        tot = tot + part[g]
    return tot / np.float32(m)


def split_like_device(X, c, split):
    """(hi, lo) BF16 parts of fl(X - c), as float64."""
    x = (X.astype(np.float32) - c).astype(np.float32)
    h = bf16(x)
    lo = bf16((x.astype(np.float64) - h).astype(np.float32)) if split else np.zeros_like(h)
    return x.astype(np.float64), h, lo


ACC_ERR = 1.5e-5  # accumulation bound per unit of sum |products| the certificate assumes


@gpu
@pytest.mark.parametrize("precision", [1, 2])
@pytest.mark.parametrize("nP,nQ", [(1, 1), (300, 700), (513, 129), (256, 3000)])
def test_tc_contraction_within_certificate_bounds(ctx, nP, nQ, precision):
    split = precision == 1
    rng = np.random.default_rng(nP * 7919 + nQ)
    A, B = fpfh_like(nP, rng), fpfh_like(nQ, rng)
    d2 = ctx.match_scores_bf16(A, B, precision=precision).astype(np.float64)
    c = center_like_device(B)
    xa, ha, la = split_like_device(A, c, split)
    xb, hb, lb = split_like_device(B, c, split)
    at, bt = ha + la, hb + lb
    # what the MMA chain computes, in exact arithmetic
    dot = ha @ hb.T + (la @ hb.T + ha @ lb.T if split else 0.0)
    ref = (bt * bt).sum(1)[None, :] - 2.0 * dot + (at * at).sum(1)[:, None]
    mag = 2.0 * (np.abs(ha) @ np.abs(hb).T + (np.abs(la) @ np.abs(hb).T + np.abs(ha) @ np.abs(lb).T if split else 0))
    mag += (bt * bt).sum(1)[None, :]
    # |a~|^2 is added in FP32 after the MMAs: allow its two roundings
    aa = (at * at).sum(1)[:, None]
    acc = np.maximum(np.abs(d2 - ref) - 1.2e-7 * (aa + np.abs(d2)), 0.0) / np.maximum(mag, 1e-30)
    assert acc.max() < ACC_ERR, acc.max()
    # the certificate's whole bound on |D~^2 - |a - b|^2|
    na, nb = np.sqrt((at * at).sum(1)), np.sqrt((bt * bt).sum(1)).max()
    eta = np.sqrt(((xa - at) ** 2).sum(1)) + 1.2e-7 * np.sqrt((xa * xa).sum(1))
    eta_b = (np.sqrt(((xb - bt) ** 2).sum(1)) + 1.2e-7 * np.sqrt((xb * xb).sum(1))).max()
    efp = ACC_ERR * (2.05 * na * nb + nb * nb) + (3.1e-5 * na * nb if split else 0.0)
    A64, B64 = A.astype(np.float64), B.astype(np.float64)
    Dx = np.sqrt(np.maximum((A64 * A64).sum(1)[:, None] + (B64 * B64).sum(1)[None] - 2.0 * A64 @ B64.T, 0.0))
    e = (eta + eta_b)[:, None]
    lo = np.maximum(Dx - e, 0.0) ** 2 - efp[:, None]
    hi = (Dx + e) ** 2 + efp[:, None]
    assert np.all((d2 >= lo) & (d2 <= hi))


def _check_same(ctx, A, B, precision=1):
    nn32, d32, fb32 = ctx.stage_match(A, B, precision=0)
    nn16, d16, fb16 = ctx.stage_match(A, B, precision=precision)
    assert fb32 == 0
    assert np.array_equal(nn16, nn32)
    assert np.array_equal(d16.view(np.uint32), d32.view(np.uint32))
    return nn16, d16, fb16


@gpu
@pytest.mark.parametrize("precision", [1, 2])
@pytest.mark.parametrize("nP,nQ", [(1, 1), (1, 9), (7, 5), (255, 8), (257, 9), (1000, 3001), (3000, 1000)])
def test_tc_match_equals_fp32_random(ctx, nP, nQ, precision):
    rng = np.random.default_rng(nP + 31 * nQ)
    A, B = fpfh_like(nP, rng), fpfh_like(nQ, rng)
    _, _, fb = _check_same(ctx, A, B, precision)
    assert 0 <= fb <= nP


@gpu
@pytest.mark.parametrize("precision", [1, 2])
def test_tc_match_ties_and_near_duplicates(ctx, precision):
    """Exact duplicate rows (ties go to the smaller index), a pair of rows 1e-6
    apart (both in the candidate chunks: the exact re-rank decides), and
    clusters of 12 rows within 1e-6 of each other, each row in a different
    32-row chunk (more near-tied chunks than the 8 candidate chunks: no BF16
    certificate is possible and the exact fallback must decide)."""
    rng = np.random.default_rng(5)
    B = fpfh_like(2400, rng)
    B[1500:1600] = B[100:200]                       # exact duplicates
    B[1600:1700] = B[200:300] + 1e-6                # near-duplicate pairs
    for c in range(20):                             # 20 clusters of 12, rows 32 apart
        B[1700 + c:1700 + c + 32 * 12:32] = B[300 + c] + 1e-7 * rng.random((12, D), dtype=np.float32)
    A = np.concatenate([B[100:200], B[200:300] + 3e-7, B[300:320] + 2e-7, fpfh_like(500, rng)])
    nn, d, fb = _check_same(ctx, A, B, precision)
    assert np.array_equal(nn[:100], np.arange(100, 200))
    assert fb >= 20  # the clustered queries cannot be certified in BF16


@gpu
@pytest.mark.parametrize("precision", [1, 2])
def test_tc_match_real_fpfh_vs_oracle(ctx, real_feats, precision):
    FP, FQ = real_feats
    nn, d, fb = _check_same(ctx, FP, FQ, precision)
    nn_ref, d1, d2 = oracle.match(FP.astype(np.float64), FQ.astype(np.float64))
    sure = (d2 - d1) > 1e-5
    assert sure.mean() > 0.5
    assert np.array_equal(nn[sure], nn_ref[sure])
    if precision == 1:  # the hi/lo split certifies nearly every real query
        assert fb < 0.1 * len(FP), fb


@gpu
@pytest.mark.parametrize("precision", [1, 2])
def test_tc_register_pair_identical(ctx, precision):
    import paper_1801_01572_gb300 as lsr
    p = make_pair(0, 0)
    prm = lsr.default_params()
    prm.n_hypotheses = 400_000
    prm.seed = p.seed
    c32 = lsr.Context(0, prm)
    prm.match_precision = precision
    c16 = lsr.Context(0, prm)
    try:
        r32 = c32.register_pair(p.P, p.Q)
        r16 = c16.register_pair(p.P, p.Q)
    finally:
        c32.close()
        c16.close()
    assert np.array_equal(r16.T, r32.T)
    assert r16.inliers == r32.inliers and r16.survivors == r32.survivors
    assert r16.match_fallbacks >= 0


@gpu
@pytest.mark.parametrize("tile", [1, 2])
@pytest.mark.parametrize("precision", [1, 2])
def test_tc_tile_shapes_equal_fp32(tile, precision):
    """Both tile shapes (128 or 256 queries per unit) return the FP32
    matcher's indices and distance bits, with ragged query units and database
    tiles, an odd number of 128-row tiles and a single row."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1801_01572_gb300 as lsr
    with lsr.Context(0, match_tile=tile) as c:
        for nP, nQ in [(1, 1), (255, 129), (257, 257), (130, 385), (1000, 3001), (3000, 1000)]:
            rng = np.random.default_rng(nP + 17 * nQ + 1000 * tile)
            A, B = fpfh_like(nP, rng), fpfh_like(nQ, rng)
            nn32, d32, _ = c.stage_match(A, B, precision=0)
            nn, d, _ = c.stage_match(A, B, precision=precision)
            assert np.array_equal(nn, nn32), (nP, nQ)
            assert np.array_equal(d.view(np.uint32), d32.view(np.uint32)), (nP, nQ)
