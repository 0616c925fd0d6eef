"""The exact FP32 matcher's projection window (Algorithm 1, feature
pre-matching): the search visits only database tiles whose projection on one
axis lies within reach of a query's current best, so these cases aim at what
could make it skip the true nearest row: ragged and one-row sets, a database
of identical rows (no principal axis), duplicate rows far apart in index
(ties go to the smaller index whatever the scan order), queries far outside
the database (the window must grow to the ends), a database whose rows differ
only across the axis, and permuted inputs (the result must follow the
permutation, as the bucket order inside the matcher does not).

Indices are compared with the FP64 oracle wherever its runner-up is more than
1e-5 behind the nearest; elsewhere the GPU's row must be a near-tie of the
oracle's minimum. The BF16 tensor-core path (an independent exact search)
must return the same indices and distance bits.
"""
import numpy as np
import pytest

import oracle

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


def fpfh_like(n, rng):
    g = rng.gamma(0.35, 1.0, size=(n, 3, 11))
    g /= g.sum(2, keepdims=True)
    return g.reshape(n, D).astype(np.float32)


def check_oracle(nn, d, A, B):
    nn_ref, d1, d2 = oracle.match(A.astype(np.float64), B.astype(np.float64))
    sure = (d2 - d1) > 1e-5
    assert np.array_equal(nn[sure], nn_ref[sure])
    D2 = ((A[~sure].astype(np.float64) - B[nn[~sure]].astype(np.float64)) ** 2).sum(1)
    assert np.all(D2 - d1[~sure] <= 1e-5)
    assert np.allclose(d, d1, atol=2e-6, rtol=1e-5)


def check_bf16(ctx, nn, d, A, B):
    nn16, d16, _ = ctx.stage_match(A, B, precision=1)
    assert np.array_equal(nn16, nn)
    assert np.array_equal(d16.view(np.uint32), d.view(np.uint32))


@gpu
@pytest.mark.parametrize("nP,nQ", [(1, 1), (1, 63), (1, 64), (1, 65), (129, 1), (300, 7), (127, 129), (5000, 130),
                                   (2000, 6000)])
def test_window_sizes(ctx, nP, nQ):
    rng = np.random.default_rng(7 * nP + nQ)
    A, B = fpfh_like(nP, rng), fpfh_like(nQ, rng)
    nn, d, _ = ctx.stage_match(A, B)
    check_oracle(nn, d, A, B)
    if nP * nQ > 1:
        check_bf16(ctx, nn, d, A, B)


@gpu
def test_window_identical_database_rows(ctx):
    rng = np.random.default_rng(1)
    B = np.repeat(fpfh_like(1, rng), 700, axis=0)
    A = fpfh_like(400, rng)
    nn, d, _ = ctx.stage_match(A, B)
    assert np.all(nn == 0)
    ref = ((A.astype(np.float64) - B[0].astype(np.float64)) ** 2).sum(1)
    assert np.allclose(d, ref, rtol=1e-5, atol=1e-7)
    # queries equal to the row: distance exactly 0, still the first index
    nn, d, _ = ctx.stage_match(B[:50], B)
    assert np.all(nn == 0) and np.all(d == 0)


@gpu
def test_window_duplicates_far_apart(ctx):
    rng = np.random.default_rng(2)
    B = fpfh_like(9000, rng)
    src = rng.choice(3000, 400, replace=False)
    dst = 6000 + rng.choice(3000, 400, replace=False)
    B[dst] = B[src]
    A = B[dst] + np.float32(0)
    nn, d, _ = ctx.stage_match(A, B)
    assert np.array_equal(nn, src) and np.all(d == 0)


@gpu
def test_window_far_queries(ctx):
    rng = np.random.default_rng(3)
    B = fpfh_like(4000, rng)
    A = np.concatenate([fpfh_like(300, rng), 5.0 * fpfh_like(100, rng), -3.0 * fpfh_like(100, rng),
                        np.full((20, D), 40.0, np.float32)])
    nn, d, _ = ctx.stage_match(A, B)
    check_oracle(nn, d, A, B)
    check_bf16(ctx, nn, d, A, B)


@gpu
def test_window_rows_differ_across_the_axis(ctx):
    """Two clusters far apart along one direction, and inside each cluster rows
    that differ only in other bins: the principal axis separates the clusters
    and says nothing about the rows within one."""
    rng = np.random.default_rng(4)
    base = fpfh_like(2, rng)
    B = np.repeat(base, 3000, axis=0)
    B += (1e-3 * rng.standard_normal(B.shape)).astype(np.float32) * (np.arange(D) % 3 == 1)
    A = B[rng.choice(len(B), 500, replace=False)] + (2e-4 * rng.standard_normal((500, D))).astype(np.float32)
    nn, d, _ = ctx.stage_match(A, B)
    check_oracle(nn, d, A, B)
    check_bf16(ctx, nn, d, A, B)


@gpu
def test_window_permutation_and_determinism(ctx):
    rng = np.random.default_rng(5)
    A, B = fpfh_like(3000, rng), fpfh_like(5000, rng)
    nn, d, _ = ctx.stage_match(A, B)
    nn2, d2, _ = ctx.stage_match(A, B)
    assert np.array_equal(nn, nn2) and np.array_equal(d.view(np.uint32), d2.view(np.uint32))
    pa, pb = rng.permutation(len(A)), rng.permutation(len(B))
    nnp, dp, _ = ctx.stage_match(A[pa], B[pb])
    # no exact ties among random rows: the nearest row is unique
    assert np.array_equal(pb[nnp], nn[pa])
    assert np.array_equal(dp.view(np.uint32), d[pa].view(np.uint32))
