"""Voxel downsampling (Algorithm 1, first line) through lsr_voxel_downsample
against the FP64 oracle: the same occupied voxels in the same order (voxel
keys are computed in FP64 on both sides, so they agree exactly), and means
within the FP32 rounding of the output (the device sums offsets as 64-bit
integers of leaf / 2^36)."""
import numpy as np
import pytest

import oracle
from synth import make_pair

gpu = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1801_01572_gb300 as lsr
    c = lsr.Context(0)
    yield c
    c.close()


@gpu
@pytest.mark.parametrize("config, leaf", [(0, 0.05), (1, 0.05), (1, 0.0137), (0, 0.25)])
def test_voxel_downsample_matches_oracle(ctx, config, leaf):
    P = make_pair(config, 0).P
    out = ctx.voxel_downsample(P, leaf)
    ref, cnt = oracle.voxel_downsample(P, leaf)
    assert len(out) == len(ref) and cnt.sum() == len(P)
    assert np.abs(out - ref).max() <= 2e-7 * max(1.0, np.abs(ref).max()), np.abs(out - ref).max()


@gpu
def test_voxel_downsample_order_independent(ctx):
    P = make_pair(1, 0).P
    perm = np.random.default_rng(0).permutation(len(P))
    a = ctx.voxel_downsample(P, 0.05)
    b = ctx.voxel_downsample(P[perm], 0.05)
    assert np.array_equal(a, b)


@gpu
def test_voxel_downsample_degenerate_inputs(ctx):
    # one point: itself; all points in one voxel: their mean; a lattice of voxel centres: unchanged, sorted
    one = np.array([[0.1234, -0.5, 2.0]], np.float32)
    assert np.allclose(ctx.voxel_downsample(one, 0.05), one, rtol=0, atol=1e-7)
    same = np.random.default_rng(3).uniform(0.0, 0.049, (1000, 3)).astype(np.float32)
    out = ctx.voxel_downsample(same, 0.05)
    assert out.shape == (1, 3) and np.allclose(out[0], same.astype(np.float64).mean(0), rtol=0, atol=1e-7)
    g = np.stack(np.meshgrid(np.arange(3), np.arange(2), np.arange(2), indexing="ij"), -1).reshape(-1, 3)
    P = ((g + 0.5) * 0.25).astype(np.float32)
    ref, _ = oracle.voxel_downsample(P[::-1], 0.25)
    assert np.allclose(ctx.voxel_downsample(P[::-1], 0.25), ref, rtol=0, atol=1e-7)
