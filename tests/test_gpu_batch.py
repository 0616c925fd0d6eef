"""Batched registration (lsr_register_batch): pairs of uneven size run
concurrently on several streams, optionally captured once as a CUDA graph and
replayed, with the tensor-core tile shape and the stream count picked by the
autotuner. Every variant must give exactly the results of registering each
pair on its own (the pipeline is deterministic), and a replayed graph must
give them again.
"""
import numpy as np
import pytest

from synth import make_pair

gpu = pytest.mark.gpu


@pytest.fixture(scope="module")
def batch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    # the batch generator's room scenes with uneven sizes, scaled down for test time
    rng = np.random.default_rng(2)
    pairs = [make_pair(2, i, n_p=int(rng.integers(6000, 30000)), n_q=int(rng.integers(6000, 30000)))
             for i in range(10)]
    P = [torch.from_numpy(p.P).cuda() for p in pairs]
    Q = [torch.from_numpy(p.Q).cuda() for p in pairs]
    return pairs, P, Q


def _single(lsr, pairs, P, Q, **kw):
    out = []
    with lsr.Context(0, **kw) as ctx:
        for i, p in enumerate(pairs):
            prm = ctx.params
            prm.pair_id = i
            ctx.set_params(prm)
            out.append(ctx.register_pair(P[i], Q[i], p.vpP, p.vpQ))
    return out


def _same(a, b):
    assert len(a) == len(b)
    for x, y in zip(a, b):
        assert np.array_equal(x.T, y.T) and x.inliers == y.inliers and x.survivors == y.survivors
        assert x.status == y.status


@gpu
@pytest.mark.parametrize("precision", [0, 1])
def test_batch_streams_graph_and_autotune_equal_single(batch, precision):
    import paper_1801_01572_gb300 as lsr
    pairs, P, Q = batch
    vp = np.concatenate([np.concatenate([p.vpP, p.vpQ]) for p in pairs]).astype(np.float32)
    common = dict(n_hypotheses=500_000, match_precision=precision, match_tile=1 if precision else 0)
    ref = _single(lsr, pairs, P, Q, **common)
    assert sum(r.status == 0 for r in ref) >= 8
    for kw in (dict(batch_streams=4), dict(batch_streams=3, batch_graph=1), dict(batch_streams=0)):
        with lsr.Context(0, **common, **kw) as ctx:
            got = ctx.register_batch(P, Q, vp)
            _same(got, ref)
            if kw.get("batch_graph"):
                l0 = lsr.launch_count()
                again = ctx.register_batch(P, Q, vp)  # replay of the captured graph
                assert lsr.launch_count() - l0 > 100 * len(pairs)
                _same(again, ref)
    # (no comparison with the generator's pose here: for small low-overlap
    # fragments the optimum of the robust objective itself lies centimetres
    # from it, the FP64 oracle's included; test_gpu_config2.py checks parity)


@gpu
def test_autotuned_tile_shapes_give_identical_matches(batch):
    """Both tensor-core tile shapes (one or two query tiles per CTA) give the
    FP32 matcher's correspondences."""
    import paper_1801_01572_gb300 as lsr
    pairs, P, Q = batch
    rng = np.random.default_rng(9)
    g = rng.gamma(0.35, 1.0, size=(3000, 3, 11))
    A = (g / g.sum(2, keepdims=True)).reshape(-1, 33).astype(np.float32)
    g = rng.gamma(0.35, 1.0, size=(5000, 3, 11))
    B = (g / g.sum(2, keepdims=True)).reshape(-1, 33).astype(np.float32)
    with lsr.Context(0) as ctx:
        nn32, d32, _ = ctx.stage_match(A, B, precision=0)
    for tile in (1, 2):
        with lsr.Context(0, match_tile=tile) as ctx:
            nn, d, _ = ctx.stage_match(A, B, precision=1)
        assert np.array_equal(nn, nn32) and np.array_equal(d.view(np.uint32), d32.view(np.uint32))
