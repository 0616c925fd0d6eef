"""Config 2, the batched workload: 256 room-fragment pairs of 10k-120k points
per cloud (overlap 30-80 %), registered with lsr_register_batch.

Parity: the three smallest pairs of the 256 (where a complete FP64 oracle
registration, all 4M hypotheses, runs in test time) registered as one batch
through the concurrent, graph-captured, BF16 tensor-core path must agree with
the oracle's registration within 0.05 deg / 0.5 mm.
"""
import numpy as np
import pytest

import oracle
from synth import make_pair, pose_error
from synth.fragments import CONFIGS, seed_of

gpu = pytest.mark.gpu


def config2_sizes(n=256):
    """(n_p, n_q) of every config-2 pair, drawn as the generator draws them."""
    lo, hi = CONFIGS[2]["n_range"]
    out = []
    for i in range(n):
        rng = np.random.default_rng(seed_of(2, i))
        out.append((int(rng.integers(lo, hi + 1)), int(rng.integers(lo, hi + 1))))
    return out


def test_config2_sizes_follow_the_generator():
    sizes = config2_sizes(8)
    for i, (a, b) in enumerate(sizes):
        p = make_pair(2, i) if i < 2 else None
        if p is not None:
            assert (len(p.P), len(p.Q)) == (a, b)
        assert 10000 <= a <= 120000 and 10000 <= b <= 120000


@gpu
def test_config2_smallest_pairs_batch_matches_oracle():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1801_01572_gb300 as lsr
    sizes = config2_sizes()
    idx = [int(i) for i in np.argsort([a + b for a, b in sizes], kind="stable")[:3]]
    pairs = [make_pair(2, i) for i in idx]
    P = [torch.from_numpy(p.P).cuda() for p in pairs]
    Q = [torch.from_numpy(p.Q).cuda() for p in pairs]
    vp = np.concatenate([np.concatenate([p.vpP, p.vpQ]) for p in pairs]).astype(np.float32)
    with lsr.Context(0, match_precision=lsr.MATCH_BF16, batch_streams=3, batch_graph=1) as ctx:
        got = ctx.register_batch(P, Q, vp)
    for k, (p, r) in enumerate(zip(pairs, got)):
        ref = oracle.register(p.P, p.Q, p.vpP, p.vpQ, seed=0, pair_id=k)
        assert r.status == ref["status"]
        if r.status == 0:
            ang, tr = pose_error(r.T, ref["T"])
            assert ang < 0.05 and tr < 5e-4, (k, ang, tr)
