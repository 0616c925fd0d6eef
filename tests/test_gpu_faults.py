"""Failure paths, made on the host so that no GPU faults or hangs.

- An injected device-allocation failure returns LSR_E_OOM, and the same
  context then registers normally.
- An injected stall of the tensor-core matcher (its producer issues no copy
  and no MMA, so nothing ever completes the epilogue's first barrier) makes
  that bounded wait run out after 20 ms: the kernel releases its tensor memory
  and returns, the call returns LSR_E_TIMEOUT, and the next call on the same
  context gives the undisturbed result.
"""
import numpy as np
import pytest

from synth import make_pair

gpu = pytest.mark.gpu


@pytest.fixture(scope="module")
def lsr():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1801_01572_gb300 as m
    return m


@pytest.fixture(scope="module")
def pair():
    return make_pair(0, 0, n_p=3000, n_q=3000)


@gpu
def test_injected_allocation_failure_returns_oom_and_context_recovers(lsr, pair):
    with lsr.Context(0, n_hypotheses=200_000) as ctx:
        ctx.debug_inject(lsr.INJECT_ALLOC, 1)
        with pytest.raises(lsr.LsrError) as e:
            ctx.register_pair(pair.P, pair.Q, pair.vpP, pair.vpQ)
        assert e.value.code == lsr.LSR_E_OOM
        assert ctx.workspace_bytes() == 0
        r = ctx.register_pair(pair.P, pair.Q, pair.vpP, pair.vpQ)
        assert r.status == lsr.STATUS_ALIGNED
    with lsr.Context(0, n_hypotheses=200_000) as ref:
        r0 = ref.register_pair(pair.P, pair.Q, pair.vpP, pair.vpQ)
    assert np.array_equal(r.T, r0.T) and r.inliers == r0.inliers


@gpu
def test_injected_allocation_failure_in_a_batch(lsr, pair):
    with lsr.Context(0, n_hypotheses=100_000, batch_streams=2) as ctx:
        ctx.debug_inject(lsr.INJECT_ALLOC, 1)
        with pytest.raises(lsr.LsrError) as e:
            ctx.register_batch([pair.P, pair.P], [pair.Q, pair.Q])
        assert e.value.code == lsr.LSR_E_OOM
        out = ctx.register_batch([pair.P, pair.P], [pair.Q, pair.Q])
    with lsr.Context(0, n_hypotheses=100_000, batch_streams=2) as ref:
        want = ref.register_batch([pair.P, pair.P], [pair.Q, pair.Q])
    for o, w in zip(out, want):
        assert o.status == w.status and np.array_equal(o.T, w.T) and o.inliers == w.inliers


@gpu
@pytest.mark.parametrize("mode", ["pair", "stage"])
def test_injected_matcher_stall_times_out_and_context_recovers(lsr, pair, mode):
    import time
    with lsr.Context(0, n_hypotheses=200_000, match_precision=lsr.MATCH_BF16) as ctx:
        good = ctx.register_pair(pair.P, pair.Q, pair.vpP, pair.vpQ)
        F = np.random.default_rng(3).uniform(0, 1, (3000, 33)).astype(np.float32)
        nn0, d0, _ = ctx.stage_match(F, F[::-1].copy(), lsr.MATCH_BF16)
        ctx.debug_inject(lsr.INJECT_MATCH_STALL, 1)
        t0 = time.perf_counter()
        with pytest.raises(lsr.LsrError) as e:
            if mode == "pair":
                ctx.register_pair(pair.P, pair.Q, pair.vpP, pair.vpQ)
            else:
                ctx.stage_match(F, F[::-1].copy(), lsr.MATCH_BF16)
        took = time.perf_counter() - t0
        assert e.value.code == lsr.LSR_E_TIMEOUT
        assert took < 1.5  # the 20 ms limit, not the normal 2 s one
        again = ctx.register_pair(pair.P, pair.Q, pair.vpP, pair.vpQ)
        assert np.array_equal(again.T, good.T) and again.inliers == good.inliers
        nn1, d1, _ = ctx.stage_match(F, F[::-1].copy(), lsr.MATCH_BF16)
        assert np.array_equal(nn0, nn1) and np.array_equal(d0, d1)


@gpu
def test_injection_arguments_are_checked():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1801_01572_gb300 as lsr
    with lsr.Context(0) as ctx:
        with pytest.raises(lsr.LsrError) as e:
            ctx.debug_inject(7, 1)
        assert e.value.code == lsr.LSR_E_ARG
        with pytest.raises(lsr.LsrError) as e:
            ctx.debug_inject(lsr.INJECT_ALLOC, -1)
        assert e.value.code == lsr.LSR_E_ARG
        ctx.debug_inject(lsr.INJECT_NONE, 0)
