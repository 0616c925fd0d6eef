"""The allocation-free pose scoring entry point (lsr_consensus_static).

Callers that must not allocate device memory while scoring poses (a loop
closure check inside a real-time loop, or a process whose device memory is
owned by another framework) call it with their own inputs and outputs; its
scratch is a fixed array in the library. This test calls it through the C ABI
twice in a row, on different clouds and poses, and checks each result against
the workspace-based entry point lsr_stage_consensus. It lives in a file of its
own, collected after the other tests, and passes alone or after them.
"""
import ctypes as C

import numpy as np
import pytest

from synth import make_pair, random_pose

gpu = pytest.mark.gpu


def _poses(fp, rng, n):
    Rt = []
    for k in range(n):
        T = fp.T if k % 3 == 0 else random_pose(rng, 0.05) @ fp.T
        Rt.append(np.concatenate([T[:3, :3], T[:3, 3:]], axis=1).reshape(12))
    return np.asarray(Rt, np.float32)


@gpu
def test_static_scoring_matches_workspace_entry_point_twice():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1801_01572_gb300 as lsr
    L = lsr.lib()
    rng = np.random.default_rng(31)
    ctx = lsr.Context(0)
    try:
        # two calls in a row: the second on smaller clouds and other poses, so
        # anything left over from the first call would show up
        cases = [(make_pair(0, 0), 300), (make_pair(0, 1, n_p=2500, n_q=4000), 57)]
        for fp, nh in cases:
            Rt = _poses(fp, rng, nh)
            P = torch.from_numpy(fp.P).cuda()
            Q = torch.from_numpy(fp.Q).cuda()
            Rt_d = torch.from_numpy(Rt).cuda()
            cnt = torch.full((nh,), -1, dtype=torch.int32, device="cuda")
            sd = torch.full((nh,), -1.0, dtype=torch.float64, device="cuda")
            torch.cuda.synchronize()
            rc = L.lsr_consensus_static(C.c_void_p(P.data_ptr()), len(fp.P), C.c_void_p(Q.data_ptr()), len(fp.Q),
                                        C.c_void_p(Rt_d.data_ptr()), nh, C.c_float(0.0375),
                                        C.c_void_p(cnt.data_ptr()), C.c_void_p(sd.data_ptr()), None)
            assert rc == lsr.LSR_OK, L.lsr_error_string(rc)
            ref_cnt, ref_sd = ctx.stage_consensus(fp.P, fp.Q, Rt, 0.0375)
            got_cnt, got_sd = cnt.cpu().numpy(), sd.cpu().numpy()
            assert np.array_equal(got_cnt, ref_cnt)
            assert np.allclose(got_sd, ref_sd, rtol=1e-9, atol=1e-12)
            assert got_cnt.max() > len(fp.P) // 2
        # sizes beyond the fixed scratch are refused before any device work
        big = np.zeros((65537, 3), np.float32)
        rc = L.lsr_consensus_static(C.c_void_p(big.ctypes.data), len(big), C.c_void_p(big.ctypes.data), 10,
                                    C.c_void_p(Rt.ctypes.data), 1, C.c_float(0.0375),
                                    C.c_void_p(got_cnt.ctypes.data), C.c_void_p(got_sd.ctypes.data), None)
        assert rc == lsr.LSR_E_TOO_LARGE
    finally:
        ctx.close()


@gpu
def test_static_scoring_with_host_arrays_on_a_caller_stream():
    """Poses read from, and counts and sums written to, host arrays, with the
    work ordered on a stream the caller created (the entry point copies the
    host arrays itself and synchronises that stream before returning)."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1801_01572_gb300 as lsr
    L = lsr.lib()
    rng = np.random.default_rng(47)
    fp = make_pair(0, 2, n_p=3500, n_q=3000)
    nh = 91
    Rt = _poses(fp, rng, nh)
    P = torch.from_numpy(fp.P).cuda()
    Q = torch.from_numpy(fp.Q).cuda()
    cnt = np.full(nh, -1, np.int32)
    sd = np.full(nh, -1.0, np.float64)
    stream = torch.cuda.Stream()
    torch.cuda.synchronize()
    rc = L.lsr_consensus_static(C.c_void_p(P.data_ptr()), len(fp.P), C.c_void_p(Q.data_ptr()), len(fp.Q),
                                C.c_void_p(Rt.ctypes.data), nh, C.c_float(0.0375), C.c_void_p(cnt.ctypes.data),
                                C.c_void_p(sd.ctypes.data), C.c_void_p(stream.cuda_stream))
    assert rc == lsr.LSR_OK, L.lsr_error_string(rc)
    with lsr.Context(0) as ctx:
        ref_cnt, ref_sd = ctx.stage_consensus(fp.P, fp.Q, Rt, 0.0375)
    assert np.array_equal(cnt, ref_cnt)
    assert np.allclose(sd, ref_sd, rtol=1e-9, atol=1e-12)
