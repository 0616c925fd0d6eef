"""Dense model correction (eq. (7)) through lsr_surfel_correct against the
FP64 oracle, on a seeded room-sized surfel map and a keyframe loop with a
drift correction growing to 1.5 deg / 6 cm.

Which keyframes observe a surfel is decided in FP32 on the device and in FP64
in the oracle. The oracle reports the surfels for which some keyframe of their
time window decides visibility within 1e-5 m of a depth limit or 1e-3 pixels of
an image edge (the FP32 transform and projection err by less); only those may
differ. Every other surfel is kept or removed by both, and where kept its
position and normal agree to FP32 rounding (1e-5).
"""
import numpy as np
import pytest

import oracle
from synth.surfels import make_surfels

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


@pytest.fixture(scope="module")
def smap():
    return make_surfels(400_000, 200, seed=9)


@gpu
def test_surfel_correction_matches_oracle(ctx, smap):
    S = smap
    p, n, keep, kept = ctx.surfel_correct(S.pos, S.nrm, S.t0, S.tu, S.T_old, S.T_new, S.t_kf, S.cam)
    pr, nr, keepr, border = oracle.surfel_correct(S.pos, S.nrm, S.t0, S.tu, S.T_old, S.T_new, S.t_kf, S.cam,
                                                  band=(1e-5, 1e-3))
    keep = keep.astype(bool)
    assert kept == keep.sum() and 0.1 < keep.mean() < 0.9
    assert border.mean() < 1e-3
    assert np.array_equal(keep[~border], keepr[~border])
    both = keep & keepr & ~border
    ep = np.linalg.norm(p[both] - pr[both], axis=1)
    en = np.linalg.norm(n[both] - nr[both], axis=1)
    assert ep.max() <= 1e-5 and en.max() <= 1e-5, (ep.max(), en.max())
    assert np.median(ep) < 2e-6
    # removed surfels come back unchanged
    assert np.array_equal(p[~keep], S.pos[~keep]) and np.array_equal(n[~keep], S.nrm[~keep])


@gpu
def test_surfel_correction_device_inputs_equal_host(ctx, smap):
    torch = pytest.importorskip("torch")
    S = smap
    a = ctx.surfel_correct(S.pos, S.nrm, S.t0, S.tu, S.T_old, S.T_new, S.t_kf, S.cam)
    d = [torch.from_numpy(x).cuda() for x in (S.pos, S.nrm, S.t0, S.tu)]
    b = ctx.surfel_correct(*d, S.T_old, S.T_new, S.t_kf, S.cam)
    assert a[3] == b[3]
    for x, y in zip(a[:3], b[:3]):
        assert np.array_equal(x, y.cpu().numpy())


@gpu
def test_surfels_outside_every_window_are_removed_unchanged(ctx, smap):
    S = smap
    n = 1000
    t0 = np.full(n, -10.0, np.float32)
    tu = np.full(n, -5.0, np.float32)  # before the first keyframe
    p, nr, keep, kept = ctx.surfel_correct(S.pos[:n], S.nrm[:n], t0, tu, S.T_old, S.T_new, S.t_kf, S.cam)
    assert kept == 0 and not keep.any()
    assert np.array_equal(p, S.pos[:n]) and np.array_equal(nr, S.nrm[:n])
