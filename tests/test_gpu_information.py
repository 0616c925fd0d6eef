"""Information matrix of a verified pair (loop verification, eq. (5)-(6))
through lsr_information_matrix, against the FP64 oracle.

The correspondence sets agree except for points whose NN distance lies within
a band of eps (FP32 and FP64 may decide those either way); each such point
changes an entry of Lambda by at most max(|p|^2, 1). Everything else agrees to
the FP32 rounding of the moved points and the per-thread sums (sums about the
centre of Q's box, FP64 across blocks): 1e-5 of the largest entry.
"""
import numpy as np
import pytest
from scipy.spatial.transform import Rotation

import oracle
from synth import make_pair

gpu = pytest.mark.gpu
EPS = 0.05


@pytest.fixture(scope="module")
def ctx():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1801_01572_gb300 as lsr
    c = lsr.Context(0)
    yield c
    c.close()


def _pose(p, perturb):
    T = p.T.copy()
    if perturb:
        rng = np.random.default_rng(11)
        dT = np.eye(4)
        dT[:3, :3] = Rotation.from_rotvec(rng.normal(0, 0.02, 3)).as_matrix()
        dT[:3, 3] = rng.normal(0, 0.01, 3)
        T = dT @ T
    return T


@gpu
@pytest.mark.parametrize("config, perturb", [(0, False), (0, True), (1, False), (1, True)])
def test_information_matrix_matches_oracle(ctx, config, perturb):
    p = make_pair(config, 0)
    T = _pose(p, perturb)
    info, n = ctx.information_matrix(p.P, p.Q, T, EPS)
    ref, n_ref, namb, amb_max = oracle.information(p.P, p.Q, T, EPS, band=2e-5)
    assert n_ref > 0.2 * len(p.P)
    assert abs(n - n_ref) <= namb, (n, n_ref, namb)
    tol = namb * max(amb_max, 1.0) + 1e-5 * np.abs(ref).max()
    assert np.abs(info - ref).max() <= tol, (np.abs(info - ref).max(), tol)
    assert np.array_equal(info, info.T)
    assert np.array_equal(info[3:, 3:], n * np.eye(3))


@gpu
def test_information_matrix_host_and_device_inputs_agree(ctx):
    torch = pytest.importorskip("torch")
    p = make_pair(0, 2)
    a, na = ctx.information_matrix(p.P, p.Q, p.T, EPS)
    b, nb = ctx.information_matrix(torch.from_numpy(p.P).cuda(), torch.from_numpy(p.Q).cuda(), p.T, EPS)
    assert na == nb and np.array_equal(a, b)


@gpu
def test_information_matrix_without_correspondences(ctx):
    """A pose that moves P far from Q: no correspondence, a zero matrix."""
    p = make_pair(0, 0)
    T = p.T.copy()
    T[0, 3] += 100.0
    info, n = ctx.information_matrix(p.P, p.Q, T, EPS)
    assert n == 0 and np.array_equal(info, np.zeros((6, 6)))
