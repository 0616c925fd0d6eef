"""Pins of the oracle's dense model correction (eq. (7)).

p' = (1/k) sum_{f in F} T_f_new T_f_old^-1 p and n' = normalize((1/k) sum R_f_new
R_f_old^-1 n) over the keyframes F with t0 < t_f < tu that observe the surfel
(in front of the camera, within the maximum depth, inside the image); k = 0
removes it. Pinned by: no correction changes nothing; one correction shared by
every keyframe moves every kept surfel by exactly that motion; hand-built
single-camera cases for each visibility and time-window condition; and the
average of two pure translations.
"""
import numpy as np
from scipy.spatial.transform import Rotation

import oracle
from synth.surfels import CAM, make_surfels


def _run(S, T_new=None):
    return oracle.surfel_correct(S.pos, S.nrm, S.t0, S.tu, S.T_old, S.T_new if T_new is None else T_new,
                                 S.t_kf, S.cam)


def test_no_correction_changes_nothing():
    S = make_surfels(20000, 60, seed=1)
    p, n, keep = _run(S, T_new=S.T_old)
    assert 0.1 < keep.mean() < 0.9
    assert np.abs(p[keep] - S.pos[keep]).max() < 1e-9
    assert np.abs(n[keep] - S.nrm[keep]).max() < 1e-6  # the float32 input normals, renormalised


def test_shared_correction_moves_every_kept_surfel_rigidly():
    S = make_surfels(20000, 60, seed=2)
    C = np.eye(4)
    C[:3, :3] = Rotation.from_rotvec([0.01, -0.02, 0.03]).as_matrix()
    C[:3, 3] = [0.05, -0.02, 0.01]
    p, n, keep = _run(S, T_new=np.einsum("ij,fjk->fik", C, S.T_old))
    P = S.pos.astype(np.float64)
    assert np.abs(p[keep] - (P[keep] @ C[:3, :3].T + C[:3, 3])).max() < 1e-9
    N = S.nrm.astype(np.float64) @ C[:3, :3].T
    N /= np.linalg.norm(N, axis=1, keepdims=True)
    assert np.abs(n[keep] - N[keep]).max() < 1e-9


def _one(points, t0, tu, T_old, T_new, t_kf):
    pts = np.asarray(points, np.float64)
    nrm = np.tile([0.0, 0.0, -1.0], (len(pts), 1))
    return oracle.surfel_correct(pts, nrm, np.full(len(pts), t0), np.full(len(pts), tu), np.asarray(T_old),
                                 np.asarray(T_new), np.asarray(t_kf, np.float64), CAM)


def test_visibility_and_time_window():
    fx, fy, cx, cy, W, H, dmax = CAM
    I = np.eye(4)
    shift = np.eye(4)
    shift[:3, 3] = [0.1, 0.0, 0.0]
    z = 2.0
    u_in, u_out = (W - 0.5 - cx) * z / fx, (W + 0.5 - cx) * z / fx
    pts = [[0, 0, z],            # in view
           [0, 0, -1.0],         # behind the camera
           [0, 0, dmax + 0.5],   # beyond the maximum depth
           [u_in, 0, z],         # just inside the right image edge
           [u_out, 0, z]]        # just outside it
    p, _, keep = _one(pts, -1.0, 1.0, [I], [shift], [0.0])
    assert keep.tolist() == [True, False, False, True, False]
    assert np.allclose(p[0], [0.1, 0, z]) and np.allclose(p[3], [u_in + 0.1, 0, z])
    # the keyframe outside (t0, tu): nothing observes the surfel
    for t0, tu in ((0.0, 1.0), (-1.0, 0.0), (0.5, 3.0)):
        _, _, keep = _one([[0, 0, z]], t0, tu, [I], [shift], [0.0])
        assert not keep[0]


def test_average_of_two_corrections():
    I = np.eye(4)
    A, B = np.eye(4), np.eye(4)
    A[:3, 3] = [0.02, 0.0, 0.0]
    B[:3, 3] = [0.0, 0.04, 0.0]
    p, _, keep = _one([[0.1, -0.1, 1.5]], -1.0, 5.0, [I, I], [A, B], [0.0, 1.0])
    assert keep[0] and np.allclose(p[0], [0.11, -0.08, 1.5], atol=1e-12)


def test_border_report_flags_only_limit_cases():
    """The band report flags a surfel whose projection sits on an image edge
    or at the maximum depth of a keyframe in its window, and nothing else; it
    changes no result."""
    cam = np.array([525.0, 525.0, 320.0, 240.0, 640.0, 480.0, 4.0])
    T = np.eye(4)[None]  # one camera at the origin looking along +z
    z = 2.0
    x_edge = (0.0 - 320.0) * z / 525.0  # u = 0 exactly
    pos = np.array([[0.0, 0.0, z], [x_edge, 0.0, z], [0.0, 0.0, 4.0], [0.1, 0.05, 3.0]])
    nrm = np.tile([0.0, 0.0, -1.0], (4, 1))
    t0, tu, tk = np.full(4, -1.0), np.full(4, 1.0), np.zeros(1)
    p, n, keep, border = oracle.surfel_correct(pos, nrm, t0, tu, T, T, tk, cam, band=(1e-5, 1e-3))
    assert border.tolist() == [False, True, True, False]
    p2, n2, keep2 = oracle.surfel_correct(pos, nrm, t0, tu, T, T, tk, cam)
    assert np.array_equal(keep, keep2) and np.array_equal(p, p2)
    # outside the time window nothing is a border case
    _, _, _, b3 = oracle.surfel_correct(pos, nrm, np.full(4, 0.5), tu, T, T, tk, cam, band=(1e-5, 1e-3))
    assert not b3.any()
