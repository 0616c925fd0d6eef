"""Pins of the oracle's voxel downsampling (Algorithm 1, first line): one point
per occupied voxel (edge leaf, aligned to the origin), the mean of its points,
ordered by (k_z, k_y, k_x). Pinned by brute-force grouping with a dictionary,
a lattice of voxel centres (comes back unchanged, sorted), a whole-leaf shift
(moves every output point by exactly that shift), and points on voxel faces
(a face belongs to the voxel above it)."""
import numpy as np

import oracle
from synth import make_pair


def test_voxel_brute_force_grouping():
    rng = np.random.default_rng(1)
    P = rng.uniform(-0.3, 0.3, (3000, 3))
    leaf = 0.05
    out, cnt = oracle.voxel_downsample(P, leaf)
    groups = {}
    for p in P:
        groups.setdefault(tuple(int(v) for v in np.floor(p / leaf)), []).append(p)
    keys = sorted(groups, key=lambda k: (k[2], k[1], k[0]))
    assert len(out) == len(keys) and cnt.sum() == len(P)
    for o, c, k in zip(out, cnt, keys):
        assert c == len(groups[k]) and np.allclose(o, np.mean(groups[k], axis=0), rtol=0, atol=1e-15)


def test_voxel_lattice_and_shift():
    leaf = 0.05
    g = np.stack(np.meshgrid(np.arange(-3, 4), np.arange(0, 5), np.arange(-2, 2), indexing="ij"), -1).reshape(-1, 3)
    P = (g + 0.5) * leaf
    out, cnt = oracle.voxel_downsample(P[::-1], leaf)
    assert np.all(cnt == 1)
    exp = P[np.lexsort((P[:, 0], P[:, 1], P[:, 2]))]
    assert np.allclose(out, exp, rtol=0, atol=1e-15)
    p = make_pair(0, 0).P.astype(np.float64)
    a, ca = oracle.voxel_downsample(p, leaf)
    b, cb = oracle.voxel_downsample(p + np.array([3, -2, 5]) * leaf, leaf)
    assert np.array_equal(ca, cb) and np.allclose(b - a, np.array([3, -2, 5]) * leaf, rtol=0, atol=1e-12)


def test_voxel_faces_belong_to_the_upper_voxel():
    leaf = 0.25  # exact in binary, so the face coordinates are exact
    P = np.array([[0.25, 0.1, 0.1], [0.2, 0.1, 0.1], [0.0, 0.0, 0.0], [-1e-17, 0.0, 0.0]])
    out, cnt = oracle.voxel_downsample(P, leaf)
    # (-1e-17 rounds to a key of -1), the origin and (0.2, ...) share voxel (0,0,0); 0.25 starts voxel 1
    assert cnt.tolist() == [1, 2, 1]
    assert np.allclose(out[1], [0.1, 0.05, 0.05]) and np.allclose(out[2], [0.25, 0.1, 0.1])
