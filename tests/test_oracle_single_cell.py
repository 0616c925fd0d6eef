"""Pins of the oracle's single-cell grid lookup (eq. (1), the O(1) search the
paper uses as its speed argument): it can only miss, never invent, an inlier
(its distance is that of a real Q point, so the exact NN is at least as close);
it equals the exact NN whenever the exact NN lies in the query's cell (brute
force); on a lattice of cell centres every query within the cell finds its
centre; a query just across a face from its only neighbour finds nothing."""
import numpy as np

import oracle
from synth import make_pair


def test_single_cell_never_beats_exact_and_matches_it_inside_the_cell():
    p = make_pair(0, 0)
    Q = p.Q.astype(np.float64)
    X = p.P.astype(np.float64) @ p.T[:3, :3].T + p.T[:3, 3]
    h, eps = 0.05, 0.05
    nn1, d1 = oracle.nn_single_cell(Q, X, h)
    nne, de = oracle.nn_within(Q, X, 10.0, brute=True)
    assert np.all(de <= d1)
    same = (nn1 >= 0)
    c = Q.mean(axis=0)
    k_x = np.floor((X - c) / h)
    k_nn = np.floor((Q[nne] - c) / h)
    inside = np.all(k_x == k_nn, axis=1)
    assert np.array_equal(nn1[inside], nne[inside]) and np.allclose(d1[inside], de[inside], rtol=0, atol=1e-15)
    assert np.all(same[inside])
    # recall of the eps inlier test is below one here (the speed mode is approximate)
    exact, approx = (de < eps * eps).sum(), (d1 < eps * eps).sum()
    assert approx <= exact and approx > 0.3 * exact


def test_single_cell_lattice_and_faces():
    h = 0.25
    g = np.stack(np.meshgrid(np.arange(4), np.arange(4), np.arange(2), indexing="ij"), -1).reshape(-1, 3)
    Q = (g + 0.5) * h  # cell centres; even counts put the centroid on a lattice corner, so the search cells are these
    rng = np.random.default_rng(2)
    X = Q + rng.uniform(-0.4, 0.4, Q.shape) * h
    nn, d2 = oracle.nn_single_cell(Q, X, h)
    assert np.array_equal(nn, np.arange(len(Q)))
    assert np.allclose(d2, ((X - Q) ** 2).sum(1))
    # one Q point (its own centroid, so it sits on the lower corner of its cell): a
    # query 1 cm below it is in the cell beneath and finds nothing; 0.7 cells above, it does
    Q1 = np.array([[0.1, 0.1, 0.1]])
    nn, _ = oracle.nn_single_cell(Q1, np.array([[0.1, 0.1, 0.09], [0.1, 0.1, 0.1 + 0.7 * h]]), h)
    assert nn.tolist() == [-1, 0]
