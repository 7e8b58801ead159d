"""Pins for the oracle's warm-start pieces (CPU only): problem features and the MLP."""
import math

import numpy as np

import oracle


def test_weighted_median_closed_forms():
    # a weight above half the total decides
    f = oracle.features(np.array([[3.0], [-1.0], [8.0], [5.0]]), np.array([1.0, 0.5, 4.0, 1.0]))
    assert f[1] == 8.0
    # equal weights, odd n: the ordinary median
    rng = np.random.default_rng(1)
    x = rng.normal(size=(9, 1)) * 10
    assert oracle.features(x, np.ones(9))[1] == np.median(x[:, 0])
    # equal weights, even n: the lower of the two middle values
    x = np.array([[4.0], [1.0], [3.0], [2.0]])
    assert oracle.features(x, np.ones(4))[1] == 2.0
    # weighted mean of one point is the point; entropy 0, largest weight 1
    f = oracle.features(np.array([[7.0, -2.0]]), np.array([0.3]))
    assert np.array_equal(f, [7.0, -2.0, 7.0, -2.0, 0.0, 1.0])


def test_weighted_median_solves_problem_1_in_one_dimension():
    rng = np.random.default_rng(2)
    for _ in range(10):
        n = int(rng.integers(3, 12))
        x = rng.uniform(0, 255, (n, 1))
        w = rng.uniform(0.1, 2.0, n)
        q = oracle.features(x, w)[1]
        F = lambda t: float(np.sum(w * np.abs(t - x[:, 0])))
        # no data point gives a smaller objective (a weighted median minimises it)
        assert all(F(q) <= F(t) + 1e-12 for t in x[:, 0])


def test_entropy_and_max_weight():
    n = 441
    f = oracle.features(np.zeros((n, 3)), np.full(n, 0.37))
    assert abs(f[6] - math.log(n)) < 1e-12 and abs(f[7] - 1.0 / n) < 1e-15
    w = np.array([1.0, 3.0])
    f = oracle.features(np.zeros((2, 1)), w)
    p = w / w.sum()
    assert abs(f[2] - (-(p * np.log(p)).sum())) < 1e-15 and f[3] == 0.75


def test_features_permutation_invariant_and_coordinatewise():
    rng = np.random.default_rng(3)
    pts = rng.uniform(0, 255, (50, 5))
    w = rng.exponential(1.0, 50)
    f = oracle.features(pts, w)
    perm = rng.permutation(50)
    assert np.allclose(oracle.features(pts[perm], w[perm]), f, rtol=0, atol=1e-9)
    for c in range(5):   # each coordinate's median is the 1-D median of that coordinate
        assert oracle.features(pts[:, c:c + 1], w)[1] == f[5 + c]


def _tiny_params(d, hidden):
    rng = np.random.default_rng(4)
    P = oracle.mlp_num_params(d, hidden)
    return rng.normal(size=P) * 0.3


def test_mlp_hand_computed_forward():
    # d = 1: F = 4 inputs, O = 2 outputs; hidden = 2
    d, Hd = 1, 2
    W1 = np.array([[1.0, 0.0, 0.0, 0.0], [0.0, -1.0, 0.0, 2.0]])
    b1 = np.array([0.5, 0.0])
    W2 = np.array([[1.0, 1.0], [-1.0, 0.0]])
    b2 = np.array([0.0, 0.25])
    W3 = np.array([[2.0, 0.0], [0.0, 3.0]])
    b3 = np.array([1.0, -1.0])
    prm = np.concatenate([W1.ravel(), b1, W2.ravel(), b2, W3.ravel(), b3])
    feats = np.array([[191.5, 63.5, math.log(441.0), 0.25]])   # normalises to x = [1, -1, 1, 0.25]
    y = oracle.mlp_forward(prm, d, feats, hidden=Hd)
    # h1 = relu([1 + 0.5, 1 + 0.5]) = [1.5, 1.5]; h2 = relu([3, -1.5 + 0.25]) = [3, 0]
    assert np.allclose(y, [[2 * 3 + 1, 0 - 1]], atol=1e-13)


def test_mlp_gradient_against_finite_differences():
    d, Hd, B = 3, 6, 5
    rng = np.random.default_rng(5)
    prm = _tiny_params(d, Hd)
    feats = np.concatenate([rng.uniform(0, 255, (B, 2 * d)), rng.uniform(2, 6, (B, 1)),
                            rng.uniform(0, 0.5, (B, 1))], axis=1)
    t = rng.normal(size=(B, d + 1))
    L, g = oracle.mlp_loss_grad(prm, d, feats, t, hidden=Hd)
    assert abs(L - oracle.mlp_loss_grad(prm, d, feats, t, hidden=Hd)[0]) == 0
    eps = 1e-6
    for i in range(prm.size):
        p1, p2 = prm.copy(), prm.copy()
        p1[i] += eps
        p2[i] -= eps
        fd = (oracle.mlp_loss_grad(p1, d, feats, t, hidden=Hd)[0] - oracle.mlp_loss_grad(p2, d, feats, t, hidden=Hd)[0]) / (2 * eps)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g[i])), (i, fd, g[i])
    # the loss is the stated weighted squared error
    y = oracle.mlp_forward(prm, d, feats, hidden=Hd)
    Lref = np.mean(np.sum((y[:, :d] - t[:, :d]) ** 2, 1) / d + (y[:, d] - t[:, d]) ** 2)
    assert abs(L - Lref) < 1e-12
