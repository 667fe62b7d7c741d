"""Pins of the learned-density oracle (host only): the gradient against central
finite differences, the Adam update against its closed form for a constant
gradient and on a quadratic, the descriptors against a single Gaussian and the
separable image sum."""
import math

import numpy as np

from oracle import mlp_oracle as M


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(0)
    nf, nh, N = 3, 5, 9
    th = rng.normal(0, 0.7, M.nparams(nf, nh))
    D = rng.normal(0, 1, (N, nf))
    t = rng.normal(0, 1, N)
    loss, g = M.loss_and_grad(th, D, t, nf, nh)
    eps = 1e-6
    for i in range(th.size):
        tp, tm = th.copy(), th.copy()
        tp[i] += eps
        tm[i] -= eps
        fd = (M.loss_and_grad(tp, D, t, nf, nh)[0] - M.loss_and_grad(tm, D, t, nf, nh)[0]) / (2 * eps)
        assert abs(fd - g[i]) < 1e-7 * max(1.0, abs(g[i])), (i, fd, g[i])
    y, _ = M.forward(th, D, nf, nh)
    assert abs(loss - np.mean((y - t) ** 2)) < 1e-15


def test_forward_of_a_hand_sized_network():
    # nf = 1, nh = 2: y = w3 . relu(relu(x W1 + b1) W2 + b2) + b3, evaluated by hand
    th = np.array([1.0, -2.0,  0.5, 0.25,  1.0, 0.0, -1.0, 3.0,  0.0, -0.5,  2.0, 1.0,  0.75])
    x = 1.5
    a1 = [max(1.0 * x + 0.5, 0.0), max(-2.0 * x + 0.25, 0.0)]          # [2.0, 0.0]
    a2 = [max(a1[0] * 1.0 + a1[1] * -1.0 + 0.0, 0.0), max(a1[0] * 0.0 + a1[1] * 3.0 - 0.5, 0.0)]
    y_hand = 2.0 * a2[0] + 1.0 * a2[1] + 0.75                          # 4.75
    y, _ = M.forward(th, np.array([[x]]), 1, 2)
    assert y[0] == y_hand == 4.75


def test_adam_constant_gradient_closed_form():
    g = np.array([0.3, -2.0, 1e-3])
    th = np.zeros(3)
    m = np.zeros(3)
    v = np.zeros(3)
    lr = 0.01
    for step in range(1, 6):
        new, m, v = M.adam(th, g, m, v, step, lr)
        # bias-corrected moments equal g and g^2 exactly for a constant gradient
        assert np.allclose(new - th, -lr * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=0)
        th = new


def test_adam_minimises_a_quadratic():
    A = np.diag([1.0, 10.0, 0.1])
    c = np.array([1.0, -2.0, 3.0])
    th = np.zeros(3)
    m = np.zeros(3)
    v = np.zeros(3)
    for step in range(1, 20001):
        g = A @ th - c
        th, m, v = M.adam(th, g, m, v, step, 0.01)
    assert np.allclose(th, np.linalg.solve(A, c), atol=1e-3)


def test_descriptors_single_gaussian_and_separable_image_sum():
    n, h = (40, 40, 40), (0.5, 0.5, 0.5)
    s = M.widths()
    assert abs(s[0] - 0.4) < 1e-15 and abs(s[-1] - 4.0) < 1e-12
    R = np.array([[0.1, -0.2, 0.3]])
    D = M.descriptors(n, h, R, s[:3])
    xs = [-10.0 + np.arange(40) * 0.5] * 3
    # narrow widths in a 20 bohr cell: the images add < 1e-30
    for node in (0, 12345, 40 * 40 * 20 + 40 * 20 + 20):
        i, j, k = node % 40, (node // 40) % 40, node // 1600
        r2 = (xs[0][i] - 0.1) ** 2 + (xs[1][j] + 0.2) ** 2 + (xs[2][k] - 0.3) ** 2
        for q in range(3):
            assert abs(D[node, q] - math.exp(-r2 / s[q] ** 2)) < 1e-15
    # wide widths on a small cell: the 27-image sum is a product of per-axis sums
    n2, h2 = (6, 5, 7), (0.9, 1.1, 0.8)
    rng = np.random.default_rng(3)
    L = np.array([n2[a] * h2[a] for a in range(3)])
    atoms = rng.uniform(-0.5, 0.5, (2, 3)) * L
    D2 = M.descriptors(n2, h2, atoms, s[-2:])
    x2 = [-0.5 * L[a] + np.arange(n2[a]) * h2[a] for a in range(3)]
    for node in range(0, n2[0] * n2[1] * n2[2], 7):
        i, j, k = node % n2[0], (node // n2[0]) % n2[1], node // (n2[0] * n2[1])
        p = (x2[0][i], x2[1][j], x2[2][k])
        for q, sk in enumerate(s[-2:]):
            ref = sum(math.prod(sum(math.exp(-(p[a] - Rj[a] - t * L[a]) ** 2 / sk ** 2) for t in (-1, 0, 1))
                                for a in range(3)) for Rj in atoms)
            assert abs(D2[node, q] - ref) < 1e-12 * max(1.0, ref)
