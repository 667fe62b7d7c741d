"""FP64 CPU oracle for the learned initial density (a project-added part: the
paper starts every SCF from a superposition of atomic densities, Section 5).

TEST INFRASTRUCTURE ONLY, like sparc_oracle.py: only the tests, the smoke check and
the benchmark's CPU baseline may import it, and it shares no code with the CUDA
library.  What it computes is textbook: atom-centred Gaussian radial descriptors,
a 3-layer perceptron with ReLU, the mean-squared-error loss, its gradient by the
chain rule (backpropagation), and the Adam update of Kingma and Ba (2015).

Definitions (also in the design notes):
  * descriptor k of grid node x: D_k(x) = sum_J sum_{T in {-1,0,1}^3 L}
    exp(-|x - R_J - T|^2 / s_k^2), widths s_k = 0.4 * 10^(k/(K-1)) bohr, K = 16;
  * network: a1 = relu(D W1 + b1), a2 = relu(a1 W2 + b2), y = a2 w3 + b3 with
    W1 [K][H], W2 [H][H], w3 [H], H = 128; relu'(0) taken as 0;
  * loss: mean over the batch of (y - t)^2;
  * Adam: m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2, theta -= lr m_hat/(sqrt(v_hat)+eps)
    with m_hat = m/(1-b1^t), v_hat = v/(1-b2^t), b1 = 0.9, b2 = 0.999, eps = 1e-8;
  * the flat parameter vector is [W1 (row-major K x H), b1, W2 (row-major H x H), b2,
    w3, b3].
"""
from __future__ import annotations

import numpy as np

NFEAT = 16
NHID = 128


def widths(k=NFEAT):
    """Descriptor widths s_k = 0.4 * 10^(k/(K-1)) bohr."""
    return 0.4 * 10.0 ** (np.arange(k) / (k - 1))


def descriptors(n, h, atoms, s):
    """D[node, k] for nodes x-fastest, by the explicit 27-image sum at every node."""
    n = tuple(n)
    L = np.array([n[a] * h[a] for a in range(3)])
    xs = [-0.5 * L[a] + np.arange(n[a]) * h[a] for a in range(3)]
    Z, Y, X = np.meshgrid(xs[2], xs[1], xs[0], indexing="ij")
    P = np.stack([X.reshape(-1), Y.reshape(-1), Z.reshape(-1)], axis=1)
    D = np.zeros((P.shape[0], len(s)))
    for R in atoms:
        for t in np.ndindex(3, 3, 3):
            d = P - R - (np.array(t) - 1) * L
            r2 = np.einsum("ij,ij->i", d, d)
            for k, sk in enumerate(s):
                D[:, k] += np.exp(-r2 / (sk * sk))
    return D


def unpack(theta, nf=NFEAT, nh=NHID):
    """Views W1, b1, W2, b2, w3, b3 of the flat parameter vector."""
    o = 0
    out = []
    for shape in ((nf, nh), (nh,), (nh, nh), (nh,), (nh,), (1,)):
        sz = int(np.prod(shape))
        out.append(theta[o:o + sz].reshape(shape))
        o += sz
    return out


def nparams(nf=NFEAT, nh=NHID):
    return nf * nh + nh + nh * nh + nh + nh + 1


def init_params(seed, nf=NFEAT, nh=NHID):
    """Glorot-uniform weights, zero biases (numpy default_rng(seed))."""
    rng = np.random.default_rng(seed)
    th = np.zeros(nparams(nf, nh))
    W1, b1, W2, b2, w3, b3 = unpack(th, nf, nh)
    W1[...] = rng.uniform(-1, 1, W1.shape) * np.sqrt(6.0 / (nf + nh))
    W2[...] = rng.uniform(-1, 1, W2.shape) * np.sqrt(6.0 / (2 * nh))
    w3[...] = rng.uniform(-1, 1, w3.shape) * np.sqrt(6.0 / (nh + 1))
    return th


def forward(theta, D, nf=NFEAT, nh=NHID):
    """y = relu(relu(D W1 + b1) W2 + b2) w3 + b3 (and the hidden activations)."""
    W1, b1, W2, b2, w3, b3 = unpack(theta, nf, nh)
    z1 = D @ W1 + b1
    a1 = np.maximum(z1, 0.0)
    z2 = a1 @ W2 + b2
    a2 = np.maximum(z2, 0.0)
    y = a2 @ w3 + b3[0]
    return y, (a1, a2)


def loss_and_grad(theta, D, t, nf=NFEAT, nh=NHID):
    """Mean-squared error and its gradient with respect to the flat parameters."""
    W1, b1, W2, b2, w3, b3 = unpack(theta, nf, nh)
    y, (a1, a2) = forward(theta, D, nf, nh)
    N = D.shape[0]
    r = y - t
    loss = float(np.mean(r * r))
    dy = 2.0 * r / N                        # dL/dy
    g = np.zeros_like(theta)
    gW1, gb1, gW2, gb2, gw3, gb3 = unpack(g, nf, nh)
    gw3[...] = a2.T @ dy
    gb3[0] = dy.sum()
    dz2 = np.outer(dy, w3) * (a2 > 0)       # dL/dz2
    gW2[...] = a1.T @ dz2
    gb2[...] = dz2.sum(axis=0)
    dz1 = (dz2 @ W2.T) * (a1 > 0)           # dL/dz1
    gW1[...] = D.T @ dz1
    gb1[...] = dz1.sum(axis=0)
    return loss, g


def adam(theta, g, m, v, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (step counts from 1); returns new (theta, m, v)."""
    m = b1 * m + (1.0 - b1) * g
    v = b2 * v + (1.0 - b2) * g * g
    mh = m / (1.0 - b1 ** step)
    vh = v / (1.0 - b2 ** step)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v
