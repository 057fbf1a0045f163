"""CPU FP64 reference of the cost model's multilayer perceptron (test infrastructure only).

The network maps a feature vector x (nin) to one output through two hidden layers with ReLU:
    h1 = relu(W1 x + b1), h2 = relu(W2 h1 + b2), y = w3 . h2 + b3,
and is trained on the mean squared error L = mean((y - t)^2). This module writes the forward
pass and the gradients of L out directly (chain rule, layer by layer) so the library's CUDA
kernels can be checked against it; its own gradients are pinned by finite differences in
tests/test_oracle.py. Parameter layout (shared with the library's flat parameter vector):
W1 (h x nin, row-major), b1 (h), W2 (h x h), b2 (h), w3 (h), b3 (1).
"""
import numpy as np


def unpack(theta, nin, h):
    theta = np.asarray(theta, dtype=np.float64)
    o = 0
    W1 = theta[o:o + h * nin].reshape(h, nin); o += h * nin
    b1 = theta[o:o + h]; o += h
    W2 = theta[o:o + h * h].reshape(h, h); o += h * h
    b2 = theta[o:o + h]; o += h
    w3 = theta[o:o + h]; o += h
    b3 = theta[o:o + 1]; o += 1
    assert o == theta.size
    return W1, b1, W2, b2, w3, b3


def nparams(nin, h):
    return h * nin + h + h * h + h + h + 1


def forward(theta, X, nin, h):
    W1, b1, W2, b2, w3, b3 = unpack(theta, nin, h)
    X = np.asarray(X, dtype=np.float64)
    z1 = X @ W1.T + b1
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ W2.T + b2
    h2 = np.maximum(z2, 0.0)
    y = h2 @ w3 + b3[0]
    return y, (X, z1, h1, z2, h2)


def loss(theta, X, t, nin, h):
    y, _ = forward(theta, X, nin, h)
    return float(np.mean((y - np.asarray(t, dtype=np.float64)) ** 2))


def gradient(theta, X, t, nin, h):
    """dL/dtheta by the chain rule, in the flat layout."""
    W1, b1, W2, b2, w3, b3 = unpack(theta, nin, h)
    y, (X, z1, h1, z2, h2) = forward(theta, X, nin, h)
    N = X.shape[0]
    dy = 2.0 * (y - np.asarray(t, dtype=np.float64)) / N          # dL/dy
    dw3 = h2.T @ dy
    db3 = np.array([dy.sum()])
    dz2 = np.outer(dy, w3) * (z2 > 0)
    dW2 = dz2.T @ h1
    db2 = dz2.sum(axis=0)
    dz1 = (dz2 @ W2) * (z1 > 0)
    dW1 = dz1.T @ X
    db1 = dz1.sum(axis=0)
    return np.concatenate([dW1.ravel(), db1, dW2.ravel(), db2, dw3, db3])
