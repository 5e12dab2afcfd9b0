"""FP64 CPU reference of the learned viscosity sensor's network (test
infrastructure only; imported by tests/ and nothing in the product).

Network: y = W3 . gelu(W2 gelu(W1 x + b1) + b2) + b3, with
gelu(z) = z/2 (1 + erf(z/sqrt 2)).  Loss: mean squared error.  Optimiser:
Adam (Kingma & Ba 2015): m <- b1 m + (1-b1) g, v <- b2 v + (1-b2) g^2,
theta <- theta - lr (m/(1-b1^t)) / (sqrt(v/(1-b2^t)) + eps).

Flat parameter vector (the library's layout): W1 [H][D] row-major, b1 [H],
W2 [H][H], b2 [H], W3 [H], b3 [1].
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erf

H = 64


def n_params(D: int, Hh: int = H) -> int:
    return Hh * D + Hh + Hh * Hh + Hh + Hh + 1


def unpack(theta: np.ndarray, D: int, Hh: int = H):
    o = 0
    W1 = theta[o:o + Hh * D].reshape(Hh, D); o += Hh * D
    b1 = theta[o:o + Hh]; o += Hh
    W2 = theta[o:o + Hh * Hh].reshape(Hh, Hh); o += Hh * Hh
    b2 = theta[o:o + Hh]; o += Hh
    W3 = theta[o:o + Hh]; o += Hh
    b3 = theta[o:o + 1]; o += 1
    return W1, b1, W2, b2, W3, b3


def gelu(z):
    return 0.5 * z * (1.0 + erf(z / math.sqrt(2.0)))


def gelu_prime(z):
    return 0.5 * (1.0 + erf(z / math.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)


def init_params(D: int, seed: int, Hh: int = H) -> np.ndarray:
    """Kaiming-uniform weights U(-sqrt(6/fan_in), +sqrt(6/fan_in)), zero biases."""
    rng = np.random.default_rng(seed)
    th = np.zeros(n_params(D, Hh))
    W1, b1, W2, b2, W3, b3 = unpack(th, D, Hh)
    W1[:] = rng.uniform(-1, 1, W1.shape) * math.sqrt(6.0 / D)
    W2[:] = rng.uniform(-1, 1, W2.shape) * math.sqrt(6.0 / Hh)
    W3[:] = rng.uniform(-1, 1, W3.shape) * math.sqrt(6.0 / Hh)
    return th


def forward(theta: np.ndarray, X: np.ndarray) -> np.ndarray:
    D = X.shape[1]
    W1, b1, W2, b2, W3, b3 = unpack(theta, D)
    a1 = gelu(X @ W1.T + b1)
    a2 = gelu(a1 @ W2.T + b2)
    return a2 @ W3 + b3[0]


def loss_and_grad(theta: np.ndarray, X: np.ndarray, y: np.ndarray):
    """MSE loss and its gradient by hand-written backpropagation."""
    n, D = X.shape
    W1, b1, W2, b2, W3, b3 = unpack(theta, D)
    z1 = X @ W1.T + b1
    a1 = gelu(z1)
    z2 = a1 @ W2.T + b2
    a2 = gelu(z2)
    yh = a2 @ W3 + b3[0]
    r = yh - y
    loss = float(np.mean(r * r))
    d3 = 2.0 * r / n                       # dL/dyh
    g = np.zeros_like(theta)
    gW1, gb1, gW2, gb2, gW3, gb3 = unpack(g, D)
    gW3[:] = a2.T @ d3
    gb3[0] = d3.sum()
    dz2 = np.outer(d3, W3) * gelu_prime(z2)
    gW2[:] = dz2.T @ a1
    gb2[:] = dz2.sum(axis=0)
    dz1 = (dz2 @ W2) * gelu_prime(z1)
    gW1[:] = dz1.T @ X
    gb1[:] = dz1.sum(axis=0)
    return loss, g


class Adam:
    def __init__(self, n: int, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
        self.m = np.zeros(n)
        self.v = np.zeros(n)
        self.t = 0
        self.lr, self.b1, self.b2, self.eps = lr, b1, b2, eps

    def step(self, theta: np.ndarray, g: np.ndarray) -> None:
        self.t += 1
        self.m = self.b1 * self.m + (1 - self.b1) * g
        self.v = self.b2 * self.v + (1 - self.b2) * g * g
        mh = self.m / (1 - self.b1 ** self.t)
        vh = self.v / (1 - self.b2 ** self.t)
        theta -= self.lr * mh / (np.sqrt(vh) + self.eps)


def train(theta: np.ndarray, X: np.ndarray, y: np.ndarray, epochs: int, batch: int, lr=1e-3) -> list:
    """Minibatch Adam over the rows in their given order; returns per-epoch mean loss."""
    opt = Adam(theta.size, lr=lr)
    hist = []
    n = len(y)
    for _ in range(epochs):
        tot = 0.0
        nb = 0
        for s in range(0, n, batch):
            loss, g = loss_and_grad(theta, X[s:s + batch], y[s:s + batch])
            opt.step(theta, g)
            tot += loss
            nb += 1
        hist.append(tot / nb)
    return hist
