"""Learned projection (MLP feature map) -- CPU oracle.

TEST INFRASTRUCTURE ONLY.  The paper suggests replacing the random
projection by a non-random hashing (Sec. 6 names learned hash functions as
a drop-in for the random projection); the learned form maps every point through
  y = W2 . gelu(W1 . x + b1) + b2        (D -> H -> D_y)
and then takes the usual sign projection (Eq. 3) of y.  Training pulls
epsilon-neighbour pairs together and pushes other pairs apart in angle:
  loss = mean over pairs of  max(0, m_pos - cos(y_i, y_j))   (label 1)
                            max(0, cos(y_i, y_j) - m_neg)   (label 0)
Everything here is float64 numpy; gelu is the exact erf form.
"""
from __future__ import annotations

import math

import numpy as np

_erf = np.vectorize(math.erf, otypes=[np.float64])


def gelu(h):
    return 0.5 * h * (1.0 + _erf(h / math.sqrt(2.0)))


def gelu_grad(h):
    cdf = 0.5 * (1.0 + _erf(h / math.sqrt(2.0)))
    pdf = np.exp(-0.5 * h * h) / math.sqrt(2.0 * math.pi)
    return cdf + h * pdf


def forward(X, W1, b1, W2, b2):
    """Returns (Y, H, A): pre-activation H, activation A, output Y."""
    X = np.asarray(X, dtype=np.float64)
    H = X @ np.asarray(W1, np.float64).T + np.asarray(b1, np.float64)
    A = gelu(H)
    Y = A @ np.asarray(W2, np.float64).T + np.asarray(b2, np.float64)
    return Y, H, A


def pair_loss(Y, ia, ib, label, m_pos, m_neg):
    """Mean hinge loss over pairs (ia[t], ib[t]) of rows of Y and dL/dY."""
    yi, yj = Y[ia], Y[ib]
    ni = np.linalg.norm(yi, axis=1)
    nj = np.linalg.norm(yj, axis=1)
    cos = np.einsum("ij,ij->i", yi, yj) / (ni * nj)
    pos = label.astype(bool)
    viol = np.where(pos, m_pos - cos, cos - m_neg)
    active = viol > 0
    B = len(ia)
    loss = np.where(active, viol, 0.0).sum() / B
    dcos = np.where(active, np.where(pos, -1.0, 1.0), 0.0) / B
    gi = dcos[:, None] * (yj / (ni * nj)[:, None] - cos[:, None] * yi / (ni * ni)[:, None])
    gj = dcos[:, None] * (yi / (ni * nj)[:, None] - cos[:, None] * yj / (nj * nj)[:, None])
    dY = np.zeros_like(Y)
    np.add.at(dY, ia, gi)
    np.add.at(dY, ib, gj)
    return loss, dY


def backward(X, W1, W2, H, A, dY):
    """Gradients of the loss with respect to W1, b1, W2, b2 given dL/dY."""
    X = np.asarray(X, np.float64)
    dW2 = dY.T @ A
    db2 = dY.sum(axis=0)
    dA = dY @ np.asarray(W2, np.float64)
    dH = dA * gelu_grad(H)
    dW1 = dH.T @ X
    db1 = dH.sum(axis=0)
    return dW1, db1, dW2, db2


def loss_and_grads(X, W1, b1, W2, b2, ia, ib, label, m_pos, m_neg):
    Y, H, A = forward(X, W1, b1, W2, b2)
    loss, dY = pair_loss(Y, ia, ib, label, m_pos, m_neg)
    return loss, backward(X, W1, W2, H, A, dY)


def adam_step(w, g, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba 2015) of w in float64; returns new
    (w, m, v).  t counts steps from 1."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mh = m / (1.0 - beta1 ** t)
    vh = v / (1.0 - beta2 ** t)
    return w - lr * mh / (np.sqrt(vh) + eps), m, v
