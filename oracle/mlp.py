"""FP64 reference of the learned angle proposer (numpy).

TEST INFRASTRUCTURE ONLY (tests, smoke check, benchmark CPU baseline).

The paper observes that optimal G-QAOA angles cluster as a function of the
instance's size and clause count (Section III.B, Fig. 2; Appendix D) and
suggests predicting angles from the problem structure, e.g. its density of
states (Section V). The proposer is a small MLP on that density of states:

  x  = [h[c] / 2^n for c = 0..d_in-3 (zero-padded), n / 32, m / 128]
  z1 = W1 x + b1,  h1 = GELU(z1)
  z2 = W2 h1 + b2, h2 = GELU(z2)
  o  = W3 h2 + b3
  angles = 2 pi sigmoid(o)     (first p entries gammas, last p betas)
  loss = mean over the batch and the 2p outputs of 2 (1 - cos(angles - labels))

The angles are 2 pi periodic (C is an integer, H_M a projector), so the loss is
the squared chord between the angles on the unit circle; it equals the squared
difference to fourth order and does not penalise a wrap through 0 = 2 pi.

GELU(x) = x Phi(x) with the exact normal CDF Phi(x) = (1 + erf(x / sqrt 2)) / 2.
Adam: m <- b1 m + (1-b1) g; v <- b2 v + (1-b2) g^2;
      theta <- theta - lr (m / (1-b1^t)) / (sqrt(v / (1-b2^t)) + eps).

Parameters are one flat vector [W1 (d_h x d_in), b1, W2 (d_h x d_h), b2,
W3 (d_out x d_h), b3], row-major, as in the CUDA library.

Pins: torch's CPU float64 Linear/gelu/sigmoid/autograd (library routines),
central finite differences, GELU identities, Adam's first-step closed form.
"""

from __future__ import annotations

import math

import numpy as np
from scipy.special import erf


def unpack(params, d_in, d_h, d_out):
    p = np.asarray(params, dtype=np.float64)
    sizes = [d_h * d_in, d_h, d_h * d_h, d_h, d_out * d_h, d_out]
    out, o = [], 0
    for s in sizes:
        out.append(p[o:o + s])
        o += s
    W1, b1, W2, b2, W3, b3 = out
    return W1.reshape(d_h, d_in), b1, W2.reshape(d_h, d_h), b2, W3.reshape(d_out, d_h), b3


def gelu(x):
    return 0.5 * x * (1.0 + erf(x / math.sqrt(2.0)))


def gelu_grad(x):
    return 0.5 * (1.0 + erf(x / math.sqrt(2.0))) + x * np.exp(-0.5 * x * x) / math.sqrt(2 * math.pi)


def features(hist, n, m, d_in=130):
    x = np.zeros(d_in)
    h = np.asarray(hist, dtype=np.float64)[: m + 1]
    x[: min(len(h), d_in - 2)] = h[: d_in - 2] / float(1 << n)
    x[d_in - 2] = n / 32.0
    x[d_in - 1] = m / 128.0
    return x


def forward(params, x, dims):
    d_in, d_h, d_out = dims
    W1, b1, W2, b2, W3, b3 = unpack(params, *dims)
    x = np.asarray(x, dtype=np.float64)
    z1 = x @ W1.T + b1
    h1 = gelu(z1)
    z2 = h1 @ W2.T + b2
    h2 = gelu(z2)
    o = h2 @ W3.T + b3
    s = 1.0 / (1.0 + np.exp(-o))
    return 2 * np.pi * s, (x, z1, h1, z2, h2, o, s)


def loss_and_grad(params, x, labels, dims):
    d_in, d_h, d_out = dims
    W1, b1, W2, b2, W3, b3 = unpack(params, *dims)
    ang, (x, z1, h1, z2, h2, o, s) = forward(params, x, dims)
    B = x.shape[0]
    diff = ang - labels
    loss = float(np.mean(2.0 * (1.0 - np.cos(diff))))
    dang = 2.0 * np.sin(diff) / (B * d_out)
    do = dang * 2 * np.pi * s * (1 - s)
    dW3 = do.T @ h2
    db3 = do.sum(0)
    dz2 = (do @ W3) * gelu_grad(z2)
    dW2 = dz2.T @ h1
    db2 = dz2.sum(0)
    dz1 = (dz2 @ W2) * gelu_grad(z1)
    dW1 = dz1.T @ x
    db1 = dz1.sum(0)
    g = np.concatenate([dW1.ravel(), db1, dW2.ravel(), db2, dW3.ravel(), db3])
    return loss, g


def adam(params, grads, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    m = b1 * m + (1 - b1) * grads
    v = b2 * v + (1 - b2) * grads * grads
    mhat = m / (1 - b1 ** t)
    vhat = v / (1 - b2 ** t)
    return params - lr * mhat / (np.sqrt(vhat) + eps), m, v
