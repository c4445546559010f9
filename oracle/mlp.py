"""Oracle for the learned-alpha network: an MLP 4 -> 32 -> 32 -> 1 with tanh hidden layers, its
mean-squared-error gradient by backpropagation and full-batch Adam (Kingma and Ba), in FP64.

Test infrastructure only (see the package docstring).  The paper has no learned component; this
follows the textbook definitions of the layers, of backpropagation and of the Adam update.
Parameters use the library's flat layout: W1[32][4], b1[32], W2[32][32], b2[32], w3[32], b3, then
the feature mean[4], std[4] and the label y_mean, y_std.
"""
from __future__ import annotations

import numpy as np

H, F = 32, 4
NPARAM = H * F + H + H * H + H + H + 1
MODEL_FLOATS = NPARAM + 2 * F + 2


def unpack(model):
    m = np.asarray(model, dtype=np.float64)
    o = 0
    W1 = m[o:o + H * F].reshape(H, F); o += H * F
    b1 = m[o:o + H]; o += H
    W2 = m[o:o + H * H].reshape(H, H); o += H * H
    b2 = m[o:o + H]; o += H
    w3 = m[o:o + H]; o += H
    b3 = m[o]; o += 1
    mean = m[o:o + F]; o += F
    std = m[o:o + F]; o += F
    ym, ys = m[o], m[o + 1]
    return W1, b1, W2, b2, w3, b3, mean, std, ym, ys


def forward(model, feats):
    """Standardised network output for every row of feats ([n, 4])."""
    W1, b1, W2, b2, w3, b3, mean, std, ym, ys = unpack(model)
    X = (np.asarray(feats, dtype=np.float64) - mean) / std
    H1 = np.tanh(X @ W1.T + b1)
    H2 = np.tanh(H1 @ W2.T + b2)
    return H2 @ w3 + b3, (X, H1, H2)


def predict(model, feats):
    """alpha = 10^(y * y_std + y_mean)."""
    *_, ym, ys = unpack(model)
    y, _ = forward(model, feats)
    return 10.0 ** (y * ys + ym)


def loss_and_grad(model, feats, labels):
    """L = mean((y - t)^2) with t = (label - y_mean)/y_std, and dL/dparams (flat, NPARAM)."""
    W1, b1, W2, b2, w3, b3, mean, std, ym, ys = unpack(model)
    y, (X, H1, H2) = forward(model, feats)
    t = (np.asarray(labels, dtype=np.float64) - ym) / ys
    n = len(t)
    r = y - t
    L = float(np.mean(r * r))
    d3 = 2.0 * r / n                        # dL/dy
    D2 = np.outer(d3, w3) * (1.0 - H2 ** 2)  # dL/dz2
    D1 = (D2 @ W2) * (1.0 - H1 ** 2)         # dL/dz1
    g = np.concatenate([(D1.T @ X).ravel(), D1.sum(0), (D2.T @ H1).ravel(), D2.sum(0),
                        H2.T @ d3, [d3.sum()]])
    return L, g


def adam_train(model, feats, labels, epochs, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """Full-batch Adam: m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2, p -= lr m^/(sqrt(v^) + eps)
    with the bias corrections m^ = m/(1-b1^t), v^ = v/(1-b2^t).  Returns (model, losses)."""
    model = np.array(model, dtype=np.float64)
    m = np.zeros(NPARAM)
    v = np.zeros(NPARAM)
    hist = []
    for t in range(1, epochs + 1):
        L, g = loss_and_grad(model, feats, labels)
        hist.append(L)
        m = beta1 * m + (1 - beta1) * g
        v = beta2 * v + (1 - beta2) * g * g
        mh = m / (1 - beta1 ** t)
        vh = v / (1 - beta2 ** t)
        model[:NPARAM] -= lr * mh / (np.sqrt(vh) + eps)
    return model, np.array(hist)
