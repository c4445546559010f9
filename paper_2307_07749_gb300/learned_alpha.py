"""Learned alpha: features, alpha sweeps run by this solver, labels, training and prediction.

The paper fixes alpha = 1e-8 (Sec. 5.2); its Theorem 1 bounds alpha from above only.  With an
FP32 preconditioner that alpha fails (rounding grows like alpha^{-(N-1)/N}), so the best alpha
depends on the problem.  This module labels each training problem from a 16-point sweep
(10^{-j/2}, j = 1..16) by the alphas that need the fewest MINRES iterations to reach the
tolerance (the centre of the widest run of them, see label), and fits the library's MLP (bltt_alpha_train) to
(log N, log M, gamma, log(tau/h^2)) -> log10(alpha).  Every solve and every network pass runs in
the library's CUDA kernels; this file only arranges inputs.
"""
from __future__ import annotations

import math
import time

import numpy as np

from . import (ALPHA_MODEL_FLOATS, ALPHA_NPARAM, ARITH_F32X2, BASIS_SPECTRAL, PREC_F32, Solver,
               bltt_alpha_predict, bltt_alpha_train)

SWEEP = [10.0 ** (-j / 2.0) for j in range(1, 17)]      # 10^-0.5 ... 10^-8
H = 32


def features(prob) -> np.ndarray:
    """(log N, log M, gamma, log(tau / h^2)); gamma := 1 for the heat equation."""
    meta = getattr(prob, "meta", {}) or {}
    gamma = float(meta.get("gamma", 1.0))
    tau = float(meta.get("tau", 1.0 / prob.N))
    h = float(prob.h[0])
    return np.array([math.log(prob.N), math.log(prob.M), gamma, math.log(tau / (h * h))])


def sweep(solver, f_dev, alphas=SWEEP, tol=1e-8, maxit=40, precision=PREC_F32,
          matvec_arith=ARITH_F32X2, basis=BASIS_SPECTRAL):
    """Solve for every alpha; returns a list of (alpha, iterations or None, seconds)."""
    out = []
    for a in alphas:
        t0 = time.perf_counter()
        _, info = solver.solve(f_dev, alpha=a, tol=tol, maxit=maxit, precision=precision,
                               basis=basis, matvec_arith=matvec_arith, raise_on_error=False,
                               rebuild=True)
        dt = time.perf_counter() - t0
        ok = info["status"] == 0 and info["relres_true"] <= tol
        out.append((a, info["iters"] if ok else None, dt))
    return out


def label(results):
    """log10 alpha label of one sweep: the fewest iterations decide; among the alphas that reach
    that count, the label is the centre (in log10 alpha) of the longest run of consecutive sweep
    points that all reach it (equal runs: the run of larger alpha).  The centre keeps the largest
    margin to the points where the count rises, on the small-alpha side often sharply (rounding of
    the FP32 form).  None if no alpha converged."""
    its = [it for _, it, _ in results if it is not None]
    if not its:
        return None
    best = min(its)
    runs, cur = [], []
    for a, it, _ in results:
        if it == best:
            cur.append(math.log10(a))
        elif cur:
            runs.append(cur)
            cur = []
    if cur:
        runs.append(cur)
    # longest run; among equally long runs the one of largest alpha
    run = max(runs, key=lambda r: (len(r), max(r)))
    return 0.5 * (min(run) + max(run))


def init_model(feats, labels, seed=0) -> np.ndarray:
    """Xavier-uniform weights from default_rng(seed), zero biases, and the standardisation of the
    training features and labels."""
    rng = np.random.default_rng(seed)
    m = np.zeros(ALPHA_MODEL_FLOATS, np.float64)
    o = 0

    def xavier(fan_in, fan_out):
        lim = math.sqrt(6.0 / (fan_in + fan_out))
        return rng.uniform(-lim, lim, fan_in * fan_out)

    m[o:o + H * 4] = xavier(4, H); o += H * 4
    o += H
    m[o:o + H * H] = xavier(H, H); o += H * H
    o += H
    m[o:o + H] = xavier(H, 1); o += H
    o += 1
    assert o == ALPHA_NPARAM
    feats = np.asarray(feats, np.float64)
    labels = np.asarray(labels, np.float64)
    m[o:o + 4] = feats.mean(0); o += 4
    m[o:o + 4] = np.maximum(feats.std(0), 1e-6); o += 4
    m[o] = labels.mean()
    m[o + 1] = max(labels.std(), 1e-6)
    return m.astype(np.float32)


def train(feats, labels, epochs=3000, lr=3e-3, seed=0):
    model = init_model(feats, labels, seed)
    return bltt_alpha_train(model, feats, labels, epochs, lr)


def predict(model, probs, lo=1e-8, hi=10.0 ** -0.5):
    """Predicted alpha per problem, clipped to the sweep's range."""
    F = np.stack([features(p) for p in probs])
    return np.clip(bltt_alpha_predict(model, F).astype(np.float64), lo, hi)


def build_dataset(problems, tol=1e-8, maxit=40, **form):
    """Sweep every (problem, rhs_factory); returns (features, labels, raw sweep results)."""
    import torch
    feats, labels, raw = [], [], []
    for prob, rf in problems:
        s = Solver(prob)
        f = torch.from_numpy(np.ascontiguousarray(rf())).cuda()
        res = sweep(s, f, tol=tol, maxit=maxit, **form)
        lab = label(res)
        raw.append(res)
        s.close()
        if lab is None:
            continue
        feats.append(features(prob))
        labels.append(lab)
    return np.array(feats), np.array(labels), raw
