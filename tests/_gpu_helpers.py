"""Shared helpers of the GPU parity tests (no oracle arithmetic here)."""
import numpy as np


def rel(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def rel_max(a, b):
    """max_i |a_i - b_i| / max_i |b_i|: the max-norm relative error.  Beside the 2-norm one it
    catches a wrong block of entries (a ragged tail, one tile) too small to move the 2-norm."""
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.max(np.abs(a - b)) / max(float(np.max(np.abs(b))), 1e-300))


def precond_tol(N, alpha, prec=64):
    """Tolerance for P_alpha^{-1} between two independent implementations (prec 96: double-float).

    The D_alpha similarity has condition number alpha^{-(N-1)/N}; each FP64 (or FP32) evaluation
    carries about eps * log2(N) * that relative error, so two of them differ by at most a small
    multiple of it.  FP64 never needs to be looser than 1e-12 when alpha is moderate.
    """
    eps = {64: 2.0 ** -52, 32: 2.0 ** -23, 96: 2.0 ** -45}[prec]
    kappa = alpha ** (-(N - 1) / N)
    floor = {64: 1e-12, 32: 1e-5, 96: 1e-12}[prec]
    return max(floor, 50.0 * eps * kappa)


def to_dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).cuda()


def to_host(t):
    return t.detach().cpu().numpy()
