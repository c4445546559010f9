"""Oracle for the ABAC preconditioner P_alpha = |C_alpha| (Sec. 3) and its inverse (Sec. 5.1).

Two independent routes:

* dense (tiny sizes): C_alpha assembled from eq. tensordef2calpha, its principal square root by a
  Schur method (Def. 2 with the principal branch; C_alpha's eigenvalues lie in the open right half
  plane, Sec. 3, so this is the square root of Def. 2), then |C_alpha| = (C^1/2)^* C^1/2 (Def. 3,
  eq. calphaabsdef) and a dense solve;
* structured (any size): the paper's three steps for (C_alpha^{-1/2})^* y, then the same three
  steps with D_alpha^{-1} F Lambda^{-1/2} F^* D_alpha for C_alpha^{-1/2} (Sec. 5.1), with the
  eigenvalues lambda_i^(k,alpha) of eq. hatcalphaieigvaldef.

Test infrastructure only (see the package docstring).
"""
from __future__ import annotations

import numpy as np
from scipy.linalg import sqrtm, solve

from .operators import apply_U, block_eigenvalues, assemble_C_alpha


def _F(x):
    """Unitary F = N^{-1/2} [theta^{(i-1)(j-1)}], theta = exp(+2 pi i/N), along axis -1 (eq. after
    hatcalphaidiagform).  F x = sqrt(N) * ifft(x)."""
    n = x.shape[-1]
    return np.fft.ifft(x, axis=-1) * np.sqrt(n)


def _F_star(x):
    """F^* x = fft(x)/sqrt(N) (the DFT with exp(-2 pi i jk/N), unitarily scaled)."""
    n = x.shape[-1]
    return np.fft.fft(x, axis=-1) / np.sqrt(n)


def d_alpha(N: int, alpha: float) -> np.ndarray:
    """Diagonal of D_alpha = diag(alpha^{(i-1)/N}), i = 1..N (eq. after hatcalphaidiagform)."""
    return alpha ** (np.arange(N) / N)


def alpha_circulant_eigs(prob, alpha: float) -> np.ndarray:
    """lambda_i^(k,alpha) = sum_j C_hat_{alpha,i}(j,1) alpha^{(j-1)/N} theta^{-(k-1)(j-1)} (eq. hatcalphaieigvaldef).

    The first column of C_hat_{alpha,i} (eq. hatcalphaidef) is (lambda_i^(0), ..., lambda_i^(N-1)).
    Returns an (M, N) complex array: row i holds the diagonal of Lambda_{alpha,i}.
    """
    lam = block_eigenvalues(prob)                  # (N, M), column i = first column of C_hat_i
    cols = lam.T                                   # Pi^T: mode-major, (M, N)
    return np.sqrt(prob.N) * _F_star(d_alpha(prob.N, alpha)[None, :] * cols)


def precond_apply(prob, alpha: float, y: np.ndarray, return_imag: bool = False):
    """z = P_alpha^{-1} y = C_alpha^{-1/2} (C_alpha^{-1/2})^* y by the steps of Sec. 5.1.

    (C_alpha^{-1/2})^* y:
      Step 1  y~ = Pi^T (I_N (x) U)^T y                      (DST of every time slice, mode-major)
      Step 2  z~ = blockdiag(D_alpha F conj(Lambda_{alpha,i})^{-1/2} F^* D_alpha^{-1}) y~
      Step 3  y^ = (I_N (x) U) Pi z~
    then C_alpha^{-1/2} y^ by the same three steps with D_alpha^{-1} F Lambda^{-1/2} F^* D_alpha
    (eq. sqrtcalphabdiagform).  Powers ^{-1/2} take the principal branch (Def. 2).  After each F
    the imaginary part is rounding only (Lemma 3.1, Lemma 3 (b)); it is discarded and its largest
    magnitude relative to the real part is returned when `return_imag`.
    """
    N, M = prob.N, prob.M
    lam = alpha_circulant_eigs(prob, alpha)        # (M, N)
    d = d_alpha(N, alpha)[None, :]
    Y = np.asarray(y, dtype=np.float64).reshape(N, M)
    imag = 0.0

    # (C_alpha^{-1/2})^* y
    yt = apply_U(prob, Y, transpose=True).T        # Steps 1: U^T per slice, then Pi^T -> (M, N)
    t = _F(np.conj(lam) ** -0.5 * _F_star(yt / d)) * d     # Step 2
    imag = max(imag, float(np.max(np.abs(t.imag))) / max(float(np.max(np.abs(t.real))), 1e-300))
    yhat = apply_U(prob, np.ascontiguousarray(t.real.T))   # Step 3: Pi, then U per slice

    # C_alpha^{-1/2} y^
    st = apply_U(prob, yhat, transpose=True).T
    s = _F(lam ** -0.5 * _F_star(st * d)) / d
    imag = max(imag, float(np.max(np.abs(s.imag))) / max(float(np.max(np.abs(s.real))), 1e-300))
    z = apply_U(prob, np.ascontiguousarray(s.real.T)).reshape(-1)
    return (z, imag) if return_imag else z


def precond_apply_one_pass_alpha1(prob, y: np.ndarray) -> np.ndarray:
    """For alpha = 1, C_1 is normal and |C_1| = Q^* |Lambda| Q (Def. 1), so
    P_1^{-1} y = (I (x) U) Pi blockdiag(F |Lambda_{1,i}|^{-1} F^*) Pi^T (I (x) U)^T y: one pass."""
    N, M = prob.N, prob.M
    lam = alpha_circulant_eigs(prob, 1.0)
    yt = apply_U(prob, np.asarray(y, dtype=np.float64).reshape(N, M), transpose=True).T
    t = _F(_F_star(yt) / np.abs(lam))
    return apply_U(prob, np.ascontiguousarray(t.real.T)).reshape(-1)


def sqrt_C_alpha_dense(prob, alpha: float) -> np.ndarray:
    """C_alpha^{1/2}: the principal square root of the dense C_alpha (Def. 2), Schur method."""
    C = assemble_C_alpha(prob, alpha)
    R = sqrtm(C)
    return R


def precond_dense(prob, alpha: float) -> np.ndarray:
    """Dense P_alpha = |C_alpha| = (C_alpha^{1/2})^* C_alpha^{1/2} (Def. 3, eqs. calphaabsdef, precdef).

    Returned as a complex array; Lemma 3 (b) says it is real (tests check the imaginary part).
    """
    R = sqrt_C_alpha_dense(prob, alpha)
    return R.conj().T @ R


def precond_dense_apply(P: np.ndarray, y: np.ndarray) -> np.ndarray:
    """P^{-1} y by a dense solve with the real part of P."""
    return solve(P.real, y, assume_a="sym")
