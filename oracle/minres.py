"""Oracle: textbook preconditioned MINRES on Y A u = Y f (Sec. 2, Sec. 4.2, Sec. 5.2).

The paper names no MINRES implementation; its convergence Lemma (Sec. 4.2) is the one of Elman,
Silvester and Wathen, whose preconditioned MINRES (Lanczos in the P^{-1} inner product plus Givens
QR) is written out here step by step, zero initial guess (Sec. 5.2).

Stopping rule (the paper's "||r_k||_2 <= 1e-6" does not say which residual or whether it is
relative): stop when the recurrence estimate |eta_j| / eta_0 <= tol, eta_j being the P^{-1}-norm
of the residual; then compute the true relative residual ||Yf - YA u_j||_2 / ||Yf||_2 and stop only
if it is <= tol as well, else keep iterating.  An iteration is one (A z, P^{-1} v) pair after the
initial P^{-1} b.  gamma_{j+1} = 0 is an exact (lucky) breakdown: stop after the x update.

Test infrastructure only (see the package docstring).
"""
from __future__ import annotations

import math

import numpy as np

from .operators import bltt_matvec
from .precond import precond_apply


class MinresError(RuntimeError):
    pass


def minres(apply_A, apply_Pinv, b, tol=1e-8, maxit=1000, true_check=True):
    """Preconditioned MINRES (ESW algorithm) for a symmetric A and SPD P, x0 = 0.

    Returns a dict: x, iters, eta_history (|eta_j|/eta_0 for j = 0..iters), relres_true,
    converged, status ("converged", "not_converged", "breakdown").
    """
    b = np.asarray(b, dtype=np.float64)
    n = b.size
    x = np.zeros(n)
    v_prev = np.zeros(n)
    v = b.copy()                           # v_1 = b - A x_0
    z = apply_Pinv(v)                      # z_1 = P^{-1} v_1
    g2 = float(np.dot(z, v))
    if not math.isfinite(g2) or g2 < 0.0:
        raise MinresError("<z_1, v_1> is negative or not finite")
    gamma = math.sqrt(g2)                  # gamma_1
    normb = float(np.linalg.norm(b))
    hist = [1.0]
    if gamma == 0.0:
        return dict(x=x, iters=0, eta_history=hist, relres_true=0.0, converged=True,
                    status="converged")
    gamma_prev = 1.0                       # gamma_0 (multiplies v_0 = 0)
    eta = gamma
    eta0 = gamma
    s_prev = s = 0.0                       # s_0, s_1
    c_prev = c = 1.0                       # c_0, c_1
    w_prev = np.zeros(n)                   # w_0
    w = np.zeros(n)                        # w_1
    relres = 1.0
    for j in range(1, maxit + 1):
        z = z / gamma                                          # z_j
        Az = apply_A(z)
        delta = float(np.dot(Az, z))                           # delta_j
        v_next = Az - (delta / gamma) * v - (gamma / gamma_prev) * v_prev
        z_next = apply_Pinv(v_next)
        g2 = float(np.dot(z_next, v_next))
        if not math.isfinite(g2) or g2 < 0.0:
            raise MinresError(f"<z_{j+1}, v_{j+1}> = {g2} is negative or not finite")
        gamma_next = math.sqrt(g2)                             # gamma_{j+1}
        a0 = c * delta - c_prev * s * gamma
        a1 = math.sqrt(a0 * a0 + gamma_next * gamma_next)
        a2 = s * delta + c_prev * c * gamma
        a3 = s_prev * gamma
        c_next = a0 / a1
        s_next = gamma_next / a1
        w_next = (z - a3 * w_prev - a2 * w) / a1
        x = x + c_next * eta * w_next
        eta = -s_next * eta
        hist.append(abs(eta) / eta0)
        # shift the recurrences
        v_prev, v = v, v_next
        z = z_next
        w_prev, w = w, w_next
        gamma_prev, gamma = gamma, gamma_next
        s_prev, s = s, s_next
        c_prev, c = c, c_next
        if gamma_next == 0.0 or abs(eta) / eta0 <= tol:
            if true_check:
                r = b - apply_A(x)
                relres = float(np.linalg.norm(r)) / normb
                if relres <= tol or gamma_next == 0.0:
                    return dict(x=x, iters=j, eta_history=hist, relres_true=relres,
                                converged=relres <= tol, status="converged")
            else:
                return dict(x=x, iters=j, eta_history=hist, relres_true=float("nan"),
                            converged=True, status="converged")
    r = b - apply_A(x)
    relres = float(np.linalg.norm(r)) / normb
    return dict(x=x, iters=maxit, eta_history=hist, relres_true=relres, converged=False,
                status="not_converged")


def solve(prob, f, alpha=1e-8, tol=1e-8, maxit=1000, precond="alpha"):
    """MINRES-P_alpha (precond="alpha"), MINRES-P_1 ("one") or MINRES-I ("none") for Y A u = Y f.

    The right-hand side is b = Y f (eq. symmetrizedblttsys); the returned x solves A u = f.
    """
    f = np.asarray(f, dtype=np.float64)
    N, M = prob.N, prob.M
    b = f.reshape(N, M)[::-1].reshape(-1).copy()
    A = lambda z: bltt_matvec(prob, z, flip=True)
    if precond == "alpha":
        P = lambda v: precond_apply(prob, alpha, v)
    elif precond == "one":
        P = lambda v: precond_apply(prob, 1.0, v)
    elif precond == "none":
        P = lambda v: v.copy()
    else:
        raise ValueError(precond)
    return minres(A, P, b, tol=tol, maxit=maxit)
