"""Pins of the oracle for general commuting symmetric blocks given as matrices (Assumption 1 (i),
Sec. 3): A_(k) need not be a_k I + b_k L; they share one orthonormal eigenbasis, which the oracle
finds itself from a generic combination of the blocks (no GPU).

Each test checks the blocks route against something else: the grid-Laplacian route of the same
operator, the dense definitions of Sec. 3 (C_alpha assembled, its principal square root, Def. 3),
the involution of Lemma 4, or an exact solve.
"""
import numpy as np
import pytest

import oracle as O
from oracle.precond import precond_dense, precond_dense_apply
from workloads import Problem, commuting_blocks_problem, fractional_problem, rhs_uniform


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def as_blocks(prob):
    """The same operator with its blocks a_k I + b_k L written out as dense matrices."""
    L = O.laplacian(prob).toarray()
    B = np.stack([prob.a[k] * np.eye(prob.M) + prob.b[k] * L for k in range(prob.N)])
    return Problem(prob.N, prob.d, prob.m, prob.h, np.zeros(prob.N), np.zeros(prob.N),
                   name=prob.name + "_blocks", meta=dict(blocks=B))


@pytest.mark.parametrize("prob", [fractional_problem(1, 15, 8, 0.5),
                                  fractional_problem(2, (3, 5), 6, 0.7)], ids=["1d", "2d"])
def test_blocks_route_reproduces_the_grid_route(prob):
    # the blocks a_k I + b_k L given as matrices: the eigenbasis found from a combination of the
    # blocks, the eigenvalues u_i^T A_(k) u_i and the block-sum matvec give the DST route's
    # matvec, P_alpha^{-1} and MINRES iterates
    q = as_blocks(prob)
    z = rhs_uniform(prob.n, 3)
    assert rel(O.bltt_matvec(q, z, flip=True), O.bltt_matvec(prob, z, flip=True)) < 1e-13
    assert abs(O.assumption_margin(q) - O.assumption_margin(prob)) < 1e-9 * O.assumption_margin(prob)
    for alpha in (1.0, 1e-3, 1e-8):
        assert rel(O.precond_apply(q, alpha, z), O.precond_apply(prob, alpha, z)) < 1e-9
    r1 = O.solve(q, z, alpha=1e-8, tol=1e-10)
    r2 = O.solve(prob, z, alpha=1e-8, tol=1e-10)
    assert r1["iters"] == r2["iters"]
    assert rel(r1["x"], r2["x"]) < 1e-8


@pytest.mark.parametrize("kind", ["modal", "poly"])
def test_common_eigenbasis_diagonalises_every_block(kind):
    p = commuting_blocks_problem(15, 6, seed=2, kind=kind)
    U = O.operators.commuting_eigh(p)
    assert np.abs(U.T @ U - np.eye(p.M)).max() < 1e-12
    B = np.asarray(p.meta["blocks"])
    scale = np.abs(B).max()
    for k in range(p.N):
        D = U.T @ B[k] @ U
        assert np.abs(D - np.diag(np.diag(D))).max() < 1e-11 * scale
    # the eigenvalues are the generator's, up to the order of the columns
    lam = O.block_eigenvalues(p)
    ref = np.asarray(p.meta["lam"])
    order_o = np.argsort(lam[0])
    order_r = np.argsort(ref[0])
    assert np.abs(lam[:, order_o] - ref[:, order_r]).max() < 1e-10 * np.abs(ref).max()


@pytest.mark.parametrize("alpha", [1.0, 1e-2, 1e-6])
def test_structured_precond_matches_dense_definition(alpha):
    # Def. 3 built densely from the assembled block alpha-circulant of the blocks themselves
    p = commuting_blocks_problem(7, 6, seed=3)
    y = rhs_uniform(p.n, 4)
    P = precond_dense(p, alpha)
    assert np.abs(P.imag).max() < 1e-8 * np.abs(P.real).max()
    z_dense = precond_dense_apply(P, y)
    assert rel(O.precond_apply(p, alpha, y), z_dense) < 1e-8


@pytest.mark.parametrize("alpha", [1.0, 1e-3])
def test_lemma4_involution_for_commuting_blocks(alpha):
    # (P_alpha^{-1} Y C_alpha)^2 = I (Lemma 4) with C_alpha assembled from the blocks
    p = commuting_blocks_problem(7, 5, seed=5, kind="poly")
    C = O.assemble_C_alpha(p, alpha)
    Y = O.assemble_Y(p.N, p.M)
    X = np.stack([O.precond_apply(p, alpha, col) for col in (Y @ C).T], axis=1)
    assert np.abs(X @ X - np.eye(p.n)).max() < 1e-8


@pytest.mark.parametrize("kind", ["modal", "poly"])
def test_minres_matches_exact_solutions(kind):
    p = commuting_blocks_problem(15, 8, seed=6, kind=kind)
    f = rhs_uniform(p.n, 7)
    u_lu = np.linalg.solve(O.assemble_A(p), f)
    u_ts = O.timestep_solve(p, f)
    assert rel(u_ts, u_lu) < 1e-12
    r = O.solve(p, f, alpha=1e-8, tol=1e-10)
    assert r["converged"] and r["iters"] <= 4
    assert rel(r["x"], u_lu) < 1e-8


def test_matvec_entry_matches_block_sum():
    p = commuting_blocks_problem(15, 8, seed=8)
    z = rhs_uniform(p.n, 9)
    y = O.bltt_matvec(p, z, flip=True)
    for n, i in [(0, 0), (3, 7), (7, 14)]:
        assert abs(O.operators.bltt_matvec_entry(p, z, n, i, flip=True) - y[n * p.M + i]) < 1e-12 * np.abs(y).max()
