"""Pins of the CPU oracle against what the paper and the mathematics fix (no GPU).

Each test names the passage it pins.  The oracle is only trusted because of these tests: every
function of it is checked against something other than itself (a definition assembled another way,
a closed form, a proved identity, a library routine, a printed result of the paper).
"""
import json
import math
import os

import numpy as np
import pytest
import scipy.sparse.linalg as spla
from scipy.linalg import sqrtm

import oracle as O
from oracle.precond import precond_dense, precond_dense_apply, sqrt_C_alpha_dense, d_alpha
from workloads import (fractional_problem, heat_bdf_problem, heat_cn_problem, l1_weights,
                       rhs_uniform, Problem)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
EPS = np.finfo(np.float64).eps


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def tiny_problems():
    return [
        fractional_problem(1, 7, 8, 0.5),
        fractional_problem(2, (3, 5), 6, 0.3),
        heat_cn_problem(2, (4, 3), 5),
        heat_bdf_problem(3, (2, 3, 2), 4),
    ]


# ---------------------------------------------------------------- U, L, mu (Sec. 3, Sec. 5.1)

@pytest.mark.parametrize("m", [1, 2, 7, 31])
def test_dst_symmetric_orthogonal(m):
    S = O.dst1_matrix(m)
    assert np.abs(S - S.T).max() < 1e-15
    assert np.abs(S @ S - np.eye(m)).max() < 1e-13


def test_U_diagonalises_L_with_closed_form_eigenvalues():
    # unequal m per axis catches axis-order mistakes
    for prob in [heat_bdf_problem(1, 9, 2), heat_bdf_problem(2, (3, 5), 2),
                 heat_bdf_problem(3, (2, 3, 4), 2, length=math.pi)]:
        L = O.laplacian(prob).toarray()
        M = prob.M
        U = O.apply_U(prob, np.eye(M)).T          # columns: U e_i
        D = U.T @ L @ U
        mu = O.laplacian_eigenvalues(prob)
        assert np.abs(D - np.diag(mu)).max() < 1e-10 * mu.max()
        # L is the SPD 2d+1 point stencil: diagonal sum_ax 2/h^2
        assert np.allclose(np.diag(L), sum(2.0 / h ** 2 for h in prob.h))


# ---------------------------------------------------------------- L1 weights (Sec. 5.2)

@pytest.mark.parametrize("gamma", [0.1, 0.5, 0.7, 0.9])
def test_l1_weights_closed_forms(gamma):
    N = 300
    l = l1_weights(gamma, N)
    g = math.gamma(2 - gamma)
    assert l[0] == pytest.approx(1.0 / g, rel=1e-15)
    # telescoping: sum_{k<N} l_k = (N^{1-g} - (N-1)^{1-g}) / Gamma(2-g) > 0
    assert l.sum() == pytest.approx((N ** (1 - gamma) - (N - 1) ** (1 - gamma)) / g, rel=1e-10)
    assert np.all(l[1:] < 0)
    assert np.abs(l[1:]).sum() < l[0]              # strict diagonal dominance of T
    # explicit k = 2 value
    assert l[2] == pytest.approx((3 ** (1 - gamma) - 2 * 2 ** (1 - gamma) + 1) / g, rel=1e-14)


def test_l1_weights_gamma_to_one_is_backward_euler():
    l = l1_weights(1.0, 6)
    assert np.array_equal(l, [1.0, -1.0, 0, 0, 0, 0])
    l2 = l1_weights(1.0 - 1e-9, 6)
    assert np.abs(l2 - l).max() < 1e-7
    p = fractional_problem(2, 5, 6, 1.0)
    q = heat_bdf_problem(2, 5, 6)
    assert np.allclose(p.a, q.a) and np.array_equal(p.b, q.b)


# ---------------------------------------------------------------- A and Y (eq. amatdef, Sec. 2)

@pytest.mark.parametrize("prob", tiny_problems(), ids=lambda p: p.name)
def test_matvec_matches_block_assembly(prob):
    A = O.assemble_A(prob)
    z = np.random.default_rng(1).standard_normal(prob.n)
    assert rel(O.bltt_matvec(prob, z), A @ z) < 1e-14
    Y = O.assemble_Y(prob.N, prob.M)
    assert rel(O.bltt_matvec(prob, z, flip=True), Y @ A @ z) < 1e-14
    from oracle.operators import bltt_matvec_entry
    full = O.bltt_matvec(prob, z, flip=True).reshape(prob.N, prob.M)
    for (n, i) in [(0, 0), (prob.N - 1, prob.M - 1), (prob.N // 2, prob.M // 2)]:
        assert bltt_matvec_entry(prob, z, n, i, flip=True) == pytest.approx(full[n, i], rel=1e-12, abs=1e-12)


@pytest.mark.parametrize("prob", tiny_problems(), ids=lambda p: p.name)
def test_YA_symmetric(prob):
    YA = O.assemble_Y(prob.N, prob.M) @ O.assemble_A(prob)
    assert np.array_equal(YA, YA.T)


def test_YA_symmetric_bilinear_moderate():
    prob = fractional_problem(2, 15, 64, 0.7)
    rng = np.random.default_rng(2)
    x, y = rng.standard_normal(prob.n), rng.standard_normal(prob.n)
    lhs = x @ O.bltt_matvec(prob, y, flip=True)
    rhs = y @ O.bltt_matvec(prob, x, flip=True)
    assert abs(lhs - rhs) <= 1e-12 * np.linalg.norm(x) * np.linalg.norm(O.bltt_matvec(prob, y))


# ---------------------------------------------------------------- preconditioner (Sec. 3, Sec. 5.1)

def precond_tol(N, alpha):
    """Rounding bound for two independent FP64 evaluations of P_alpha^{-1}: the D_alpha similarity
    has condition number alpha^{-(N-1)/N}, so the FFT route carries ~eps * that (times log N)."""
    return max(1e-12, 50 * EPS * alpha ** (-(N - 1) / N))


@pytest.mark.parametrize("prob", tiny_problems(), ids=lambda p: p.name)
@pytest.mark.parametrize("alpha", [1.0, 0.1, 1e-2, 1e-4, 1e-8])
def test_precond_structured_matches_dense(prob, alpha):
    P = precond_dense(prob, alpha)
    y = np.random.default_rng(3).standard_normal(prob.n)
    zd = precond_dense_apply(P, y)
    zs, imag = O.precond_apply(prob, alpha, y, return_imag=True)
    assert rel(zs, zd) <= precond_tol(prob.N, alpha)
    assert imag < 1e-6


@pytest.mark.parametrize("prob", tiny_problems()[:3], ids=lambda p: p.name)
@pytest.mark.parametrize("alpha", [1.0, 1e-3])
def test_lemma3_sqrt_real_and_YC_half_symmetric(prob, alpha):
    R = sqrt_C_alpha_dense(prob, alpha)
    assert np.abs(np.imag(R)).max() <= 1e-10 * np.abs(R).max()        # Lemma 3 (b)
    Y = O.assemble_Y(prob.N, prob.M)
    YR = Y @ np.real(R)
    assert np.abs(YR - YR.T).max() <= 1e-9 * np.abs(YR).max()         # Lemma 3 (c)
    assert np.linalg.matrix_rank(np.real(R)) == prob.n                # Lemma 3 (a)


@pytest.mark.parametrize("prob", tiny_problems()[:3], ids=lambda p: p.name)
@pytest.mark.parametrize("alpha", [1.0, 1e-2, 1e-5])
def test_precond_spd(prob, alpha):
    P = np.real(precond_dense(prob, alpha))
    assert np.abs(P - P.T).max() <= 1e-10 * np.abs(P).max()
    assert np.linalg.eigvalsh(0.5 * (P + P.T)).min() > 0


@pytest.mark.parametrize("prob", tiny_problems()[:3], ids=lambda p: p.name)
@pytest.mark.parametrize("alpha", [1.0, 1e-2, 1e-4])
def test_lemma4_preconditioned_circulant_is_involution(prob, alpha):
    # (P^{-1} Y C_alpha)^2 = I
    C = O.assemble_C_alpha(prob, alpha)
    Y = O.assemble_Y(prob.N, prob.M)
    y = np.random.default_rng(4).standard_normal(prob.n)
    t = O.precond_apply(prob, alpha, Y @ (C @ y))
    t = O.precond_apply(prob, alpha, Y @ (C @ t))
    assert rel(t, y) <= 100 * precond_tol(prob.N, alpha)


def test_lemma11_spectrum_clusters_at_pm1_linearly_in_alpha():
    prob = fractional_problem(1, 7, 8, 0.7)
    A = O.assemble_A(prob)
    YA = O.assemble_Y(prob.N, prob.M) @ A
    dist = {}
    for alpha in [1e-3, 1e-4, 1e-5]:
        P = np.real(precond_dense(prob, alpha))
        ev = np.linalg.eigvals(np.linalg.solve(P, YA))
        assert np.abs(ev.imag).max() < 1e-6                       # similar to a symmetric matrix
        ev = ev.real
        dist[alpha] = np.abs(np.abs(ev) - 1.0).max()
        assert (ev < 0).sum() > 0 and (ev > 0).sum() > 0          # indefinite: both clusters
    assert dist[1e-3] < 1e-1
    for a, b in [(1e-3, 1e-4), (1e-4, 1e-5)]:
        assert 4.0 < dist[a] / dist[b] < 25.0                     # distance proportional to alpha


@pytest.mark.parametrize("prob", tiny_problems(), ids=lambda p: p.name)
def test_alpha1_two_pass_equals_one_pass(prob):
    y = np.random.default_rng(5).standard_normal(prob.n)
    assert rel(O.precond_apply(prob, 1.0, y), O.precond_apply_one_pass_alpha1(prob, y)) < 1e-13


@pytest.mark.parametrize("alpha", [1.0, 1e-3, 1e-8])
def test_eigenvalue_conjugate_symmetry(alpha):
    prob = fractional_problem(2, (3, 4), 9, 0.4)
    lam = O.alpha_circulant_eigs(prob, alpha)                     # (M, N)
    assert np.abs(lam[:, 0].imag).max() <= 1e-14 * np.abs(lam).max()
    assert lam[:, 0].real.min() > 0
    N = prob.N
    for k in range(1, N):
        assert np.abs(lam[:, N - k] - np.conj(lam[:, k])).max() <= 1e-13 * np.abs(lam).max()
    assert lam.real.min() > 0                                     # right half plane (Sec. 3)


def test_eigenvalues_match_dense_circulant_block():
    # lambda^(k,alpha) of eq. hatcalphaieigvaldef are the eigenvalues of C_hat_{alpha,i}
    prob = fractional_problem(1, 3, 7, 0.6)
    alpha = 0.05
    lam_blocks = O.block_eigenvalues(prob)                        # (N, M)
    lam = O.alpha_circulant_eigs(prob, alpha)
    N = prob.N
    for i in range(prob.M):
        c = lam_blocks[:, i]
        Ch = np.zeros((N, N))
        for r in range(N):
            for q in range(N):
                Ch[r, q] = c[r - q] if r >= q else alpha * c[N + r - q]
        ev = np.sort_complex(np.linalg.eigvals(Ch))
        assert np.abs(ev - np.sort_complex(lam[i])).max() < 1e-10 * np.abs(ev).max()


def test_assumption_margin():
    for p in tiny_problems():
        assert O.assumption_margin(p) > 0
    bad = fractional_problem(1, 7, 8, 0.5)
    bad.b = bad.b.copy()
    bad.b[1] = -2.0          # |A_(1)| outweighs A_(0) on the high modes
    assert O.assumption_margin(bad) <= 0


# ---------------------------------------------------------------- MINRES (Sec. 4.2, Sec. 5.2)

@pytest.mark.parametrize("precond", ["alpha", "one", "none"])
def test_minres_iterates_match_scipy(precond):
    prob = fractional_problem(1, 7, 8, 0.5)
    f = rhs_uniform(prob.n, 6)
    b = f.reshape(prob.N, prob.M)[::-1].reshape(-1)
    A = lambda z: O.bltt_matvec(prob, z, flip=True)
    alpha = {"alpha": 1e-2, "one": 1.0, "none": None}[precond]
    Pinv = (lambda v: v.copy()) if alpha is None else (lambda v: O.precond_apply(prob, alpha, v))
    Aop = spla.LinearOperator((prob.n, prob.n), matvec=A, dtype=np.float64)
    Mop = spla.LinearOperator((prob.n, prob.n), matvec=Pinv, dtype=np.float64)
    for k in [1, 2, 3, 4]:
        ours = O.minres(A, Pinv, b, tol=0.0, maxit=k)
        ref, _ = spla.minres(Aop, b, M=Mop, rtol=1e-30, maxiter=k)
        assert ours["iters"] == k
        assert rel(ours["x"], ref) < 1e-9


@pytest.mark.parametrize("prob", tiny_problems(), ids=lambda p: p.name)
def test_minres_matches_dense_lu(prob):
    f = rhs_uniform(prob.n, 7)
    r = O.solve(prob, f, alpha=1e-8, tol=1e-8)
    assert r["converged"] and r["relres_true"] <= 1e-8
    u = np.linalg.solve(O.assemble_A(prob), f)
    assert rel(r["x"], u) < 1e-6
    h = r["eta_history"]
    assert all(h[j + 1] <= h[j] * (1 + 1e-12) for j in range(len(h) - 1))   # monotone


def test_minres_matches_time_stepping():
    prob = fractional_problem(2, 15, 48, 0.6)
    f = rhs_uniform(prob.n, 8)
    r = O.solve(prob, f, alpha=1e-8, tol=1e-8)
    u = O.timestep_solve(prob, f)
    assert r["relres_true"] <= 1e-8
    assert rel(r["x"], u) < 1e-6
    assert rel(O.bltt_matvec(prob, u), f) < 1e-12              # time stepping solves A u = f


def _golden_problem(c):
    m = c["m_plus_1"] - 1
    L = c["domain_length"]
    if c["example"] == "heat_bdf":
        return heat_bdf_problem(2, m, c["N"], length=L)
    if c["example"] == "heat_cn":
        return heat_cn_problem(2, m, c["N"], length=L)
    return fractional_problem(2, m, c["N"], c["gamma"], length=L)


def test_paper_iteration_counts():
    g = json.load(open(os.path.join(GOLDEN, "paper_iteration_counts.json")))
    for c in g["cases"]:
        prob = _golden_problem(c)
        assert prob.n == c["dof"]
        f = rhs_uniform(prob.n, 11)
        r = O.solve(prob, f, alpha=g["alpha"], tol=g["tol"])
        assert r["iters"] == c["iters"], (c, r["iters"])


def test_theorem1_rate_bound_tiny():
    # Lemma 11 / Theorem 1 constants from the dense S(A): alpha = 1e-8 <= zeta for delta = 1/2,
    # and the preconditioned residual obeys ||r_k|| <= 2 delta^{k-1} ||r_0||.
    prob = fractional_problem(1, 5, 6, 0.5)
    A = O.assemble_A(prob)
    SA = np.real(sqrtm(A))
    lmin = np.linalg.eigvalsh(SA.T @ SA).min()
    c0 = O.assumption_margin(prob)
    lam0 = O.block_eigenvalues(prob)[0]
    A0norm = float(lam0.max())
    SAn = np.linalg.norm(SA, 2)
    nu = min(1.0, 2 * c0 * lmin / (4 * math.sqrt(c0) * (A0norm - c0) * SAn + (A0norm - c0) ** 2))
    mu = 2 * (A0norm - c0) / lmin
    delta = 0.5
    zeta = min(delta ** 2 / mu, nu)
    alpha = min(1e-8, zeta)
    assert zeta >= 1e-8
    f = rhs_uniform(prob.n, 12)
    b = f.reshape(prob.N, prob.M)[::-1].reshape(-1)
    Afn = lambda z: O.bltt_matvec(prob, z, flip=True)
    Pinv = lambda v: O.precond_apply(prob, alpha, v)
    r0 = np.linalg.norm(Pinv(b))
    for k in [1, 2, 3]:
        x = O.minres(Afn, Pinv, b, tol=0.0, maxit=k)["x"]
        rk = np.linalg.norm(Pinv(Afn(x) - b))
        assert rk <= 2 * delta ** (k - 1) * r0 * (1 + 1e-8) + 1e-12 * r0


# ------------------------------------------- variable coefficient (Sec. 5.2, Example heateqvarcoeff)

def _var1d(m, coef):
    """1-D problem on (0, 1) whose L is L_a for the coefficient function coef (faces at (f+1/2)h)."""
    from workloads import Problem
    p = heat_cn_problem(1, m, 4)
    h = p.h[0]
    faces = coef((np.arange(m + 1) + 0.5) * h)
    return Problem(p.N, p.d, p.m, p.h, p.a, p.b, name="var1d",
                   meta=dict(faces=(faces,), abar=float(np.mean(coef((np.arange(m) + 1.0) * h)))))


def test_variable_laplacian_exact_on_quadratics():
    # The conservative central difference is exact when the flux a u' is quadratic: with a(x) = x
    # and u = x (1 - x) (zero at both ends), -(a u')' = 4x - 1 at every interior point.
    m = 31
    p = _var1d(m, lambda x: x)
    x = (np.arange(m) + 1.0) / (m + 1)
    Lu = O.laplacian(p) @ (x * (1 - x))
    assert np.max(np.abs(Lu - (4 * x - 1))) < 1e-10


def test_variable_laplacian_properties():
    from workloads import heat_cn_varcoeff_problem
    import copy
    p = heat_cn_varcoeff_problem(7, 4)
    L = O.laplacian(p)
    assert abs(L - L.T).max() == 0.0
    assert np.linalg.eigvalsh(L.toarray()).min() > 0                   # -Delta_{a,h} is SPD
    one = copy.deepcopy(p)
    one.meta["faces"] = tuple(np.ones_like(f) for f in p.meta["faces"])
    plain = copy.deepcopy(p)
    plain.meta.pop("faces")
    assert abs(O.laplacian(one) - O.laplacian(plain)).max() == 0.0     # a = 1 gives Delta_h
    # the block sum entry by entry agrees with the Toeplitz-product matvec
    from oracle.operators import bltt_matvec_entry
    z = np.random.default_rng(3).standard_normal(p.n)
    y = O.bltt_matvec(p, z, flip=True)
    e = np.array([bltt_matvec_entry(p, z, n, i, flip=True) for n in range(p.N) for i in range(p.M)])
    assert rel(e, y) < 1e-14
    # the preconditioner is that of the mean-coefficient blocks (eq. meancoeffheateqtsmat)
    lam = O.block_eigenvalues(p)
    mu = O.laplacian_eigenvalues(p)
    assert np.allclose(lam[0], p.a[0] + p.meta["abar"] * p.b[0] * mu, rtol=1e-15)


def test_paper_iteration_counts_varcoeff():
    from workloads import heat_cn_varcoeff_problem
    g = json.load(open(os.path.join(GOLDEN, "paper_iteration_counts_varcoeff.json")))
    for c in g["cases"]:
        prob = heat_cn_varcoeff_problem(c["m_plus_1"] - 1, c["N"])
        assert prob.n == c["dof"]
        f = rhs_uniform(prob.n, 11)
        r = O.solve(prob, f, alpha=g["alpha"], tol=g["tol"])
        assert r["iters"] == c["iters"], (c, r["iters"])


def _paper_rhs(c):
    """The paper's own right-hand side of a golden case (its examples' data)."""
    from workloads import heat_cn_varcoeff_problem, paper_data_fractional, paper_data_heat_var
    if c["example"] == "heat_cn_var":
        prob = heat_cn_varcoeff_problem(c["m_plus_1"] - 1, c["N"])
        F, u0 = paper_data_heat_var(prob)
        tau = 1.0 / prob.N
        # CN first block: f^(1/2) - (1/tau) L_{a,2} u_0 with L_{a,2} = -I - (tau/2) Delta_{a,h}
        F[0] += u0 / tau - 0.5 * (O.laplacian(prob) @ u0)
        return prob, F.reshape(-1)
    prob = fractional_problem(2, c["m_plus_1"] - 1, c["N"], c["gamma"], length=math.pi)
    return prob, paper_data_fractional(prob, c["gamma"])


def test_paper_iteration_counts_with_paper_data():
    # both preconditioners on the paper's own data: MINRES-P_alpha and the comparison MINRES-P_1
    g = json.load(open(os.path.join(GOLDEN, "paper_iteration_counts_paper_data.json")))
    for c in g["cases"]:
        prob, f = _paper_rhs(c)
        r = O.solve(prob, f, alpha=g["alpha"], tol=g["tol"], precond=c["precond"], maxit=2000)
        assert abs(r["iters"] - c["iters"]) <= c["slack"], (c, r["iters"])


def _example4_cases():
    g = json.load(open(os.path.join(GOLDEN, "paper_iteration_counts_example4.json")))
    return g, g["cases"]


@pytest.mark.parametrize("case", _example4_cases()[1],
                         ids=[f"{c['table']}_g{c['gamma']}_N{c['N']}_m{c['m_plus_1']}_{c['precond']}"
                              for c in _example4_cases()[1]])
def test_example4_paper_counts(case):
    # Example 4 (variable coefficient a = 35 + x^3.5 + y^3.5, L1 fractional) on its own data:
    # Tables 7-9 print 8 iterations for MINRES-P_alpha at every size and order, and 8 to 10 for
    # MINRES-P_1; the mean-coefficient preconditioner reproduces them
    from workloads import fractional_varcoeff_problem, paper_data_frac_var
    g = _example4_cases()[0]
    prob = fractional_varcoeff_problem(case["m_plus_1"] - 1, case["N"], case["gamma"])
    f = paper_data_frac_var(prob, case["gamma"])
    alpha = g["alpha"] if case["precond"] == "alpha" else 1.0
    r = O.solve(prob, f, alpha=alpha, tol=g["tol"], precond=case["precond"], maxit=500)
    assert abs(r["iters"] - case["iters"]) <= case["slack"], (case, r["iters"])


# ------------------------------------- dense commuting blocks (Sec. 3: A_(k) = a_k I + b_k K)

def _with_K(p, K):
    from workloads import Problem
    return Problem(p.N, p.d, p.m, p.h, p.a, p.b, name=p.name + "_K", meta=dict(p.meta, K=K))


def test_dense_operator_reproduces_the_dst_path():
    # K = the finite-difference Laplacian as a dense matrix: its eigenvectors span the DST basis,
    # so every operator of the method must agree with the DST path
    p = fractional_problem(2, (7, 5), 16, 0.6)
    pk = _with_K(p, O.laplacian(p).toarray())
    z = np.random.default_rng(71).standard_normal(p.n)
    assert rel(O.bltt_matvec(pk, z, flip=True), O.bltt_matvec(p, z, flip=True)) < 1e-14
    assert np.allclose(np.sort(O.laplacian_eigenvalues(pk)), np.sort(O.laplacian_eigenvalues(p)),
                       rtol=1e-12)
    for alpha in (1.0, 1e-2, 1e-8):
        # two FP64 evaluations differ by a few eps times kappa(D_alpha) = alpha^{-(N-1)/N}
        tol = max(1e-12, 100 * 2.0 ** -52 * alpha ** (-(p.N - 1) / p.N))
        assert rel(O.precond_apply(pk, alpha, z), O.precond_apply(p, alpha, z)) < tol
    f = rhs_uniform(p.n, 72)
    r, rk = O.solve(p, f, alpha=1e-8, tol=1e-10), O.solve(pk, f, alpha=1e-8, tol=1e-10)
    assert r["iters"] == rk["iters"] and rel(rk["x"], r["x"]) < 1e-9


def test_dense_operator_precond_matches_dense_definition():
    # a random SPD K on a tiny problem: the steps of Sec. 5.1 against P_alpha of Def. 3 built
    # densely from the blocks a_k I + b_k K
    p = fractional_problem(1, 5, 6, 0.5)
    G = np.random.default_rng(73).standard_normal((p.M, p.M))
    pk = _with_K(p, G @ G.T + p.M * np.eye(p.M))
    v = np.random.default_rng(74).standard_normal(p.n)
    for alpha in (1.0, 1e-2):
        P = precond_dense(pk, alpha)
        assert rel(O.precond_apply(pk, alpha, v), precond_dense_apply(P, v)) < 1e-9


def test_dense_operator_exact_preconditioner_for_variable_coefficient():
    # with K = L_a the preconditioner is P_alpha of the true blocks (no mean-coefficient
    # approximation): the clustered spectrum of Theorem 1 gives a few iterations instead of 10
    from workloads import heat_cn_varcoeff_problem
    p = heat_cn_varcoeff_problem(15, 32)
    meta = {k: v for k, v in p.meta.items() if k not in ("faces", "abar")}
    from workloads import Problem
    pk = Problem(p.N, p.d, p.m, p.h, p.a, p.b, name="cnvar_K", meta=dict(meta, K=O.laplacian(p).toarray()))
    f = rhs_uniform(p.n, 75)
    r_mean = O.solve(p, f, alpha=1e-8, tol=1e-6)
    r_exact = O.solve(pk, f, alpha=1e-8, tol=1e-6)
    assert r_mean["iters"] == 10 and r_exact["iters"] <= 3
    assert rel(O.bltt_matvec(pk, r_exact["x"]), f) <= 1e-6
