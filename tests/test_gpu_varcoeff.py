"""Variable-coefficient blocks (Sec. 5.2, Example heateqvarcoeff) against the oracle: the matvec with
L_a = -Delta_{a,h} on the direct (Crank-Nicolson) and FFT (L1 fractional) paths, the
mean-coefficient preconditioner, solves in the physical basis (Table 3's iteration count), and the
combinations the library declines."""
import copy

import numpy as np
import pytest

import oracle as O
from workloads import Problem, fractional_problem, heat_cn_problem, heat_cn_varcoeff_problem, rhs_uniform
from _gpu_helpers import precond_tol, rel, to_dev, to_host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    from paper_2307_07749_gb300 import build
    build.build()
    import paper_2307_07749_gb300 as mod
    return mod


def frac_var(m=31, N=32, gamma=0.7):
    """L1 fractional blocks (b = e_0, the FFT matvec) with the coefficient of Example
    heateqvarcoeff on (0,1)^2: the paper's non-local evolutionary equation form."""
    p = fractional_problem(2, m, N, gamma)
    q = heat_cn_varcoeff_problem(m, N)
    return Problem(p.N, p.d, p.m, p.h, p.a, p.b, name=f"fracvar2d_N{N}_m{m}",
                   meta=dict(p.meta, faces=q.meta["faces"], abar=q.meta["abar"]))


def var_problems():
    return [heat_cn_varcoeff_problem(31, 32), heat_cn_varcoeff_problem(15, 64), frac_var()]


VIDS = [p.name for p in var_problems()]


@pytest.mark.parametrize("prob", var_problems(), ids=VIDS)
@pytest.mark.parametrize("flip", [0, 1])
@pytest.mark.parametrize("arith", [1, 2], ids=["f64", "f32x2"])
def test_varcoeff_matvec_parity(B, prob, flip, arith):
    s = B.Solver(prob)
    s.set_matvec_arith(arith)
    z = np.random.default_rng(61).standard_normal(prob.n)
    y = to_host(s.matvec(to_dev(z), flip=bool(flip)))
    assert rel(y, O.bltt_matvec(prob, z, flip=bool(flip))) <= 1e-12


@pytest.mark.parametrize("prob", var_problems(), ids=VIDS)
@pytest.mark.parametrize("alpha", [1.0, 1e-8])
def test_varcoeff_precond_parity(B, prob, alpha):
    s = B.Solver(prob)
    v = np.random.default_rng(62).standard_normal(prob.n)
    z = to_host(s.precond_apply(alpha, to_dev(v), precision=64))
    assert rel(z, O.precond_apply(prob, alpha, v)) <= precond_tol(prob.N, alpha)


def test_varcoeff_unit_coefficient_is_the_constant_problem(B):
    p = heat_cn_problem(2, 15, 16)
    q = copy.deepcopy(p)
    q.meta["faces"] = (np.ones((15, 16)), np.ones((16, 15)))
    q.meta["abar"] = 1.0
    z = to_dev(np.random.default_rng(63).standard_normal(p.n))
    sp, sq = B.Solver(p), B.Solver(q)
    assert np.array_equal(to_host(sp.matvec(z)), to_host(sq.matvec(z)))
    f = to_dev(rhs_uniform(p.n, 64))
    up, ip = sp.solve(f, alpha=1e-8, tol=1e-8, basis=2)
    uq, iq = sq.solve(f, alpha=1e-8, tol=1e-8)        # AUTO: the physical basis
    assert ip["iters"] == iq["iters"] and np.array_equal(to_host(up), to_host(uq))


def test_varcoeff_table3_iterations(B):
    # Table 3: MINRES-P_alpha, alpha = 1e-8, tolerance 1e-6: 10 iterations (oracle: 10)
    prob = heat_cn_varcoeff_problem(31, 32)
    f = rhs_uniform(prob.n, 11)
    ref = O.solve(prob, f, alpha=1e-8, tol=1e-6)
    u, info = B.Solver(prob).solve(to_dev(f), alpha=1e-8, tol=1e-6, maxit=100, precision=64)
    assert info["status"] == 0 and info["basis"] == 2
    assert info["iters"] == ref["iters"] == 10
    assert rel(O.bltt_matvec(prob, to_host(u)), f) <= 1e-6


@pytest.mark.parametrize("prob", var_problems()[1:], ids=VIDS[1:])
@pytest.mark.parametrize("form", [dict(precision=64, alpha=1e-8), dict(precision=32, alpha=1e-3)],
                         ids=["f64", "f32"])
def test_varcoeff_solve(B, prob, form):
    f = rhs_uniform(prob.n, 65)
    ref = O.solve(prob, f, alpha=1e-8, tol=1e-8)
    u, info = B.Solver(prob).solve(to_dev(f), tol=1e-8, maxit=200, **form)
    assert info["status"] == 0, info
    if form["precision"] == 64:
        assert abs(info["iters"] - ref["iters"]) <= 1, (info["iters"], ref["iters"])
    uh = to_host(u)
    assert info["relres_true"] <= 1e-8 and rel(O.bltt_matvec(prob, uh), f) <= 1e-8
    assert rel(uh, ref["x"]) <= 1e-6


def test_varcoeff_declined(B):
    prob = heat_cn_varcoeff_problem(15, 16)
    s = B.Solver(prob)
    with pytest.raises(B.BlttError) as e:
        s.solve(to_dev(rhs_uniform(prob.n, 66)), basis=1)      # the DST basis
    assert e.value.status == 8
    fv = frac_var(m=15, N=128)
    with pytest.raises(B.BlttError) as e:
        B.Solver(fv).set_matvec_arith(3)                         # the tensor-core product
    assert e.value.status == 8
    bad = copy.deepcopy(prob)
    bad.meta["faces"] = (-bad.meta["faces"][0], bad.meta["faces"][1])
    with pytest.raises(B.BlttError) as e:
        B.Solver(bad)
    assert e.value.status == 1


@pytest.mark.parametrize("precond,alpha,printed,slack", [("alpha", 1e-8, 10, 0), ("one", 1.0, 217, 1)],
                         ids=["P_alpha", "P_1"])
def test_varcoeff_paper_data_counts(B, precond, alpha, printed, slack):
    # Table 3 on the example's own data (exact solution e^t x1(1-x1) x2(1-x2), u_0 in the CN first
    # block): MINRES-P_alpha 10 iterations, MINRES-P_1 (alpha = 1) 217 printed
    from workloads import paper_data_heat_var
    prob = heat_cn_varcoeff_problem(31, 32)
    F, u0 = paper_data_heat_var(prob)
    F[0] += u0 * prob.N - 0.5 * (O.laplacian(prob) @ u0)
    f = F.reshape(-1)
    ref = O.solve(prob, f, alpha=alpha, tol=1e-6, maxit=1000, precond=precond)
    u, info = B.Solver(prob).solve(to_dev(f), alpha=alpha, tol=1e-6, maxit=1000, precision=64)
    assert info["status"] == 0
    assert abs(info["iters"] - printed) <= slack and abs(info["iters"] - ref["iters"]) <= 1
    assert rel(to_host(u), ref["x"]) <= 1e-5


def _example4_cases():
    import json
    import os
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden",
                                    "paper_iteration_counts_example4.json")))
    cases = list(g["cases"])
    # the largest size of Tables 7-9 (N = 256, m + 1 = 256: 16.6 M unknowns), GPU only
    for table, gamma, p1 in (("Table 7", 0.3, 8), ("Table 8", 0.6, 10), ("Table 9", 0.9, 10)):
        cases.append(dict(table=table, gamma=gamma, N=256, m_plus_1=256, precond="alpha", iters=8,
                          slack=0))
        cases.append(dict(table=table, gamma=gamma, N=256, m_plus_1=256, precond="one", iters=p1,
                          slack=1))
    return g, cases


@pytest.mark.parametrize("case", _example4_cases()[1],
                         ids=[f"{c['table']}_g{c['gamma']}_N{c['N']}_m{c['m_plus_1']}_{c['precond']}"
                              for c in _example4_cases()[1]])
def test_example4_paper_counts(B, case):
    # Tables 7-9 (Example 4: L1 fractional, a = 35 + x^3.5 + y^3.5) on the example's own data:
    # MINRES-P_alpha 8 iterations everywhere, MINRES-P_1 8 to 10 as printed
    from workloads import fractional_varcoeff_problem, paper_data_frac_var
    g = _example4_cases()[0]
    prob = fractional_varcoeff_problem(case["m_plus_1"] - 1, case["N"], case["gamma"])
    f = paper_data_frac_var(prob, case["gamma"])
    alpha = g["alpha"] if case["precond"] == "alpha" else 1.0
    u, info = B.Solver(prob).solve(to_dev(f), alpha=alpha, tol=g["tol"], maxit=500, precision=64)
    assert info["status"] == 0 and info["basis"] == 2
    assert abs(info["iters"] - case["iters"]) <= case["slack"], (case, info["iters"])
    assert info["relres_true"] <= g["tol"]
