"""Parity at the workloads' full sizes, in the configurations bench.py times.

2-D L1 fractional, N = 1024, m = 255 (66.6 M unknowns): sampled matvec entries against the oracle's
block sum, the whole preconditioner apply against the oracle's structured route, and whole solves
whose true residual is recomputed by the oracle's own matvec.
3-D backward-Euler heat, N = 256, m = 127 (524 M unknowns): sampled matvec entries and a sampled
estimate of the solve's true residual (the oracle's full operators do not fit a few seconds here).
"""
import json
import os

import numpy as np
import pytest

import oracle as O
from oracle.operators import bltt_matvec_entry
from workloads import heat_bdf_problem, rhs_smoothed_field, workload
from _gpu_helpers import precond_tol, rel, rel_max, to_dev, to_host

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                      "oracle_solve_counts.json")


def oracle_count(name, alpha, tol=1e-8):
    """The FP64 oracle's MINRES count on a named workload (stored by
    tests/golden/make_oracle_solve_counts.py, which calls only the oracle)."""
    with open(GOLDEN) as fh:
        for c in json.load(fh)["cases"]:
            if c["workload"] == name and c["alpha"] == alpha and c["tol"] == tol:
                return c["iters"]
    raise KeyError((name, alpha, tol))

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def B():
    from paper_2307_07749_gb300 import build
    build.build()
    import paper_2307_07749_gb300 as mod
    return mod


@pytest.fixture(scope="module")
def frac2d(B):
    prob, rf = workload("frac2d_N1024_m255_g0.7")
    f = rf()
    return prob, f, B.Solver(prob)


def _samples(prob, k, seed):
    rng = np.random.default_rng(seed)
    return rng.integers(0, prob.N, k), rng.integers(0, prob.M, k)


@pytest.mark.parametrize("arith", [1, 2], ids=["f64", "f32x2"])
def test_frac2d_matvec_sampled(B, frac2d, arith):
    prob, f, s = frac2d
    s.set_matvec_arith(arith)
    y = to_host(s.matvec(to_dev(f), flip=True)).reshape(prob.N, prob.M)
    ns, is_ = _samples(prob, 300, 50)
    got = np.array([y[n, i] for n, i in zip(ns, is_)])
    ref = np.array([bltt_matvec_entry(prob, f, n, i, flip=True) for n, i in zip(ns, is_)])
    assert rel(got, ref) <= 1e-12
    s.set_matvec_arith(1)


def test_frac2d_precond_full(B, frac2d):
    prob, f, s = frac2d
    alpha = 1e-3
    ref = O.precond_apply(prob, alpha, f)
    for prec in (64, 96, 32):
        z = to_host(s.precond_apply(alpha, to_dev(f), precision=prec))
        assert rel(z, ref) <= precond_tol(prob.N, alpha, prec)
        assert rel_max(z, ref) <= precond_tol(prob.N, alpha, prec)


@pytest.mark.parametrize("form", [
    dict(alpha=1e-8, precision=64, basis=1, matvec_arith=1),      # plain FP64
    dict(alpha=1e-2, precision=32, basis=1, matvec_arith=2),      # the bench's FP32-preconditioner form
    dict(alpha=1e-3, precision=32, basis=1, matvec_arith=2),
    dict(alpha=1e-3, precision=32, basis=2, matvec_arith=2),
    dict(alpha=1e-6, precision=96, basis=1, matvec_arith=2),      # double-float preconditioner
], ids=["plain_f64", "f32_a1e-2", "f32_a1e-3", "f32_a1e-3_physical", "f32x2_a1e-6"])
def test_frac2d_solve(B, frac2d, form):
    prob, f, s = frac2d
    u, info = s.solve(to_dev(f), tol=1e-8, maxit=100, rebuild=True, **form)
    assert info["status"] == 0, info
    assert info["relres_true"] <= 1e-8
    r = f - O.bltt_matvec(prob, to_host(u))
    assert np.linalg.norm(r) / np.linalg.norm(f) <= 1e-8


def test_frac2d_iterations_vs_oracle(B, frac2d):
    # the oracle's textbook MINRES on the same workload (about a minute of CPU)
    prob, f, s = frac2d
    ref = O.solve(prob, f, alpha=1e-8, tol=1e-8)
    u, info = s.solve(to_dev(f), alpha=1e-8, tol=1e-8, maxit=100, precision=64, basis=1)
    assert abs(info["iters"] - ref["iters"]) <= 1, (info["iters"], ref["iters"])
    assert rel(to_host(u), ref["x"]) <= 1e-6


# Each precision form against the FP64 oracle's count at the same alpha (stored oracle runs of this
# workload).  The FP32 preconditioner perturbs P_alpha^{-1} by about eps_32 log2(N) kappa(D_alpha),
# kappa(D_alpha) = alpha^{-(N-1)/N}: at N = 1024 and alpha = 1e-3 (kappa ~ 1e3) that costs exactly two
# iterations (6 against the oracle's 4); at alpha = 1e-2 none (6 and 6).  The double-float
# preconditioner (about 2^-47 per operation) costs none at alpha = 1e-6 (2 and 2).
@pytest.mark.parametrize("form,delta", [
    (dict(alpha=1e-2, precision=32, basis=1, matvec_arith=2), 0),
    (dict(alpha=1e-3, precision=32, basis=1, matvec_arith=2), 2),
    (dict(alpha=1e-6, precision=96, basis=1, matvec_arith=2), 0),
    (dict(alpha=1e-8, precision=64, basis=1, matvec_arith=1), 0),
], ids=["f32_a1e-2", "f32_a1e-3", "f32x2_a1e-6", "f64_a1e-8"])
def test_frac2d_form_iterations_vs_stored_oracle(B, frac2d, form, delta):
    prob, f, s = frac2d
    u, info = s.solve(to_dev(f), tol=1e-8, maxit=100, rebuild=True, **form)
    assert info["status"] == 0, info
    ref = oracle_count("frac2d_N1024_m255_g0.7", form["alpha"])
    assert info["iters"] == ref + delta, (info["iters"], ref)


@pytest.fixture(scope="module")
def heat3d(B):
    prob, rf = workload("heat3d_bdf_N256_m127")
    f = rf()
    return prob, f, B.Solver(prob)


def test_heat3d_matvec_sampled(B, heat3d):
    prob, f, s = heat3d
    fd = to_dev(f)
    y = s.matvec(fd, flip=True)
    ns, is_ = _samples(prob, 300, 51)
    yh = y.view(prob.N, prob.M)
    got = np.array([float(yh[n, i]) for n, i in zip(ns, is_)])
    ref = np.array([bltt_matvec_entry(prob, f, n, i, flip=True) for n, i in zip(ns, is_)])
    assert rel(got, ref) <= 1e-12
    del y


@pytest.mark.parametrize("form", [
    dict(alpha=1e-8, precision=64, basis=1, matvec_arith=1),
    dict(alpha=1e-3, precision=32, basis=2, matvec_arith=1),
    dict(alpha=1e-2, precision=32, basis=1, matvec_arith=2),      # the bench's forms
    dict(alpha=1e-3, precision=32, basis=1, matvec_arith=2),
    dict(alpha=1e-6, precision=96, basis=1, matvec_arith=2),
], ids=["plain_f64", "f32_physical", "f32_a1e-2", "f32_a1e-3", "f32x2_a1e-6"])
def test_heat3d_solve_sampled_residual(B, heat3d, form):
    prob, f, s = heat3d
    fd = to_dev(f)
    u, info = s.solve(fd, tol=1e-8, maxit=100, **form)
    assert info["status"] == 0, info
    assert info["relres_true"] <= 1e-8
    # sampled residual entries recomputed by the oracle's block sum: an unbiased estimate of
    # ||f - A u||^2 / n from 4000 entries, held to 3x the tolerance
    uh = to_host(u)
    ns, is_ = _samples(prob, 4000, 52)
    r2 = sum((f[n * prob.M + i] - bltt_matvec_entry(prob, uh, n, i)) ** 2 for n, i in zip(ns, is_))
    est = np.sqrt(r2 / len(ns) * prob.n) / np.linalg.norm(f)
    assert est <= 3e-8, est


@pytest.fixture(scope="module")
def heat3d_m63(B):
    # the 3-D backward-Euler heat family at m = 63 (65 M unknowns): small enough for the oracle's
    # whole solves, whose counts are stored
    prob = heat_bdf_problem(3, 63, 256)
    f = rhs_smoothed_field(prob.N, 3, prob.m, 3)
    return prob, f, B.Solver(prob)


# On this family the FP32 preconditioner costs no iteration at alpha = 1e-3 or 1e-2 (N = 256:
# kappa(D_alpha) = alpha^{-255/256}), and the double-float one none at alpha = 1e-6.
@pytest.mark.parametrize("form", [
    dict(alpha=1e-2, precision=32, basis=1, matvec_arith=2),
    dict(alpha=1e-3, precision=32, basis=1, matvec_arith=2),
    dict(alpha=1e-6, precision=96, basis=1, matvec_arith=2),
    dict(alpha=1e-8, precision=64, basis=1, matvec_arith=1),
], ids=["f32_a1e-2", "f32_a1e-3", "f32x2_a1e-6", "f64_a1e-8"])
def test_heat3d_m63_form_iterations_vs_stored_oracle(B, heat3d_m63, form):
    prob, f, s = heat3d_m63
    u, info = s.solve(to_dev(f), tol=1e-8, maxit=100, rebuild=True, **form)
    assert info["status"] == 0, info
    assert info["relres_true"] <= 1e-8
    assert info["iters"] == oracle_count("heat3d_bdf_N256_m63", form["alpha"]), info["iters"]
