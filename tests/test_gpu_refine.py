"""Mixed-precision iterative refinement (bltt_solve_opts.refine), the fallback of the precision
forms: with an FP32 preconditioner at a small alpha the FP32 rounding, amplified by
kappa(D_alpha) = alpha^{-(N-1)/N}, stalls MINRES or breaks it down (P^{-1} no longer positive
definite); the refinement corrects from fresh FP64-accurate residuals with double-float inner
solves and reaches the tolerance.  A solve that converges on its own is unchanged."""
import numpy as np
import pytest

import oracle as O
from workloads import fractional_problem, rhs_uniform

from _gpu_helpers import rel, to_dev, to_host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    import paper_2307_07749_gb300 as B
    return B


F32 = dict(precision=32, basis=1, matvec_arith=2)


def test_refine_leaves_a_converging_solve_unchanged(B):
    prob = fractional_problem(2, 31, 64, 0.7)
    f = to_dev(rhs_uniform(prob.n, 60))
    s = B.Solver(prob)
    u0, i0 = s.solve(f, alpha=1e-2, tol=1e-8, maxit=100, **F32)
    u1, i1 = s.solve(f, alpha=1e-2, tol=1e-8, maxit=100, refine=4, **F32)
    assert i0["status"] == i1["status"] == 0 and i1["refinements"] == 0
    assert i0["iters"] == i1["iters"]
    assert np.array_equal(to_host(u0), to_host(u1))


@pytest.mark.parametrize("alpha", [1e-7, 1e-8])
def test_refine_recovers_a_stalled_fp32_solve(B, alpha):
    # 2-D L1 blocks, N = 256, m = 63: without refinement MINRES with the FP32 preconditioner
    # stalls near 1e-4 (alpha = 1e-7) or breaks down (1e-8) within 100 iterations
    prob = fractional_problem(2, 63, 256, 0.7)
    fh = rhs_uniform(prob.n, 5)
    f = to_dev(fh)
    s = B.Solver(prob)
    u0, i0 = s.solve(f, alpha=alpha, tol=1e-8, maxit=100, raise_on_error=False, **F32)
    assert i0["status"] != 0
    u1, i1 = s.solve(f, alpha=alpha, tol=1e-8, maxit=100, refine=8, **F32)
    assert i1["status"] == 0 and i1["refinements"] >= 1 and i1["iters"] <= 100
    assert i1["relres_true"] <= 1e-8
    # the reported residual is a fresh one: the oracle's block sum agrees
    r = rel(O.bltt_matvec(prob, to_host(u1)), fh)
    assert r <= 1e-8 and abs(r - i1["relres_true"]) <= 1e-12


def test_refine_against_the_oracle_solution(B):
    # a case small enough for the oracle's own FP64 solve (N = 64, m = 31, alpha = 1e-8)
    prob = fractional_problem(2, 31, 64, 0.6)
    fh = rhs_uniform(prob.n, 61)
    s = B.Solver(prob)
    u, info = s.solve(to_dev(fh), alpha=1e-8, tol=1e-10, maxit=100, refine=8, **F32)
    assert info["status"] == 0 and info["relres_true"] <= 1e-10
    ref = O.solve(prob, fh, alpha=1e-8, tol=1e-10)
    assert rel(to_host(u), ref["x"]) <= 1e-8


def test_refine_host_buffers_and_refusals(B):
    import torch
    prob = fractional_problem(2, 31, 64, 0.7)
    fh = rhs_uniform(prob.n, 62)
    s = B.Solver(prob)
    form = dict(alpha=1e-8, tol=1e-9, maxit=100, refine=8, **F32)
    ud, idev = s.solve(to_dev(fh), **form)
    uh, ih = s.solve_host(torch.from_numpy(fh).pin_memory(), **form)
    assert idev["status"] == ih["status"] == 0 and idev["iters"] == ih["iters"]
    assert np.array_equal(uh.numpy(), to_host(ud))
    # the budget: maxit covers every inner solve
    u2, i2 = s.solve(to_dev(fh), alpha=1e-8, tol=1e-14, maxit=12, refine=3, raise_on_error=False,
                     **F32)
    assert i2["iters"] <= 12
    # a dense operator: no physical-basis product to refine with
    from workloads import nonlocal_diffusion_problem
    pd = nonlocal_diffusion_problem(7, 16, 0.5)
    sd = B.Solver(pd)
    with pytest.raises(B.BlttError) as e:
        sd.solve(to_dev(rhs_uniform(pd.n, 63)), alpha=1e-2, refine=2, **F32)
    assert e.value.status == 8
