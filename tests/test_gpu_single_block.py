"""The whole solve by one block (one kernel launch per solve) for problems whose every phase is
one FFT tile, the smallest workload (1-D L1 fractional, N = 64, m = 63: 4032 unknowns) first:
against the oracle, against the multi-launch solve, at maxit, and the problems it declines."""
import numpy as np
import pytest

import oracle as O
from workloads import fractional_problem, heat_cn_problem, rhs_uniform, workload
from _gpu_helpers import rel, to_dev, to_host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    from paper_2307_07749_gb300 import build
    build.build()
    import paper_2307_07749_gb300 as mod
    return mod


def one_tile_problems():
    return [workload("frac1d_N64_m63_g0.5")[0],              # 4032 unknowns
            fractional_problem(1, 31, 128, 0.3),               # longer time axis
            fractional_problem(2, 7, 32, 0.7),                 # 2-D, two DST axes
            fractional_problem(3, 3, 16, 0.9)]                 # 3-D


PIDS = [p.name for p in one_tile_problems()]


@pytest.mark.parametrize("prob", one_tile_problems(), ids=PIDS)
@pytest.mark.parametrize("alpha", [1e-8, 1.0])
def test_single_block_matches_oracle(B, prob, alpha):
    f = rhs_uniform(prob.n, 101)
    ref = O.solve(prob, f, alpha=alpha, tol=1e-10, maxit=300)
    u, info = B.Solver(prob).solve(to_dev(f), alpha=alpha, tol=1e-10, maxit=300, precision=64,
                                   basis=1, single_block=True)
    assert info["status"] == 0, info
    assert abs(info["iters"] - ref["iters"]) <= 1, (info["iters"], ref["iters"])
    uh = to_host(u)
    assert info["relres_true"] <= 1e-10
    assert rel(O.bltt_matvec(prob, uh), f) <= 1e-9
    assert rel(uh, ref["x"]) <= 1e-7
    # one launch for the solve itself (plus the per-alpha table set-up)
    assert info["kernel_launches"] <= 2


@pytest.mark.parametrize("prob", one_tile_problems(), ids=PIDS)
def test_single_block_matches_multi_launch_solve(B, prob):
    f = to_dev(rhs_uniform(prob.n, 102))
    s = B.Solver(prob)
    u1, i1 = s.solve(f, alpha=1e-8, tol=1e-10, precision=64, basis=1, matvec_arith=1, graph=False)
    u2, i2 = s.solve(f, alpha=1e-8, tol=1e-10, precision=64, basis=1, matvec_arith=1,
                     single_block=True)
    assert i1["status"] == i2["status"] == 0 and i1["iters"] == i2["iters"]
    assert rel(to_host(u2), to_host(u1)) <= 1e-12


# the chosen form: FP32 preconditioner (alpha = 1e-3), double-float product and DSTs
@pytest.mark.parametrize("prob", one_tile_problems(), ids=PIDS)
def test_single_block_chosen_form(B, prob):
    f = rhs_uniform(prob.n, 107)
    ref = O.solve(prob, f, alpha=1e-8, tol=1e-10, maxit=300)
    s = B.Solver(prob)
    form = dict(alpha=1e-3, tol=1e-10, maxit=300, precision=32, basis=1, matvec_arith=2)
    u1, i1 = s.solve(to_dev(f), graph=False, **form)
    u2, i2 = s.solve(to_dev(f), single_block=True, **form)
    assert i1["status"] == i2["status"] == 0, (i1, i2)
    assert abs(i1["iters"] - i2["iters"]) <= 1
    uh = to_host(u2)
    assert i2["relres_true"] <= 1e-10 and rel(O.bltt_matvec(prob, uh), f) <= 1e-9
    assert rel(uh, ref["x"]) <= 1e-7 and rel(uh, to_host(u1)) <= 1e-7
    assert i2["kernel_launches"] <= 2


def test_single_block_maxit(B):
    prob = one_tile_problems()[0]
    f = to_dev(rhs_uniform(prob.n, 103))
    u, info = B.Solver(prob).solve(f, alpha=1.0, tol=1e-14, maxit=3, precision=64, basis=1,
                                   single_block=True, raise_on_error=False)
    assert info["status"] == 6 and info["iters"] == 3
    assert np.all(np.isfinite(to_host(u)))


def test_single_block_declined(B):
    prob = one_tile_problems()[0]
    s = B.Solver(prob)
    f = to_dev(rhs_uniform(prob.n, 104))
    for kw in (dict(precision=32), dict(basis=2), dict(matvec_arith=2),
               dict(precision=96, matvec_arith=2)):
        with pytest.raises(B.BlttError) as e:
            s.solve(f, single_block=True, **kw)
        assert e.value.status == 8, kw
    heat = heat_cn_problem(1, 63, 64)                          # the direct product
    with pytest.raises(B.BlttError) as e:
        B.Solver(heat).solve(to_dev(rhs_uniform(heat.n, 105)), single_block=True)
    assert e.value.status == 8
    big = fractional_problem(2, 31, 64, 0.5)                   # more than one tile
    with pytest.raises(B.BlttError) as e:
        B.Solver(big).solve(to_dev(rhs_uniform(big.n, 106)), single_block=True)
    assert e.value.status == 8
