"""Deferred solution update (defer_window): the first S iterations keep their preconditioned
vectors and form x (and the two latest w vectors) from them only when needed.  The Lanczos
vectors and scalars are the same bits with or without the window, so the iteration counts agree;
x agrees to rounding.  Every other GPU test runs with the default window (S = 8) against the
oracle; these tests compare it with the per-iteration update and cover its edges: stops inside
and at the end of the window, iterations past it, window sizes, graph blocks, the resumed
iterations after a failed host check, host buffers."""
import numpy as np
import pytest

import oracle as O
from workloads import fractional_problem, heat_bdf_problem, heat_cn_problem, rhs_uniform

from _gpu_helpers import rel, to_dev, to_host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    import paper_2307_07749_gb300 as B
    return B


FORMS = {
    "f64_spectral": dict(precision=64, basis=1, matvec_arith=1, alpha=1e-8),
    "f32_spectral": dict(precision=32, basis=1, matvec_arith=2, alpha=1e-2),
    "f32x2_spectral": dict(precision=96, basis=1, matvec_arith=2, alpha=1e-6),
    "f32_physical": dict(precision=32, basis=2, matvec_arith=2, alpha=1e-3),
    "f64_physical": dict(precision=64, basis=2, matvec_arith=1, alpha=1e-8),
}


def _pair(B, prob, f, form, window, **kw):
    import torch
    st = torch.cuda.Stream()
    s = B.Solver(prob, stream=st)
    with torch.cuda.stream(st):
        u0, i0 = s.solve(f, tol=1e-8, defer_window=-1, **form, **kw)
        u1, i1 = s.solve(f, tol=1e-8, defer_window=window, **form, **kw)
    torch.cuda.synchronize()
    return to_host(u0), i0, to_host(u1), i1


@pytest.mark.parametrize("form", list(FORMS), ids=list(FORMS))
@pytest.mark.parametrize("window", [0, 2, 4, 16])
def test_window_matches_per_iteration_update(B, form, window):
    # 2-D L1 fractional blocks (FFT product): stops inside the window, at its end, or after it
    prob = fractional_problem(2, 31, 64, 0.7)
    f = to_dev(rhs_uniform(prob.n, 41))
    u0, i0, u1, i1 = _pair(B, prob, f, FORMS[form], window, maxit=100)
    assert i0["status"] == i1["status"] == 0
    assert i0["iters"] == i1["iters"], (i0["iters"], i1["iters"])
    assert rel(u1, u0) <= 1e-12
    assert i1["relres_true"] <= 1e-8
    assert rel(O.bltt_matvec(prob, u1), to_host(f)) <= 1e-8


@pytest.mark.parametrize("precond,alpha", [(0, 1.0), (1, 0.0)], ids=["P_1", "I"])
@pytest.mark.parametrize("window", [0, 4])
def test_window_long_solves(B, precond, alpha, window):
    # MINRES-P_1 and MINRES-I run tens to hundreds of iterations: the window's w vectors hand over
    # to the per-iteration update; the count stays the oracle's and x the per-iteration one's
    prob = fractional_problem(1, 15, 32, 0.5)
    fh = rhs_uniform(prob.n, 33)
    ref = O.solve(prob, fh, alpha=alpha if precond == 0 else 1.0, tol=1e-8, maxit=2000,
                  precond="one" if precond == 0 else "none")
    u0, i0, u1, i1 = _pair(B, prob, to_dev(fh), dict(precision=64, basis=2, alpha=alpha,
                                                      precond=precond), window, maxit=2000)
    assert i0["status"] == i1["status"] == 0
    assert i1["iters"] == i0["iters"]
    assert abs(i1["iters"] - ref["iters"]) <= max(1, ref["iters"] // 50)
    assert rel(u1, u0) <= 1e-9
    assert rel(u1, ref["x"]) <= 1e-6


@pytest.mark.parametrize("maker", [heat_bdf_problem, heat_cn_problem], ids=["bdf", "cn"])
@pytest.mark.parametrize("form", ["f64_spectral", "f32_spectral", "f32_physical"])
def test_window_direct_product(B, maker, form):
    # heat blocks (direct product): the true residual is checked inside the iterations, so a
    # check that fails at the window's last iteration hands the w vectors over from there
    prob = maker(2, 31, 64)
    f = to_dev(rhs_uniform(prob.n, 42))
    u0, i0, u1, i1 = _pair(B, prob, f, FORMS[form], 0, maxit=100)
    assert i0["status"] == i1["status"] == 0 and i0["iters"] == i1["iters"]
    assert rel(u1, u0) <= 1e-12
    assert rel(O.bltt_matvec(prob, u1), to_host(f)) <= 1e-8


@pytest.mark.parametrize("window", [-1, 0, 2, 4, 6])
@pytest.mark.parametrize("sync_every", [2, 4])
def test_window_resume_after_failed_checks(B, window, sync_every):
    # a tolerance the true residual cannot reach: every host check fails and the iterations
    # resume with direct launches (inside the window, at its end, or after it); the iterate after
    # 24 iterations is the one of a run that never stops early (tol = 0), bit for bit
    import torch
    prob = fractional_problem(2, 31, 32, 0.7)
    f = to_dev(rhs_uniform(prob.n, 40))
    st = torch.cuda.Stream()
    s = B.Solver(prob, stream=st)
    form = dict(precision=32, basis=1, matvec_arith=2, alpha=1e-3, maxit=24, graph=True,
                raise_on_error=False, defer_window=window, sync_every=sync_every)
    with torch.cuda.stream(st):
        u0, i0 = s.solve(f, tol=0.0, **form)
        u1, i1 = s.solve(f, tol=1e-15, **form)
        u2, i2 = s.solve(f, tol=0.0, **dict(form, graph=False))
    torch.cuda.synchronize()
    assert i0["status"] == i1["status"] == 6 and i0["iters"] == i1["iters"] == 24
    assert torch.equal(u0, u1) and torch.equal(u0, u2)


def test_window_every_stop_iteration(B):
    # maxit = 1 .. 10 stops the solve at every position relative to an S = 4 window (inside, at
    # its end, past it); each stop's x equals the per-iteration update's to rounding
    import torch
    prob = fractional_problem(1, 31, 64, 0.5)
    f = to_dev(rhs_uniform(prob.n, 43))
    s = B.Solver(prob)
    form = dict(precision=64, basis=2, alpha=1.0, tol=0.0, raise_on_error=False)
    for maxit in range(1, 11):
        u0, i0 = s.solve(f, maxit=maxit, defer_window=-1, **form)
        u1, i1 = s.solve(f, maxit=maxit, defer_window=4, **form)
        assert i0["iters"] == i1["iters"] == maxit
        assert rel(to_host(u1), to_host(u0)) <= 1e-12, maxit
    torch.cuda.synchronize()


def test_window_host_buffers(B):
    import torch
    prob = fractional_problem(2, 31, 32, 0.7)
    fh = rhs_uniform(prob.n, 44)
    s = B.Solver(prob)
    form = dict(precision=32, basis=1, matvec_arith=2, alpha=1e-2, tol=1e-8, maxit=50)
    ud, idev = s.solve(to_dev(fh), **form)
    uh, ih = s.solve_host(torch.from_numpy(fh).pin_memory(), **form)
    assert ih["status"] == 0 and ih["iters"] == idev["iters"]
    assert np.array_equal(uh.numpy(), to_host(ud))
