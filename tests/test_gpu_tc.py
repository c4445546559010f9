"""The tensor-core time product (BLTT_ARITH_TC) against the oracle: matvec parity in both
orientations over ragged strips and every supported N, MINRES solves in the DST basis, graph
replay, and the problems it declines."""
import numpy as np
import pytest

import oracle as O
from workloads import Problem, fractional_problem, heat_bdf_problem, rhs_uniform
from _gpu_helpers import rel, to_dev, to_host

pytestmark = pytest.mark.gpu

ARITH_TC = 3


@pytest.fixture(scope="module")
def B():
    from paper_2307_07749_gb300 import build
    build.build()
    import paper_2307_07749_gb300 as mod
    return mod


def tc_problems():
    return [
        fractional_problem(1, 63, 128, 0.5),           # one strip, 65 padded lines
        fractional_problem(2, (31, 15), 256, 0.7),     # M = 465: four strips, ragged tail
        fractional_problem(2, 31, 512, 0.3),           # M = 961: eight strips, ragged
        fractional_problem(1, 255, 1024, 0.9),         # longest N, two strips
        fractional_problem(3, (7, 7, 3), 128, 0.6),    # 3-D, M = 147
    ]


TC_IDS = [p.name for p in tc_problems()]


def bound(prob, z):
    """Per-element error bound of the five-digit fixed-point product: a few 2^-40 of
    max|a| sum_k |z_k| on each spatial line (taken at its largest), with a safety factor."""
    Z = np.abs(z.reshape(prob.N, -1))
    return 64 * 2.0 ** -40 * np.max(np.abs(prob.a)) * Z.sum(axis=0).max()


@pytest.mark.parametrize("prob", tc_problems(), ids=TC_IDS)
@pytest.mark.parametrize("flip", [0, 1])
def test_tc_matvec_parity(B, prob, flip):
    s = B.Solver(prob)
    s.set_matvec_arith(ARITH_TC)
    rng = np.random.default_rng(41)
    # lines of very different scale: the digits are relative to each line's own bound
    z = (rng.standard_normal((prob.N, prob.M)) * np.exp(rng.uniform(-6, 6, prob.M))[None, :]).ravel()
    y = to_host(s.matvec(to_dev(z), flip=bool(flip)))
    ref = O.bltt_matvec(prob, z, flip=bool(flip))
    assert np.max(np.abs(y - ref)) <= bound(prob, z)
    assert rel(y, ref) <= 1e-10


@pytest.mark.parametrize("prob", tc_problems()[:2], ids=TC_IDS[:2])
def test_tc_matvec_special_inputs(B, prob):
    s = B.Solver(prob)
    s.set_matvec_arith(ARITH_TC)
    # zero vector, one impulse per line, a line of zeros next to a line of ones
    z0 = np.zeros(prob.n)
    assert np.all(to_host(s.matvec(to_dev(z0))) == 0.0)
    imp = np.zeros((prob.N, prob.M))
    imp[np.arange(prob.M) % prob.N, np.arange(prob.M)] = 1.0
    imp = imp.ravel()
    y = to_host(s.matvec(to_dev(imp)))
    assert np.max(np.abs(y - O.bltt_matvec(prob, imp, flip=True))) <= bound(prob, imp)
    mix = np.zeros((prob.N, prob.M))
    mix[:, ::2] = 1.0
    mix = mix.ravel()
    y = to_host(s.matvec(to_dev(mix)))
    assert np.max(np.abs(y - O.bltt_matvec(prob, mix, flip=True))) <= bound(prob, mix)


@pytest.mark.parametrize("prob", tc_problems()[1:4], ids=TC_IDS[1:4])
@pytest.mark.parametrize("precision", [64, 32], ids=["f64", "f32"])
def test_tc_solve_parity(B, prob, precision):
    f = rhs_uniform(prob.n, 43)
    ref = O.solve(prob, f, alpha=1e-8, tol=1e-8)
    alpha = 1e-8 if precision == 64 else 1e-3
    s = B.Solver(prob)
    u, info = s.solve(to_dev(f), alpha=alpha, tol=1e-8, maxit=100, precision=precision, basis=1,
                      matvec_arith=ARITH_TC)
    assert info["status"] == 0, info
    if precision == 64:
        assert abs(info["iters"] - ref["iters"]) <= 1, (info["iters"], ref["iters"])
    assert info["relres_true"] <= 1e-8
    uh = to_host(u)
    assert rel(O.bltt_matvec(prob, uh), f) <= 1e-8
    assert rel(uh, ref["x"]) <= 1e-6
    # the same solve with the double-float product: same iterations, nearby solution
    u2, i2 = s.solve(to_dev(f), alpha=alpha, tol=1e-8, maxit=100, precision=precision, basis=1,
                     matvec_arith=2)
    assert abs(i2["iters"] - info["iters"]) <= 1
    assert rel(uh, to_host(u2)) <= 1e-7


def test_tc_graph_replay(B):
    import torch
    prob = tc_problems()[1]
    f = to_dev(rhs_uniform(prob.n, 44))
    st = torch.cuda.Stream()
    s = B.Solver(prob, stream=st)
    form = dict(precision=32, basis=1, matvec_arith=ARITH_TC, alpha=1e-3)
    with torch.cuda.stream(st):
        u1, i1 = s.solve(f, tol=1e-8, maxit=50, graph=True, **form)
        u2, i2 = s.solve(f, tol=1e-8, maxit=50, graph=False, **form)
    torch.cuda.synchronize()
    assert i1["status"] == i2["status"] == 0 and i1["iters"] == i2["iters"]
    assert torch.equal(u1, u2)


def test_tc_unsupported(B):
    heat = heat_bdf_problem(2, (15, 15), 128)               # direct taps
    with pytest.raises(B.BlttError) as e:
        B.Solver(heat).set_matvec_arith(ARITH_TC)
    assert e.value.status == 8
    big = fractional_problem(1, 7, 2048, 0.5)               # N beyond 1024
    with pytest.raises(B.BlttError) as e:
        B.Solver(big).set_matvec_arith(ARITH_TC)
    assert e.value.status == 8
    p = fractional_problem(1, 15, 128, 0.5)                 # general b
    b = 0.3 * (0.5 ** np.arange(p.N))
    b[0] = 1.0
    genb = Problem(p.N, p.d, p.m, p.h, p.a, b, name="genb", meta={})
    s = B.Solver(genb)
    with pytest.raises(B.BlttError) as e:
        s.solve(to_dev(rhs_uniform(genb.n, 45)), matvec_arith=ARITH_TC)
    assert e.value.status == 8


def test_tc_bounded_wait_gives_up_and_the_context_stays_usable(B, monkeypatch):
    """Failure detection without a fault: BLTT_TC_WAIT_CYCLES = 0 makes the tensor-core kernel's
    waits for progress (a stage's copy landed, its MMAs done, the accumulators read) give up at
    the first miss.  The block then sets its error flag, writes NaN partials, waits (with the
    default limit) for its own copies and MMAs and frees its tensor memory; the solve returns
    BLTT_ERR_TIMEOUT (7).  Without the setting the next solve on the same handle is correct."""
    prob = fractional_problem(2, 63, 512, 0.6)          # M = 3969: many units per block
    f = rhs_uniform(prob.n, 71)
    s = B.Solver(prob)
    monkeypatch.setenv("BLTT_TC_WAIT_CYCLES", "0")
    _, info = s.solve(to_dev(f), alpha=1e-2, tol=1e-8, maxit=20, precision=32, basis=1,
                      matvec_arith=ARITH_TC, graph=False, raise_on_error=False)
    assert info["status"] == 7, info
    monkeypatch.delenv("BLTT_TC_WAIT_CYCLES")
    u, info = s.solve(to_dev(f), alpha=1e-2, tol=1e-8, maxit=50, precision=32, basis=1,
                      matvec_arith=ARITH_TC, graph=False)
    assert info["status"] == 0 and info["relres_true"] <= 1e-8
    assert rel(O.bltt_matvec(prob, to_host(u)), f) <= 1e-8
