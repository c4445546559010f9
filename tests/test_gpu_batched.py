"""Batched solves: many systems of uneven N and M with several right-hand sides each, in one
launch per MINRES phase under a CUDA graph.  Every item is compared with the oracle's own solve."""
import numpy as np
import pytest

import oracle as O
from workloads import fractional_problem, rhs_uniform
from _gpu_helpers import rel, to_dev, to_host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    from paper_2307_07749_gb300 import build
    build.build()
    import paper_2307_07749_gb300 as mod
    return mod


def small_batch(seed=7):
    rng = np.random.default_rng(seed)
    probs = []
    for s in range(8):
        d = int(rng.choice([1, 2]))
        m = int(rng.choice([7, 15, 31] if d == 2 else [15, 31, 63, 127]))
        N = int(rng.choice([16, 32, 64, 128]))
        probs.append(fractional_problem(d, m, N, float(rng.uniform(0.2, 0.9))))
    fs = [[rhs_uniform(p.n, 1000 * s + r) for r in range(2)] for s, p in enumerate(probs)]
    return probs, fs


@pytest.mark.parametrize("form", [
    dict(precision=64, matvec_arith=1, alpha=1e-8),
    dict(precision=32, matvec_arith=2, alpha=1e-3),
    dict(precision=96, matvec_arith=2, alpha=1e-5),
], ids=["f64", "f32_prec", "f32x2"])
def test_batched_matches_oracle(B, form):
    probs, fs = small_batch()
    fd = [[to_dev(f) for f in row] for row in fs]
    ud = [[to_dev(np.zeros_like(f)) for f in row] for row in fs]
    st, infos = B.bltt_solve_batched(probs, fd, ud, alpha=[form["alpha"]] * len(probs), tol=1e-8,
                                     maxit=100, precision=form["precision"],
                                     matvec_arith=form["matvec_arith"])
    assert st == 0, [i["status"] for i in infos]
    k = 0
    for s, p in enumerate(probs):
        for r, f in enumerate(fs[s]):
            info = infos[k]
            k += 1
            ref = O.solve(p, f, alpha=form["alpha"], tol=1e-8)
            u = to_host(ud[s][r])
            assert info["relres_true"] <= 1e-8
            assert rel(O.bltt_matvec(p, u), f) <= 1e-8
            # every form within one iteration of the FP64 oracle at the same alpha (N <= 128
            # here, where neither the FP32 nor the double-float rounding costs an iteration)
            assert abs(info["iters"] - ref["iters"]) <= 1, (s, r, info["iters"], ref["iters"])
            assert rel(u, ref["x"]) <= 1e-6


def test_batched_equals_single_solves_and_splits_waves(B, monkeypatch):
    probs, fs = small_batch(seed=8)
    fd = [[to_dev(f) for f in row] for row in fs]
    ud = [[to_dev(np.zeros_like(f)) for f in row] for row in fs]
    # a workspace cap of ~3 items forces several waves
    sizes = sorted((9 * p.n * 8 for p in probs), reverse=True)
    monkeypatch.setenv("BLTT_BATCH_MAX_BYTES", str(int(sizes[0] * 2.5)))
    st, infos = B.bltt_solve_batched(probs, fd, ud, tol=1e-8, maxit=100)
    assert st == 0
    k = 0
    for s, p in enumerate(probs):
        sol = B.Solver(p)
        for r in range(2):
            u1, inf1 = sol.solve(fd[s][r], alpha=1e-8, tol=1e-8, maxit=100, precision=64, basis=1)
            assert infos[k]["iters"] == inf1["iters"]
            assert rel(to_host(ud[s][r]), to_host(u1)) <= 1e-12
            k += 1


@pytest.mark.parametrize("form", [
    dict(precision=64, matvec_arith=1, alpha=1e-8),
    dict(precision=32, matvec_arith=2, alpha=1e-3),
], ids=["f64", "f32_prec"])
def test_batched_big_and_small_items_equal_single_solves(B, form):
    """Items of at least 2^21 unknowns run their FFT phases as single-item launches inside the
    batched graph, the smaller ones share the multi-item launches: both kinds reproduce the single
    solves (same iterations, same solution)."""
    # (the N = 1024 item takes the wide FP32 time-pass tile in its single-item launches)
    probs = [fractional_problem(2, 127, 256, 0.6), fractional_problem(2, 63, 1024, 0.7),
             fractional_problem(1, 63, 64, 0.4), fractional_problem(2, 31, 128, 0.8)]
    assert probs[0].n >= 1 << 21 and probs[1].n >= 1 << 21
    assert probs[2].n < 1 << 21 and probs[3].n < 1 << 21
    fs = [[rhs_uniform(p.n, 50 + 10 * s + r) for r in range(2)] for s, p in enumerate(probs)]
    fd = [[to_dev(f) for f in row] for row in fs]
    ud = [[to_dev(np.zeros_like(f)) for f in row] for row in fs]
    st, infos = B.bltt_solve_batched(probs, fd, ud, alpha=[form["alpha"]] * len(probs), tol=1e-8,
                                     maxit=100, precision=form["precision"],
                                     matvec_arith=form["matvec_arith"])
    assert st == 0, [i["status"] for i in infos]
    k = 0
    for s, p in enumerate(probs):
        sol = B.Solver(p)
        for r in range(2):
            u1, inf1 = sol.solve(fd[s][r], alpha=form["alpha"], tol=1e-8, maxit=100,
                                 precision=form["precision"], basis=1,
                                 matvec_arith=form["matvec_arith"])
            assert infos[k]["relres_true"] <= 1e-8
            assert infos[k]["iters"] == inf1["iters"], (s, r, infos[k]["iters"], inf1["iters"])
            assert rel(to_host(ud[s][r]), to_host(u1)) <= 1e-10
            k += 1


def test_batched_memory_cap_below_one_item_reports_oom(B, monkeypatch):
    """A workspace budget smaller than one item's vectors: the call returns BLTT_ERR_OOM (3)
    before any iteration, leaves the outputs untouched, and the library stays usable."""
    probs, fs = small_batch(seed=9)
    fd = [[to_dev(f) for f in row] for row in fs]
    ud = [[to_dev(np.full_like(f, 7.0)) for f in row] for row in fs]
    monkeypatch.setenv("BLTT_BATCH_MAX_BYTES", "4096")
    st, infos = B.bltt_solve_batched(probs, fd, ud, tol=1e-8, maxit=100)
    assert st == 3
    assert all(float(u.min()) == 7.0 == float(u.max()) for row in ud for u in row)
    monkeypatch.delenv("BLTT_BATCH_MAX_BYTES")
    st, infos = B.bltt_solve_batched(probs, fd, ud, tol=1e-8, maxit=100)
    assert st == 0 and all(i["relres_true"] <= 1e-8 for i in infos)


@pytest.mark.parametrize("form", [
    dict(precision=64, matvec_arith=1, alpha=1e-8),
    dict(precision=32, matvec_arith=2, alpha=1e-2),
    dict(precision=96, matvec_arith=2, alpha=1e-6),
], ids=["f64", "f32_prec", "f32x2_prec"])
def test_batched_workload_sample_vs_stored_oracle(B, form):
    """The small systems of the 96-system batched workload (M <= 3969, at most 600,000 unknowns:
    24 systems, 96 items) solved in one batched call; every item's count against the FP64
    oracle's stored count at the same alpha (tests/golden/make_oracle_solve_counts.py)."""
    import json
    import os
    from workloads import batched_systems
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                           "oracle_counts_batched_sample.json")) as fh:
        golden = {(c["system"], c["rhs"], c["alpha"]): c["iters"] for c in json.load(fh)["cases"]}
    sysl = batched_systems(96, 4, seed=4)
    sample = [s for s, (p, _) in enumerate(sysl) if p.M <= 3969 and p.n <= 600_000]
    assert len(sample) == 24
    probs = [sysl[s][0] for s in sample]
    fd = [[to_dev(rf()) for rf in sysl[s][1]] for s in sample]
    ud = [[to_dev(np.zeros(p.n)) for _ in range(4)] for p in probs]
    st, infos = B.bltt_solve_batched(probs, fd, ud, alpha=[form["alpha"]] * len(probs), tol=1e-8,
                                     maxit=100, precision=form["precision"],
                                     matvec_arith=form["matvec_arith"])
    assert st == 0
    deltas = []
    for j, s in enumerate(sample):
        for r in range(4):
            info = infos[4 * j + r]
            assert info["relres_true"] <= 1e-8
            deltas.append(info["iters"] - golden[(s, r, form["alpha"])])
    assert max(abs(d) for d in deltas) <= 1, deltas


@pytest.mark.parametrize("form", [
    dict(precision=64, matvec_arith=1, alpha=1e-8),
    dict(precision=32, matvec_arith=2, alpha=1e-2),
    dict(precision=64, matvec_arith=1, alpha=1.0),
], ids=["f64", "f32_prec", "f64_P1"])
def test_batched_deferred_window_matches_per_iteration_update(B, form):
    """The batched items defer their (w, x) update over the first iterations as single solves do;
    with the per-iteration update instead (defer_window = -1) every item takes the same iterations
    and the same solution to rounding, also past the window (alpha = 1: tens of iterations)."""
    probs = [fractional_problem(2, 127, 256, 0.6), fractional_problem(2, 31, 128, 0.8),
             fractional_problem(1, 63, 64, 0.4)]
    fs = [[rhs_uniform(p.n, 70 + 10 * s + r) for r in range(2)] for s, p in enumerate(probs)]
    fd = [[to_dev(f) for f in row] for row in fs]
    res = []
    for win in (0, -1):
        ud = [[to_dev(np.zeros_like(f)) for f in row] for row in fs]
        st, infos = B.bltt_solve_batched(probs, fd, ud, alpha=[form["alpha"]] * len(probs),
                                         tol=1e-8, maxit=300, precision=form["precision"],
                                         matvec_arith=form["matvec_arith"], defer_window=win)
        assert st == 0
        res.append((infos, [to_host(u) for row in ud for u in row]))
    (i0, u0), (i1, u1) = res
    assert [i["iters"] for i in i0] == [i["iters"] for i in i1]
    if form["alpha"] == 1.0:
        assert min(i["iters"] for i in i0) > 8
    for a, b in zip(u0, u1):
        assert rel(a, b) <= 1e-10
