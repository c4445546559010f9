"""Dense commuting blocks a_k I + b_k K (Sec. 3) against the oracle: the matvec and the
preconditioner through K's eigenbasis, MINRES solves there (device and host buffers, graph and
direct launches), K = the Laplacian against the DST path, K = L_a as the exact preconditioner of
the variable-coefficient blocks, and the combinations the library declines."""
import numpy as np
import pytest

import oracle as O
from workloads import (Problem, fractional_problem, heat_cn_problem, heat_cn_varcoeff_problem,
                       rhs_uniform)
from _gpu_helpers import precond_tol, rel, to_dev, to_host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    from paper_2307_07749_gb300 import build
    build.build()
    import paper_2307_07749_gb300 as mod
    return mod


def with_K(p, K, tag):
    meta = {k: v for k, v in p.meta.items() if k not in ("faces", "abar")}
    return Problem(p.N, p.d, p.m, p.h, p.a, p.b, name=f"{p.name}_{tag}", meta=dict(meta, K=K))


def spd(M, seed, scale):
    """A random SPD operator with eigenvalues spread over about [scale, 5 scale]."""
    G = np.random.default_rng(seed).standard_normal((M, M))
    return scale * (G @ G.T / M + np.eye(M))


def dense_problems():
    f2 = fractional_problem(2, (15, 7), 64, 0.6)          # FFT matvec, M = 105
    h2 = heat_cn_problem(2, 15, 32)                        # direct matvec, M = 225
    h3 = heat_cn_problem(3, 7, 16)                         # 3-D, M = 343
    f1 = fractional_problem(1, 63, 1024, 0.7)              # N = 1024: the wide time-pass tiles
    return [with_K(f2, O.laplacian(f2).toarray(), "lap"),
            with_K(h2, O.laplacian(h2).toarray(), "lap"),
            with_K(h3, O.laplacian(h3).toarray(), "lap"),
            with_K(f2, spd(f2.M, 81, 400.0), "spd"),
            with_K(f1, spd(f1.M, 82, 1000.0), "spd")]


DPS = dense_problems()
DIDS = [p.name for p in DPS]


@pytest.mark.parametrize("prob", DPS, ids=DIDS)
@pytest.mark.parametrize("flip", [0, 1])
@pytest.mark.parametrize("arith", [1, 2], ids=["f64", "f32x2"])
def test_dense_matvec_parity(B, prob, flip, arith):
    s = B.Solver(prob)
    s.set_matvec_arith(arith)
    z = np.random.default_rng(83).standard_normal(prob.n)
    y = to_host(s.matvec(to_dev(z), flip=bool(flip)))
    # two GEMMs move x into K's eigenbasis and back: FP64 (cuBLAS) with the FP64 matvec, double-float
    # with the double-float one; a few eps sqrt(M) of rounding, or about 2^-47 per multiply-add
    assert rel(y, O.bltt_matvec(prob, z, flip=bool(flip))) <= 1e-11


@pytest.mark.parametrize("prob", DPS, ids=DIDS)
@pytest.mark.parametrize("alpha", [1.0, 1e-3, 1e-8])
@pytest.mark.parametrize("precision", [64, 96, 32], ids=["f64", "df", "f32"])
@pytest.mark.parametrize("arith", [1, 2], ids=["gemm64", "gemmdf"])
def test_dense_precond_parity(B, prob, alpha, precision, arith):
    # the basis changes follow the handle's matvec arithmetic: FP64 GEMMs, or double-float GEMMs
    # on the FP32 pipes (about 2^-47 per multiply-add, within the 1e-11 floor)
    s = B.Solver(prob)
    s.set_matvec_arith(arith)
    v = np.random.default_rng(84).standard_normal(prob.n)
    z = to_host(s.precond_apply(alpha, to_dev(v), precision=precision))
    tol = max(precond_tol(prob.N, alpha, precision), 1e-11)
    assert rel(z, O.precond_apply(prob, alpha, v)) <= tol


@pytest.mark.parametrize("prob", DPS, ids=DIDS)
@pytest.mark.parametrize("form", [dict(precision=64, alpha=1e-8), dict(precision=64, alpha=1.0),
                                  dict(precision=32, alpha=1e-3), dict(precision=96, alpha=1e-8),
                                  dict(precision=32, alpha=1e-3, matvec_arith=2)],
                         ids=["f64", "f64_P1", "f32", "df", "chosen"])
def test_dense_solve(B, prob, form):
    f = rhs_uniform(prob.n, 85)
    # alpha = 1 (P_1): 8 to 34 iterations on these problems; alpha = 1e-8: 2
    ref = O.solve(prob, f, alpha=form["alpha"] if form["precision"] != 32 else 1e-8, tol=1e-8,
                  maxit=300)
    u, info = B.Solver(prob).solve(to_dev(f), tol=1e-8, maxit=300, **form)
    assert info["status"] == 0, info
    assert info["basis"] == 1                               # K's eigenbasis
    if form["precision"] == 64:
        assert abs(info["iters"] - ref["iters"]) <= 1, (info["iters"], ref["iters"])
    elif form["precision"] == 96:
        # double-float rounding (~2^-47) amplified by the D_alpha conditioning alpha^{-(N-1)/N}
        # (7e7 here): up to two more iterations than the FP64 oracle at alpha = 1e-8
        assert ref["iters"] - 1 <= info["iters"] <= ref["iters"] + 2, (info["iters"], ref["iters"])
    uh = to_host(u)
    # the iterations checked the residual in the eigenbasis; the oracle checks it physically
    assert info["relres_true"] <= 1e-8 and rel(O.bltt_matvec(prob, uh), f) <= 2e-8
    assert rel(uh, ref["x"]) <= 1e-6


def test_dense_laplacian_is_the_dst_path(B):
    # K = the dense Laplacian: the same iterations and solution as the DST-basis solve
    p = fractional_problem(2, (15, 7), 64, 0.6)
    pk = with_K(p, O.laplacian(p).toarray(), "lap")
    f = to_dev(rhs_uniform(p.n, 86))
    u0, i0 = B.Solver(p).solve(f, alpha=1e-8, tol=1e-10, basis=1)
    u1, i1 = B.Solver(pk).solve(f, alpha=1e-8, tol=1e-10)
    assert i0["status"] == i1["status"] == 0 and i0["iters"] == i1["iters"]
    assert rel(to_host(u1), to_host(u0)) <= 1e-9


def test_dense_exact_preconditioner_for_variable_coefficient(B):
    # K = L_a: P_alpha of the true blocks, not the mean-coefficient one; Table 3's problem needs 10
    # iterations with the mean coefficient and a few with the exact preconditioner
    p = heat_cn_varcoeff_problem(15, 32)
    pk = with_K(p, O.laplacian(p).toarray(), "La")
    f = rhs_uniform(p.n, 75)
    ref = O.solve(pk, f, alpha=1e-8, tol=1e-6)
    _, im = B.Solver(p).solve(to_dev(f), alpha=1e-8, tol=1e-6)
    u, ik = B.Solver(pk).solve(to_dev(f), alpha=1e-8, tol=1e-6)
    assert im["iters"] == 10 and ik["iters"] <= 3 and abs(ik["iters"] - ref["iters"]) <= 1
    assert rel(O.bltt_matvec(pk, to_host(u)), f) <= 1e-6


def test_dense_host_buffers_and_graph_replay(B):
    import torch
    prob = DPS[3]
    fh = rhs_uniform(prob.n, 87)
    st = torch.cuda.Stream()
    s = B.Solver(prob, stream=st)
    form = dict(precision=32, alpha=1e-3, tol=1e-8, maxit=100)
    with torch.cuda.stream(st):
        u1, i1 = s.solve(to_dev(fh), graph=True, **form)
        u2, i2 = s.solve(to_dev(fh), graph=False, **form)
    torch.cuda.synchronize()
    assert i1["status"] == i2["status"] == 0 and i1["iters"] == i2["iters"]
    assert torch.equal(u1, u2)
    uh, ih = s.solve_host(torch.from_numpy(fh), **form)
    assert ih["iters"] == i1["iters"] and np.array_equal(uh.numpy(), to_host(u1))


def test_dense_replace_and_keep_on_failure(B):
    p = fractional_problem(1, 31, 32, 0.5)
    K1, K2 = spd(p.M, 88, 200.0), spd(p.M, 89, 300.0)
    s = B.Solver(with_K(p, K1, "k1"))
    z = np.random.default_rng(90).standard_normal(p.n)
    y1 = to_host(s.matvec(to_dev(z)))
    assert rel(y1, O.bltt_matvec(with_K(p, K1, "k1"), z, flip=True)) <= 1e-11
    # a K whose eigenvalues break Assumption 1 (ii): refused, the handle keeps K1
    with pytest.raises(B.BlttError) as e:
        B.bltt_set_dense_operator(s.handle, -K1)
    assert e.value.status == 2
    assert np.array_equal(to_host(s.matvec(to_dev(z))), y1)
    B.bltt_set_dense_operator(s.handle, K2)
    y2 = to_host(s.matvec(to_dev(z)))
    assert rel(y2, O.bltt_matvec(with_K(p, K2, "k2"), z, flip=True)) <= 1e-11


def test_dense_declined(B):
    p = fractional_problem(1, 31, 128, 0.5)
    pk = with_K(p, spd(p.M, 91, 100.0), "spd")
    s = B.Solver(pk)
    f = to_dev(rhs_uniform(p.n, 92))
    with pytest.raises(B.BlttError) as e:
        s.solve(f, basis=2)                                   # the physical basis
    assert e.value.status == 8
    with pytest.raises(B.BlttError) as e:
        s.set_matvec_arith(3)                                 # the tensor-core product
    assert e.value.status == 8
    with pytest.raises(B.BlttError) as e:
        s.solve(f, matvec_arith=3)
    assert e.value.status == 8
    q = heat_cn_varcoeff_problem(15, 16)                      # variable coefficient already set
    with pytest.raises(B.BlttError) as e:
        B.bltt_set_dense_operator(B.Solver(q).handle, np.eye(q.M))
    assert e.value.status == 8
    s2 = B.Solver(p)
    bad = spd(p.M, 93, 100.0)
    bad[0, 1] += 1.0                                          # not symmetric
    with pytest.raises(B.BlttError) as e:
        B.bltt_set_dense_operator(s2.handle, bad)
    assert e.value.status == 1
    nan = spd(p.M, 94, 100.0)
    nan[3, 3] = np.nan
    with pytest.raises(B.BlttError) as e:
        B.bltt_set_dense_operator(s2.handle, nan)
    assert e.value.status == 1
    # a TC handle takes no dense operator
    s3 = B.Solver(fractional_problem(1, 31, 128, 0.5))
    s3.set_matvec_arith(3)
    with pytest.raises(B.BlttError) as e:
        B.bltt_set_dense_operator(s3.handle, np.eye(31) * 100.0)
    assert e.value.status == 8
    # a dense handle takes no variable coefficient
    with pytest.raises(B.BlttError) as e:
        B.bltt_set_variable_coefficient(s.handle, (np.ones(32),), 1.0)
    assert e.value.status == 8
