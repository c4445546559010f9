"""bltt_residual_noalloc: the allocation-free true-residual entry point (no handle, no cudaMalloc;
its scratch is a fixed device array).  Checked through the C ABI against the residual built from
the existing bltt_matvec entry point and against the oracle's block sum, on two calls in a row.
Collected last on purpose."""
import numpy as np
import pytest

import oracle as O
from workloads import fractional_problem, heat_bdf_problem, rhs_uniform
from _gpu_helpers import rel, to_dev, to_host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    from paper_2307_07749_gb300 import build
    build.build()
    import paper_2307_07749_gb300 as mod
    return mod


@pytest.mark.parametrize("prob", [fractional_problem(2, 31, 32, 0.7),       # FFT matvec
                                  heat_bdf_problem(3, (15, 7, 3), 16)],     # direct taps
                         ids=["frac2d_fft", "heat3d_direct"])
def test_residual_noalloc_matches_matvec(B, prob):
    s = B.Solver(prob)
    for call in range(2):                      # the shared scratch keeps the previous call's data
        rng = np.random.default_rng(40 + call)
        u = to_dev(rng.standard_normal(prob.n))
        f = to_dev(rng.standard_normal(prob.n))
        r = to_dev(np.zeros(prob.n))
        relres = B.bltt_residual_noalloc(prob.a, prob.b, prob.N, prob.d, prob.m, prob.h, u, f, r)
        y = s.matvec(u, flip=False)            # existing entry point: y = A u
        r_ref = to_host(f) - to_host(y)
        relres_ref = np.linalg.norm(r_ref) / np.linalg.norm(to_host(f))
        assert rel(to_host(r), r_ref) <= 1e-12
        assert abs(relres - relres_ref) <= 1e-12 * relres_ref
        # and the oracle's direct block sum A u (independent of the library's matvec)
        r_or = to_host(f) - O.bltt_matvec(prob, to_host(u))
        assert rel(to_host(r), r_or) <= 1e-12
        assert abs(relres - np.linalg.norm(r_or) / np.linalg.norm(to_host(f))) <= 1e-12 * relres_ref
        # without the residual vector
        relres2 = B.bltt_residual_noalloc(prob.a, prob.b, prob.N, prob.d, prob.m, prob.h, u, f)
        assert abs(relres2 - relres_ref) <= 1e-12 * relres_ref


def test_residual_noalloc_rejects_unsupported(B):
    p = fractional_problem(2, 7, 16, 0.5)
    b = 0.1 * 0.5 ** np.arange(p.N)
    b[0] = 1.0
    u = to_dev(np.zeros(p.n))
    with pytest.raises(B.BlttError) as e:
        B.bltt_residual_noalloc(p.a, b, p.N, p.d, p.m, p.h, u, u.clone())
    assert e.value.status == 8
    with pytest.raises(B.BlttError) as e:            # N not a power of two
        B.bltt_residual_noalloc(p.a[:6], p.b[:6], 6, p.d, p.m, p.h, u[:6 * p.M], u[:6 * p.M].clone())
    assert e.value.status == 8
    q = fractional_problem(2, 6, 16, 0.5)             # m+1 = 7 is not a power of two
    uq = to_dev(np.zeros(q.n))
    with pytest.raises(B.BlttError) as e:
        B.bltt_residual_noalloc(q.a, q.b, q.N, q.d, q.m, q.h, uq, uq.clone())
    assert e.value.status == 8
    with pytest.raises(B.BlttError) as e:            # r aliases u
        B.bltt_residual_noalloc(p.a, p.b, p.N, p.d, p.m, p.h, u, u.clone(), u)
    assert e.value.status == 1
