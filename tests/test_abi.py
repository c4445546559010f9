"""The C ABI without a GPU: the library builds and loads, exports every declared symbol, and
rejects bad arguments on the host before touching the device."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    inc = os.path.join(ROOT, "include")
    for f in os.listdir(inc):
        if f.endswith(".h"):
            txt = open(os.path.join(inc, f)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(bltt_[a-z0-9_]+)\s*\(", txt))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_2307_07749_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_exports_every_declared_symbol(lib):
    syms = declared_symbols()
    assert "bltt_create" in syms and "bltt_minres_solve" in syms
    for s in syms:
        assert hasattr(lib, s), s


def test_version(lib):
    import paper_2307_07749_gb300 as B
    assert "sm_103a" in B.bltt_version()


def _create(a, b, N, d, m, h):
    import paper_2307_07749_gb300 as B
    with pytest.raises(B.BlttError) as ei:
        B.bltt_create(a, b, N, d, m, h)
    return ei.value.status


def test_host_validation(lib):
    from workloads import fractional_problem
    p = fractional_problem(1, 7, 8, 0.5)
    # N not a power of two
    assert _create(np.ones(6), np.r_[1.0, np.zeros(5)], 6, 1, (7,), (0.125,)) == 8
    # m + 1 not a power of two
    assert _create(p.a, p.b, 8, 1, (6,), (1 / 7,)) == 8
    # bad dimension
    assert _create(p.a, p.b, 8, 4, (7,), (0.125,)) == 1
    # Assumption 1 (ii) violated: |A_(1)| outweighs A_(0) on the high modes
    b = p.b.copy()
    b[1] = -2.0
    assert _create(p.a, b, 8, 1, (7,), (0.125,)) == 2
    # beyond the largest FFT a tile holds (N = 4096, m + 1 = 4096)
    assert _create(np.r_[1.0, np.zeros(4095)], np.r_[1.0, np.zeros(4095)], 4096, 1, (7,), (0.125,)) == 8
    assert _create(p.a, p.b, 8, 1, (4095,), (1 / 4096,)) == 8
    # non-finite coefficient
    a = p.a.copy()
    a[3] = np.nan
    assert _create(a, p.b, 8, 1, (7,), (0.125,)) == 5


def test_null_handle_calls(lib):
    import paper_2307_07749_gb300 as B
    L = B.lib()
    assert L.bltt_destroy(None) == 0
    assert L.bltt_matvec(None, None, None, 1) == 1
    assert L.bltt_precond_apply(None, 0.5, None, None, 64) == 1
    assert L.bltt_set_stream(None, None) == 1
    assert L.bltt_set_matvec_arith(None, 1) == 1
    assert L.bltt_set_variable_coefficient(None, None, 1.0) == 1
    assert L.bltt_set_dense_operator(None, None) == 1
    # guard bands and the refinement path refuse a null handle before touching the device
    import ctypes
    n = ctypes.c_int(-1)
    assert L.bltt_check_guards(None, ctypes.byref(n)) == 1
    assert L.bltt_guard_poke(None, 0) == 1
    opts = B.bltt_solve_opts(32, 1, 0, 0, 0, 2, 0, 0, 0, 4)
    info = B.bltt_solve_info()
    assert L.bltt_minres_solve_ex(None, None, 1e-2, 1e-8, 10, ctypes.byref(opts), None,
                                  ctypes.byref(info)) == 1
    assert L.bltt_minres_solve_host(None, None, 1e-2, 1e-8, 10, ctypes.byref(opts), None,
                                    ctypes.byref(info)) == 1


def test_alpha_label_rule(lib):
    """Sweep labels: the fewest iterations decide; the label is the centre (log10) of the longest
    run of consecutive sweep points reaching that count, equal runs going to larger alpha."""
    from paper_2307_07749_gb300 import learned_alpha as LA
    a = [10.0 ** (-j / 2.0) for j in range(1, 9)]          # 10^-0.5 .. 10^-4

    def res(its):
        return [(x, it, 0.0) for x, it in zip(a, its)]

    # plateau of 5s over 10^-1.5 .. 10^-2.5, a cliff below it
    assert LA.label(res([9, 7, 5, 5, 5, None, None, None])) == pytest.approx(-2.0)
    # a single minimum beats a longer plateau of higher counts
    assert LA.label(res([6, 6, 6, 6, 5, 6, 12, None])) == pytest.approx(-2.5)
    # two equally long runs: the one of larger alpha
    assert LA.label(res([4, 4, 6, 4, 4, 7, None, None])) == pytest.approx(-0.75)
    assert LA.label(res([None] * 8)) is None
