"""Guard bands (BLTT_GUARD_BANDS=1), the substitute for a memory checker: every workspace vector
and deferred-update slot sits between bands of a fixed NaN pattern, read back after the solves of
every form; a band written from the host is reported.  Runs in a child process, so that the
environment variable is set before the library allocates any workspace."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import sys
sys.path.insert(0, ROOT)
sys.path.insert(0, ROOT + "/tests")
import numpy as np, torch
import paper_2307_07749_gb300 as B
import oracle as O
from workloads import fractional_problem, heat_cn_problem, rhs_uniform
from _gpu_helpers import rel, to_dev, to_host
forms = [dict(precision=64, basis=1, matvec_arith=1, alpha=1e-8),
         dict(precision=32, basis=1, matvec_arith=2, alpha=1e-2),
         dict(precision=96, basis=1, matvec_arith=2, alpha=1e-6),
         dict(precision=32, basis=2, matvec_arith=2, alpha=1e-3),
         dict(precision=64, basis=2, matvec_arith=1, alpha=1.0)]
checked = 0
for prob in (fractional_problem(2, 31, 64, 0.7), heat_cn_problem(2, 31, 64), fractional_problem(1, 63, 128, 0.4)):
    fh = rhs_uniform(prob.n, 64)
    s = B.Solver(prob)
    for form in forms:
        u, info = s.solve(to_dev(fh), tol=1e-8, maxit=300, **form)
        assert info["status"] == 0, info
        assert rel(O.bltt_matvec(prob, to_host(u)), fh) <= 1e-8
        n = B.bltt_check_guards(s.handle)
        assert n == 11 + 8, n        # 10 workspace vectors and 7 window slots: 11 + 8 bands
        checked += n
    u, info = s.solve(to_dev(fh), tol=1e-8, maxit=300, refine=4, precision=32, basis=1,
                      matvec_arith=2, alpha=1e-8)
    assert B.bltt_check_guards(s.handle) == 19
B.bltt_guard_poke(s.handle, 3)
try:
    B.bltt_check_guards(s.handle)
    raise SystemExit("a written band went unreported")
except B.BlttError as e:
    assert "guard band 3" in str(e) or "guard band 3" in B.lib().bltt_last_error(s.handle).decode(), e
print("GUARDS_OK", checked)
""".replace("ROOT", repr(ROOT))


def test_guard_bands_stay_intact_and_a_written_band_is_reported():
    env = dict(os.environ, BLTT_GUARD_BANDS="1")
    r = subprocess.run([sys.executable, "-c", CHILD], env=env, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0 and "GUARDS_OK" in r.stdout, r.stdout[-2000:] + r.stderr[-4000:]
