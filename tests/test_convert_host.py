"""The integer-pipe FP64 <-> FP32 conversions of the kernels (convert.cuh), compiled for the host
with g++ and checked against IEEE conversions (numpy's float32 casts) on a few million values:
ordinary values, exact ties, powers of two, the ends of the FP32 range, zeros, Inf and NaN."""
import os
import shutil
import subprocess
import tempfile

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
HDR = os.path.join(HERE, "..", "paper_2307_07749_gb300", "csrc", "convert.cuh")

SRC = r'''
#include <cstdio>
#include <cstdint>
#include <vector>
#include "convert.cuh"
using namespace bltt;
int main(int argc, char** argv) {
  FILE* fi = fopen(argv[1], "rb");
  FILE* fo = fopen(argv[2], "wb");
  std::vector<double> x;
  double v;
  while (fread(&v, 8, 1, fi) == 1) x.push_back(v);
  for (double d : x) {
    float a = d2f_bits(d), b = d2f_fast(d);
    double c = f2d_bits(a), e = f2d_fast(a);
    fwrite(&a, 4, 1, fo); fwrite(&b, 4, 1, fo); fwrite(&c, 8, 1, fo); fwrite(&e, 8, 1, fo);
  }
  fclose(fo);
  return 0;
}
'''


@pytest.fixture(scope="module")
def conv_tool():
    if shutil.which("g++") is None:
        pytest.skip("g++ not available")
    d = tempfile.mkdtemp()
    src = os.path.join(d, "conv.cpp")
    exe = os.path.join(d, "conv")
    with open(src, "w") as fh:
        fh.write(SRC)
    subprocess.run(["g++", "-O1", "-std=c++17", "-I", os.path.dirname(HDR), src, "-o", exe],
                   check=True)
    yield exe
    shutil.rmtree(d, ignore_errors=True)


def run(exe, x):
    d = tempfile.mkdtemp()
    try:
        fi, fo = os.path.join(d, "in"), os.path.join(d, "out")
        np.asarray(x, np.float64).tofile(fi)
        subprocess.run([exe, fi, fo], check=True)
        rec = np.fromfile(fo, dtype=np.dtype([("a", "<f4"), ("b", "<f4"), ("c", "<f8"), ("e", "<f8")]))
        return rec["a"], rec["b"], rec["c"], rec["e"]
    finally:
        shutil.rmtree(d, ignore_errors=True)


def values():
    rng = np.random.default_rng(0)
    x = [rng.standard_normal(1 << 20) * 10.0 ** rng.uniform(-30, 30, 1 << 20),
         rng.uniform(-1, 1, 1 << 20)]
    # exact ties between two FP32 neighbours, and their neighbours
    f = rng.standard_normal(1 << 18).astype(np.float32)
    up = np.nextafter(f, np.float32(np.inf))
    mid = (f.astype(np.float64) + up.astype(np.float64)) / 2.0
    x += [mid, np.nextafter(mid, np.inf), np.nextafter(mid, -np.inf)]
    x.append(2.0 ** np.arange(-125, 128).astype(np.float64))
    x.append(np.array([0.0, -0.0, 1.0, -1.0, float(np.finfo(np.float32).max),
                       float(np.finfo(np.float32).tiny)]))
    return np.concatenate(x)


def test_rne_conversions_are_exact(conv_tool):
    x = values()
    a, _, c, _ = run(conv_tool, x)
    ref = x.astype(np.float32)
    assert np.array_equal(a.view(np.uint32), ref.view(np.uint32))
    assert np.array_equal(c, ref.astype(np.float64))


def test_fast_conversions(conv_tool):
    x = values()
    _, b, _, e = run(conv_tool, x)
    ref = x.astype(np.float32)
    exact = b.view(np.uint32) == ref.view(np.uint32)
    # d2f_fast rounds ties away from zero: the only differences are exact ties, by one ulp
    ties = ~exact
    assert np.all(np.abs(b[ties].astype(np.float64)) > np.abs(ref[ties].astype(np.float64)))
    gap = np.abs(np.nextafter(ref[ties], np.float32(np.inf)) - ref[ties]).astype(np.float64)
    assert np.allclose(np.abs(x[ties]) - np.abs(ref[ties].astype(np.float64)), gap / 2, rtol=0, atol=0)
    assert ties.sum() <= (1 << 18) + 10                         # the ties block and nothing else
    # f2d_fast (applied to the IEEE-rounded floats) is exact on every normal or zero float
    a = ref
    fin = np.isfinite(a) & ((np.abs(a) >= np.finfo(np.float32).tiny) | (a == 0))
    assert np.array_equal(e[fin], a[fin].astype(np.float64))
    assert np.array_equal(np.signbit(e[fin]), np.signbit(a[fin]))


def test_fast_conversions_keep_non_finite_visible(conv_tool):
    x = np.array([np.inf, -np.inf, np.nan, 1e300, -3e38 * 2, 1e-300, -1e-300])
    a, b, _, e = run(conv_tool, x)
    assert np.all(np.isnan(b[:5]))
    assert np.all(b[5:] == 0.0) and np.signbit(b[6]) and not np.signbit(b[5])
    # f2d_fast of the IEEE floats: Inf and NaN (the first five, after d2f_bits) stay non-finite
    assert not np.any(np.isfinite(e[:5]))
