// common.cuh - device building blocks shared by the libbltt kernels: complex arithmetic, the
// shared-memory Stockham FFT engine, block reductions and the tile geometry of a batch of lines.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace bltt {

// ------------------------------------------------------------------------------------------
// complex numbers as CUDA vector types
template <typename T> struct cplx;
template <> struct cplx<double> { using t = double2; };
template <> struct cplx<float> { using t = float2; };
template <typename T> using C = typename cplx<T>::t;

template <typename T> __device__ __forceinline__ C<T> mk(T re, T im) { C<T> r; r.x = re; r.y = im; return r; }
template <typename T> __device__ __forceinline__ C<T> cadd(C<T> a, C<T> b) { return mk<T>(a.x + b.x, a.y + b.y); }
template <typename T> __device__ __forceinline__ C<T> csub(C<T> a, C<T> b) { return mk<T>(a.x - b.x, a.y - b.y); }
template <typename T> __device__ __forceinline__ C<T> cconj(C<T> a) { return mk<T>(a.x, -a.y); }
// a * b
template <typename T> __device__ __forceinline__ C<T> cmul(C<T> a, C<T> b) {
  return mk<T>(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
// a * conj(b)
template <typename T> __device__ __forceinline__ C<T> cmulc(C<T> a, C<T> b) {
  return mk<T>(fma(a.x, b.x, a.y * b.y), fma(a.y, b.x, -a.x * b.y));
}
// multiply by -i (forward) or +i (inverse)
template <typename T, bool INV> __device__ __forceinline__ C<T> rot(C<T> a) {
  return INV ? mk<T>(-a.y, a.x) : mk<T>(a.y, -a.x);
}

// ------------------------------------------------------------------------------------------
// Shared-memory Stockham FFT (self-sorting, radix 4 with one radix-2 pass when log2 L is odd).
//
// buf holds NC independent complex columns of length L, element (p, c) at buf[p * NC + c].
// tw is the table w_L^k = exp(-2 pi i k / L), k < L.  Forward: X_k = sum_j x_j w^{jk};
// inverse (INV): the same with conjugate twiddles and no 1/L scaling.
// Every pass first loads all of its butterfly inputs into registers, synchronises, then writes;
// so the transform runs in place in buf.  CAP bounds NC*L; the block has NT threads.
template <typename T, int NT, int CAP, bool INV>
__device__ void fft_columns(C<T>* buf, int L, int log2L, int NC, const C<T>* __restrict__ tw) {
  constexpr int IPT4 = (CAP / 4 + NT - 1) / NT;   // radix-4 butterflies per thread
  const int tid = threadIdx.x;
  int Ns = 1;
  if (log2L & 1) {
    // radix-2 pass with Ns = 1: no twiddles; out[2j + r] = DFT2(in[j], in[j + L/2])
    const int half = L >> 1;
    const int total = NC * half;
    C<T> v[2 * IPT4][2];
#pragma unroll
    for (int s = 0; s < 2 * IPT4; ++s) {
      int it = tid + s * NT;
      if (it < total) {
        int c = it % NC, j = it / NC;
        v[s][0] = buf[j * NC + c];
        v[s][1] = buf[(j + half) * NC + c];
      }
    }
    __syncthreads();
#pragma unroll
    for (int s = 0; s < 2 * IPT4; ++s) {
      int it = tid + s * NT;
      if (it < total) {
        int c = it % NC, j = it / NC;
        buf[(2 * j) * NC + c] = cadd<T>(v[s][0], v[s][1]);
        buf[(2 * j + 1) * NC + c] = csub<T>(v[s][0], v[s][1]);
      }
    }
    __syncthreads();
    Ns = 2;
  }
  const int quarter = L >> 2;
  const int total = NC * quarter;
  for (; Ns < L; Ns <<= 2) {
    const int tstep = L / (4 * Ns);   // twiddle index stride: w_{4Ns}^{rk} = w_L^{rk L/(4Ns)}
    C<T> v[IPT4][4];
#pragma unroll
    for (int s = 0; s < IPT4; ++s) {
      int it = tid + s * NT;
      if (it < total) {
        int c = it % NC, j = it / NC;
#pragma unroll
        for (int r = 0; r < 4; ++r) v[s][r] = buf[(j + r * quarter) * NC + c];
      }
    }
    __syncthreads();
#pragma unroll
    for (int s = 0; s < IPT4; ++s) {
      int it = tid + s * NT;
      if (it < total) {
        int c = it % NC, j = it / NC;
        int k = j & (Ns - 1);
        if (k != 0) {
          int e = k * tstep;
#pragma unroll
          for (int r = 1; r < 4; ++r) {
            C<T> w = __ldg(&tw[r * e]);
            v[s][r] = INV ? cmulc<T>(v[s][r], w) : cmul<T>(v[s][r], w);
          }
        }
        C<T> t0 = cadd<T>(v[s][0], v[s][2]);
        C<T> t1 = csub<T>(v[s][0], v[s][2]);
        C<T> t2 = cadd<T>(v[s][1], v[s][3]);
        C<T> t3 = rot<T, INV>(csub<T>(v[s][1], v[s][3]));
        int o = (j - k) * 4 + k;   // (j / Ns) * 4Ns + k
        buf[o * NC + c] = cadd<T>(t0, t2);
        buf[(o + Ns) * NC + c] = cadd<T>(t1, t3);
        buf[(o + 2 * Ns) * NC + c] = csub<T>(t0, t2);
        buf[(o + 3 * Ns) * NC + c] = csub<T>(t1, t3);
      }
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------------------------------------
// block-wide sum of one double per thread; result valid in thread 0.  scratch: >= 32 doubles.
template <int NT>
__device__ __forceinline__ double block_sum(double v, double* scratch) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) scratch[warp] = v;
  __syncthreads();
  double r = 0.0;
  if (warp == 0) {
    r = (lane < NT / 32) ? scratch[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) r += __shfl_down_sync(0xffffffffu, r, o);
  }
  return r;
}

// ------------------------------------------------------------------------------------------
// A batch of lines inside a time-major array: line g has elements at base(g) + p * inner,
// p < len, with base(g) = (g / inner) * (len * inner) + g % inner.  Time lines: len = N,
// inner = M.  DST lines along spatial axis ax: len = m_ax, inner = m_0 ... m_{ax-1}.
struct Lines {
  long long nlines;
  int len;
  long long inner;
  __device__ __forceinline__ long long base(long long g) const {
    return (g / inner) * ((long long)len * inner) + (g % inner);
  }
};

}  // namespace bltt
