// dfgemm.cu - the basis changes of the dense-operator form (Sec. 3: commuting blocks share K's
// eigenvectors U) as double-float GEMMs on the FP32 pipes: C = A X with A = U or U^T (M x M), X
// and C time-major vectors (column-major M x N).  GB300's FP64 rate is a small fraction of its
// FP32 rate, so a product carried as hi + lo float pairs (about 48 significant bits, the
// precision of the double-float matvec) runs faster than the FP64 GEMM.
//
// Arithmetic per multiply-add, acc += a b with a = ah + al, b = bh + bl:
//   p = ah bh, e = fma(ah, bh, -p) (the exact rounding error of p), e += ah bl + al bh;
//   (s, t) = TwoSum(acc_hi, p) (Knuth's error-free sum), t += acc_lo + e, renormalised by
//   Fast2Sum.  The dropped al bl and the roundings of e and t give about 2^-47 relative error per
//   step.
#include "internal.h"

namespace bltt {

namespace {

constexpr int kBM = 64, kBN = 64, kBK = 16, kGemmThreads = 256;

__device__ __forceinline__ void df_mac(float& hi, float& lo, float2 a, float2 b) {
  const float p = a.x * b.x;
  float e = fmaf(a.x, b.x, -p);
  e = fmaf(a.x, b.y, e);
  e = fmaf(a.y, b.x, e);
  const float s = hi + p;
  const float z = s - hi;
  float t = (hi - (s - z)) + (p - z);
  t += lo + e;
  hi = s + t;
  lo = t - (hi - s);
}

__device__ __forceinline__ float2 split_d(double x) {
  const float h = (float)x;
  return make_float2(h, (float)(x - (double)h));
}

// hi/lo planes of U and of U^T, both column-major (A[i + k M]) for the GEMM's A operand
__global__ void k_df_planes(const double* __restrict__ U, long long M, float* __restrict__ Uh,
                            float* __restrict__ Ul, float* __restrict__ Th, float* __restrict__ Tl) {
  const long long total = M * M;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long k = e / M, i = e - k * M;           // U[i + k M] = U_ik
    const float2 v = split_d(U[e]);
    Uh[e] = v.x;
    Ul[e] = v.y;
    Th[k + i * M] = v.x;                                // (U^T)_ki
    Tl[k + i * M] = v.y;
  }
}

// one 64 x 64 tile of C per block; thread (tx, ty) owns rows i0 + tx + 16 r, columns t0 + ty + 16 c
__global__ void __launch_bounds__(kGemmThreads)
k_df_gemm(const float* __restrict__ Ah, const float* __restrict__ Al, const double* __restrict__ X,
          double* __restrict__ C, int M, int N) {
  __shared__ float2 sA[kBK][kBM];
  __shared__ float2 sB[kBK][kBN];
  const int i0 = blockIdx.x * kBM, t0 = blockIdx.y * kBN;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  float hi[4][4], lo[4][4];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) hi[r][c] = lo[r][c] = 0.f;
  for (int k0 = 0; k0 < M; k0 += kBK) {
    // A tile: for each k, 64 consecutive rows (coalesced along i)
    for (int e = threadIdx.x; e < kBK * kBM; e += kGemmThreads) {
      const int k = e / kBM, i = e - k * kBM;
      float2 v = make_float2(0.f, 0.f);
      if (i0 + i < M && k0 + k < M) {
        const long long idx = (long long)(k0 + k) * M + i0 + i;
        v = make_float2(Ah[idx], Al[idx]);
      }
      sA[k][i] = v;
    }
    // X tile: for each time t, 16 consecutive k (one 128-byte run of the vector)
    for (int e = threadIdx.x; e < kBK * kBN; e += kGemmThreads) {
      const int t = e / kBK, k = e - t * kBK;
      float2 v = make_float2(0.f, 0.f);
      if (t0 + t < N && k0 + k < M) v = split_d(__ldg(X + (long long)(t0 + t) * M + k0 + k));
      sB[k][t] = v;
    }
    __syncthreads();
#pragma unroll 4
    for (int k = 0; k < kBK; ++k) {
      float2 a[4], b[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) a[r] = sA[k][tx + 16 * r];
#pragma unroll
      for (int c = 0; c < 4; ++c) b[c] = sB[k][ty + 16 * c];
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) df_mac(hi[r][c], lo[r][c], a[r], b[c]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const int t = t0 + ty + 16 * c;
    if (t >= N) continue;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int i = i0 + tx + 16 * r;
      if (i < M) C[(long long)t * M + i] = (double)hi[r][c] + (double)lo[r][c];
    }
  }
}

}  // namespace

cudaError_t launch_df_planes(const double* U, long long M, float* Uh, float* Ul, float* Th,
                             float* Tl, cudaStream_t st) {
  if (M <= 0) return cudaSuccess;
  const long long total = M * M;
  const int grid = (int)((total + 255) / 256 < 4096 ? (total + 255) / 256 : 4096);
  k_df_planes<<<grid, 256, 0, st>>>(U, M, Uh, Ul, Th, Tl);
  return cudaGetLastError();
}

cudaError_t launch_df_gemm(const float* Ah, const float* Al, const double* X, double* C, int M,
                           int N, cudaStream_t st) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  if (N > 65535 * kBN) return cudaErrorInvalidValue;
  dim3 grid((M + kBM - 1) / kBM, (N + kBN - 1) / kBN);
  k_df_gemm<<<grid, kGemmThreads, 0, st>>>(Ah, Al, X, C, M, N);
  return cudaGetLastError();
}

}  // namespace bltt
