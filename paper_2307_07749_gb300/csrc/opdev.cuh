// opdev.cuh - device helpers on the operator tables shared by the kernel translation units:
// the phase gate of graph-replayed launches, the eigenvalues of L per spatial mode and the
// finite-difference stencil of L.
#pragma once
#include "internal.h"

namespace bltt {

// a launch whose MINRES phase differs from `want` does nothing (replayed graphs keep launching
// after the solve has stopped)
__device__ __forceinline__ bool skip_phase(const int* phase, int want) {
  return phase != nullptr && *phase != want;
}

// eigenvalue of L for spatial mode i (x fastest): sum over axes of the 1-D eigenvalues
__device__ __forceinline__ double mode_mu(const OpTables& op, long long i) {
  long long r = i / op.m[0];
  double mu = op.mu_axis[0][i - r * op.m[0]];
  if (op.d > 1) {
    long long r2 = r / op.m[1];
    mu += op.mu_axis[1][r - r2 * op.m[1]];
    if (op.d > 2) mu += op.mu_axis[2][r2];
  }
  return mu;
}
__device__ __forceinline__ float mode_mu32(const OpTables& op, long long i) {
  long long r = i / op.m[0];
  float mu = op.mu_axis32[0][i - r * op.m[0]];
  if (op.d > 1) {
    long long r2 = r / op.m[1];
    mu += op.mu_axis32[1][r - r2 * op.m[1]];
    if (op.d > 2) mu += op.mu_axis32[2][r2];
  }
  return mu;
}

// (L x)[i] on the time slice starting at x_t: the 2d+1 point Dirichlet stencil (Sec. 5.2)
__device__ __forceinline__ double stencil_at(const OpTables& op, const double* __restrict__ x_t,
                                             long long i) {
  const double xi = x_t[i];
  double acc = 0.0;
  long long r = i, stride = 1;
#pragma unroll 1
  for (int ax = 0; ax < op.d; ++ax) {
    const int mm = op.m[ax];
    long long q = r / mm;
    int c = (int)(r - q * mm);
    r = q;
    double s = 2.0 * xi;
    if (c > 0) s -= x_t[i - stride];
    if (c < mm - 1) s -= x_t[i + stride];
    acc = fma(s, op.h2inv[ax], acc);
    stride *= mm;
  }
  return acc;
}

}  // namespace bltt
