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

// eigenvalue of L for spatial mode i (x fastest): sum over axes of the 1-D eigenvalues, or the
// dense operator's eigenvalue from its table
__device__ __forceinline__ double mode_mu(const OpTables& op, long long i) {
  if (op.mu_tab) return op.mu_tab[i];
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
  if (op.mu_tab32) return op.mu_tab32[i];
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

// coordinates (ix, iy, iz) of spatial index i (x fastest)
__device__ __forceinline__ void mode_coords(const OpTables& op, long long i, int& ix, int& iy,
                                            int& iz) {
  const long long r1 = i / op.m[0];
  ix = (int)(i - r1 * op.m[0]);
  iy = 0;
  iz = 0;
  if (op.d > 1) {
    const long long r2 = r1 / op.m[1];
    iy = (int)(r1 - r2 * op.m[1]);
    iz = (int)r2;
  }
}

// (L_a x)[i] on the time slice x_t with the coefficient at the cell faces (op.kf): per axis
// [a_lo (x_i - x_{i-s}) + a_hi (x_i - x_{i+s})] / h^2 with zero Dirichlet values, the central-
// difference discretisation of -div(a grad) (Sec. 5.2, the paper's Delta_{a,h}).  Face (.., f, ..)
// of axis ax sits between points f-1 and f of its line.
__device__ __forceinline__ double stencil_faces(const OpTables& op, const double* __restrict__ x_t,
                                                long long i, int ix, int iy, int iz) {
  const double xi = x_t[i];
  const long long m0 = op.m[0], m1 = op.d > 1 ? op.m[1] : 1;
  double acc = 0.0;
  long long stride = 1;
  for (int ax = 0; ax < op.d; ++ax) {
    const int c = ax == 0 ? ix : (ax == 1 ? iy : iz);
    const int mm = op.m[ax];
    long long lo, hi;
    if (ax == 0) { lo = ((long long)iz * m1 + iy) * (m0 + 1) + ix; hi = lo + 1; }
    else if (ax == 1) { lo = ((long long)iz * (m1 + 1) + iy) * m0 + ix; hi = lo + m0; }
    else { lo = ((long long)iz * m1 + iy) * m0 + ix; hi = lo + m1 * m0; }
    const double alo = op.kf[ax][lo], ahi = op.kf[ax][hi];
    double s = (alo + ahi) * xi;
    if (c > 0) s -= alo * x_t[i - stride];
    if (c < mm - 1) s -= ahi * x_t[i + stride];
    acc = fma(s, op.h2inv[ax], acc);
    stride *= mm;
  }
  return acc;
}

}  // namespace bltt
