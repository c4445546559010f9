// spec_conv.cu - the BLTT matvec tile kernel (k_conv) compiled for N = 2^9 .. 2^11 with the
// transform length and the column count as constants.
#include "tiles.cuh"
#include "spec.h"
#include "launch_util.h"

namespace bltt {
namespace {

template <class A, int L2N>
cudaError_t conv_attr() {
  static std::atomic<unsigned long long> done{0};
  return once_per_device(done, [] {
    return set_smem(k_conv<A, L2N>, TileCfg<A>::CAP * sizeof(typename A::V));
  });
}

template <class A, int L2N>
cudaError_t run_conv(unsigned grid, size_t smem, cudaStream_t st, const OpTables& op, int spectral,
                     int which, const double* x, const double* xscale, double* y, int flip,
                     int mode, const double* rhs, double* partials, const int* phase, int want,
                     const double* st_src) {
  cudaError_t e = conv_attr<A, L2N>();
  if (e != cudaSuccess) return e;
  k_conv<A, L2N><<<grid, TileCfg<A>::NT, smem, st>>>(op, spectral, which, x, xscale, y, flip, mode,
                                                     rhs, partials, phase, want, st_src,
                                                     ilog2c(TileCfg<A>::CAP) - L2N - 1);
  return cudaGetLastError();
}

template <class A>
cudaError_t all_attr() {
  cudaError_t e = conv_attr<A, 9>();
  if (e == cudaSuccess) e = conv_attr<A, 10>();
  if (e == cudaSuccess) e = conv_attr<A, 11>();
  return e;
}

}  // namespace

static_assert(kSpecLog2NMin == 9 && kSpecLog2NMax == 11, "the instantiations below");

bool spec_conv(int prec, int log2N, int log2NC, unsigned grid, size_t smem, cudaStream_t st,
               const OpTables& op, int spectral, int which, const double* x, const double* xscale,
               double* y, int flip, int mode, const double* rhs, double* partials,
               const int* phase, int want, const double* st_src, cudaError_t* err) {
  if (log2N < kSpecLog2NMin || log2N > kSpecLog2NMax || log2NC != ilog2c(kCap) - log2N - 1)
    return false;
#define BLTT_CONV(A_, L_) \
  run_conv<A_, L_>(grid, smem, st, op, spectral, which, x, xscale, y, flip, mode, rhs, partials, \
                   phase, want, st_src)
  if (prec == PREC_DF) {
    *err = log2N == 9 ? BLTT_CONV(ArithDF, 9) : log2N == 10 ? BLTT_CONV(ArithDF, 10)
                                                             : BLTT_CONV(ArithDF, 11);
  } else if (prec == PREC_F64) {
    *err = log2N == 9 ? BLTT_CONV(ArithD, 9) : log2N == 10 ? BLTT_CONV(ArithD, 10)
                                                            : BLTT_CONV(ArithD, 11);
  } else {
    return false;
  }
#undef BLTT_CONV
  return true;
}

cudaError_t spec_prepare_conv_attributes() {
  cudaError_t e = all_attr<ArithD>();
  if (e == cudaSuccess) e = all_attr<ArithDF>();
  return e;
}

}  // namespace bltt
