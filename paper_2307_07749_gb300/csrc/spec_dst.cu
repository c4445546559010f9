// spec_dst.cu - the DST-I tile kernel (k_dst) compiled for P = m + 1 = 2^7 and 2^8 with P, m and
// the column count as constants, in FP64, FP32 and double-float, for contiguous and strided lines.
#include "tiles.cuh"
#include "spec.h"
#include "launch_util.h"

namespace bltt {
namespace {

template <class A, bool SWZ, int L2P>
cudaError_t dst_attr() {
  static std::atomic<unsigned long long> done{0};
  return once_per_device(done, [] {
    return set_smem(k_dst<A, SWZ, L2P>, TileCfg<A>::CAP * sizeof(typename A::V));
  });
}

template <class A, bool SWZ, int L2P>
cudaError_t run_dst(unsigned grid, size_t smem, cudaStream_t st, long long nlines, int m,
                    long long inner, const Combine& cb, double* out, int flip, int N, long long M,
                    const double* dot_with, double* partials, const void* tw, const int* phase,
                    int want) {
  cudaError_t e = dst_attr<A, SWZ, L2P>();
  if (e != cudaSuccess) return e;
  k_dst<A, SWZ, L2P><<<grid, TileCfg<A>::NT, smem, st>>>(
      nlines, m, inner, 1 << L2P, L2P, ilog2c(TileCfg<A>::CAP) - L2P, cb, out, flip, N, M,
      dot_with, partials, static_cast<const typename A::V*>(tw), phase, want);
  return cudaGetLastError();
}

template <class A, int L2P>
cudaError_t run_dst2(bool contiguous, unsigned grid, size_t smem, cudaStream_t st,
                     long long nlines, int m, long long inner, const Combine& cb, double* out,
                     int flip, int N, long long M, const double* dot_with, double* partials,
                     const void* tw, const int* phase, int want) {
  // contiguous lines take the swizzled shared-memory layout, as in the run-time-sized launcher
  return contiguous ? run_dst<A, true, L2P>(grid, smem, st, nlines, m, inner, cb, out, flip, N, M,
                                            dot_with, partials, tw, phase, want)
                    : run_dst<A, false, L2P>(grid, smem, st, nlines, m, inner, cb, out, flip, N,
                                             M, dot_with, partials, tw, phase, want);
}

template <class A>
cudaError_t all_attr() {
  cudaError_t e = dst_attr<A, true, 7>();
  if (e == cudaSuccess) e = dst_attr<A, false, 7>();
  if (e == cudaSuccess) e = dst_attr<A, true, 8>();
  if (e == cudaSuccess) e = dst_attr<A, false, 8>();
  return e;
}

}  // namespace

static_assert(kSpecLog2PMin == 7 && kSpecLog2PMax == 8, "the instantiations below");

bool spec_dst(int prec, bool contiguous, int log2P, int log2NC, unsigned grid, size_t smem,
              cudaStream_t st, long long nlines, int m, long long inner, const Combine& cb,
              double* out, int flip, int N, long long M, const double* dot_with,
              double* partials, const void* tw, const int* phase, int want, cudaError_t* err) {
  if (log2P < kSpecLog2PMin || log2P > kSpecLog2PMax || m != (1 << log2P) - 1) return false;
  if (log2NC != ilog2c(kCap) - log2P) return false;
#define BLTT_DST(A_) \
  (log2P == 7 ? run_dst2<A_, 7>(contiguous, grid, smem, st, nlines, m, inner, cb, out, flip, N, \
                                M, dot_with, partials, tw, phase, want)                        \
              : run_dst2<A_, 8>(contiguous, grid, smem, st, nlines, m, inner, cb, out, flip, N, \
                                M, dot_with, partials, tw, phase, want))
  if (prec == PREC_DF) *err = BLTT_DST(ArithDF);
  else if (prec == PREC_F64) *err = BLTT_DST(ArithD);
  else if (prec == PREC_F32) *err = BLTT_DST(ArithF);
  else return false;
#undef BLTT_DST
  return true;
}

cudaError_t spec_prepare_dst_attributes() {
  cudaError_t e = all_attr<ArithD>();
  if (e == cudaSuccess) e = all_attr<ArithF>();
  if (e == cudaSuccess) e = all_attr<ArithDF>();
  return e;
}

}  // namespace bltt
