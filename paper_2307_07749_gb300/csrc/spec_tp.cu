// spec_tp.cu - the time-pass tile kernel (k_timepass) compiled for N = 2^9 .. 2^11 with the
// transform length and the column count as constants: FP64 and double-float on the 4096-point
// tile, FP32 on the 4096-point tile for N = 512 and on the 8192-point one above.
#include "tiles.cuh"
#include "spec.h"
#include "launch_util.h"

namespace bltt {
namespace {

template <class A, class Cfg, int L2N>
cudaError_t tp_attr() {
  static std::atomic<unsigned long long> done{0};
  return once_per_device(done, [] {
    return set_smem(k_timepass<A, Cfg, L2N>,
                    Cfg::CAP * sizeof(typename A::V) + tp_stage_bytes<A>(kCap));
  });
}

template <class A, class Cfg, int L2N>
cudaError_t run_tp(unsigned grid, size_t smem, cudaStream_t st, const OpTables& op,
                   const PrecTables& pt, const Combine& cb, double* out, const double* dot_with,
                   double* partials, const int* phase, int want, const void* tw) {
  cudaError_t e = tp_attr<A, Cfg, L2N>();
  if (e != cudaSuccess) return e;
  k_timepass<A, Cfg, L2N><<<grid, Cfg::NT, smem, st>>>(
      op, pt, cb, out, dot_with, partials, phase, want, ilog2c(Cfg::CAP) - L2N,
      static_cast<const typename A::V*>(tw));
  return cudaGetLastError();
}

}  // namespace

static_assert(kSpecLog2NMin == 9 && kSpecLog2NMax == 11, "the instantiations below");

bool spec_timepass(int prec, bool wide, int log2N, int log2NC, unsigned grid, size_t smem,
                   cudaStream_t st, const OpTables& op, const PrecTables& pt, const Combine& cb,
                   double* out, const double* dot_with, double* partials, const int* phase,
                   int want, const void* tw, cudaError_t* err) {
  if (log2N < kSpecLog2NMin || log2N > kSpecLog2NMax) return false;
  // the FP32 tile of the run-time-sized launcher: 8192 points for N >= 1024
  if (prec == PREC_F32 && wide != (log2N >= 10)) return false;
  const int cap = (prec == PREC_F32 && wide) ? WideTileF::CAP : kCap;
  if (log2NC != ilog2c(cap) - log2N) return false;
#define BLTT_TP(A_, C_, L_) \
  run_tp<A_, C_, L_>(grid, smem, st, op, pt, cb, out, dot_with, partials, phase, want, tw)
  if (prec == PREC_DF) {
    using C = TileCfg<ArithDF>;
    *err = log2N == 9 ? BLTT_TP(ArithDF, C, 9) : log2N == 10 ? BLTT_TP(ArithDF, C, 10)
                                                              : BLTT_TP(ArithDF, C, 11);
  } else if (prec == PREC_F64) {
    using C = TileCfg<ArithD>;
    *err = log2N == 9 ? BLTT_TP(ArithD, C, 9) : log2N == 10 ? BLTT_TP(ArithD, C, 10)
                                                             : BLTT_TP(ArithD, C, 11);
  } else if (prec == PREC_F32) {
    *err = log2N == 9 ? BLTT_TP(ArithF, TileCfg<ArithF>, 9)
         : log2N == 10 ? BLTT_TP(ArithF, WideTileF, 10) : BLTT_TP(ArithF, WideTileF, 11);
  } else {
    return false;
  }
#undef BLTT_TP
  return true;
}

cudaError_t spec_prepare_tp_attributes() {
  cudaError_t e = tp_attr<ArithD, TileCfg<ArithD>, 9>();
  if (e == cudaSuccess) e = tp_attr<ArithD, TileCfg<ArithD>, 10>();
  if (e == cudaSuccess) e = tp_attr<ArithD, TileCfg<ArithD>, 11>();
  if (e == cudaSuccess) e = tp_attr<ArithDF, TileCfg<ArithDF>, 9>();
  if (e == cudaSuccess) e = tp_attr<ArithDF, TileCfg<ArithDF>, 10>();
  if (e == cudaSuccess) e = tp_attr<ArithDF, TileCfg<ArithDF>, 11>();
  if (e == cudaSuccess) e = tp_attr<ArithF, TileCfg<ArithF>, 9>();
  if (e == cudaSuccess) e = tp_attr<ArithF, WideTileF, 10>();
  if (e == cudaSuccess) e = tp_attr<ArithF, WideTileF, 11>();
  return e;
}

}  // namespace bltt
