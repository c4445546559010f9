// spec.h - launches of the compile-time-sized tile kernels (spec_conv.cu, spec_tp.cu,
// spec_dst.cu).  For the common transform lengths the FFT tile kernels are also compiled with the
// length and the tile's column count as constants: their passes unroll, their shared-memory
// addresses fold into immediate offsets and their divisions become multiplications, which cuts
// the integer and uniform-pipe instructions of the double-float matvec by about a third.
//
// Each spec_* call launches such a kernel when one exists for the given sizes (a full-width tile:
// log2NC the largest the tile allows) and returns true with *err the launch status; otherwise it
// launches nothing and returns false, and the caller runs the run-time-sized kernel.
#pragma once
#include <cuda_runtime.h>
#include "internal.h"

namespace bltt {

// lengths with compile-time-sized kernels: N = 2^9 .. 2^11 for the matvec and the time pass,
// P = m + 1 = 2^7, 2^8 for the DST
constexpr int kSpecLog2NMin = 9, kSpecLog2NMax = 11;
constexpr int kSpecLog2PMin = 7, kSpecLog2PMax = 8;

// k_conv: prec PREC_F64 (FP64) or PREC_DF (double-float)
bool spec_conv(int prec, int log2N, int log2NC, unsigned grid, size_t smem, cudaStream_t st,
               const OpTables& op, int spectral, int which, const double* x, const double* xscale,
               double* y, int flip, int mode, const double* rhs, double* partials,
               const int* phase, int want, const double* st_src, cudaError_t* err);

// k_timepass: prec PREC_F64, PREC_DF or PREC_F32 (wide: the 8192-point FP32 tile); tw is the
// length-N twiddle table in the arithmetic of prec
bool spec_timepass(int prec, bool wide, int log2N, int log2NC, unsigned grid, size_t smem,
                   cudaStream_t st, const OpTables& op, const PrecTables& pt, const Combine& cb,
                   double* out, const double* dot_with, double* partials, const int* phase,
                   int want, const void* tw, cudaError_t* err);

// k_dst: contiguous lines (inner == 1) or strided ones; tw is the length-2P twiddle table
bool spec_dst(int prec, bool contiguous, int log2P, int log2NC, unsigned grid, size_t smem,
              cudaStream_t st, long long nlines, int m, long long inner, const Combine& cb,
              double* out, int flip, int N, long long M, const double* dot_with,
              double* partials, const void* tw, const int* phase, int want, cudaError_t* err);

// shared-memory limits of the compile-time-sized kernels on the current device
cudaError_t spec_prepare_conv_attributes();
cudaError_t spec_prepare_tp_attributes();
cudaError_t spec_prepare_dst_attributes();

}  // namespace bltt
