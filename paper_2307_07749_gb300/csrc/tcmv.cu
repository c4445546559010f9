// tcmv.cu - the time product of the BLTT matvec (Sec. 5.1: y = Y (T (x) I) x with T the lower
// triangular Toeplitz matrix of a, plus the b_0 (I (x) L) term) on the tcgen05 tensor cores.
//
// Arithmetic (fixed point with exact tensor-core sums).  Every operand is split into kTcDigits = 5
// balanced base-256 digits: x / 2^e = 2^-7 sum_p d_p 2^(-8p) + r with |d_p| <= 128 and
// |r| <= 2^-40, e a power-of-two bound of the spatial line of x (of all of a for the
// coefficients).  A digit times 2^(-8p) is exact in bf16, the product of two digits is exact in
// FP32, and a sum of up to 1024 products of leading digits stays within 2^24, so the FP32
// accumulation of the tensor core is exact for it.  Three accumulators keep the products apart
// by weight: digit pairs (i, j) of weight 2^-8(i+j) = 2^0 (exact), 2^-8 (exact to one bit) and
// 2^-16..2^-32 (rounded).  The fifteen pairs with i + j <= 4 are formed; the rest are left out.
// The error of an output element is then a few 2^-40 of max|a| sum_k |x_k| (fixed point: the
// digits of a small coefficient are as fine as those of the largest); the b_0 term, the scale by
// s and everything after the accumulators are double-float (FP64-accurate).
//
// Layout.  With the time flip Y, output time n = N-1-t and input time k meet through a'_{n+k}
// (a'_j = a_{N-1-j}, zero past N-1): a Hankel matrix.  As the tensor core's B operand (K-major,
// no swizzle) an 8x8 core matrix then depends only on the sum of its block indices, so the
// whole operand is 16 N/128 + 15 distinct core matrices per digit plane (92 KB for N = 1024),
// resident in shared memory and addressed by a descriptor whose two strides are both one core.
// The A operand is the digit planes of x for 128 spatial lines and 16 input times, written
// beforehand by k_tc_digits in the exact shared-memory image and brought in with one bulk copy
// per stage.  One work unit is 128 lines x 128 output times: M = 128, N = 128, K = 16 MMAs over
// the input times that reach it, fifteen digit pairs per K step, FP32 accumulators in TMEM.
//
// Roles (persistent blocks, one per SM): warp 0 issues the bulk copies, warp 1 owns TMEM and
// issues the MMAs, warps 2..17 read the accumulators (tcgen05.ld) and run the epilogue.  Every
// wait on an mbarrier is bounded (about one second); a block that gives up sets *tc_err,
// writes NaN partials, lets its copies and MMAs finish and frees its TMEM.
#include <atomic>
#include <cstdlib>
#include <math.h>
#include <stdint.h>
#include <string.h>
#include <vector>

#include "common.cuh"
#include "internal.h"
#include "opdev.cuh"

namespace bltt {
namespace {

constexpr int kRows = 128;                       // spatial lines per unit (MMA M)
constexpr int kCols = 128;                       // output times per unit (MMA N)
constexpr int kKs = 16;                          // input times per K step (MMA K)
constexpr int kStages = 6;
constexpr int kPlaneBytes = kRows * kKs * 2;     // one digit plane of one stage: 4 KB
constexpr int kStageBytes = kTcDigits * kPlaneBytes;
constexpr int kEpiWarps = 16;
constexpr int kThreadsMv = 32 * (2 + kEpiWarps);
constexpr int kGroup = 32;                       // strips whose units run together (L2 reuse)
constexpr long long kWaitCycles = 2000000000LL;  // about one second at the SM clock
constexpr int kMaxCores = 16 * 8 + 15;           // N <= 1024
constexpr int kHankBytesMax = kTcDigits * kMaxCores * 128;
constexpr int kSmemMv = kHankBytesMax + kStages * kStageBytes;

// instruction descriptor of tcgen05.mma kind::f16: D FP32 (bits 4-5 = 1), A and B bf16 (bits
// 7-9 and 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 at bit 17, M >> 4 at bit 24
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) |
                            ((uint32_t)(kCols >> 3) << 17) | ((uint32_t)(kRows >> 4) << 24);

// ------------------------------------------------------------------------------------------
// digits (host and device)

// balanced base-256 digits of F = round(x 2^(39-e)), |x| < 2^e: x = 2^(e-7) sum_p d[p] 2^(-8p)
// + r, |r| <= 2^(e-40), |d[p]| <= 128.  Zeros and subnormals give zero digits.
BLTT_HD void tc_split(double x, int e, int d[kTcDigits]) {
  static_assert(kTcDigits == 5, "the scale 2^(39-e) is for five digits");
  const uint64_t b = bits_d(x);
  const int E = (int)((b >> 52) & 0x7FF);
  int64_t F = 0;
  if (E != 0) {
    const uint64_t m = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
    const int sh = 1075 + e - 39 - E;            // >= 14 because E - 1023 < e
    if (sh < 64) F = (int64_t)((m + (1ull << (sh - 1))) >> sh);
    if (b >> 63) F = -F;
  }
  // two digits off the 64-bit value, the rest in 32 bits (|F| <= 2^39, <= 2^23 after two)
  const int d4 = (int)(((uint32_t)F + 128u) & 255u) - 128;
  F = (F - d4) >> 8;
  const int d3 = (int)(((uint32_t)F + 128u) & 255u) - 128;
  int32_t f = (int32_t)((F - d3) >> 8);
  const int d2 = ((f + 128) & 255) - 128;
  f = (f - d2) >> 8;
  const int d1 = ((f + 128) & 255) - 128;
  f = (f - d1) >> 8;
  d[0] = f;
  d[1] = d1;
  d[2] = d2;
  d[3] = d3;
  d[4] = d4;
}

// bf16 bit pattern of d 2^(-8p) (exact: |d| <= 128)
BLTT_HD uint32_t tc_bf16(int d, int p) { return bits_f(ldexpf((float)d, -8 * p)) >> 16; }

// exponent bound: smallest e with |x| < 2^e for the largest biased exponent E of a set
BLTT_HD int tc_exp_bound(int Emax) { return Emax == 0 ? 0 : Emax - 1022; }

// ------------------------------------------------------------------------------------------
// PTX wrappers (tcgen05, mbarrier, bulk copy)

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
// wait for the phase of the given parity to complete; false after `limit` SM cycles (about a
// second by default)
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity,
                                          long long limit = kWaitCycles) {
  const long long t0 = clock64();
  for (;;) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
    if (clock64() - t0 > limit) return false;
  }
}
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes,
                                         uint32_t bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
      "l"(src), "r"(bytes), "r"(bar)
      : "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void tc_after_sync() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_before_sync() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tmem_alloc(uint32_t dst_smem, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst_smem),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
               : "memory");
}
// shared-memory matrix descriptor, no swizzle: start, leading (K-direction core stride) and
// stride (M/N-direction core stride) byte offsets, fixed field 0b001 at bit 46
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}
__device__ __forceinline__ void mma_bf16(uint32_t d, uint64_t a, uint64_t b, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(kIdesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
               : "memory");
}
// 16 consecutive FP32 columns of this thread's TMEM lane; the wait is part of the statement so
// that no use of the registers can move above it
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,"
      "%15}, [%16];\n tcgen05.wait::ld.sync.aligned;\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// ------------------------------------------------------------------------------------------
// float -> double with a power-of-two scale, on the integer pipes

// f 2^k as a double (exact); k moves the exponent field, zero stays zero
__device__ __forceinline__ double f2d_shift(float f, int k) {
  const double d = f2d_bits(f);
  if (f == 0.0f) return d;
  return from_bits_d(bits_d(d) + ((uint64_t)(int64_t)k << 52));
}

// ------------------------------------------------------------------------------------------
// digit planes of s x (s = *xscale, 1 when null): block = 32 lines (a quarter strip) x all N
// times, 256 threads.  Pass 1 takes the largest exponent of each line of x, which with that of s
// bounds the line of s x (one bit loose at most); pass 2 writes the digits in the A-operand image:
// per (strip, K step, plane) 128 lines x 16 times, core matrix (line/8, time/8) at byte
// (line/8) 128 + (time/8) 2048, row line%8 at 16 bytes, time%8 at 2 bytes.
__global__ void __launch_bounds__(256) k_tc_digits(const double* __restrict__ x,
                                                   const double* __restrict__ xscale, int N,
                                                   long long M, uint16_t* __restrict__ xd,
                                                   int* __restrict__ xe, const int* phase) {
  if (skip_phase(phase, PH_RUN)) return;
  const double sc = xscale ? *xscale : 1.0;
  const int es = tc_exp_bound((int)((bits_d(sc) >> 52) & 0x7FF));   // |s| < 2^es
  __shared__ int s_e[8][32];
  const int c = threadIdx.x & 31, r0 = threadIdx.x >> 5;
  const long long j = (long long)blockIdx.x * 32 + c;
  const bool valid = j < M;
  int emax = 0;
  if (valid)
    for (int t = r0; t < N; t += 8) {
      const uint32_t hw = (uint32_t)(bits_d(__ldcg(x + (long long)t * M + j)) >> 32);
      emax = max(emax, (int)((hw >> 20) & 0x7FFu));
    }
  s_e[r0][c] = emax;
  __syncthreads();
  if (r0 == 0) {
    for (int r = 1; r < 8; ++r) emax = max(emax, s_e[r][c]);
    s_e[0][c] = emax;
    xe[j] = (emax == 0) ? 0 : tc_exp_bound(emax) + es;
  }
  __syncthreads();
  const int e = (s_e[0][c] == 0) ? 0 : tc_exp_bound(s_e[0][c]) + es;
  const long long strip = j >> 7;
  const int jj = (int)(j & 127);
  const int NKS = N / kKs;
  uint16_t* base = xd + (strip * NKS) * (long long)(kStageBytes / 2) + (jj >> 3) * 64 + (jj & 7) * 8;
  for (int kg = r0; kg < N / 8; kg += 8) {
    double v[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = valid ? sc * __ldcs(x + (long long)(8 * kg + i) * M + j) : 0.0;
    uint32_t w[kTcDigits][4];
#pragma unroll
    for (int i = 0; i < 8; i += 2) {
      int d0[kTcDigits], d1[kTcDigits];
      tc_split(v[i], e, d0);
      tc_split(v[i + 1], e, d1);
#pragma unroll
      for (int p = 0; p < kTcDigits; ++p) w[p][i >> 1] = tc_bf16(d0[p], p) | (tc_bf16(d1[p], p) << 16);
    }
    uint16_t* dst = base + (long long)(kg >> 1) * (kStageBytes / 2) + (kg & 1) * 1024;
#pragma unroll
    for (int p = 0; p < kTcDigits; ++p)
      *reinterpret_cast<uint4*>(dst + p * (kPlaneBytes / 2)) = make_uint4(w[p][0], w[p][1], w[p][2], w[p][3]);
  }
}

// ------------------------------------------------------------------------------------------
// the product kernel

struct MvParams {
  OpTables op;
  const double* x;
  const double* xscale;
  double* y;
  double* partials;
  const int* phase;
  int flip, spectral, nstrips, NB, nunits;
  // limit of the waits for progress (copies landed, MMAs done, accumulators read); the waits
  // that drain the block's own copies and MMAs before TMEM is freed keep kWaitCycles
  long long wait_cycles;
};

// unit u -> (strip, row block): groups of kGroup strips, row blocks in order inside a group
// (row block 0 has the most K steps), strips fastest
__device__ __forceinline__ void unit_of(int u, int nstrips, int NB, int& strip, int& rb) {
  const int g = u / (kGroup * NB);
  const int gsz = min(kGroup, nstrips - g * kGroup);
  const int r = u - g * kGroup * NB;
  rb = r / gsz;
  strip = g * kGroup + (r - rb * gsz);
}

// the fifteen digit pairs (i of a', j of x) with i + j <= 4, their accumulator and whether they
// open it (first product into the accumulator in a unit's first K step)
// (pairs in order of weight g = i + j, i rising inside a weight)
constexpr int kPairs = 15;
struct Pair {
  int i, j, acc, open;
};
__host__ __device__ constexpr Pair pair_of(int q) {
  const int g = q < 1 ? 0 : q < 3 ? 1 : q < 6 ? 2 : q < 10 ? 3 : 4;
  const int i = q - g * (g + 1) / 2;
  return Pair{i, g - i, g < 2 ? g : 2, (i == 0 && g <= 2) ? 1 : 0};
}

__global__ void __launch_bounds__(kThreadsMv, 1) k_tc_mv(const MvParams p) {
  if (skip_phase(p.phase, PH_RUN)) return;
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) uint64_t s_bar[2 * kStages + 3];
  __shared__ uint32_t s_tmem;
  __shared__ int s_err;
  __shared__ double s_red[32];
  const OpTables& op = p.op;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int N = op.N, NB = p.NB, NKS = N / kKs;
  const long long M = op.M;
  const int ncores = op.tc_ncores;
  const int hank_bytes = kTcDigits * ncores * 128;
  unsigned char* s_hank = smem;
  unsigned char* s_stage = smem + kHankBytesMax;

  // Hankel digit cores into shared memory (generic proxy; fenced for the tensor core below)
  {
    const uint4* src = reinterpret_cast<const uint4*>(op.tc_hank);
    uint4* dst = reinterpret_cast<uint4*>(s_hank);
    for (int i = threadIdx.x; i < hank_bytes / 16; i += blockDim.x) dst[i] = src[i];
  }
  const uint32_t bar0 = smem_u32(s_bar);
  auto full_bar = [&](int s) { return bar0 + 8u * s; };
  auto empty_bar = [&](int s) { return bar0 + 8u * (kStages + s); };
  const uint32_t tfull = bar0 + 8u * (2 * kStages), tempty = tfull + 8u, done_bar = tfull + 16u;
  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(full_bar(s), 1);
      mbar_init(empty_bar(s), 1);
    }
    mbar_init(tfull, 1);
    mbar_init(tempty, kEpiWarps);
    mbar_init(done_bar, 1);
    s_err = 0;
    fence_mbar_init();
  }
  __syncwarp();
  if (warp == 1) tmem_alloc(smem_u32(&s_tmem), 512);
  fence_proxy_async();
  tc_before_sync();
  __syncthreads();
  tc_after_sync();
  const uint32_t tmem = s_tmem;
  const uint32_t stage0 = smem_u32(s_stage), hank0 = smem_u32(s_hank);
  const unsigned char* xd = reinterpret_cast<const unsigned char*>(op.tc_xd);
  volatile int* err = &s_err;
  double dot = 0.0;

  if (warp == 0) {
    if (lane == 0) {
      // producer: one bulk copy (all digit planes of one K step) per stage
      uint32_t it = 0;
      for (int u = blockIdx.x; u < p.nunits && !*err; u += gridDim.x) {
        int strip, rb;
        unit_of(u, p.nstrips, NB, strip, rb);
        const int nks = 8 * (NB - rb);
        const unsigned char* src = xd + (size_t)strip * NKS * kStageBytes;
        for (int ks = 0; ks < nks; ++ks, ++it) {
          const int s = (int)(it % kStages);
          if (it >= (uint32_t)kStages &&
              !mbar_wait(empty_bar(s), ((it / kStages) & 1u) ^ 1u, p.wait_cycles)) {
            *err = 1;
            break;
          }
          mbar_expect_tx(full_bar(s), kStageBytes);
          bulk_g2s(stage0 + s * kStageBytes, src + (size_t)ks * kStageBytes, kStageBytes, full_bar(s));
        }
      }
      // the last copy into each stage has landed before the block may exit
      for (uint32_t q = (it > (uint32_t)kStages ? it - kStages : 0); q < it; ++q)
        if (!mbar_wait(full_bar((int)(q % kStages)), (q / kStages) & 1u)) *err = 1;
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // MMA issuer.  Descriptors are built once; a start address moves by adding its offset
      // (in 16-byte units) to the low field, which stays below 2^14 inside shared memory.
      const uint64_t adesc0 = sdesc(stage0, 2048, 128), bdesc0 = sdesc(hank0, 128, 128);
      uint64_t bplane[kTcDigits];
#pragma unroll
      for (int i = 0; i < kTcDigits; ++i) bplane[i] = (uint64_t)(i * ncores * 8);
      uint32_t it = 0, ui = 0;
      for (int u = blockIdx.x; u < p.nunits && !*err; u += gridDim.x, ++ui) {
        if (ui > 0 && !mbar_wait(tempty, (ui - 1) & 1u, p.wait_cycles)) { *err = 1; break; }
        tc_after_sync();
        int strip, rb;
        unit_of(u, p.nstrips, NB, strip, rb);
        const int nks = 8 * (NB - rb);
        bool ok = true;
        for (int ks = 0; ks < nks; ++ks, ++it) {
          const int s = (int)(it % kStages);
          if (!mbar_wait(full_bar(s), (it / kStages) & 1u, p.wait_cycles)) { ok = false; break; }
          tc_after_sync();
          const uint64_t ad = adesc0 + (uint64_t)(s * (kStageBytes / 16));
          const uint64_t bd = bdesc0 + (uint64_t)((16 * rb + 2 * ks) * 8);
          const uint32_t keep = ks > 0 ? 1u : 0u;
#pragma unroll
          for (int q = 0; q < kPairs; ++q) {
            const Pair pq = pair_of(q);
            mma_bf16(tmem + 128u * pq.acc, ad + (uint64_t)(pq.j * (kPlaneBytes / 16)),
                     bd + bplane[pq.i], pq.open ? keep : 1u);
          }
          mma_commit(empty_bar(s));
        }
        if (!ok) { *err = 1; break; }
        mma_commit(tfull);
      }
      // every MMA issued by this thread has completed before TMEM is freed
      mma_commit(done_bar);
      if (!mbar_wait(done_bar, 0)) *err = 1;
    }
  } else {
    // epilogue: warp w reads TMEM lanes 32 (w % 4) ..: line jj, 32 output times per warp.  The
    // three accumulators are folded into a double-float value per output and TMEM is released
    // at once, so that the next unit's MMAs run while this unit's outputs are finished.
    const int q = warp & 3, chunk = (warp - 2) >> 2;
    const int jj = 32 * q + lane;
    const double s = p.xscale ? *p.xscale : 1.0;
    uint32_t ui = 0;
    for (int u = blockIdx.x; u < p.nunits; u += gridDim.x, ++ui) {
      if (*err || !mbar_wait(tfull, ui & 1u, p.wait_cycles)) { *err = 1; break; }
      tc_after_sync();
      float hh[32], ll[32];
#pragma unroll
      for (int half = 0; half < 2; ++half) {
        const uint32_t ta = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(32 * chunk + 16 * half);
        float a0[16], a1[16], a2[16];
        __syncwarp();
        tmem_ld16(ta, a0);
        tmem_ld16(ta + 128u, a1);
        tmem_ld16(ta + 256u, a2);
#pragma unroll
        for (int cc = 0; cc < 16; ++cc) {
          // (h, l) = a0 + a1 + a2: two-sum of the exact parts, the rounded part folded in
          const float h = __fadd_rn(a0[cc], a1[cc]);
          const float bb = __fsub_rn(h, a0[cc]);
          const float l = __fadd_rn(__fsub_rn(a0[cc], __fsub_rn(h, bb)), __fsub_rn(a1[cc], bb));
          hh[16 * half + cc] = h;
          ll[16 * half + cc] = __fadd_rn(l, a2[cc]);
        }
      }
      tc_before_sync();
      __syncwarp();
      if (lane == 0) mbar_arrive(tempty);
      int strip, rb;
      unit_of(u, p.nstrips, NB, strip, rb);
      const long long j = (long long)strip * kRows + jj;
      if (j >= M) continue;
      const int kx = op.tc_eT + op.tc_xe[j] - 14;  // s x (T) x = accumulators x 2^kx
      const double c = p.spectral ? op.b0 * mode_mu(op, j) * s : op.b0 * s;
      const int n0 = kCols * rb + 32 * chunk;    // flipped time of the first Hankel row
      double dot_u = 0.0;
      // batches of four outputs: every load of a batch is issued before its first store
#pragma unroll
      for (int b0 = 0; b0 < 32; b0 += 4) {
        double xt[4], xs[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int n = n0 + b0 + i, t = N - 1 - n;
          const int srow = p.flip ? n : t;
          xt[i] = p.spectral ? __ldg(p.x + (long long)t * M + j) : 0.0;
          xs[i] = p.partials ? __ldg(p.x + (long long)srow * M + j) : 0.0;
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int n = n0 + b0 + i, t = N - 1 - n;
          const int srow = p.flip ? n : t;
          // time product in FP64 (exact sum of the two parts), then the b_0 term
          const double tp = f2d_shift(hh[b0 + i], kx) + f2d_shift(ll[b0 + i], kx);
          const double lx = p.spectral ? xt[i] : stencil_at(op, p.x + (long long)t * M, j);
          const double val = fma(c, lx, tp);
          p.y[(long long)srow * M + j] = val;
          dot_u = fma(val, xs[i], dot_u);
        }
      }
      dot += dot_u;
    }
  }
  __syncthreads();
  if (p.partials) {
    const double sum = block_sum<kThreadsMv>(dot, s_red);
    if (threadIdx.x == 0) {
      const double s = p.xscale ? *p.xscale : 1.0;
      p.partials[blockIdx.x] = *err ? __longlong_as_double(0x7FF8000000000000LL) : sum * s;
    }
  }
  if (threadIdx.x == 0 && *err) atomicExch(op.tc_err, 1);
  if (warp == 1) {
    __syncwarp();
    tc_after_sync();
    tmem_dealloc(tmem, 512);
  }
}

// SM count of each device on which k_tc_mv's shared-memory attribute has been set (0: not yet);
// cudaFuncSetAttribute acts on the current device only
constexpr int kTcMaxDevices = 64;
std::atomic<int> g_num_sms[kTcMaxDevices];

}  // namespace

// ------------------------------------------------------------------------------------------
// host side

bool tc_eligible(const OpTables& op) {
  return op.ntaps == 0 && op.b_kind == 0 && op.N >= 128 && op.N <= 1024 &&
         (op.N & (op.N - 1)) == 0;
}

int tc_strips(long long M) { return (int)((M + kRows - 1) / kRows); }

size_t tc_workspace_bytes(int N, long long M) {
  return (size_t)tc_strips(M) * (N / kKs) * kStageBytes;
}

void tc_hankel_digits(const double* a, int N, uint16_t* out, int* eT, int* ncores) {
  const int nc = 16 * (N / kCols) + 15;
  int Emax = 0;
  for (int k = 0; k < N; ++k) {
    const int E = (int)((bits_d(a[k]) >> 52) & 0x7FF);
    Emax = E > Emax ? E : Emax;
  }
  const int e = tc_exp_bound(Emax);
  for (int c = 0; c < nc; ++c)
    for (int r = 0; r < 8; ++r)
      for (int q = 0; q < 8; ++q) {
        const int jn = 8 * c + r + q;                 // a'_{jn} = a_{N-1-jn}, zero past N-1
        const double v = (jn <= N - 1) ? a[N - 1 - jn] : 0.0;
        int d[kTcDigits];
        tc_split(v, e, d);
        for (int p = 0; p < kTcDigits; ++p)
          out[((size_t)p * nc + c) * 64 + r * 8 + q] = (uint16_t)tc_bf16(d[p], p);
      }
  *eT = e;
  *ncores = nc;
}

cudaError_t launch_tc_digits(const OpTables& op, const double* x, const double* xscale,
                             const int* phase, cudaStream_t st) {
  if (!tc_eligible(op) || !op.tc_xd || !op.tc_xe) return cudaErrorInvalidValue;
  const int nstrips = tc_strips(op.M);
  k_tc_digits<<<(unsigned)(nstrips * (kRows / 32)), 256, 0, st>>>(x, xscale, op.N, op.M,
                                                                    op.tc_xd, op.tc_xe, phase);
  return cudaGetLastError();
}

cudaError_t launch_tc_product(const OpTables& op, int spectral, const double* x,
                              const double* xscale, double* y, int flip, double* partials,
                              int* nparts, const int* phase, cudaStream_t st) {
  if (!tc_eligible(op) || !op.tc_hank || !op.tc_xd || !op.tc_xe || !op.tc_err)
    return cudaErrorInvalidValue;
  int dev = 0;
  cudaError_t ed = cudaGetDevice(&dev);
  if (ed != cudaSuccess) return ed;
  if (dev < 0 || dev >= kTcMaxDevices) return cudaErrorInvalidDevice;
  int num_sms = g_num_sms[dev].load(std::memory_order_acquire);
  if (num_sms == 0) {
    int n = 0;
    cudaError_t e = cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_tc_mv, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemMv);
    if (e != cudaSuccess) return e;
    g_num_sms[dev].store(n, std::memory_order_release);
    num_sms = n;
  }
  const int nstrips = tc_strips(op.M);
  MvParams prm;
  prm.op = op;
  prm.x = x;
  prm.xscale = xscale;
  prm.y = y;
  prm.partials = partials;
  prm.phase = phase;
  prm.flip = flip;
  prm.spectral = spectral;
  prm.nstrips = nstrips;
  // BLTT_TC_WAIT_CYCLES (environment, SM cycles >= 0) shortens the progress waits, so that a
  // test can make them give up; the default is about a second
  prm.wait_cycles = kWaitCycles;
  if (const char* w = std::getenv("BLTT_TC_WAIT_CYCLES")) {
    char* end = nullptr;
    const long long v = std::strtoll(w, &end, 10);
    if (end != w && v >= 0 && v < kWaitCycles) prm.wait_cycles = v;
  }
  prm.NB = op.N / kCols;
  prm.nunits = nstrips * prm.NB;
  const int grid = prm.nunits < num_sms ? prm.nunits : num_sms;
  if (nparts) *nparts = grid;
  k_tc_mv<<<grid, kThreadsMv, kSmemMv, st>>>(prm);
  return cudaGetLastError();
}

cudaError_t launch_tc_matvec(const OpTables& op, int spectral, const double* x,
                             const double* xscale, double* y, int flip, double* partials,
                             int* nparts, const int* phase, cudaStream_t st) {
  cudaError_t e = launch_tc_digits(op, x, xscale, phase, st);
  if (e != cudaSuccess) return e;
  return launch_tc_product(op, spectral, x, xscale, y, flip, partials, nparts, phase, st);
}

}  // namespace bltt
