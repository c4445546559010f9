// tiles.cuh - the FFT tile bodies of libbltt and their kernels: DST-I along a spatial axis,
// the alpha-scaled time pass of the ABAC preconditioner and the BLTT matvec by the 2N circulant
// embedding.  Included by the translation units that instantiate them: kernels.cu (the
// run-time-sized kernels and the multi-item ones) and the compile-time-sized ones (spec_*.cu).
#pragma once
#include <type_traits>
#include "common.cuh"
#include "internal.h"
#include "opdev.cuh"

namespace bltt {

// ============================================================================================
// helpers
__device__ __forceinline__ void load_coef(const Combine& cb, double& c0, double& c1, double& c2) {
  c0 = 1.0;
  if (cb.coef) { c1 = cb.coef[1]; c2 = cb.coef[2]; }
  else { c1 = 0.0; c2 = 0.0; }
}

// v = in0[e] + c1 in1[e] + c2 in2[e] (FP64); optionally stored to vout[e] (vout may alias
// in1/in2: the same thread reads before it writes).  The vector loads bypass L1 (which keeps the
// tables: twiddles, spectra, row scales); when v is stored, the inputs are streamed (evict-first)
// so that v itself is more likely to stay in L2 for the dot product at the end of the tile.
__device__ __forceinline__ double combine_at(const Combine& cb, long long e, double, double c1,
                                             double c2) {
  if (!cb.vout) {
    double v = __ldcg(cb.in0 + e);
    if (cb.in1) v = fma(c1, __ldcg(cb.in1 + e), v);
    if (cb.in2) v = fma(c2, __ldcg(cb.in2 + e), v);
    return v;
  }
  double v = __ldcs(cb.in0 + e);
  if (cb.in1) v = fma(c1, __ldcs(cb.in1 + e), v);
  if (cb.in2) v = fma(c2, __ldcs(cb.in2 + e), v);
  cb.vout[e] = v;
  return v;
}

// principal (x + i y)^{-1/2} for x > 0, by the half-angle form of the square root:
// sqrt(z) = s + i y/(2s), s = sqrt((|z| + x)/2), and 1/sqrt(z) = conj(sqrt(z)) / |z|.
template <typename T>
__device__ __forceinline__ C<T> inv_sqrt_principal(T x, T y) {
  T r = hypot(x, y);
  T s = sqrt(T(0.5) * (r + x));
  T t = y / (T(2) * s);
  T ir = T(1) / r;
  return mk<T>(s * ir, -t * ir);
}

// the same in FP32 with the hardware reciprocal square root (a few ulp): |z|^2 = x^2 + y^2 must
// stay inside the normal FP32 range, else the accurate form above is taken
__device__ __forceinline__ float2 inv_sqrt_principal_fast(float x, float y) {
  const float rr = fmaf(x, x, y * y);
  if (!(rr > 1e-36f && rr < 1e36f)) return inv_sqrt_principal<float>(x, y);
  const float ir = rsqrtf(rr);        // 1/|z|
  const float h = 0.5f * fmaf(rr, ir, x);   // s^2 = (|z| + x)/2
  const float is = rsqrtf(h);         // 1/s
  const float t = 0.5f * y * is;      // y/(2s)
  return make_float2(h * is * ir, -t * ir);
}

// e / m for 0 <= e < 2^22 without an integer division (float reciprocal, one correction step)
__device__ __forceinline__ int fast_div(int e, int m, float inv_m) {
  int c = __float2int_rz((float)e * inv_m);
  int r = e - c * m;
  if (r < 0) --c;
  else if (r >= m) ++c;
  return c;
}

constexpr int kBatch = 8;   // independent global loads in flight per thread in the tile loaders

// threads per tile block and complex points per tile, per arithmetic: 256 threads and 4096 points
// (32 KB of FP32, 64 KB of FP64 / double-float shared memory) let two to four independent blocks
// share an SM, so that one block's loads, stores and barriers overlap another block's arithmetic
template <class A> struct TileCfg {
  static constexpr int NT = kThreads, CAP = kCap;
  // resident blocks per SM the register budget is held to: 128 registers per thread for FP64, 64
  // for FP32
  static constexpr int MINB = sizeof(typename A::V) == 8 ? 4 : 2;
};
// double-float: 512 threads on the 4096 points (8 per thread, radix-8 passes) at 64 registers,
// two blocks per SM: twice the warps of the FP64 tile and about a third of its transform code
template <> struct TileCfg<ArithDF> {
  static constexpr int NT = 2 * kThreads, CAP = kCap;
  static constexpr int MINB = 2;
};
// a wide FP32 tile for the single-item time pass at long N: 8192 points and 512 threads (16 points
// each, two blocks per SM), so that a tile spans twice the lines and every row of a vector is read
// and written in runs twice as long (at N = 1024: 16 lines, 128 B, against 8 lines, 64 B)
struct WideTileF {
  static constexpr int NT = 2 * kThreads, CAP = 2 * kCap;
  static constexpr int MINB = 2;
};

// ============================================================================================
// DST-I along one spatial axis (Steps 1 and 3 of Sec. 5.1), by one real FFT of length P = m+1 per
// line.  With S_k = sum_{j=1}^{m} x_j sin(pi j k/P), y_j = sin(pi j/P)(x_j + x_{P-j}) +
// (x_j - x_{P-j})/2 (x_0 = x_P = 0) and Y = FFT_P(y):
//   S_{2k} = -Im Y_k,   S_{2k+1} - S_{2k-1} = Re Y_k   (S_{-1} = -S_1, so S_1 = Re Y_0 / 2),
// because sin(a+b) - sin(a-b) = 2 cos(a) sin(b), and in each sum over j the part that is odd under
// j -> P-j cancels.  The orthonormal DST-I is sqrt(2/P) S.  Two lines share one complex FFT of
// x_a + i x_b: R_k = (F_k + F_{P-k})/2 carries (Re Ya_k, Re Yb_k) and E_k = i (F_k - F_{P-k})/2
// carries (-Im Ya_k, -Im Yb_k); the odd outputs are prefix sums of R along k, per column, taken
// in shared memory.  The FFT reads the length-2P twiddle table at stride 2, and sin(pi j/P) is
// -Im w_{2P}^j from the same table.
// Lines: line g has elements base(g) + p*inner, base(g) = (g/inner)*(m*inner) + g%inner.
// LOG2P > 0: a full-width tile for P = 2^LOG2P, with P, m and the column count compile-time
// constants (the FFT passes unroll, the divisions by m become multiplications); LOG2P = 0 takes
// them from the arguments
template <class A, bool SWZ, int LOG2P = 0>
__device__ __forceinline__ void dst_tile(long long nlines, int m_rt, long long inner, int P_rt,
                                         int log2P_rt, int log2NC_rt, const Combine& cb,
                                         double* out, int flip, int N, long long M,
                                         const double* dot_with, double* partials,
                                         const typename A::V* __restrict__ tw, long long tile) {
  constexpr int NT = TileCfg<A>::NT, CAP = TileCfg<A>::CAP;
  static_assert(LOG2P == 0 || (1 << LOG2P) <= CAP, "the transform must fit one tile");
  const int log2P = LOG2P ? LOG2P : log2P_rt;
  const int P = LOG2P ? (1 << LOG2P) : P_rt;
  const int m = LOG2P ? P - 1 : m_rt;
  const int log2NC = LOG2P ? ilog2c(CAP) - LOG2P : log2NC_rt;
  constexpr int CH = 8;                           // rows per prefix-sum chunk
  constexpr int IPT = (CAP / 2 + NT - 1) / NT;    // (k, column) items per thread, k < P/2
  using V = typename A::V;
  using Sc = typename A::Sc;
  __syncthreads();   // the previous tile of a persistent block may still read shared memory
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* buf = reinterpret_cast<V*>(smem_raw);
  __shared__ double red[32];
  __shared__ long long s_in[kMaxCols], s_out[kMaxCols];
  __shared__ V s_tot[NT];                         // prefix-sum chunk totals
  const int NC = 1 << log2NC, W = 2 * NC, half = P >> 1;
  const long long g0 = tile * W;
  for (int c = threadIdx.x; c < W; c += NT) {
    long long g = g0 + c;
    long long b = -1, o = -1;
    if (g < nlines) {
      b = (g / inner) * ((long long)m * inner) + (g % inner);
      o = b;
      if (flip) o += (long long)(N - 1 - 2 * (b / M)) * M;
    }
    s_in[c] = b;
    s_out[c] = o;
  }
  const int cmask = NC - 1;
  auto at = [&](int p, int cc) { return p * NC + (SWZ ? (cc ^ (p & cmask)) : cc); };
  for (int cc = threadIdx.x; cc < NC; cc += NT) buf[at(0, cc)] = A::zero();   // x_0 = 0
  __syncthreads();
  double c0, c1, c2;
  load_coef(cb, c0, c1, c2);
  const bool contiguous = (inner == 1);
  const float inv_m = 1.0f / (float)m;
  // e / m: a multiply-high by a constant where m is one, else the float-reciprocal division
  auto divm = [&](int e) { return LOG2P ? (int)((unsigned)e / (unsigned)m) : fast_div(e, m, inv_m); };
  const int total = m * W, log2W = log2NC + 1;
  // x_j (j = p + 1) of line c into row j, column c/2, component c%2
  for (int e0 = threadIdx.x; e0 < total; e0 += kBatch * NT) {
    double v[kBatch];
    int cs[kBatch], ps[kBatch];
#pragma unroll
    for (int u = 0; u < kBatch; ++u) {
      const int e = e0 + u * NT;
      int c = 0, p = 0;
      if (contiguous) { c = divm(e); p = e - c * m; }
      else { p = e >> log2W; c = e & (W - 1); }
      cs[u] = c; ps[u] = p;
      v[u] = 0.0;
      if (e < total) {
        const long long b = s_in[c];
        if (b >= 0) v[u] = combine_at(cb, b + (long long)p * inner, c0, c1, c2);
      }
    }
#pragma unroll
    for (int u = 0; u < kBatch; ++u) {
      const int e = e0 + u * NT;
      if (e < total) A::put(buf, at(ps[u] + 1, cs[u] >> 1), cs[u] & 1, v[u]);
    }
  }
  __syncthreads();
  // y_j and y_{P-j} from x_j and x_{P-j}, in place (each item owns both rows)
  const Sc halfsc = A::make_sc(0.5);
  for (int it = threadIdx.x; it < (half << log2NC); it += NT) {
    const int cc = it & cmask, j = 1 + (it >> log2NC), jm = P - j;
    const V xa = buf[at(j, cc)], xb = buf[at(jm, cc)];
    const V sm = A::scale_sc(A::add(xa, xb), A::neg_imag_sc(tw[j]));   // sin(pi j/P) (x_j + x_{P-j})
    const V df = A::scale_sc(A::sub(xa, xb), halfsc);
    buf[at(j, cc)] = A::add(sm, df);
    if (jm != j) buf[at(jm, cc)] = A::sub(sm, df);
  }
  __syncthreads();
  fft_columns<A, NT, CAP, false, SWZ>(buf, P, log2P, log2NC, tw, false, 1);   // w_P = w_{2P}^2
  // R_k into rows k < P/2 (R_0 = F_0/2: the halved first term of the odd outputs), E_k into
  // rows P/2 + k; all reads before the barrier, all writes after
  {
    V rr[IPT], ee[IPT];
#pragma unroll
    for (int s = 0; s < IPT; ++s) {
      const int it = threadIdx.x + s * NT;
      if (it < (half << log2NC)) {
        const int cc = it & cmask, k = it >> log2NC;
        const V fk = buf[at(k, cc)], fm = buf[at((P - k) & (P - 1), cc)];
        rr[s] = A::scale_sc(k == 0 ? fk : A::add(fk, fm), halfsc);
        ee[s] = A::template rot<true>(A::scale_sc(A::sub(fk, fm), halfsc));
      }
    }
    __syncthreads();
#pragma unroll
    for (int s = 0; s < IPT; ++s) {
      const int it = threadIdx.x + s * NT;
      if (it < (half << log2NC)) {
        const int cc = it & cmask, k = it >> log2NC;
        buf[at(k, cc)] = rr[s];
        buf[at(half + k, cc)] = ee[s];
      }
    }
  }
  __syncthreads();
  // inclusive prefix sums of R along k in every column: chunks of ch rows (one per thread), the
  // chunk totals scanned per column in order, then added back
  const int ch = half < CH ? half : CH;
  const int cpc = half / ch;                      // chunks per column
  const int nchunks = cpc << log2NC;              // <= NT: P NC <= CAP
  const int t = threadIdx.x;
  const int tcc = t & cmask, tq = t >> log2NC;
  if (t < nchunks) {
    V run = A::zero();
    for (int i = 0; i < ch; ++i) {
      const int k = tq * ch + i;
      run = A::add(run, buf[at(k, tcc)]);
      buf[at(k, tcc)] = run;
    }
    s_tot[t] = run;
  }
  __syncthreads();
  if (t < NC) {
    V off = A::zero();
    for (int q = 0; q < cpc; ++q) {
      const int idx = (q << log2NC) + t;
      const V tv = s_tot[idx];
      s_tot[idx] = off;
      off = A::add(off, tv);
    }
  }
  __syncthreads();
  if (t < nchunks && tq > 0) {
    const V off = s_tot[t];
    for (int i = 0; i < ch; ++i) {
      const int k = tq * ch + i;
      buf[at(k, tcc)] = A::add(buf[at(k, tcc)], off);
    }
  }
  __syncthreads();
  // sqrt(2/P) for P = 2^log2P: a power of two (log2P odd) or sqrt(2) times one, without the
  // FP64 square root and division every thread would otherwise run
  const Sc scale = A::make_sc((log2P & 1) ? ldexp(1.0, (1 - log2P) / 2)
                                          : ldexp(1.4142135623730951, -(log2P / 2)));
  // read-out in batches: the global loads of a batch (the dot-product partner) are all issued
  // before the first use, so that their latencies overlap.  dot_with == out asks for ||out||^2.
  // Output j = p + 1: S_j from row j/2 (j odd: the prefix sums) or row P/2 + j/2 (j even).
  const bool self_dot = (dot_with == out);
  const double* dwsrc = self_dot ? nullptr : dot_with;
  double acc = 0.0;
  for (int e0 = threadIdx.x; e0 < total; e0 += kBatch * NT) {
    double dw[kBatch];
    long long ix[kBatch];
    int cs[kBatch], ks[kBatch];
#pragma unroll
    for (int u = 0; u < kBatch; ++u) {
      const int e = e0 + u * NT;
      int c = 0, k = 0;
      if (contiguous) { c = divm(e); k = e - c * m; }
      else { k = e >> log2W; c = e & (W - 1); }
      cs[u] = c; ks[u] = k;
      ix[u] = -1;
      dw[u] = 0.0;
      if (e < total) {
        const long long o = s_out[c];
        if (o >= 0) {
          ix[u] = o + (long long)k * inner;
          if (dwsrc) dw[u] = __ldcs(dwsrc + ix[u]);
        }
      }
    }
#pragma unroll
    for (int u = 0; u < kBatch; ++u) {
      if (ix[u] >= 0) {
        const int c = cs[u], j = ks[u] + 1;
        const V z = buf[at((j & 1) ? (j >> 1) : half + (j >> 1), c >> 1)];
        const double val = A::part_sc(z, c & 1, scale);
        out[ix[u]] = val;
        if (partials) acc = fma(val, self_dot ? val : dw[u], acc);   // FP64 pipe: only if asked
      }
    }
  }
  if (partials) {
    double s = block_sum<NT>(acc, red);
    if (threadIdx.x == 0) partials[tile] = s;
  }
}

template <class A, bool SWZ, int LOG2P = 0>
__global__ void __launch_bounds__(TileCfg<A>::NT, TileCfg<A>::MINB)
k_dst(long long nlines, int m, long long inner, int P, int log2P, int log2NC, Combine cb,
      double* out, int flip, int N, long long M, const double* dot_with, double* partials,
      const typename A::V* __restrict__ tw, const int* phase, int want) {
  if (skip_phase(phase, want)) return;
  dst_tile<A, SWZ, LOG2P>(nlines, m, inner, P, log2P, log2NC, cb, out, flip, N, M, dot_with,
                          partials, tw, blockIdx.x);
}

// ============================================================================================
// Time pass of P_alpha^{-1} for a tile of 2*NC spatial modes (Step 2 and its second half,
// Sec. 5.1): per mode, s1 = v/d, s2 = F conj(Lambda)^{-1/2} F^* s1, s3 = d^2 s2,
// s4 = F Lambda^{-1/2} F^* s3, z = s4/d.  Two real modes share one complex FFT of length N; the
// per-mode spectra are split and re-merged in the frequency domain (Lemma 3.1 makes each mode's
// spectrum conjugate-symmetric, so both inverse transforms are real).

// per-row scale factors (1/d_j and d_j^2) in the arithmetic of the kernel
template <class A> struct RowSc;
template <> struct RowSc<ArithD> {
  static __device__ __forceinline__ double dinv(const PrecTables& pt, int p) { return pt.dinv[p]; }
  static __device__ __forceinline__ double d2(const PrecTables& pt, int p) { return pt.d2[p]; }
};
template <> struct RowSc<ArithF> {
  static __device__ __forceinline__ float dinv(const PrecTables& pt, int p) { return pt.dinv32[p]; }
  static __device__ __forceinline__ float d2(const PrecTables& pt, int p) { return pt.d232[p]; }
};
template <> struct RowSc<ArithDF> {
  static __device__ __forceinline__ dfl dinv(const PrecTables& pt, int p) { return ArithDF::row_sc(pt.dinv_df, p); }
  static __device__ __forceinline__ dfl d2(const PrecTables& pt, int p) { return ArithDF::row_sc(pt.d2_df, p); }
};

// G for mode i at frequency k: lambda^{-1/2}/(2N), lambda = ahat_k + bhat_k mu_i.  FP64 and
// double-float read the per-(frequency, mode) table built at set-up; FP32 evaluates it where it is
// used, from the N/2+1 entries of ahat and bhat (two reciprocal square roots), which spares a
// table's 8 bytes per unknown of DRAM reads and their latency
template <class A> struct GSrc;
template <> struct GSrc<ArithDF> {
  static __device__ __forceinline__ float4 get(const OpTables& op, const PrecTables& pt, int k,
                                              long long i, float) {
    return pt.gdf[(long long)k * op.M + i];
  }
};
template <> struct GSrc<ArithD> {
  static __device__ __forceinline__ double2 get(const OpTables& op, const PrecTables& pt, int k,
                                               long long i, float) {
    return pt.g64[(long long)k * op.M + i];
  }
};
template <> struct GSrc<ArithF> {
  static __device__ __forceinline__ float2 get(const OpTables& op, const PrecTables& pt, int k,
                                              long long i, float mu32) {
    if (pt.g32) return pt.g32[(long long)k * op.M + i];   // general commuting blocks
    const float2 a = pt.ahat32[k], b = pt.bhat32[k];
    const float2 g = inv_sqrt_principal_fast(fmaf(b.x, mu32, a.x), fmaf(b.y, mu32, a.y));
    const float sc = 0.5f / (float)op.N;
    return make_float2(g.x * sc, g.y * sc);
  }
};

template <class A, bool CONJ, class Cfg>
__device__ __forceinline__ void tp_freq_mul(typename A::V* buf, const OpTables& op,
                                            const PrecTables& pt, int N, int log2NC, long long g0,
                                            const float* s_mu) {
  constexpr int NT = Cfg::NT;
  using V = typename A::V;
  const int half = N >> 1, NC = 1 << log2NC;
  const int items = (half + 1) << log2NC;
  for (int it = threadIdx.x; it < items; it += NT) {
    const int cc = it & (NC - 1), k = it >> log2NC;
    const long long ia = g0 + 2 * cc, ib = ia + 1;
    V Ga = A::zero(), Gb = A::zero();
    if (ia < op.M) Ga = GSrc<A>::get(op, pt, k, ia, s_mu[2 * cc]);
    if (ib < op.M) Gb = GSrc<A>::get(op, pt, k, ib, s_mu[2 * cc + 1]);
    if (CONJ) { Ga = A::conj(Ga); Gb = A::conj(Gb); }
    const int kb = (N - k) & (N - 1);
    const V Av = buf[k * NC + cc], Bc = A::conj(buf[kb * NC + cc]);
    const V U1 = A::mul(Ga, A::add(Av, Bc));
    const V U2 = A::mul(Gb, A::sub(Av, Bc));
    buf[k * NC + cc] = A::add(U1, U2);
    if (kb != k) buf[kb * NC + cc] = A::conj(A::sub(U1, U2));
  }
}

// LOG2N > 0: a full-width tile for N = 2^LOG2N with the transform length and column count
// compile-time constants (as in conv_tile); LOG2N = 0 takes them from op.log2N and log2NC_rt
template <class A, class Cfg = TileCfg<A>, bool TWS = false, int LOG2N = 0>
__device__ __forceinline__ void timepass_tile(const OpTables& op, const PrecTables& pt,
                                              const Combine& cb, double* out,
                                              const double* dot_with, double* partials,
                                              int log2NC_rt, const typename A::V* __restrict__ tw,
                                              long long tile) {
  constexpr int NT = Cfg::NT, CAP = Cfg::CAP;
  static_assert(LOG2N == 0 || (1 << LOG2N) <= CAP, "the transform must fit one tile");
  const int log2N = LOG2N ? LOG2N : op.log2N;
  const int log2NC = LOG2N ? ilog2c(CAP) - LOG2N : log2NC_rt;
  using V = typename A::V;
  __syncthreads();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* buf = reinterpret_cast<V*>(smem_raw);
  __shared__ double red[32];
  __shared__ float s_mu[kMaxCols];   // FP32 mode eigenvalues, used by the FP32 G
  // TWS (FP32): the length-N twiddles, the N/2+1 entries of ahat and bhat and the N row scalings
  // D^{-1} and D^2 staged in shared memory behind the tile, so that the FFT passes, the spectral
  // products and the scalings read them with shared-memory latency instead of through L1
  const V* twp = tw;
  PrecTables pts = pt;
  if constexpr (TWS) {
    const int n = 1 << log2N, nh = n / 2 + 1;
    V* tws = buf + CAP;
    float2* sa = reinterpret_cast<float2*>(tws + n);
    float2* sb = sa + nh;
    float* sdi = reinterpret_cast<float*>(sb + nh);
    float* sd2 = sdi + n;
    for (int i = threadIdx.x; i < n; i += NT) {
      tws[i] = tw[i];
      sdi[i] = pt.dinv32[i];
      sd2[i] = pt.d232[i];
    }
    for (int i = threadIdx.x; i < nh; i += NT) {
      sa[i] = pt.ahat32[i];
      sb[i] = pt.bhat32[i];
    }
    twp = tws;
    pts.ahat32 = sa;
    pts.bhat32 = sb;
    pts.dinv32 = sdi;
    pts.d232 = sd2;
    // the load loop below reads the staged row scalings written by other threads
    __syncthreads();
  }
  const int N = 1 << log2N, NC = 1 << log2NC, W = 2 * NC, log2W = log2NC + 1;
  const long long M = op.M;
  const long long g0 = tile * W;
  if (std::is_same<A, ArithF>::value)
    for (int c = threadIdx.x; c < W; c += NT) s_mu[c] = (g0 + c < M) ? mode_mu32(op, g0 + c) : 0.f;
  double c0, c1, c2;
  load_coef(cb, c0, c1, c2);
  const int total = N * W;
  // the Lanczos combine v = in0 + c1 in1 + c2 in2 (stored to vout) for a batch of elements: all
  // loads of the batch first, then the combines and stores (vout may alias in1 or in2, element by
  // element, so the compiler could not move one element's loads above another's store)
  constexpr int kCB = 4;   // elements per batch: 12 loads in flight per thread
  for (int e0 = threadIdx.x; e0 < total; e0 += kCB * NT) {
    double v[kCB], a1[kCB], a2[kCB];
#pragma unroll
    for (int u = 0; u < kCB; ++u) {
      const int e = e0 + u * NT;
      const int p = e >> log2W, c = e & (W - 1);
      v[u] = 0.0; a1[u] = 0.0; a2[u] = 0.0;
      if (e < total && g0 + c < M) {
        const long long idx = (long long)p * M + g0 + c;
        if (cb.vout) {
          v[u] = __ldcs(cb.in0 + idx);
          if (cb.in1) a1[u] = __ldcs(cb.in1 + idx);
          if (cb.in2) a2[u] = __ldcs(cb.in2 + idx);
        } else {
          v[u] = __ldcg(cb.in0 + idx);
          if (cb.in1) a1[u] = __ldcg(cb.in1 + idx);
          if (cb.in2) a2[u] = __ldcg(cb.in2 + idx);
        }
      }
    }
#pragma unroll
    for (int u = 0; u < kCB; ++u) {
      const int e = e0 + u * NT;
      if (e < total) {
        const int p = e >> log2W, c = e & (W - 1);
        if (cb.in1) v[u] = fma(c1, a1[u], v[u]);
        if (cb.in2) v[u] = fma(c2, a2[u], v[u]);
        if (cb.vout && g0 + c < M) cb.vout[(long long)p * M + g0 + c] = v[u];
        A::put_sc(buf, p * NC + (c >> 1), c & 1, v[u], RowSc<A>::dinv(pts, p));
      }
    }
  }
  __syncthreads();
  fft_columns<A, NT, CAP, false>(buf, N, log2N, log2NC, twp);
  tp_freq_mul<A, true, Cfg>(buf, op, pts, N, log2NC, g0, s_mu);
  __syncthreads();
  fft_columns<A, NT, CAP, true>(buf, N, log2N, log2NC, twp);
  for (int e = threadIdx.x; e < N * NC; e += NT)
    buf[e] = A::scale_sc(buf[e], RowSc<A>::d2(pts, e >> log2NC));
  __syncthreads();
  fft_columns<A, NT, CAP, false>(buf, N, log2N, log2NC, twp);
  tp_freq_mul<A, false, Cfg>(buf, op, pts, N, log2NC, g0, s_mu);
  __syncthreads();
  fft_columns<A, NT, CAP, true>(buf, N, log2N, log2NC, twp);
  // read-out in batches: the dot-product partner of a whole batch is loaded before its first use;
  // dot_with == out asks for ||out||^2
  const bool self_dot = (dot_with == out);
  const double* dwsrc = self_dot ? nullptr : dot_with;
  double acc = 0.0;
  for (int e0 = threadIdx.x; e0 < total; e0 += kBatch * NT) {
    double dw[kBatch];
#pragma unroll
    for (int u = 0; u < kBatch; ++u) {
      const int e = e0 + u * NT;
      const int p = e >> log2W, c = e & (W - 1);
      dw[u] = 0.0;
      if (dwsrc && e < total && g0 + c < M) dw[u] = __ldcs(dwsrc + (long long)p * M + g0 + c);
    }
#pragma unroll
    for (int u = 0; u < kBatch; ++u) {
      const int e = e0 + u * NT;
      const int p = e >> log2W, c = e & (W - 1);
      if (e < total && g0 + c < M) {
        const long long idx = (long long)p * M + g0 + c;
        const double z = A::part_sc(buf[p * NC + (c >> 1)], c & 1, RowSc<A>::dinv(pts, p));
        out[idx] = z;
        acc = fma(z, self_dot ? z : dw[u], acc);
      }
    }
  }
  if (partials) {
    double s = block_sum<NT>(acc, red);
    if (threadIdx.x == 0) partials[tile] = s;
  }
}

// shared memory the FP32 time pass stages behind its tile: N twiddles and 2 (N/2+1) spectrum
// entries (float2), N values of each row scaling (float)
template <class A> constexpr size_t tp_stage_bytes(int n) {
  return std::is_same<A, ArithF>::value
             ? (size_t)(n + 2 * (n / 2 + 1)) * sizeof(float2) + 2 * (size_t)n * sizeof(float)
             : 0;
}

template <class A, class Cfg = TileCfg<A>, int LOG2N = 0>
__global__ void __launch_bounds__(Cfg::NT, Cfg::MINB)
k_timepass(OpTables op, PrecTables pt, Combine cb, double* out, const double* dot_with,
           double* partials, const int* phase, int want, int log2NC,
           const typename A::V* __restrict__ tw) {
  if (skip_phase(phase, want)) return;
  timepass_tile<A, Cfg, std::is_same<A, ArithF>::value, LOG2N>(op, pt, cb, out, dot_with,
                                                               partials, log2NC, tw, blockIdx.x);
}


// ============================================================================================
// BLTT matvec along time by the 2N zero-padded circulant embedding (Sec. 5.1): per spatial point,
// y = first N entries of IFFT_2N(H .* FFT_2N([x; 0])), H = FFT_2N([a; 0]) (+ mu_i FFT_2N([b;0]) in
// the spectral basis).  Two real columns share one complex FFT.  The flip Y, the b_0 L (or b_0 mu)
// term, the normalisation of x and the dot product / residual are fused into load and store.
//   spectral: 1 -> lines are DST modes (matvec of (I (x) U) A (I (x) U)), 0 -> physical points.
//   which:    0 -> y = conv_a + extra term; 1 -> y = conv_b only (physical general-b first pass).
//   st_src:   source of the physical stencil term (x itself when b = b0 e_0, else conv_b(x)).
// A = ArithD runs on the FP64 pipe; A = ArithDF carries every value as a double-float pair on the
// FP32 pipes (about 2^-47 relative rounding per operation).
template <class A> struct ConvTables;
template <> struct ConvTables<ArithD> {
  static __device__ __forceinline__ const double2* tw(const OpTables& op) { return op.tw_2N; }
  static __device__ __forceinline__ const double2* H(const OpTables& op, int which) { return which ? op.Bhat : op.Ahat; }
  // per-mode spectrum, halved for the split of the packed pair: (A + mu B)/2 (general b) or
  // A/2 + sh (b = b0 e_0: B = 1/(2N) is a constant, so sh = b0 mu / (4N) is precomputed)
  static __device__ __forceinline__ double2 Hmode(const double2 a, const double2 b, double mu_or_sh, bool genb) {
    if (genb) return make_double2(0.5 * fma(mu_or_sh, b.x, a.x), 0.5 * fma(mu_or_sh, b.y, a.y));
    return make_double2(fma(0.5, a.x, mu_or_sh), 0.5 * a.y);
  }
  static __device__ __forceinline__ double sc_mu(double v) { return v; }
  static __device__ __forceinline__ const double2* Hm(const OpTables& op) { return op.Hm64; }
  static __device__ __forceinline__ double2 half(double2 v) { return make_double2(0.5 * v.x, 0.5 * v.y); }
};
template <> struct ConvTables<ArithDF> {
  static __device__ __forceinline__ const float4* tw(const OpTables& op) { return op.tw_2N_df; }
  static __device__ __forceinline__ const float4* H(const OpTables& op, int which) { return which ? op.Bhat_df : op.Ahat_df; }
  static __device__ __forceinline__ float4 Hmode(const float4 a, const float4 b, dfl mu_or_sh, bool genb) {
    const dfl ar = {0.5f * a.x, 0.5f * a.y}, ai = {0.5f * a.z, 0.5f * a.w};   // exact halving
    if (genb) {
      const dfl br = {0.5f * b.x, 0.5f * b.y}, bi = {0.5f * b.z, 0.5f * b.w};
      return ArithDF::pack(df_add(ar, df_mul(mu_or_sh, br)), df_add(ai, df_mul(mu_or_sh, bi)));
    }
    return ArithDF::pack(df_add(ar, mu_or_sh), ai);
  }
  static __device__ __forceinline__ const float4* Hm(const OpTables& op) { return op.Hmdf; }
  static __device__ __forceinline__ float4 half(float4 v) {   // exact halving of every part
    return make_float4(0.5f * v.x, 0.5f * v.y, 0.5f * v.z, 0.5f * v.w);
  }
};
template <class A> struct MuT;
template <> struct MuT<ArithD> { using t = double; static __device__ __forceinline__ double make(double v) { return v; } };
template <> struct MuT<ArithDF> { using t = dfl; static __device__ __forceinline__ dfl make(double v) { return df_from(v); } };

// LOG2N > 0: a tile of the full width for N = 2^LOG2N, with the transform length and the column
// count compile-time constants, so that the FFT passes unroll and their shared-memory addresses
// fold into immediate offsets; LOG2N = 0 takes both from op.log2N and log2NC_rt
template <class A, int LOG2N = 0>
__device__ __forceinline__ void conv_tile(const OpTables& op, int spectral, int which,
                                          const double* x, const double* xscale, double* y,
                                          int flip, int mode, const double* rhs,
                                          double* partials, const double* st_src, int log2NC_rt,
                                          long long tile) {
  constexpr int NT = TileCfg<A>::NT, CAP = TileCfg<A>::CAP;
  static_assert(LOG2N == 0 || (2 << LOG2N) <= CAP, "the transform must fit one tile");
  const int log2N = LOG2N ? LOG2N : op.log2N;
  const int log2NC = LOG2N ? ilog2c(CAP) - LOG2N - 1 : log2NC_rt;
  using V = typename A::V;
  __syncthreads();
  using MT = typename MuT<A>::t;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* buf = reinterpret_cast<V*>(smem_raw);
  __shared__ double red[32];
  __shared__ MT s_mu[kMaxCols];
  __shared__ double s_kmu[kMaxCols];
  __shared__ int s_nb[kMaxCols];
  const int N = 1 << log2N, L = 2 * N, NC = 1 << log2NC, W = 2 * NC, log2W = log2NC + 1;
  const long long M = op.M;
  const long long g0 = tile * W;
  const double s = xscale ? *xscale : 1.0;
  const bool genb = (op.b_kind == 1);
  const bool extra_st = !spectral && which == 0 && st_src != nullptr;
  // DST basis with b = b0 e_0: every mode's spectrum is FFT_2N([a;0]) plus the constant b0 mu_i,
  // so the packed pair is multiplied by the common spectrum (no split) and the b0 mu_i s x term
  // is added in the time domain at read-out
  const V* __restrict__ Hm = ConvTables<A>::Hm(op);     // per-mode spectra (general blocks)
  const bool common = spectral && !genb && Hm == nullptr;
  for (int c = threadIdx.x; c < W; c += NT) {
    const long long i = g0 + c;
    double mu = 0.0;
    int nb = 0;
    if (i < M) {
      if (spectral) mu = genb ? mode_mu(op, i) : op.b0 * mode_mu(op, i);
      long long r = i;
      for (int ax = 0; ax < op.d; ++ax) {
        const long long q = r / op.m[ax];
        const int cx = (int)(r - q * op.m[ax]);
        r = q;
        if (cx > 0) nb |= 1 << (2 * ax);
        if (cx < op.m[ax] - 1) nb |= 2 << (2 * ax);
      }
    }
    s_mu[c] = MuT<A>::make(mu);
    s_kmu[c] = mu * s;
    s_nb[c] = nb;
  }
  const typename A::Sc ssc = A::make_sc(s);
  const bool odd = ((log2N + 1) & 1) != 0;
  const int total = N * W;
  for (int e0 = threadIdx.x; e0 < total; e0 += kBatch * NT) {
    double v[kBatch];
#pragma unroll
    for (int u = 0; u < kBatch; ++u) {
      const int e = e0 + u * NT;
      const int p = e >> log2W, c = e & (W - 1);
      v[u] = (e < total && g0 + c < M) ? __ldcg(x + (long long)p * M + g0 + c) : 0.0;   // L2 only
    }
#pragma unroll
    for (int u = 0; u < kBatch; ++u) {
      const int e = e0 + u * NT;
      if (e < total) {
        const int p = e >> log2W, c = e & (W - 1);
        if (odd) {
          // the first radix-2 pass pairs x_p with the zero x_{p+N}: both outputs equal x_p
          A::put_sc2(buf, (2 * p) * NC + (c >> 1), (2 * p + 1) * NC + (c >> 1), c & 1, v[u], ssc);
        } else {
          A::put_sc(buf, p * NC + (c >> 1), c & 1, v[u], ssc);
        }
      }
    }
  }
  if (!odd)
    for (int e = threadIdx.x; e < N * NC; e += NT) buf[N * NC + e] = A::zero();
  __syncthreads();
  const V* __restrict__ tw = ConvTables<A>::tw(op);
  fft_columns<A, NT, CAP, false>(buf, L, log2N + 1, log2NC, tw, odd);
  if (!spectral || common) {
    const V* __restrict__ H = ConvTables<A>::H(op, which);
    for (int e = threadIdx.x; e < L * NC; e += NT) {
      const int k = e >> log2NC;
      const V h = (k <= N) ? H[k] : A::conj(H[L - k]);
      buf[e] = A::mul(buf[e], h);
    }
  } else {
    // per-mode spectrum H_i = FFT_2N([a;0] + mu_i [b;0]) / (2N); the packed pair is split
    const V* __restrict__ HA = ConvTables<A>::H(op, 0);
    const V* __restrict__ HB = ConvTables<A>::H(op, 1);
    const int items = (N + 1) << log2NC;
    for (int it = threadIdx.x; it < items; it += NT) {
      const int cc = it & (NC - 1), k = it >> log2NC;
      V Ha, Hb;
      if (Hm) {
        // general commuting blocks: the modes' own spectra, halved for the split
        const long long ia = g0 + 2 * cc;
        Ha = ia < M ? ConvTables<A>::half(Hm[(long long)k * M + ia]) : A::zero();
        Hb = ia + 1 < M ? ConvTables<A>::half(Hm[(long long)k * M + ia + 1]) : A::zero();
      } else {
        const V a_ = HA[k], b_ = HB[k];
        Ha = ConvTables<A>::Hmode(a_, b_, s_mu[2 * cc], true);
        Hb = ConvTables<A>::Hmode(a_, b_, s_mu[2 * cc + 1], true);
      }
      const int kb = (L - k) & (L - 1);
      const V Av = buf[k * NC + cc], Bc = A::conj(buf[kb * NC + cc]);
      const V U1 = A::mul(Ha, A::add(Av, Bc));
      const V U2 = A::mul(Hb, A::sub(Av, Bc));
      buf[k * NC + cc] = A::add(U1, U2);
      if (kb != k) buf[kb * NC + cc] = A::conj(A::sub(U1, U2));
    }
  }
  __syncthreads();
  // only the first N of the 2N outputs are kept: the last pass skips the others
  fft_columns<A, NT, CAP, true>(buf, L, log2N + 1, log2NC, tw, false, 0, true);
  double acc = 0.0;
  if (common) {
    // read-out of the time pairs (t, N-1-t) of one column: the two x values serve both the
    // b0 mu_i s x term (at t) and the dot-product partner (at the flipped index)
    constexpr int PB = kBatch / 2;
    const int half_total = (N >> 1) * W;
    for (int e0 = threadIdx.x; e0 < half_total; e0 += PB * NT) {
      double xa[PB], xb[PB], ra[PB], rb[PB];
#pragma unroll
      for (int u = 0; u < PB; ++u) {
        const int e = e0 + u * NT;
        const int t = e >> log2W, c = e & (W - 1);
        xa[u] = 0.0; xb[u] = 0.0; ra[u] = 0.0; rb[u] = 0.0;
        if (e < half_total && g0 + c < M) {
          const long long ia = (long long)t * M + g0 + c, ib = (long long)(N - 1 - t) * M + g0 + c;
          xa[u] = __ldcs(x + ia);
          xb[u] = __ldcs(x + ib);
          if (mode != MV_STORE) { ra[u] = __ldcs(rhs + ia); rb[u] = __ldcs(rhs + ib); }
        }
      }
#pragma unroll
      for (int u = 0; u < PB; ++u) {
        const int e = e0 + u * NT;
        const int t = e >> log2W, c = e & (W - 1);
        if (e >= half_total || g0 + c >= M) continue;
        const int t2 = N - 1 - t;
        const double k = s_kmu[c];
        // (A z)_t and (A z)_{N-1-t}, z = s x
        const double va = fma(k, xa[u], A::part(buf[t * NC + (c >> 1)], c & 1));
        const double vb = fma(k, xb[u], A::part(buf[t2 * NC + (c >> 1)], c & 1));
        // output time of (A z)_t is N-1-t with the flip
        const long long ia = (long long)(flip ? t2 : t) * M + g0 + c;
        const long long ib = (long long)(flip ? t : t2) * M + g0 + c;
        if (mode == MV_STORE) {
          if (y) { y[ia] = va; y[ib] = vb; }
          // partner of the output at index ia is x there: x_{t2} with the flip, else x_t
          acc = fma(va, flip ? xb[u] : xa[u], acc);
          acc = fma(vb, flip ? xa[u] : xb[u], acc);
        } else {
          const double r1 = (flip ? rb[u] : ra[u]) - va, r2 = (flip ? ra[u] : rb[u]) - vb;
          if (y) { y[ia] = r1; y[ib] = r2; }
          acc = fma(r1, r1, acc);
          acc = fma(r2, r2, acc);
        }
      }
    }
  } else {
    const double st_coef = (op.b_kind == 0) ? op.b0 * s : 1.0;
    const long long s1 = op.m[0], s2 = (long long)op.m[0] * op.m[1];
    // read-out in batches: the global operand of each output (x for the dot product, or the
    // right-hand side) is loaded for a whole batch before its first use
    for (int e0 = threadIdx.x; e0 < total; e0 += kBatch * NT) {
      double pre[kBatch];
#pragma unroll
      for (int u = 0; u < kBatch; ++u) {
        const int e = e0 + u * NT;
        const int t = e >> log2W, c = e & (W - 1);
        pre[u] = 0.0;
        if (e < total && g0 + c < M) {
          const int to = flip ? (N - 1 - t) : t;
          const long long idx = (long long)to * M + g0 + c;
          if (mode != MV_STORE) pre[u] = __ldcs(rhs + idx);
          else if (partials) pre[u] = __ldcs(x + idx);
        }
      }
#pragma unroll
      for (int u = 0; u < kBatch; ++u) {
        const int e = e0 + u * NT;
        const int t = e >> log2W, c = e & (W - 1);
        const long long i = g0 + c;
        if (e >= total || i >= M) continue;
        double val = A::part(buf[t * NC + (c >> 1)], c & 1);
        if (extra_st && op.kf[0]) {
          int ix, iy, iz;
          mode_coords(op, i, ix, iy, iz);
          val = fma(st_coef, stencil_faces(op, st_src + (long long)t * M, i, ix, iy, iz), val);
        } else if (extra_st) {
          const double* xt = st_src + (long long)t * M;
          const int nb = s_nb[c];
          const double xi2 = 2.0 * xt[i];
          double sx = xi2;
          if (nb & 1) sx -= xt[i - 1];
          if (nb & 2) sx -= xt[i + 1];
          double lap = sx * op.h2inv[0];
          if (op.d > 1) {
            double sy = xi2;
            if (nb & 4) sy -= xt[i - s1];
            if (nb & 8) sy -= xt[i + s1];
            lap = fma(sy, op.h2inv[1], lap);
            if (op.d > 2) {
              double sz = xi2;
              if (nb & 16) sz -= xt[i - s2];
              if (nb & 32) sz -= xt[i + s2];
              lap = fma(sz, op.h2inv[2], lap);
            }
          }
          val = fma(st_coef, lap, val);
        }
        const int to = flip ? (N - 1 - t) : t;
        const long long idx = (long long)to * M + i;
        if (mode == MV_STORE) {
          y[idx] = val;
          acc = fma(val, pre[u], acc);     // times s once per block below
        } else {
          const double r = pre[u] - val;
          if (y) y[idx] = r;
          acc = fma(r, r, acc);
        }
      }
    }
  }
  if (partials) {
    double sum = block_sum<NT>(acc, red);
    if (threadIdx.x == 0) partials[tile] = (mode == MV_STORE) ? sum * s : sum;
  }
}

template <class A, int LOG2N = 0>
__global__ void __launch_bounds__(TileCfg<A>::NT, TileCfg<A>::MINB)
k_conv(OpTables op, int spectral, int which, const double* x, const double* xscale, double* y,
       int flip, int mode, const double* rhs, double* partials, const int* phase, int want,
       const double* st_src, int log2NC) {
  if (skip_phase(phase, want)) return;
  conv_tile<A, LOG2N>(op, spectral, which, x, xscale, y, flip, mode, rhs, partials, st_src,
                      log2NC, blockIdx.x);
}

}  // namespace bltt
