// kernels.cu - sm_103a kernels of libbltt: DST-I along a spatial axis, the alpha-scaled time pass
// of the ABAC preconditioner, the BLTT matvec (2N circulant embedding or direct taps), the
// preconditioner set-up and the MINRES vector/scalar kernels.
#include <atomic>
#include <math.h>
#include <algorithm>
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

template <typename K>
static cudaError_t set_smem(K kern, size_t bytes) {
  return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

static int ilog2(long long v) { int l = 0; while ((1LL << l) < v) ++l; return l; }

// complex columns per FFT tile: fill the tile (kCap points) but keep at most kMaxCols real lines
// and, when the batch is small, at least two tiles per SM
int tile_columns(long long nlines, int Lfft, int cap) {
  int nc = cap / Lfft;
  if (nc < 1) nc = 1;
  if (nc > kMaxCols / 2) nc = kMaxCols / 2;
  long long pairs = (nlines + 1) / 2;
  while (nc > 1 && (pairs + nc - 1) / nc < 2 * 152) nc >>= 1;
  return nc;
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
template <class A, bool SWZ>
__device__ __forceinline__ void dst_tile(long long nlines, int m, long long inner, int P, int log2P,
                                         int log2NC, const Combine& cb, double* out, int flip,
                                         int N, long long M, const double* dot_with,
                                         double* partials, const typename A::V* __restrict__ tw,
                                         long long tile) {
  constexpr int NT = TileCfg<A>::NT, CAP = TileCfg<A>::CAP;
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
  const int total = m * W, log2W = log2NC + 1;
  // x_j (j = p + 1) of line c into row j, column c/2, component c%2
  for (int e0 = threadIdx.x; e0 < total; e0 += kBatch * NT) {
    double v[kBatch];
    int cs[kBatch], ps[kBatch];
#pragma unroll
    for (int u = 0; u < kBatch; ++u) {
      const int e = e0 + u * NT;
      int c = 0, p = 0;
      if (contiguous) { c = fast_div(e, m, inv_m); p = e - c * m; }
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
      if (contiguous) { c = fast_div(e, m, inv_m); k = e - c * m; }
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
        acc = fma(val, self_dot ? val : dw[u], acc);
      }
    }
  }
  if (partials) {
    double s = block_sum<NT>(acc, red);
    if (threadIdx.x == 0) partials[tile] = s;
  }
}

template <class A, bool SWZ>
__global__ void __launch_bounds__(TileCfg<A>::NT, TileCfg<A>::MINB)
k_dst(long long nlines, int m, long long inner, int P, int log2P, int log2NC, Combine cb,
      double* out, int flip, int N, long long M, const double* dot_with, double* partials,
      const typename A::V* __restrict__ tw, const int* phase, int want) {
  if (skip_phase(phase, want)) return;
  dst_tile<A, SWZ>(nlines, m, inner, P, log2P, log2NC, cb, out, flip, N, M, dot_with, partials,
                   tw, blockIdx.x);
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
                                            const PrecTables& pt, int log2NC, long long g0,
                                            const float* s_mu) {
  constexpr int NT = Cfg::NT;
  using V = typename A::V;
  const int N = op.N, half = N >> 1, NC = 1 << log2NC;
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

template <class A, class Cfg = TileCfg<A>, bool TWS = false>
__device__ __forceinline__ void timepass_tile(const OpTables& op, const PrecTables& pt,
                                              const Combine& cb, double* out,
                                              const double* dot_with, double* partials,
                                              int log2NC, const typename A::V* __restrict__ tw,
                                              long long tile) {
  constexpr int NT = Cfg::NT, CAP = Cfg::CAP;
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
    const int n = op.N, nh = n / 2 + 1;
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
  const int N = op.N, NC = 1 << log2NC, W = 2 * NC, log2W = log2NC + 1;
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
  fft_columns<A, NT, CAP, false>(buf, N, op.log2N, log2NC, twp);
  tp_freq_mul<A, true, Cfg>(buf, op, pts, log2NC, g0, s_mu);
  __syncthreads();
  fft_columns<A, NT, CAP, true>(buf, N, op.log2N, log2NC, twp);
  for (int e = threadIdx.x; e < N * NC; e += NT)
    buf[e] = A::scale_sc(buf[e], RowSc<A>::d2(pts, e >> log2NC));
  __syncthreads();
  fft_columns<A, NT, CAP, false>(buf, N, op.log2N, log2NC, twp);
  tp_freq_mul<A, false, Cfg>(buf, op, pts, log2NC, g0, s_mu);
  __syncthreads();
  fft_columns<A, NT, CAP, true>(buf, N, op.log2N, log2NC, twp);
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

template <class A, class Cfg = TileCfg<A>>
__global__ void __launch_bounds__(Cfg::NT, Cfg::MINB)
k_timepass(OpTables op, PrecTables pt, Combine cb, double* out, const double* dot_with,
           double* partials, const int* phase, int want, int log2NC,
           const typename A::V* __restrict__ tw) {
  if (skip_phase(phase, want)) return;
  timepass_tile<A, Cfg, std::is_same<A, ArithF>::value>(op, pt, cb, out, dot_with, partials,
                                                        log2NC, tw, blockIdx.x);
}

// identity preconditioner (MINRES-I): z = v, with the same fused load and dot
__global__ void k_precond_identity(Combine cb, double* out, long long n, const double* dot_with,
                                   double* partials, const int* phase, int want) {
  if (skip_phase(phase, want)) return;
  __shared__ double red[32];
  double c0, c1, c2;
  load_coef(cb, c0, c1, c2);
  double acc = 0.0;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x) {
    double v = combine_at(cb, e, c0, c1, c2);
    out[e] = v;
    if (dot_with) acc = fma(v, dot_with[e], acc);
  }
  if (partials) {
    double s = block_sum<256>(acc, red);
    if (threadIdx.x == 0) partials[blockIdx.x] = s;
  }
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

template <class A>
__device__ __forceinline__ void conv_tile(const OpTables& op, int spectral, int which,
                                          const double* x, const double* xscale, double* y,
                                          int flip, int mode, const double* rhs,
                                          double* partials, const double* st_src, int log2NC,
                                          long long tile) {
  constexpr int NT = TileCfg<A>::NT, CAP = TileCfg<A>::CAP;
  using V = typename A::V;
  __syncthreads();
  using MT = typename MuT<A>::t;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* buf = reinterpret_cast<V*>(smem_raw);
  __shared__ double red[32];
  __shared__ MT s_mu[kMaxCols];
  __shared__ double s_kmu[kMaxCols];
  __shared__ int s_nb[kMaxCols];
  const int N = op.N, L = 2 * N, NC = 1 << log2NC, W = 2 * NC, log2W = log2NC + 1;
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
  const bool odd = ((op.log2N + 1) & 1) != 0;
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
  fft_columns<A, NT, CAP, false>(buf, L, op.log2N + 1, log2NC, tw, odd);
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
  fft_columns<A, NT, CAP, true>(buf, L, op.log2N + 1, log2NC, tw, false, 0, true);
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

template <class A>
__global__ void __launch_bounds__(TileCfg<A>::NT, TileCfg<A>::MINB)
k_conv(OpTables op, int spectral, int which, const double* x, const double* xscale, double* y,
       int flip, int mode, const double* rhs, double* partials, const int* phase, int want,
       const double* st_src, int log2NC) {
  if (skip_phase(phase, want)) return;
  conv_tile<A>(op, spectral, which, x, xscale, y, flip, mode, rhs, partials, st_src, log2NC,
               blockIdx.x);
}

// Direct matvec for blocks that vanish beyond ntaps (heat BDF / CN): y_t = sum_{k<ntaps}
// (a_k x_{t-k} + b_k [mu_i | L] x_{t-k}), same fused epilogues as k_conv.  A thread owns one
// spatial point and walks it through all N time steps: its coefficients s (a_k + b_k mu_i) are
// formed once, the K-1 earlier x (and, in the physical basis, L x) stay in registers, and each
// output costs K FP64 multiply-adds plus the fused dot product (GB300 runs FP64 at 2 FMA per
// clock per SM, so the FP64 operation count, not the bytes, bounds this kernel).
constexpr int kDirectThreads = 256;
constexpr int kDirectPts = 4;      // points per thread, kDirectThreads apart: 8 KB rows per block

// per-point stencil weights of L (or L_a): w0 x_i - sum_n wn x_{i + off_n}; a neighbour outside
// the grid has weight 0 and offset 0 (so its load stays in bounds)
template <int D2>
struct PointStencil {
  double w0;
  double wn[D2];
  int off[D2];
};
template <int D2>
__device__ __forceinline__ PointStencil<D2> point_stencil(const OpTables& op, int ix, int iy, int iz) {
  PointStencil<D2> ps;
  ps.w0 = 0.0;
  const long long m0 = op.m[0], m1 = op.d > 1 ? op.m[1] : 1;
  long long stride = 1;
#pragma unroll
  for (int ax = 0; ax < D2 / 2; ++ax) {
    double alo = 1.0, ahi = 1.0;
    int c = 0, mm = 1;
    if (ax < op.d) {
      c = ax == 0 ? ix : (ax == 1 ? iy : iz);
      mm = op.m[ax];
      if (op.kf[0]) {
        long long lo, hi;
        if (ax == 0) { lo = ((long long)iz * m1 + iy) * (m0 + 1) + ix; hi = lo + 1; }
        else if (ax == 1) { lo = ((long long)iz * (m1 + 1) + iy) * m0 + ix; hi = lo + m0; }
        else { lo = ((long long)iz * m1 + iy) * m0 + ix; hi = lo + m1 * m0; }
        alo = op.kf[ax][lo];
        ahi = op.kf[ax][hi];
      }
      const double h2 = op.h2inv[ax];
      ps.w0 = fma(alo + ahi, h2, ps.w0);
      ps.wn[2 * ax] = c > 0 ? alo * h2 : 0.0;
      ps.off[2 * ax] = c > 0 ? (int)-stride : 0;
      ps.wn[2 * ax + 1] = c < mm - 1 ? ahi * h2 : 0.0;
      ps.off[2 * ax + 1] = c < mm - 1 ? (int)stride : 0;
      stride *= mm;
    } else {
      ps.wn[2 * ax] = ps.wn[2 * ax + 1] = 0.0;
      ps.off[2 * ax] = ps.off[2 * ax + 1] = 0;
    }
  }
  return ps;
}
template <int D2>
__device__ __forceinline__ double apply_stencil(const PointStencil<D2>& ps,
                                                const double* __restrict__ x_ti) {
  double v = ps.w0 * x_ti[0];
#pragma unroll
  for (int n = 0; n < D2; ++n)
    if (ps.wn[n] != 0.0) v = fma(-ps.wn[n], x_ti[ps.off[n]], v);   // absent axes and boundaries
  return v;
}

constexpr int kDirectChunk = 32;   // time steps a thread walks per work unit

// One work unit: a group of kDirectThreads x P consecutive points (P per thread, kDirectThreads
// apart) over a chunk of kDirectChunk time steps; the K-1 earlier values (and their L x in the
// physical basis) are loaded at the chunk's start.  Units run point groups fastest, so that the
// blocks in flight read neighbouring runs of the same rows.
template <int K, bool SPECTRAL>
__global__ void __launch_bounds__(kDirectThreads)
k_direct(OpTables op, const double* __restrict__ x, const double* xscale, double* y, int flip,
         int mode, const double* rhs, double* partials, const int* phase, int want) {
  if (skip_phase(phase, want)) return;
  constexpr bool spectral = SPECTRAL;
  constexpr int P = SPECTRAL ? kDirectPts : 1;
  constexpr int D2 = SPECTRAL ? 1 : 6;          // stencil neighbours kept per point
  __shared__ double red[32];
  const int N = op.N;
  const long long M = op.M;
  const double s = xscale ? *xscale : 1.0;
  bool any_b = false;
#pragma unroll
  for (int k = 0; k < K; ++k) any_b |= (op.b_dev[k] != 0.0);
  const bool lap = !spectral && any_b;
  const long long groups = (M + P * kDirectThreads - 1) / (P * kDirectThreads);
  const long long units = groups * ((N + kDirectChunk - 1) / kDirectChunk);
  double acc = 0.0;
  for (long long u = blockIdx.x; u < units; u += gridDim.x) {
    const int chunk = (int)(u / groups);
    const long long c0 = (u - (long long)chunk * groups) * (P * kDirectThreads);
    const int t0 = chunk * kDirectChunk, t1 = min(N, t0 + kDirectChunk);
    long long ip[P];
    double ca[P][K], cb[P][K], xp[P][K], lp[P][K];
    PointStencil<D2> pst[P];
#pragma unroll
    for (int q = 0; q < P; ++q) {
      ip[q] = c0 + q * kDirectThreads + threadIdx.x;
      const long long i = ip[q] < M ? ip[q] : M - 1;     // tail points compute, never store
      int cx, cy, cz;
      mode_coords(op, i, cx, cy, cz);
      if (!spectral && lap) pst[q] = point_stencil<D2>(op, cx, cy, cz);
      // per-point coefficients: spectral s (a_k + b_k mu_i); physical s a_k and s b_k
      const double mu = spectral ? mode_mu(op, i) : 0.0;
#pragma unroll
      for (int k = 0; k < K; ++k) {
        const double ak = op.a_dev[k], bk = op.b_dev[k];
        ca[q][k] = spectral ? s * fma(bk, mu, ak) : s * ak;
        cb[q][k] = spectral ? 0.0 : s * bk;
        // the chunk's earlier steps t0 - k (zero before the first step)
        const int tk = t0 - k;
        xp[q][k] = 0.0;
        lp[q][k] = 0.0;
        if (k > 0 && tk >= 0) {
          const double* xt = x + (long long)tk * M + i;
          // stored one slot ahead: the step loop shifts before it uses them
          xp[q][k - 1] = xt[0];
          if (!spectral && lap) lp[q][k - 1] = apply_stencil<D2>(pst[q], xt);
        }
      }
    }
    for (int t = t0; t < t1; ++t) {
      const long long row = (long long)t * M;
      const long long orow = (long long)(flip ? (N - 1 - t) : t) * M;
      double xs[P], pr[P];
#pragma unroll
      for (int q = 0; q < P; ++q) {
        const long long i = ip[q] < M ? ip[q] : M - 1;
        xs[q] = x[row + i];
        pr[q] = (mode != MV_STORE) ? rhs[orow + i] : (partials ? x[orow + i] : 0.0);
      }
#pragma unroll
      for (int q = 0; q < P; ++q) {
        const long long i = ip[q] < M ? ip[q] : M - 1;
#pragma unroll
        for (int k = K - 1; k > 0; --k) { xp[q][k] = xp[q][k - 1]; lp[q][k] = lp[q][k - 1]; }
        xp[q][0] = xs[q];
        if (!spectral && lap) lp[q][0] = apply_stencil<D2>(pst[q], x + row + i);
        double val = 0.0;
#pragma unroll
        for (int k = 0; k < K; ++k) {
          val = fma(ca[q][k], xp[q][k], val);
          if (!spectral) val = fma(cb[q][k], lp[q][k], val);
        }
        if (ip[q] < M) {
          if (mode == MV_STORE) {
            y[orow + i] = val;
            acc = fma(val, pr[q], acc);               // times s once per block below
          } else {
            const double r = pr[q] - val;
            if (y) y[orow + i] = r;
            acc = fma(r, r, acc);
          }
        }
      }
    }
  }
  if (partials) {
    double sum = block_sum<kDirectThreads>(acc, red);
    if (threadIdx.x == 0) partials[blockIdx.x] = (mode == MV_STORE) ? sum * s : sum;
  }
}

// physical general-b second pass: y += L tmp (only used when b has more than one nonzero and the
// FFT matvec is chosen; the stencil term is then folded in by k_conv with st_src = tmp)

// ============================================================================================
// Set-up of the FP64 time-pass table: g(k, i) = lambda_i(k)^{-1/2} / (2N), k = 0..N/2, with
// lambda_i(k) = ahat_k + bhat_k mu_i the eigenvalues of eq. hatcalphaieigvaldef (principal branch,
// Def. 2; Re lambda > 0 by diagonal dominance, Sec. 3).
__global__ void k_setup_g64(OpTables op, const double2* ahat, const double2* bhat, double2* g,
                            float4* gdf) {
  const int half = op.N / 2;
  const long long total = (long long)(half + 1) * op.M;
  const double sc = 0.5 / op.N;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int k = (int)(e / op.M);
    const long long i = e - (long long)k * op.M;
    const double mu = mode_mu(op, i);
    const double2 a = ahat[k], b = bhat[k];
    double2 v = inv_sqrt_principal<double>(fma(b.x, mu, a.x), fma(b.y, mu, a.y));
    const double gr = v.x * sc, gi = v.y * sc;
    if (g) g[e] = make_double2(gr, gi);
    if (gdf) {
      const dfl r = df_from(gr), im = df_from(gi);
      gdf[e] = make_float4(r.hi, r.lo, im.hi, im.lo);
    }
  }
}

// Set-up of the FP32 and double-float time-pass tables without FP64 arithmetic: g0 is the
// principal lambda^{-1/2} in FP32 (half-angle form); the double-float value takes one Newton
// step for z^{-1/2}, g1 = g0 (3 - lambda g0^2) / 2, in double-float (the error squares: 2^-24 ->
// about 2^-47), with lambda = ahat_k + bhat_k mu_i formed in double-float.
__global__ void k_setup_gdf(OpTables op, const float2* ahat32, const float2* bhat32,
                            const float4* ahatdf, const float4* bhatdf, float4* gdf) {
  const int half = op.N / 2;
  const long long total = (long long)(half + 1) * op.M;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int k = (int)(e / op.M);
    const long long i = e - (long long)k * op.M;
    const float mu = mode_mu32(op, i);
    const float2 a = ahat32[k], b = bhat32[k];
    const float2 g0 = inv_sqrt_principal<float>(fmaf(b.x, mu, a.x), fmaf(b.y, mu, a.y));
    const float4 A4 = ahatdf[k], B4 = bhatdf[k];
    // mu_i as double-float: sum of the per-axis FP64 eigenvalues (or the dense operator's)
    dfl m_;
    if (op.mu_tab) {
      m_ = df_from(op.mu_tab[i]);
    } else {
      long long r = i / op.m[0];
      m_ = df_from(op.mu_axis[0][i - r * op.m[0]]);
      if (op.d > 1) {
        long long r2 = r / op.m[1];
        m_ = df_add(m_, df_from(op.mu_axis[1][r - r2 * op.m[1]]));
        if (op.d > 2) m_ = df_add(m_, df_from(op.mu_axis[2][r2]));
      }
    }
    const float4 lam = ArithDF::pack(df_add(dfl{A4.x, A4.y}, df_mul(m_, dfl{B4.x, B4.y})),
                                     df_add(dfl{A4.z, A4.w}, df_mul(m_, dfl{B4.z, B4.w})));
    const float4 g = make_float4(g0.x, 0.f, g0.y, 0.f);
    const float4 t = ArithDF::mul(lam, ArithDF::mul(g, g));          // lambda g0^2 ~ 1
    const float4 three_m = ArithDF::sub(make_float4(3.f, 0.f, 0.f, 0.f), t);
    const float4 g1 = ArithDF::mul(g, three_m);                        // 2 g1
    const dfl s2 = {0.25f / (float)op.N, 0.f};                         // (1/2) (1/(2N)), exact
    gdf[e] = ArithDF::pack(df_mul(dfl{g1.x, g1.y}, s2), df_mul(dfl{g1.z, g1.w}, s2));
  }
}

// b = Y f (time reversal, Sec. 2) and partial sums of ||b||^2
__global__ void k_flip_copy(const double* f, double* b, int N, long long M, double* partials) {
  __shared__ double red[32];
  const long long n = (long long)N * M;
  double acc = 0.0;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x) {
    const int t = (int)(e / M);
    const long long i = e - (long long)t * M;
    const double v = f[(long long)(N - 1 - t) * M + i];
    b[e] = v;
    acc = fma(v, v, acc);
  }
  double s = block_sum<256>(acc, red);
  if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

// ============================================================================================
// MINRES scalar recurrences (one block; partial sums reduced in a fixed order)
__device__ double reduce_partials(const double* p, int n, double* scratch) {
  double acc = 0.0;
  for (int i = threadIdx.x; i < n; i += 256) acc += p[i];
  return block_sum<256>(acc, scratch);
}

__device__ __forceinline__ void scalar_init(MinresDev* st, const double* pzv, int nzv,
                                            const double* pb, int nb) {
  __shared__ double red[32];
  double g2 = reduce_partials(pzv, nzv, red);
  __syncthreads();
  double nb2 = reduce_partials(pb, nb, red);
  if (threadIdx.x != 0) return;
  st->normb = sqrt(nb2);
  st->iter = 0;
  st->wpending = 0;
  st->relres_est = 1.0;
  st->relres_true = 1.0;
  st->gamma_new = 0.0;
  if (!(g2 >= 0.0) || !isfinite(g2) || !isfinite(nb2)) {
    st->phase = PH_FAIL; st->status = 5; return;
  }
  const double g = sqrt(g2);
  st->gamma = g; st->gamma_prev = 1.0; st->eta = g; st->eta0 = g;
  st->s = 0.0; st->s_prev = 0.0; st->c = 1.0; st->c_prev = 1.0;
  st->inv_gamma = g > 0.0 ? 1.0 / g : 0.0;
  st->status = 0;
  if (g == 0.0) { st->phase = PH_DONE; st->relres_est = 0.0; st->relres_true = 0.0; }
  else st->phase = PH_RUN;
}

__device__ __forceinline__ void scalar_delta(MinresDev* st, const double* p, int np) {
  if (st->phase != PH_RUN) return;
  __shared__ double red[32];
  double delta = reduce_partials(p, np, red);
  if (threadIdx.x != 0) return;
  if (!isfinite(delta)) { st->phase = PH_FAIL; st->status = 5; return; }
  st->delta = delta;
  st->coef[0] = 1.0;
  st->coef[1] = -delta / st->gamma;
  st->coef[2] = -st->gamma / st->gamma_prev;
}

__device__ __forceinline__ void scalar_gamma(MinresDev* st, const double* p, int np) {
  if (st->phase != PH_RUN) return;
  __shared__ double red[32];
  double g2 = reduce_partials(p, np, red);
  if (threadIdx.x != 0) return;
  if (!(g2 >= 0.0) || !isfinite(g2)) { st->phase = PH_FAIL; st->status = 5; return; }
  const double gn = sqrt(g2);
  const double delta = st->delta, gamma = st->gamma;
  const double c = st->c, c_prev = st->c_prev, s = st->s, s_prev = st->s_prev;
  const double a0 = c * delta - c_prev * s * gamma;
  const double a1 = sqrt(a0 * a0 + gn * gn);
  const double a2 = s * delta + c_prev * c * gamma;
  const double a3 = s_prev * gamma;
  const double cn = a0 / a1, sn = gn / a1;
  st->w_inv_gamma = st->inv_gamma;
  st->w_a1inv = 1.0 / a1;
  st->w_a2 = a2;
  st->w_a3 = a3;
  st->w_ceta = cn * st->eta;
  st->w_cz = st->inv_gamma / a1;
  st->w_cwp = -a3 / a1;
  st->w_cw = -a2 / a1;
  st->eta = -sn * st->eta;
  st->gamma_prev = gamma;
  st->gamma = gn;
  st->gamma_new = gn;
  st->inv_gamma = gn > 0.0 ? 1.0 / gn : 0.0;
  st->s_prev = s; st->s = sn;
  st->c_prev = c; st->c = cn;
  st->iter += 1;
  st->wpending = 1;
  st->relres_est = fabs(st->eta) / st->eta0;
  if (gn == 0.0 || st->relres_est <= st->tol || st->iter >= st->maxit) st->phase = PH_CHECK;
}

__device__ __forceinline__ void scalar_check(MinresDev* st, const double* p, int np) {
  __shared__ double red[32];
  const bool check = (st->phase == PH_CHECK);
  double r2 = check ? reduce_partials(p, np, red) : 0.0;
  if (threadIdx.x != 0) return;
  st->wpending = 0;
  if (!check) return;
  const double rr = sqrt(r2) / st->normb;
  st->relres_true = rr;
  if (!isfinite(rr)) { st->phase = PH_FAIL; st->status = 5; return; }
  if (rr <= st->tol || st->gamma_new == 0.0) {
    st->phase = PH_DONE; st->status = (rr <= st->tol) ? 0 : 6;
  } else if (st->iter >= st->maxit) {
    st->phase = PH_MAXIT; st->status = 6;
  } else {
    st->phase = PH_RUN;
  }
}

__global__ void __launch_bounds__(256) k_scalar_init(MinresDev* st, const double* pzv, int nzv,
                                                     const double* pb, int nb) {
  scalar_init(st, pzv, nzv, pb, nb);
}
__global__ void __launch_bounds__(256) k_scalar_delta(MinresDev* st, const double* p, int np) {
  scalar_delta(st, p, np);
}
__global__ void __launch_bounds__(256) k_scalar_gamma(MinresDev* st, const double* p, int np) {
  scalar_gamma(st, p, np);
}
__global__ void __launch_bounds__(256) k_scalar_check(MinresDev* st, const double* p, int np) {
  scalar_check(st, p, np);
}
// the true-residual check left to the host: an estimate that met the stopping rule halts the
// iterations (PH_VERIFY) instead of launching the residual product here
__global__ void k_scalar_defer(MinresDev* st) {
  st->wpending = 0;
  if (st->phase == PH_CHECK) st->phase = PH_VERIFY;
}

// w_{j+1} = (z_j - a3 w_{j-1} - a2 w_j)/a1 (written over w_{j-1}); x += c_{j+1} eta w_{j+1}.
// The coefficients are folded (w_cz = 1/(gamma_j a1), ...) so that each element costs four FP64
// operations: GB300 runs FP64 at 1/64 of its FP32 rate and this kernel is bound by that pipe.
__device__ __forceinline__ void w_update_elem(const double* __restrict__ z, double* w_prev,
                                              const double* __restrict__ w, double* x, long long e,
                                              double cz, double cwp, double cw, double ce) {
  const double wn = fma(cz, __ldcs(z + e), fma(cwp, __ldcs(w_prev + e), cw * __ldcs(w + e)));
  __stcs(w_prev + e, wn);
  __stcs(x + e, fma(ce, wn, __ldcs(x + e)));
}

// elements e0, e0 + stride, ... < n of one update; pairs of elements as 16-byte accesses when
// every vector is 16-byte aligned, with all loads of four pairs issued before the first store (the
// stores alias nothing that the loads read, but the compiler cannot know that)
__device__ __forceinline__ void w_update_range(const double* z, double* w_prev, const double* w,
                                               double* x, long long n, long long e,
                                               long long stride, double cz, double cwp,
                                               double cw, double ce) {
  const bool vec = ((n & 1) == 0) &&
                   ((((uintptr_t)z | (uintptr_t)w_prev | (uintptr_t)w | (uintptr_t)x) & 15) == 0);
  if (vec) {
    const double2* z2 = reinterpret_cast<const double2*>(z);
    double2* wp2 = reinterpret_cast<double2*>(w_prev);
    const double2* w2 = reinterpret_cast<const double2*>(w);
    double2* x2 = reinterpret_cast<double2*>(x);
    const long long n2 = n >> 1;
    for (; e + 3 * stride < n2; e += 4 * stride) {
      double2 a[4], b[4], c[4], d[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const long long i = e + u * stride;
        a[u] = __ldcs(z2 + i); b[u] = __ldcs(wp2 + i); c[u] = __ldcs(w2 + i); d[u] = __ldcs(x2 + i);
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const long long i = e + u * stride;
        double2 wn, xn;
        wn.x = fma(cz, a[u].x, fma(cwp, b[u].x, cw * c[u].x));
        wn.y = fma(cz, a[u].y, fma(cwp, b[u].y, cw * c[u].y));
        xn.x = fma(ce, wn.x, d[u].x);
        xn.y = fma(ce, wn.y, d[u].y);
        __stcs(wp2 + i, wn);
        __stcs(x2 + i, xn);
      }
    }
    for (; e < n2; e += stride) {
      w_update_elem(z, w_prev, w, x, 2 * e, cz, cwp, cw, ce);
      w_update_elem(z, w_prev, w, x, 2 * e + 1, cz, cwp, cw, ce);
    }
    return;
  }
  for (; e + 3 * stride < n; e += 4 * stride) {          // four independent elements in flight
#pragma unroll
    for (int u = 0; u < 4; ++u) w_update_elem(z, w_prev, w, x, e + u * stride, cz, cwp, cw, ce);
  }
  for (; e < n; e += stride) w_update_elem(z, w_prev, w, x, e, cz, cwp, cw, ce);
}

__global__ void __launch_bounds__(256) k_w_update(const MinresDev* st, const double* z,
                                                  double* w_prev, const double* w, double* x,
                                                  long long n) {
  if (!st->wpending) return;
  w_update_range(z, w_prev, w, x, n, blockIdx.x * (long long)blockDim.x + threadIdx.x,
                 (long long)gridDim.x * blockDim.x, st->w_cz, st->w_cwp, st->w_cw, st->w_ceta);
}

__global__ void __launch_bounds__(256) k_sum_partials(const double* p, int np, double* out) {
  __shared__ double red[32];
  double s = reduce_partials(p, np, red);
  if (threadIdx.x == 0) *out = s;
}

// ============================================================================================
// The whole solve by one block (A5 for the smallest workload, 4032 unknowns): entry DST, the
// MINRES iterations with the residual check inside the loop (DST basis), exit DST.  The phases are
// the tile functions of the multi-block kernels, each called on its one tile; the partial sums
// they write (one per tile, so the totals) are read after a barrier, which orders global memory
// within the block.  The loop is bounded by maxit.  Two arithmetic forms: FP64 throughout (256
// threads), and the chosen form (double-float product and DSTs, FP32 time pass; 512 threads), whose
// work runs on the FP32 pipes: one SM's FP64 rate is 1/64 of its FP32 rate.
struct OneF64 {
  using Conv = ArithD;
  using Tp = ArithD;
  using TpCfg = TileCfg<ArithD>;
  using Dst = ArithD;
  static constexpr int NT = kThreads;
  static __device__ __forceinline__ const double2* tw_tp(const OpTables& op) { return op.tw_N; }
  static __device__ __forceinline__ const double2* tw_dst(const OpTables& op, int ax) { return op.tw_dst[ax]; }
};
struct OneChosen {
  using Conv = ArithDF;
  using Tp = ArithF;
  using TpCfg = WideTileF;
  using Dst = ArithDF;
  static constexpr int NT = 2 * kThreads;
  static __device__ __forceinline__ const float2* tw_tp(const OpTables& op) { return op.tw_N32; }
  static __device__ __forceinline__ const float4* tw_dst(const OpTables& op, int ax) { return op.tw_dst_df[ax]; }
};

template <class F, bool SWZ>
__device__ __forceinline__ void one_dst(const OneSolve& s, int ax, const double* in, double* out,
                                        int flip, const double* dot_with, double* partials) {
  const OpTables& op = s.op;
  const int m = op.m[ax];
  long long inner = 1;
  for (int a = 0; a < ax; ++a) inner *= op.m[a];
  const long long nlines = (long long)op.N * op.M / m;
  const int P = m + 1;
  Combine c{};
  c.in0 = in;
  dst_tile<typename F::Dst, SWZ>(nlines, m, inner, P, __ffs(P) - 1, s.log2NC_dst[ax], c, out, flip,
                                 op.N, op.M, dot_with, partials, F::tw_dst(op, ax), 0);
}

// out = (I (x) U) in over every axis (flip on the first), ||out||^2 into partials[0] if asked
template <class F>
__device__ __forceinline__ void one_dst_all(const OneSolve& s, const double* in, double* out,
                                            int flip, double* partials) {
  for (int ax = 0; ax < s.op.d; ++ax) {
    const bool last = (ax == s.op.d - 1);
    const double* src = (ax == 0) ? in : out;
    double* dw = (last && partials) ? out : nullptr;
    if (ax == 0) one_dst<F, true>(s, ax, src, out, flip, dw, last ? partials : nullptr);
    else one_dst<F, false>(s, ax, src, out, 0, dw, last ? partials : nullptr);
    __syncthreads();
  }
}

template <class F>
__global__ void __launch_bounds__(F::NT) k_solve_one(OneSolve s) {
  constexpr int NT = F::NT;
  static_assert(TileCfg<typename F::Conv>::NT == NT && F::TpCfg::NT == NT &&
                TileCfg<typename F::Dst>::NT == NT, "one block size for every phase");
  const OpTables& op = s.op;
  MinresDev* st = s.st;
  const long long n = (long long)op.N * op.M;
  double* const P_B = s.part + 0;     // ||b||^2
  double* const P_ZV = s.part + 1;    // <z, v>
  double* const P_D = s.part + 2;     // delta
  double* const P_R = s.part + 3;     // ||r||^2
  // b = Y (I (x) U) f with ||b||^2
  one_dst_all<F>(s, s.f, s.b, 1, P_B);
  // v_1 = b, z_1 = P^{-1} v_1, <z_1, v_1>
  {
    Combine c{};
    c.in0 = s.b;
    c.vout = s.v[0];
    timepass_tile<typename F::Tp, typename F::TpCfg>(op, s.pt, c, s.z[0], s.v[0], P_ZV,
                                                     s.log2NC_tp, F::tw_tp(op), 0);
  }
  for (long long e = threadIdx.x; e < n; e += NT) {
    s.x[e] = 0.0;
    s.v[1][e] = 0.0;
    s.w[0][e] = 0.0;
    s.w[1][e] = 0.0;
  }
  __syncthreads();
  scalar_init(st, P_ZV, 1, P_B, 1);
  __syncthreads();
  double *vc = s.v[0], *vp = s.v[1], *zc = s.z[0], *zp = s.z[1], *wc = s.w[0], *wp = s.w[1];
  for (int it = 0; it < s.maxit && st->phase == PH_RUN; ++it) {
    // q = Y A z_j (z_j = z_u / gamma_j), delta = <q, z_j>
    conv_tile<typename F::Conv>(op, 1, 0, zc, &st->inv_gamma, s.q, 1, MV_STORE, nullptr, P_D,
                                nullptr, s.log2NC_conv, 0);
    __syncthreads();
    scalar_delta(st, P_D, 1);
    __syncthreads();
    if (st->phase != PH_RUN) break;
    // v_{j+1} = q - (delta/gamma) v_j - (gamma/gamma_prev) v_{j-1} (over v_{j-1}); z_{j+1}; <z, v>
    Combine c{};
    c.in0 = s.q;
    c.in1 = vc;
    c.in2 = vp;
    c.coef = st->coef;
    c.vout = vp;
    timepass_tile<typename F::Tp, typename F::TpCfg>(op, s.pt, c, zp, vp, P_ZV, s.log2NC_tp,
                                                     F::tw_tp(op), 0);
    __syncthreads();
    scalar_gamma(st, P_ZV, 1);
    __syncthreads();
    if (st->wpending)
      w_update_range(zc, wp, wc, s.x, n, threadIdx.x, NT, st->w_cz, st->w_cwp, st->w_cw,
                     st->w_ceta);
    __syncthreads();
    // the true residual ||b - Y A x|| when the estimate met the stopping rule
    if (st->phase == PH_CHECK)
      conv_tile<typename F::Conv>(op, 1, 0, s.x, nullptr, nullptr, 1, MV_RESID, s.b, P_R, nullptr,
                                  s.log2NC_conv, 0);
    __syncthreads();
    scalar_check(st, P_R, 1);
    __syncthreads();
    double* t;
    t = vc; vc = vp; vp = t;
    t = zc; zc = zp; zp = t;
    t = wc; wc = wp; wp = t;
  }
  // u = (I (x) U) x
  one_dst_all<F>(s, s.x, s.u, 0, nullptr);
}

int one_tile_columns(long long nlines, int Lfft, int cap_points) {
  int cap = cap_points / Lfft;
  if (cap > kMaxCols / 2) cap = kMaxCols / 2;
  const long long pairs = (nlines + 1) / 2;
  if (cap < 1 || pairs > cap) return 0;
  int nc = 1;
  while (nc < pairs) nc <<= 1;
  return nc;
}

// ============================================================================================
// launchers
static int grid_stream(long long n, int threads) {
  long long g = (n + threads - 1) / threads;
  long long cap = 152LL * 8;
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return (int)g;
}

// cudaFuncSetAttribute acts on the current device only, so each helper below records, per device
// (bit d of a mask), that its attributes are set.  Setting them twice is harmless, so two threads
// racing on a first call only repeat the work; devices beyond 63 set them on every call.
template <class F> static cudaError_t once_per_device(std::atomic<unsigned long long>& mask, F&& f) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const unsigned long long bit = (dev >= 0 && dev < 64) ? (1ull << dev) : 0ull;
  if (bit && (mask.load(std::memory_order_acquire) & bit)) return cudaSuccess;
  e = f();
  if (e == cudaSuccess && bit) mask.fetch_or(bit, std::memory_order_acq_rel);
  return e;
}

template <class A> static cudaError_t ensure_smem_dst() {
  static std::atomic<unsigned long long> done{0};
  return once_per_device(done, [] {
    cudaError_t e = set_smem(k_dst<A, false>, TileCfg<A>::CAP * sizeof(typename A::V));
    if (e == cudaSuccess) e = set_smem(k_dst<A, true>, TileCfg<A>::CAP * sizeof(typename A::V));
    return e;
  });
}

template <class A>
static void run_dst(const OpTables& op, long long grid, long long nlines, int m, long long inner,
                    int P, int log2NC, const Combine& in, double* out, int flip,
                    const double* dot_with, double* partials, const typename A::V* tw,
                    const int* phase, cudaStream_t st) {
  const size_t smem = TileCfg<A>::CAP * sizeof(typename A::V);
  if (inner == 1)
    k_dst<A, true><<<(unsigned)grid, TileCfg<A>::NT, smem, st>>>(nlines, m, inner, P, ilog2(P), log2NC,
        in, out, flip, op.N, op.M, dot_with, partials, tw, phase, PH_RUN);
  else
    k_dst<A, false><<<(unsigned)grid, TileCfg<A>::NT, smem, st>>>(nlines, m, inner, P, ilog2(P), log2NC,
        in, out, flip, op.N, op.M, dot_with, partials, tw, phase, PH_RUN);
}
// shared memory the FP32 time pass stages behind its tile: N twiddles and 2 (N/2+1) spectrum
// entries (float2), N values of each row scaling (float)
template <class A> constexpr size_t tp_stage_bytes(int n) {
  return std::is_same<A, ArithF>::value
             ? (size_t)(n + 2 * (n / 2 + 1)) * sizeof(float2) + 2 * (size_t)n * sizeof(float)
             : 0;
}
template <class A, class Cfg = TileCfg<A>> static cudaError_t ensure_smem_tp() {
  static std::atomic<unsigned long long> done{0};
  return once_per_device(done, [] {
    return set_smem(k_timepass<A, Cfg>, Cfg::CAP * sizeof(typename A::V) + tp_stage_bytes<A>(kCap));
  });
}
template <class A> static cudaError_t ensure_smem_conv() {
  static std::atomic<unsigned long long> done{0};
  return once_per_device(done, [] { return set_smem(k_conv<A>, TileCfg<A>::CAP * sizeof(typename A::V)); });
}

cudaError_t prepare_kernel_attributes() {
  cudaError_t e = ensure_smem_dst<ArithD>();
  if (e == cudaSuccess) e = ensure_smem_dst<ArithF>();
  if (e == cudaSuccess) e = ensure_smem_dst<ArithDF>();
  if (e == cudaSuccess) e = ensure_smem_tp<ArithD>();
  if (e == cudaSuccess) e = ensure_smem_tp<ArithF>();
  if (e == cudaSuccess) e = ensure_smem_tp<ArithF, WideTileF>();
  if (e == cudaSuccess) e = ensure_smem_tp<ArithDF>();
  if (e == cudaSuccess) e = ensure_smem_conv<ArithD>();
  if (e == cudaSuccess) e = ensure_smem_conv<ArithDF>();
  return e;
}

cudaError_t launch_dst(const OpTables& op, int axis, int prec, const Combine& in, double* out,
                       int flip, const double* dot_with, double* partials, int* nparts,
                       const int* phase, cudaStream_t st) {
  const int m = op.m[axis];
  long long inner = 1;
  for (int a = 0; a < axis; ++a) inner *= op.m[a];
  const long long nlines = (long long)op.N * op.M / m;
  const int P = m + 1;
  if (P > kCap) return cudaErrorInvalidValue;      // the FFT (length P) must fit one tile
  const int NC = tile_columns(nlines, P);
  const int log2NC = ilog2(NC);
  const long long grid = (nlines + 2 * NC - 1) / (2 * NC);
  if (nparts) *nparts = (int)grid;
  cudaError_t e;
  if (prec == PREC_F64) {
    if ((e = ensure_smem_dst<ArithD>()) != cudaSuccess) return e;
    run_dst<ArithD>(op, grid, nlines, m, inner, P, log2NC, in, out, flip, dot_with, partials,
                    op.tw_dst[axis], phase, st);
  } else if (prec == PREC_DF) {
    if ((e = ensure_smem_dst<ArithDF>()) != cudaSuccess) return e;
    run_dst<ArithDF>(op, grid, nlines, m, inner, P, log2NC, in, out, flip, dot_with, partials,
                     op.tw_dst_df[axis], phase, st);
  } else {
    if ((e = ensure_smem_dst<ArithF>()) != cudaSuccess) return e;
    run_dst<ArithF>(op, grid, nlines, m, inner, P, log2NC, in, out, flip, dot_with, partials,
                    op.tw_dst32[axis], phase, st);
  }
  return cudaGetLastError();
}

// tile choice of the single-item time pass (shared by launch_timepass and timepass_tiles)
static bool tp_wide(const OpTables& op, int prec) {
  return prec == PREC_F32 && 2 * (kCap / op.N) < 16 && op.N <= WideTileF::CAP;
}

long long timepass_tiles(const OpTables& op, int prec) {
  const int NC = tile_columns(op.M, op.N, tp_wide(op, prec) ? WideTileF::CAP : kCap);
  return (op.M + 2 * NC - 1) / (2 * NC);
}

cudaError_t launch_timepass(const OpTables& op, const PrecTables& pt, int prec, const Combine& in,
                            double* out, const double* dot_with, double* partials, int* nparts,
                            const int* phase, cudaStream_t st) {
  if (pt.none) {
    long long n = (long long)op.N * op.M;
    int g = grid_stream(n, 256);
    if (nparts) *nparts = g;
    k_precond_identity<<<g, 256, 0, st>>>(in, out, n, dot_with, partials, phase, PH_RUN);
    return cudaGetLastError();
  }
  if (op.N > kCap) return cudaErrorInvalidValue;   // the FFT must fit one tile
  auto run = [&](auto arith, auto cfg, const auto* tw) -> cudaError_t {
    using A = decltype(arith);
    using Cfg = decltype(cfg);
    cudaError_t e = ensure_smem_tp<A, Cfg>();
    if (e != cudaSuccess) return e;
    const int NC = tile_columns(op.M, op.N, Cfg::CAP);
    const int log2NC = ilog2(NC);
    const long long grid = (op.M + 2 * NC - 1) / (2 * NC);
    if (nparts) *nparts = (int)grid;
    const size_t smem = Cfg::CAP * sizeof(typename A::V) + tp_stage_bytes<A>(op.N);
    k_timepass<A, Cfg><<<(unsigned)grid, Cfg::NT, smem, st>>>(
        op, pt, in, out, dot_with, partials, phase, PH_RUN, log2NC, tw);
    return cudaGetLastError();
  };
  if (prec == PREC_F64) return run(ArithD{}, TileCfg<ArithD>{}, op.tw_N);
  if (prec == PREC_DF) return run(ArithDF{}, TileCfg<ArithDF>{}, op.tw_N_df);
  // FP32: the wide tile where the common one would span fewer than 16 lines (N >= 1024)
  if (tp_wide(op, PREC_F32)) return run(ArithF{}, WideTileF{}, op.tw_N32);
  return run(ArithF{}, TileCfg<ArithF>{}, op.tw_N32);
}

template <class A>
static cudaError_t launch_conv_t(const OpTables& op, int spectral, const double* x,
                                 const double* xscale, double* y, int flip, int mode,
                                 const double* rhs, double* partials, int* nparts,
                                 const int* phase, int want, double* tmp, cudaStream_t st) {
  if (2 * op.N > kCap) return cudaErrorInvalidValue;   // the FFT must fit one tile
  cudaError_t e = ensure_smem_conv<A>();
  if (e != cudaSuccess) return e;
  const int NC = tile_columns(op.M, 2 * op.N);
  const int log2NC = ilog2(NC);
  const long long grid = (op.M + 2 * NC - 1) / (2 * NC);
  if (nparts) *nparts = (int)grid;
  const size_t smem = kCap * sizeof(typename A::V);
  const double* st_src = x;
  if (!spectral && op.b_kind == 1) {
    // conv_b(x) first (scaled like x), then y = conv_a(x) + L conv_b(x)
    k_conv<A><<<(unsigned)grid, TileCfg<A>::NT, smem, st>>>(op, 0, 1, x, xscale, tmp, 0, MV_STORE,
                                                     nullptr, nullptr, phase, want, nullptr, log2NC);
    st_src = tmp;
  }
  k_conv<A><<<(unsigned)grid, TileCfg<A>::NT, smem, st>>>(op, spectral, 0, x, xscale, y, flip, mode, rhs,
                                                   partials, phase, want, st_src, log2NC);
  return cudaGetLastError();
}

cudaError_t launch_matvec(const OpTables& op, int spectral, const double* x, const double* xscale,
                          double* y, int flip, int mode, const double* rhs, double* partials,
                          int* nparts, const int* phase, double* tmp, cudaStream_t st) {
  const int want = (mode == MV_RESID) ? PH_CHECK : PH_RUN;
  if (op.ntaps > 0) {
    const long long per = (long long)(spectral ? kDirectPts : 1) * kDirectThreads;
    long long g = (op.M + per - 1) / per * ((op.N + kDirectChunk - 1) / kDirectChunk);
    if (g > 152LL * 8) g = 152LL * 8;
    if (nparts) *nparts = (int)g;
#define BLTT_DIRECT(K_)                                                                         \
  (spectral ? k_direct<K_, true><<<(unsigned)g, kDirectThreads, 0, st>>>(                      \
                  op, x, xscale, y, flip, mode, rhs, partials, phase, want)                     \
            : k_direct<K_, false><<<(unsigned)g, kDirectThreads, 0, st>>>(                     \
                  op, x, xscale, y, flip, mode, rhs, partials, phase, want))
    switch (op.ntaps) {
      case 1: BLTT_DIRECT(1); break;
      case 2: BLTT_DIRECT(2); break;
      case 3: BLTT_DIRECT(3); break;
      default: BLTT_DIRECT(4); break;
    }
#undef BLTT_DIRECT
    return cudaGetLastError();
  }
  if (op.mv_arith == 2 && mode == MV_STORE)
    return launch_tc_matvec(op, spectral, x, xscale, y, flip, partials, nparts, phase, st);
  if (op.mv_arith >= 1)
    return launch_conv_t<ArithDF>(op, spectral, x, xscale, y, flip, mode, rhs, partials, nparts,
                                  phase, want, tmp, st);
  return launch_conv_t<ArithD>(op, spectral, x, xscale, y, flip, mode, rhs, partials, nparts,
                               phase, want, tmp, st);
}

cudaError_t launch_setup_g64(const OpTables& op, const double2* ahat, const double2* bhat,
                             double2* g64, float4* gdf, cudaStream_t st) {
  long long total = (long long)(op.N / 2 + 1) * op.M;
  k_setup_g64<<<grid_stream(total, 256), 256, 0, st>>>(op, ahat, bhat, g64, gdf);
  return cudaGetLastError();
}

cudaError_t launch_setup_gdf(const OpTables& op, const float2* ahat32, const float2* bhat32,
                             const float4* ahatdf, const float4* bhatdf, float4* gdf,
                             cudaStream_t st) {
  long long total = (long long)(op.N / 2 + 1) * op.M;
  k_setup_gdf<<<grid_stream(total, 256), 256, 0, st>>>(op, ahat32, bhat32, ahatdf, bhatdf, gdf);
  return cudaGetLastError();
}

cudaError_t launch_flip_copy(const double* f, double* b, int N, long long M, double* partials,
                             int* nparts, cudaStream_t st) {
  long long n = (long long)N * M;
  int g = grid_stream(n, 256);
  if (nparts) *nparts = g;
  k_flip_copy<<<g, 256, 0, st>>>(f, b, N, M, partials);
  return cudaGetLastError();
}

cudaError_t launch_scalar_init(MinresDev* s, const double* pzv, int nzv, const double* pb, int nb,
                               cudaStream_t st) {
  k_scalar_init<<<1, 256, 0, st>>>(s, pzv, nzv, pb, nb);
  return cudaGetLastError();
}
cudaError_t launch_scalar_delta(MinresDev* s, const double* p, int np, cudaStream_t st) {
  k_scalar_delta<<<1, 256, 0, st>>>(s, p, np);
  return cudaGetLastError();
}
cudaError_t launch_scalar_gamma(MinresDev* s, const double* p, int np, cudaStream_t st) {
  k_scalar_gamma<<<1, 256, 0, st>>>(s, p, np);
  return cudaGetLastError();
}
cudaError_t launch_scalar_check(MinresDev* s, const double* p, int np, cudaStream_t st) {
  k_scalar_check<<<1, 256, 0, st>>>(s, p, np);
  return cudaGetLastError();
}

cudaError_t launch_scalar_defer(MinresDev* s, cudaStream_t st) {
  k_scalar_defer<<<1, 1, 0, st>>>(s);
  return cudaGetLastError();
}
cudaError_t launch_solve_one(const OneSolve& s, bool chosen, cudaStream_t st) {
  // both forms stage a tile of 64 KB: kCap double2 (FP64), kCap float4 (double-float), 8192 float2
  static_assert(kCap * sizeof(double2) == kCap * sizeof(float4) &&
                kCap * sizeof(float4) == WideTileF::CAP * sizeof(float2), "one tile size");
  const size_t smem = kCap * sizeof(double2);
  static std::atomic<unsigned long long> attr{0};
  cudaError_t ea = once_per_device(attr, [smem] {
    cudaError_t e = set_smem(k_solve_one<OneF64>, smem);
    if (e == cudaSuccess) e = set_smem(k_solve_one<OneChosen>, smem);
    return e;
  });
  if (ea != cudaSuccess) return ea;
  if (chosen) k_solve_one<OneChosen><<<1, OneChosen::NT, smem, st>>>(s);
  else k_solve_one<OneF64><<<1, OneF64::NT, smem, st>>>(s);
  return cudaGetLastError();
}
cudaError_t launch_w_update(MinresDev* s, const double* z, double* w_prev, const double* w,
                            double* x, long long n, cudaStream_t st) {
  k_w_update<<<grid_stream(n, 256), 256, 0, st>>>(s, z, w_prev, w, x, n);
  return cudaGetLastError();
}
cudaError_t launch_sum_partials(const double* partials, int np, double* out, cudaStream_t st) {
  k_sum_partials<<<1, 256, 0, st>>>(partials, np, out);
  return cudaGetLastError();
}

// ============================================================================================
// Multi-item kernels (batched solves).  They keep the full register budget: their tile bodies
// read the item tables through memory rather than from kernel parameters and need more registers.
__device__ __forceinline__ int find_item(const long long* prefix, int nitems, long long t) {
  int lo = 0, hi = nitems - 1;           // largest i with prefix[i] <= t
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (prefix[mid] <= t) lo = mid; else hi = mid - 1;
  }
  return lo;
}

template <class A>
__global__ void __launch_bounds__(TileCfg<A>::NT)
k_conv_multi(const ConvItem* __restrict__ items, const long long* __restrict__ prefix, int nitems,
             long long total) {
  for (long long t = blockIdx.x; t < total; t += gridDim.x) {
    const int it = find_item(prefix, nitems, t);
    const ConvItem& ci = items[it];
    if (ci.phase && *ci.phase != ci.want) continue;
    conv_tile<A>(ci.op, ci.spectral, 0, ci.x, ci.xscale, ci.y, ci.flip, ci.mode, ci.rhs,
                 ci.partials, ci.spectral ? nullptr : ci.x, ci.log2NC, t - prefix[it]);
  }
}

template <class A>
__global__ void __launch_bounds__(TileCfg<A>::NT)
k_timepass_multi(const TpItem* __restrict__ items, const long long* __restrict__ prefix,
                 int nitems, long long total) {
  for (long long t = blockIdx.x; t < total; t += gridDim.x) {
    const int it = find_item(prefix, nitems, t);
    const TpItem& ti = items[it];
    if (ti.phase && *ti.phase != ti.want) continue;
    const typename A::V* tw = reinterpret_cast<const typename A::V*>(
        sizeof(typename A::V) == 16 ? (std::is_same<A, ArithDF>::value ? (const void*)ti.op.tw_N_df
                                                                        : (const void*)ti.op.tw_N)
                                    : (const void*)ti.op.tw_N32);
    timepass_tile<A>(ti.op, ti.pt, ti.cb, ti.out, ti.dot_with, ti.partials, ti.log2NC, tw,
                     t - prefix[it]);
  }
}

template <class A>
__global__ void __launch_bounds__(TileCfg<A>::NT)
k_dst_multi(const DstItem* __restrict__ items, const long long* __restrict__ prefix, int nitems,
            long long total) {
  for (long long t = blockIdx.x; t < total; t += gridDim.x) {
    const int it = find_item(prefix, nitems, t);
    const DstItem& di = items[it];
    const typename A::V* tw = reinterpret_cast<const typename A::V*>(di.tw);
    if (di.inner == 1)
      dst_tile<A, true>(di.nlines, di.m, di.inner, di.P, di.log2P, di.log2NC, di.cb, di.out,
                        di.flip, (int)di.N, di.M, di.dot_with, di.partials, tw, t - prefix[it]);
    else
      dst_tile<A, false>(di.nlines, di.m, di.inner, di.P, di.log2P, di.log2NC, di.cb, di.out,
                         di.flip, (int)di.N, di.M, di.dot_with, di.partials, tw, t - prefix[it]);
  }
}

// one block row of items per blockIdx.y; elements grid-strided over blockIdx.x
__global__ void __launch_bounds__(256) k_w_update_multi(const VecItem* __restrict__ items) {
  const VecItem& vi = items[blockIdx.y];
  if (!vi.st->wpending) return;
  const MinresDev* st = vi.st;
  w_update_range(vi.z, vi.w_prev, vi.w, vi.x, vi.n, blockIdx.x * (long long)blockDim.x + threadIdx.x,
                 (long long)gridDim.x * blockDim.x, st->w_cz, st->w_cwp, st->w_cw, st->w_ceta);
}

__global__ void __launch_bounds__(256) k_scalar_multi(int which, const ScalItem* __restrict__ items) {
  const ScalItem& si = items[blockIdx.x];
  switch (which) {
    case 0: scalar_init(si.st, si.p0, si.n0, si.p1, si.n1); break;
    case 1: scalar_delta(si.st, si.p0, si.n0); break;
    case 2: scalar_gamma(si.st, si.p0, si.n0); break;
    default: scalar_check(si.st, si.p0, si.n0); break;
  }
}

__global__ void k_count_running(const ScalItem* __restrict__ items, int nitems, int* out) {
  int c = 0;
  for (int i = threadIdx.x; i < nitems; i += blockDim.x) {
    const int ph = items[i].st->phase;
    c += (ph == PH_RUN || ph == PH_CHECK) ? 1 : 0;
  }
  for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
  if (threadIdx.x == 0) *out = c;
}

int persistent_grid(int kind, int prec) {
  int dev = 0, sms = 152, per = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  size_t smem = (prec == PREC_F32 ? sizeof(float2) : sizeof(double2)) * kCap;
  if (kind == 0) {
    if (prec == PREC_DF) { set_smem(k_conv_multi<ArithDF>, smem);
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_conv_multi<ArithDF>, TileCfg<ArithDF>::NT, smem); }
    else { set_smem(k_conv_multi<ArithD>, smem);
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_conv_multi<ArithD>, TileCfg<ArithD>::NT, smem); }
  } else if (kind == 1) {
    if (prec == PREC_F32) { set_smem(k_timepass_multi<ArithF>, smem);
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_timepass_multi<ArithF>, TileCfg<ArithF>::NT, smem); }
    else if (prec == PREC_DF) { set_smem(k_timepass_multi<ArithDF>, smem);
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_timepass_multi<ArithDF>, TileCfg<ArithDF>::NT, smem); }
    else { set_smem(k_timepass_multi<ArithD>, smem);
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_timepass_multi<ArithD>, TileCfg<ArithD>::NT, smem); }
  } else {
    if (prec == PREC_DF) { set_smem(k_dst_multi<ArithDF>, smem);
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_dst_multi<ArithDF>, TileCfg<ArithDF>::NT, smem); }
    else { set_smem(k_dst_multi<ArithD>, smem);
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_dst_multi<ArithD>, TileCfg<ArithD>::NT, smem); }
  }
  if (per < 1) per = 1;
  return sms * per;
}

cudaError_t launch_conv_multi(int arith, const ConvItem* items, const long long* prefix,
                              int nitems, long long total, cudaStream_t st) {
  const int g = (int)std::min<long long>(persistent_grid(0, arith ? PREC_DF : PREC_F64), total);
  if (g <= 0) return cudaSuccess;
  if (arith)
    k_conv_multi<ArithDF><<<g, TileCfg<ArithDF>::NT, kCap * sizeof(float4), st>>>(items, prefix, nitems, total);
  else
    k_conv_multi<ArithD><<<g, TileCfg<ArithD>::NT, kCap * sizeof(double2), st>>>(items, prefix, nitems, total);
  return cudaGetLastError();
}

cudaError_t launch_timepass_multi(int prec, const TpItem* items, const long long* prefix,
                                  int nitems, long long total, cudaStream_t st) {
  const int g = (int)std::min<long long>(persistent_grid(1, prec), total);
  if (g <= 0) return cudaSuccess;
  if (prec == PREC_F32)
    k_timepass_multi<ArithF><<<g, TileCfg<ArithF>::NT, kCap * sizeof(float2), st>>>(items, prefix, nitems, total);
  else if (prec == PREC_DF)
    k_timepass_multi<ArithDF><<<g, TileCfg<ArithDF>::NT, kCap * sizeof(float4), st>>>(items, prefix, nitems, total);
  else
    k_timepass_multi<ArithD><<<g, TileCfg<ArithD>::NT, kCap * sizeof(double2), st>>>(items, prefix, nitems, total);
  return cudaGetLastError();
}

cudaError_t launch_dst_multi(int prec, const DstItem* items, const long long* prefix, int nitems,
                             long long total, cudaStream_t st) {
  const int g = (int)std::min<long long>(persistent_grid(2, prec), total);
  if (g <= 0) return cudaSuccess;
  if (prec == PREC_DF)
    k_dst_multi<ArithDF><<<g, TileCfg<ArithDF>::NT, kCap * sizeof(float4), st>>>(items, prefix, nitems, total);
  else
    k_dst_multi<ArithD><<<g, TileCfg<ArithD>::NT, kCap * sizeof(double2), st>>>(items, prefix, nitems, total);
  return cudaGetLastError();
}

cudaError_t launch_w_update_multi(const VecItem* items, int nitems, cudaStream_t st) {
  if (nitems <= 0) return cudaSuccess;
  dim3 grid(std::max(1, 152 * 8 / std::max(1, nitems)), nitems);
  k_w_update_multi<<<grid, 256, 0, st>>>(items);
  return cudaGetLastError();
}

cudaError_t launch_scalar_multi(int which, const ScalItem* items, int nitems, cudaStream_t st) {
  if (nitems <= 0) return cudaSuccess;
  k_scalar_multi<<<nitems, 256, 0, st>>>(which, items);
  return cudaGetLastError();
}

cudaError_t launch_count_running(const ScalItem* items, int nitems, int* out, cudaStream_t st) {
  k_count_running<<<1, 32, 0, st>>>(items, nitems, out);
  return cudaGetLastError();
}

}  // namespace bltt
