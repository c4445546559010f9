// noalloc.cu - bltt_residual_noalloc: the true relative residual ||f - A u|| / ||f|| of a
// candidate solution, computed without a handle and without allocating device or pinned memory.
//
// Everything the kernels need besides the caller's vectors (operator tables, per-block partial
// sums, the two reduced scalars) lives in one file-scope device array of kNoAllocBytes.  Host
// code never dereferences that array's name: on the first call on a device the code below asks
// the runtime for its device address with cudaGetSymbolAddress (with that device current) and
// hands that address to the kernels from then on.
#include <cmath>
#include <complex>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/bltt.h"
#include "internal.h"

using namespace bltt;

namespace {

constexpr size_t kNoAllocBytes = 2u << 20;          // 2 MiB of device scratch, shared by all calls
constexpr int kNoAllocPartials = 131072;            // per-block partial sums (1 MiB of the scratch)
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {nullptr};

// this entry point reports through its status code only (the message is for debuggers)
bltt_status na_fail(bltt_status s, const std::string& msg) {
  (void)msg;
  return s;
}

// device address of the scratch array for the current device (looked up once per device)
bltt_status scratch_address(unsigned char** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return na_fail(BLTT_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return na_fail(BLTT_ERR_UNSUPPORTED, "device index out of range");
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr)
      return na_fail(BLTT_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    g_scratch_ptr[dev] = p;
  }
  *out = static_cast<unsigned char*>(g_scratch_ptr[dev]);
  return BLTT_OK;
}

// host tables (FP64): twiddles w_L^k and the 2N-embedding spectra, as the handle builds them
void na_twiddles(int L, std::vector<double2>& out) {
  out.resize(L);
  const long double two_pi = 6.283185307179586476925286766559005768L;
  for (int k = 0; k < L; ++k) {
    long double ang = two_pi * (long double)k / (long double)L;
    out[k] = make_double2((double)cosl(ang), (double)(-sinl(ang)));
  }
}

void na_fft(std::vector<std::complex<double>>& a) {
  const int n = (int)a.size();
  for (int i = 1, j = 0; i < n; ++i) {
    int bit = n >> 1;
    for (; j & bit; bit >>= 1) j ^= bit;
    j ^= bit;
    if (i < j) std::swap(a[i], a[j]);
  }
  std::vector<double2> tw;
  na_twiddles(n, tw);
  for (int len = 2; len <= n; len <<= 1) {
    const int step = n / len;
    for (int i = 0; i < n; i += len)
      for (int k = 0; k < len / 2; ++k) {
        std::complex<double> w(tw[k * step].x, tw[k * step].y);
        std::complex<double> u = a[i + k], v = a[i + k + len / 2] * w;
        a[i + k] = u + v;
        a[i + k + len / 2] = u - v;
      }
  }
}

bool pow2(long long v) { return v > 0 && (v & (v - 1)) == 0; }

__global__ void k_sumsq_noalloc(const double* __restrict__ f, long long n, double* partials) {
  __shared__ double red[32];
  double acc = 0.0;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x)
    acc = fma(f[e], f[e], acc);
  double s = acc;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    double r = (threadIdx.x < blockDim.x / 32) ? red[threadIdx.x] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) r += __shfl_down_sync(0xffffffffu, r, o);
    if (threadIdx.x == 0) partials[blockIdx.x] = r;
  }
}

}  // namespace

extern "C" bltt_status bltt_residual_noalloc(const bltt_blocks* blocks, int N, long long M,
                                             const double* u_dev, const double* f_dev,
                                             double* r_dev, void* cuda_stream,
                                             double* relres_out) {
  if (!blocks || !blocks->a || !blocks->b || !u_dev || !f_dev || !relres_out)
    return na_fail(BLTT_ERR_INVALID_ARG, "null argument");
  if (blocks->N != N || N < 2) return na_fail(BLTT_ERR_INVALID_ARG, "N mismatch or N < 2");
  const bltt_space& sp = blocks->space;
  if (sp.ndim < 1 || sp.ndim > 3) return na_fail(BLTT_ERR_INVALID_ARG, "ndim must be 1, 2 or 3");
  long long prodm = 1;
  for (int ax = 0; ax < sp.ndim; ++ax) {
    if (sp.m[ax] < 1 || !(sp.h[ax] > 0.0)) return na_fail(BLTT_ERR_INVALID_ARG, "bad m or h");
    prodm *= sp.m[ax];
  }
  if (prodm != M) return na_fail(BLTT_ERR_INVALID_ARG, "M != prod(m)");
  // the sizes bltt_create accepts: every FFT (2N along time, 2(m+1) along each axis) fits a tile
  if (!pow2(N) || 2 * N > kCap) return na_fail(BLTT_ERR_UNSUPPORTED, "N must be a power of two <= 2048");
  for (int ax = 0; ax < sp.ndim; ++ax)
    if (!pow2(sp.m[ax] + 1) || 2 * (sp.m[ax] + 1) > kCap)
      return na_fail(BLTT_ERR_UNSUPPORTED, "m+1 must be a power of two <= 2048");
  for (int k = 0; k < N; ++k)
    if (!std::isfinite(blocks->a[k]) || !std::isfinite(blocks->b[k]))
      return na_fail(BLTT_ERR_NUMERIC, "non-finite block coefficient");
  if (r_dev && (r_dev == u_dev || r_dev == f_dev))
    return na_fail(BLTT_ERR_INVALID_ARG, "r must not alias u or f");

  OpTables op{};
  op.N = N; op.d = sp.ndim; op.M = M;
  { int l = 0; while ((1 << l) < N) ++l; op.log2N = l; }
  for (int ax = 0; ax < 3; ++ax) {
    op.m[ax] = ax < sp.ndim ? sp.m[ax] : 1;
    const double h = ax < sp.ndim ? sp.h[ax] : 1.0;
    op.h2inv[ax] = 1.0 / (h * h);
  }
  bool b_e0 = true;
  int last_nz = 0;
  for (int k = 0; k < N; ++k) {
    if (k > 0 && blocks->b[k] != 0.0) b_e0 = false;
    if (blocks->a[k] != 0.0 || blocks->b[k] != 0.0) last_nz = k;
  }
  op.b_kind = b_e0 ? 0 : 1;
  op.b0 = blocks->b[0];
  op.ntaps = (last_nz < 4) ? last_nz + 1 : 0;
  op.mv_arith = 0;
  if (op.ntaps == 0 && op.b_kind == 1)
    return na_fail(BLTT_ERR_UNSUPPORTED,
                   "blocks with more than 4 nonzero coefficients and b != b0 e_0 need an N*M "
                   "temporary; use bltt_matvec");
  const int NC = tile_columns(M, 2 * N);
  const long long tiles = (M + 2 * NC - 1) / (2 * NC);
  if (op.ntaps == 0 && tiles > kNoAllocPartials)
    return na_fail(BLTT_ERR_UNSUPPORTED, "too many spatial modes for the fixed partial-sum scratch");

  // scratch layout (byte offsets, each 256-aligned)
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t o = off; off += (bytes + 255) & ~size_t(255); return o; };
  const size_t o_part = take(sizeof(double) * kNoAllocPartials);
  const size_t o_part2 = take(sizeof(double) * 2048);
  const size_t o_scal = take(sizeof(double) * 2);
  const size_t o_tw = take(sizeof(double2) * 2 * N);
  const size_t o_A = take(sizeof(double2) * (N + 1));
  const size_t o_B = take(sizeof(double2) * (N + 1));
  const size_t o_a = take(sizeof(double) * N);
  const size_t o_b = take(sizeof(double) * N);
  size_t o_mu[3];
  for (int ax = 0; ax < 3; ++ax) o_mu[ax] = take(sizeof(double) * (ax < sp.ndim ? op.m[ax] : 1));
  if (off > kNoAllocBytes) return na_fail(BLTT_ERR_UNSUPPORTED, "tables exceed the fixed scratch size");

  unsigned char* base = nullptr;
  bltt_status s = scratch_address(&base);
  if (s != BLTT_OK) return s;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(cuda_stream);

  // host tables
  std::vector<double2> tw;
  na_twiddles(2 * N, tw);
  std::vector<std::complex<double>> A2(2 * N, 0.0), B2(2 * N, 0.0);
  for (int k = 0; k < N; ++k) { A2[k] = blocks->a[k]; B2[k] = blocks->b[k]; }
  na_fft(A2);
  na_fft(B2);
  std::vector<double2> Ah(N + 1), Bh(N + 1);
  for (int k = 0; k <= N; ++k) {
    Ah[k] = make_double2(A2[k].real() / (2.0 * N), A2[k].imag() / (2.0 * N));
    Bh[k] = make_double2(B2[k].real() / (2.0 * N), B2[k].imag() / (2.0 * N));
  }
  std::vector<std::vector<double>> mu(3);
  for (int ax = 0; ax < sp.ndim; ++ax) {
    mu[ax].resize(op.m[ax]);
    for (int k = 0; k < op.m[ax]; ++k) {
      long double sn = sinl(3.141592653589793238462643383279502884L * (k + 1) / (2.0L * (op.m[ax] + 1)));
      mu[ax][k] = (double)(4.0L / ((long double)sp.h[ax] * sp.h[ax]) * sn * sn);
    }
  }
  cudaError_t e = cudaSuccess;
  auto put = [&](size_t o, const void* src, size_t bytes) {
    if (e == cudaSuccess) e = cudaMemcpyAsync(base + o, src, bytes, cudaMemcpyHostToDevice, st);
  };
  put(o_tw, tw.data(), tw.size() * sizeof(double2));
  put(o_A, Ah.data(), Ah.size() * sizeof(double2));
  put(o_B, Bh.data(), Bh.size() * sizeof(double2));
  put(o_a, blocks->a, N * sizeof(double));
  put(o_b, blocks->b, N * sizeof(double));
  for (int ax = 0; ax < sp.ndim; ++ax) put(o_mu[ax], mu[ax].data(), mu[ax].size() * sizeof(double));
  op.tw_2N = reinterpret_cast<const double2*>(base + o_tw);
  op.Ahat = reinterpret_cast<const double2*>(base + o_A);
  op.Bhat = reinterpret_cast<const double2*>(base + o_B);
  op.a_dev = reinterpret_cast<const double*>(base + o_a);
  op.b_dev = reinterpret_cast<const double*>(base + o_b);
  for (int ax = 0; ax < sp.ndim; ++ax) op.mu_axis[ax] = reinterpret_cast<const double*>(base + o_mu[ax]);
  double* partials = reinterpret_cast<double*>(base + o_part);
  double* partials2 = reinterpret_cast<double*>(base + o_part2);
  double* scal = reinterpret_cast<double*>(base + o_scal);

  // r = f - A u with per-block partial sums of r^2; ||f||^2 by a grid-stride sum
  int np = 0;
  if (e == cudaSuccess)
    e = launch_matvec(op, 0, u_dev, nullptr, r_dev, 0, MV_RESID, f_dev, partials, &np, nullptr,
                      nullptr, st);
  const long long n = (long long)N * M;
  const int g2 = 1024;
  if (e == cudaSuccess) {
    k_sumsq_noalloc<<<g2, 256, 0, st>>>(f_dev, n, partials2);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = launch_sum_partials(partials, np, scal, st);
  if (e == cudaSuccess) e = launch_sum_partials(partials2, g2, scal + 1, st);
  double host[2] = {0.0, 0.0};
  if (e == cudaSuccess) e = cudaMemcpyAsync(host, scal, sizeof host, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);   // host tables and host[] are locals
  if (e != cudaSuccess) return na_fail(BLTT_ERR_CUDA, std::string("bltt_residual_noalloc: ") + cudaGetErrorString(e));
  if (!std::isfinite(host[0]) || !std::isfinite(host[1])) return na_fail(BLTT_ERR_NUMERIC, "non-finite residual");
  *relres_out = host[1] > 0.0 ? std::sqrt(host[0] / host[1]) : std::sqrt(host[0]);
  return BLTT_OK;
}
