// bltt_api.cu - the C ABI of libbltt (declared in include/bltt.h): handle life cycle, set-up of
// the spectral tables, the physical-basis matvec and preconditioner entry points and the MINRES
// driver (device-resident scalar state, host checks every few iterations).
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include <cublas_v2.h>
#include <cusolverDn.h>
#include <nvtx3/nvToolsExt.h>

#include "internal.h"

using namespace bltt;
using cd = std::complex<double>;

namespace {

thread_local std::string g_create_error;

// ---------------------------------------------------------------------------------------------
// host-side transforms for the set-up (O(N log N), FP64 with long-double twiddles)
void twiddle_table(int L, std::vector<double2>& out) {
  out.resize(L);
  const long double two_pi = 6.283185307179586476925286766559005768L;
  for (int k = 0; k < L; ++k) {
    long double ang = two_pi * (long double)k / (long double)L;
    out[k] = make_double2((double)cosl(ang), (double)(-sinl(ang)));
  }
}

// the table of one length, computed once per process (long double is a software format on some
// hosts, so the per-alpha set-up must not recompute it)
const std::vector<double2>& twiddles(int L) {
  static std::mutex mu;
  static std::map<int, std::vector<double2>> cache;   // nodes do not move: references stay valid
  std::lock_guard<std::mutex> lk(mu);
  auto it = cache.find(L);
  if (it == cache.end()) {
    std::vector<double2> t;
    twiddle_table(L, t);
    it = cache.emplace(L, std::move(t)).first;
  }
  return it->second;
}

// forward DFT X_k = sum_j x_j exp(-2 pi i jk/L), L a power of two (iterative radix 2)
void host_fft(std::vector<cd>& a) {
  const int n = (int)a.size();
  for (int i = 1, j = 0; i < n; ++i) {
    int bit = n >> 1;
    for (; j & bit; bit >>= 1) j ^= bit;
    j ^= bit;
    if (i < j) std::swap(a[i], a[j]);
  }
  const std::vector<double2>& tw = twiddles(n);
  for (int len = 2; len <= n; len <<= 1) {
    const int step = n / len;
    for (int i = 0; i < n; i += len)
      for (int k = 0; k < len / 2; ++k) {
        const double wr = tw[k * step].x, wi = tw[k * step].y;
        const cd u = a[i + k], b = a[i + k + len / 2];
        const cd v(b.real() * wr - b.imag() * wi, b.real() * wi + b.imag() * wr);   // b * w
        a[i + k] = u + v;
        a[i + k + len / 2] = u - v;
      }
  }
}

bool is_pow2(long long v) { return v > 0 && (v & (v - 1)) == 0; }
int ilog2i(long long v) { int l = 0; while ((1LL << l) < v) ++l; return l; }

}  // namespace

// ---------------------------------------------------------------------------------------------
struct bltt_ctx {
  struct Pending { const char* name; cudaEvent_t a, b; };
  int N = 0, d = 0, m[3] = {1, 1, 1};
  long long M = 0, n = 0;
  double h[3] = {1, 1, 1};
  std::vector<double> a, b;
  double pc_bscale = 1.0;     // the preconditioner's blocks are a_k I + pc_bscale b_k L (abar)
  bool var_coef = false;      // the matvec's L is L_a = -Delta_{a,h} (faces in op.kf)
  bool dense = false;         // L is a dense symmetric K: eigenbasis U (dU, columns), op.mu_tab
  bool spectra = false;       // general commuting blocks given by U and their eigenvalues (lam)
  std::vector<double> lam;    // [k][i] eigenvalues of the blocks (spectra), kept for the per-alpha set-up
  int spectra_b_kind = 0, spectra_ntaps = 0;   // the op fields the blocks a, b gave
  double* dU = nullptr;
  float* dUp[4] = {nullptr, nullptr, nullptr, nullptr};   // double-float planes: U hi, lo; U^T hi, lo
  cublasHandle_t blas = nullptr;
  cudaStream_t stream = nullptr;
  std::string err;
  OpTables op{};
  // owned device allocations
  std::vector<void*> allocs;
  // workspace
  double* ws = nullptr;          // 10 vectors of n doubles
  size_t ws_vectors = 0;
  double* partials[2] = {nullptr, nullptr};
  MinresDev* state = nullptr;
  MinresDev* state_host = nullptr;   // pinned
  double* scal = nullptr;            // device scalar scratch
  double* scal_host = nullptr;       // pinned
  // per-alpha preconditioner cache
  double pc_alpha = -1.0;
  bool pc_has64 = false, pc_has32 = false;
  double* pc_dinv = nullptr;
  double* pc_d2 = nullptr;
  float* pc_dinv32 = nullptr;
  float* pc_d232 = nullptr;
  float2* pc_dinv_df = nullptr;
  float2* pc_d2_df = nullptr;
  float4* pc_gdf = nullptr;
  float4* pc_ahatdf = nullptr;
  float4* pc_bhatdf = nullptr;
  bool pc_hasdf = false;
  double2* pc_g64 = nullptr;
  float2* pc_g32 = nullptr;    // general commuting blocks: the FP32 time pass reads a table too
  float2* pc_ahat32 = nullptr;
  float2* pc_bhat32 = nullptr;
  double2* pc_ahat64 = nullptr;
  double2* pc_bhat64 = nullptr;
  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
  long long launches = 0;
  // cached CUDA graph of the MINRES iterations and the key it was captured for; when captured
  // with profiling on, its event-record nodes (graph_prof) are read after every replay
  cudaGraphExec_t gexec = nullptr;
  const void* gkey[14] = {nullptr};
  std::vector<Pending> graph_prof;
  // with a deferred-update window, the window's iteration blocks have graphs of their own (their
  // z slots differ from block to block); gexec above serves the iterations after the window
  struct WinGraph { cudaGraphExec_t exec = nullptr; std::vector<Pending> prof; };
  std::vector<WinGraph> win_graphs;
  // the window's z slots beyond the two of the workspace (S - 1 vectors of n doubles)
  double* win_ws = nullptr;
  int win_vectors = 0;
  size_t guard = 0;   // doubles of each guard band (0: none)
  int ahead_blocks = 0;   // graph blocks the last solve needed: the next one's first burst
  bool capturing = false;
  // per-launch profiling
  bool prof = false;
  std::vector<cudaEvent_t> ev_pool;
  size_t ev_used = 0;
  std::vector<Pending> pending;
  // per kernel family: every launch's duration, so that "active" (longer than a quarter of the
  // family's longest launch) is decided against the final maximum when the counters are read
  struct Stat { long long launches = 0; double ms = 0; double max_ms = 0; std::vector<float> each; };
  std::map<std::string, Stat> stats;
  // host-buffer solves: device staging of f and u, a copy stream and its event
  double* io_f = nullptr;
  double* io_u = nullptr;
  // iterative refinement: the residual and the correction
  double* ir_r = nullptr;
  double* ir_d = nullptr;
  cudaStream_t io_stream = nullptr;
  cudaEvent_t io_ev = nullptr;
  cudaEvent_t io_chunk_ev[4] = {nullptr, nullptr, nullptr, nullptr};

  ~bltt_ctx() {
    if (stream_sync_ok) cudaStreamSynchronize(stream);
    if (io_stream) { cudaStreamSynchronize(io_stream); cudaStreamDestroy(io_stream); }
    if (io_ev) cudaEventDestroy(io_ev);
    if (blas) cublasDestroy(blas);
    for (cudaEvent_t e : io_chunk_ev)
      if (e) cudaEventDestroy(e);
    for (void* p : allocs) cudaFree(p);
    if (state_host) cudaFreeHost(state_host);
    if (scal_host) cudaFreeHost(scal_host);
    for (auto& e : ev) if (e) cudaEventDestroy(e);
    for (auto& e : ev_pool) cudaEventDestroy(e);
    if (gexec) cudaGraphExecDestroy(gexec);
    for (auto& p : graph_prof) { cudaEventDestroy(p.a); cudaEventDestroy(p.b); }
    for (auto& w : win_graphs) {
      if (w.exec) cudaGraphExecDestroy(w.exec);
      for (auto& p : w.prof) { cudaEventDestroy(p.a); cudaEventDestroy(p.b); }
    }
  }
  bool stream_sync_ok = true;

  template <typename T>
  cudaError_t alloc(T** p, size_t count) {
    void* q = nullptr;
    cudaError_t e = cudaMalloc(&q, std::max<size_t>(count, 1) * sizeof(T));
    if (e != cudaSuccess) { *p = nullptr; return e; }
    allocs.push_back(q);
    *p = reinterpret_cast<T*>(q);
    return cudaSuccess;
  }
  void release(void* p) {
    if (!p) return;
    auto it = std::find(allocs.begin(), allocs.end(), p);
    if (it != allocs.end()) { cudaFree(p); allocs.erase(it); }
  }
};

namespace {

// NVTX ranges of a solve's phases (visible under nsys / ncu; free when no tool is attached): a
// range started by start() ends at end() or when the holder goes out of scope
struct NvtxSpan {
  nvtxRangeId_t id = 0;
  bool open = false;
  NvtxSpan() = default;
  explicit NvtxSpan(const char* name) { start(name); }
  void start(const char* name) { end(); id = nvtxRangeStartA(name); open = true; }
  void end() { if (open) { nvtxRangeEnd(id); open = false; } }
  ~NvtxSpan() { end(); }
};

bltt_status fail(bltt_ctx* h, bltt_status s, const std::string& msg) {
  if (h) h->err = msg; else g_create_error = msg;
  return s;
}
bltt_status cuda_fail(bltt_ctx* h, cudaError_t e, const char* where) {
  bltt_status s = (e == cudaErrorMemoryAllocation) ? BLTT_ERR_OOM : BLTT_ERR_CUDA;
  return fail(h, s, std::string(where) + ": " + cudaGetErrorString(e));
}
#define CK(h, call, where)                                   \
  do {                                                       \
    cudaError_t e__ = (call);                                \
    if (e__ != cudaSuccess) return cuda_fail((h), e__, where); \
  } while (0)

cudaEvent_t prof_begin(bltt_ctx* h);
void prof_end(bltt_ctx* h, const char* name, cudaEvent_t a);
#define PCK(h, name, call, where)                            \
  do {                                                       \
    cudaEvent_t pa__ = prof_begin(h);                        \
    cudaError_t e__ = (call);                                \
    if (e__ != cudaSuccess) return cuda_fail((h), e__, where); \
    prof_end((h), (name), pa__);                             \
  } while (0)

template <typename T>
cudaError_t upload(bltt_ctx* h, T** dst, const T* src, size_t count) {
  cudaError_t e = h->alloc(dst, count);
  if (e != cudaSuccess) return e;
  return cudaMemcpy(*dst, src, count * sizeof(T), cudaMemcpyHostToDevice);
}

float4 split_df(double re, double im) {
  float rh = (float)re, ih = (float)im;
  return make_float4(rh, (float)(re - (double)rh), ih, (float)(im - (double)ih));
}

cudaError_t upload_df(bltt_ctx* h, const std::vector<double2>& src, const float4** dst) {
  std::vector<float4> v(src.size());
  for (size_t k = 0; k < src.size(); ++k) v[k] = split_df(src[k].x, src[k].y);
  float4* p;
  cudaError_t e = upload(h, &p, v.data(), v.size());
  *dst = p;
  return e;
}

cudaError_t upload_twiddles(bltt_ctx* h, int L, const double2** d64, const float2** d32) {
  const std::vector<double2>& tw = twiddles(L);
  std::vector<float2> tw32(L);
  for (int k = 0; k < L; ++k) tw32[k] = make_float2((float)tw[k].x, (float)tw[k].y);
  double2* p64;
  float2* p32;
  cudaError_t e = upload(h, &p64, tw.data(), L);
  if (e != cudaSuccess) return e;
  e = upload(h, &p32, tw32.data(), L);
  if (e != cudaSuccess) return e;
  *d64 = p64;
  if (d32) *d32 = p32;
  return cudaSuccess;
}

// ensure the tensor-core matvec workspace: digit planes, column exponents, the error flag
bltt_status ensure_tc(bltt_ctx* h) {
  if (h->var_coef || h->dense)
    return fail(h, BLTT_ERR_UNSUPPORTED, "the tensor-core matvec has no variable coefficient or dense operator");
  if (!tc_eligible(h->op) || !h->op.tc_hank)
    return fail(h, BLTT_ERR_UNSUPPORTED,
                "the tensor-core matvec needs b = b0 e_0, more than 4 nonzeros in a and N in "
                "{128, 256, 512, 1024}");
  if (h->op.tc_xd) return BLTT_OK;
  uint16_t* xd = nullptr;
  int *xe = nullptr, *err = nullptr;
  CK(h, h->alloc(&xd, tc_workspace_bytes(h->N, h->M) / sizeof(uint16_t)), "digit planes");
  CK(h, h->alloc(&xe, (size_t)tc_strips(h->M) * 128), "column exponents");
  CK(h, h->alloc(&err, 1), "error flag");
  CK(h, cudaMemset(err, 0, sizeof(int)), "error flag");
  h->op.tc_xd = xd;
  h->op.tc_xe = xe;
  h->op.tc_err = err;
  return BLTT_OK;
}

// basis changes of the dense-operator form: out = (I (x) U^T) in (to the eigenbasis) or
// out = (I (x) U) in; a time-major vector is a column-major M x N matrix.  FP64 GEMM (cuBLAS), or
// with df the double-float GEMM on the FP32 pipes (the precision of the double-float matvec)
bltt_status eigen_transform(bltt_ctx* h, const double* in, double* out, bool to_eigen, bool df) {
  const double one = 1.0, zero = 0.0;
  const int M = (int)h->M;
  if (df) {
    cudaEvent_t pa = prof_begin(h);
    const float* Ah = to_eigen ? h->dUp[2] : h->dUp[0];
    const float* Al = to_eigen ? h->dUp[3] : h->dUp[1];
    CK(h, launch_df_gemm(Ah, Al, in, out, M, h->N, h->stream), "double-float basis change");
    prof_end(h, "basis_gemm_df", pa);
    h->launches++;
    return BLTT_OK;
  }
  cudaEvent_t pa = prof_begin(h);
  if (cublasSetStream(h->blas, h->stream) != CUBLAS_STATUS_SUCCESS ||
      cublasDgemm(h->blas, to_eigen ? CUBLAS_OP_T : CUBLAS_OP_N, CUBLAS_OP_N, M, h->N, M, &one,
                  h->dU, M, in, M, &zero, out, M) != CUBLAS_STATUS_SUCCESS)
    return fail(h, BLTT_ERR_CUDA, "cuBLAS basis change failed");
  prof_end(h, "basis_gemm", pa);
  h->launches++;
  return BLTT_OK;
}

// guard bands (BLTT_GUARD_BANDS=1 in the environment when the workspace is first allocated): a
// band of kGuard doubles with a fixed bit pattern before, between and after the workspace vectors
// and the window slots; bltt_check_guards reports a band that a kernel wrote into
constexpr size_t kGuard = 256;                        // 2 KB: vectors stay 16-byte aligned
constexpr uint64_t kGuardBits = 0x7FF4C0FFEEC0FFEEull;  // a NaN no kernel writes
size_t guard_of(bltt_ctx* h) {
  if (!h->ws && !h->win_ws) {
    const char* e = std::getenv("BLTT_GUARD_BANDS");
    h->guard = (e && std::atoi(e) > 0) ? kGuard : 0;
  }
  return h->guard;
}
// fill the nvec + 1 bands of a region of nvec vectors
cudaError_t fill_guards(bltt_ctx* h, double* base, size_t nvec) {
  if (!h->guard) return cudaSuccess;
  std::vector<uint64_t> pat(h->guard, kGuardBits);
  for (size_t k = 0; k <= nvec; ++k) {
    cudaError_t e = cudaMemcpy(base + k * (h->n + h->guard), pat.data(), h->guard * 8,
                               cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// ensure the solve workspace: 10 vectors of n doubles, partial sums, device scalar state
bltt_status ensure_workspace(bltt_ctx* h) {
  if (h->ws) return BLTT_OK;
  const size_t nv = 10;
  const size_t g = guard_of(h);
  CK(h, h->alloc(&h->ws, nv * ((size_t)h->n + g) + g + 2), "workspace allocation");
  CK(h, fill_guards(h, h->ws, nv), "guard bands");
  h->ws_vectors = nv;
  CK(h, h->alloc(&h->partials[0], (size_t)kMaxPartials), "partials");
  CK(h, h->alloc(&h->partials[1], (size_t)kMaxPartials), "partials");
  CK(h, h->alloc(&h->state, 1), "state");
  CK(h, h->alloc(&h->scal, 8), "scalars");
  if (!h->state_host) CK(h, cudaMallocHost(&h->state_host, sizeof(MinresDev)), "pinned state");
  if (!h->scal_host) CK(h, cudaMallocHost(&h->scal_host, 8 * sizeof(double)), "pinned scalars");
  return BLTT_OK;
}

double* vec(bltt_ctx* h, int k) { return h->ws + h->guard + (size_t)k * ((size_t)h->n + h->guard); }
// window slot j (0 .. win_vectors - 1)
double* win_vec(bltt_ctx* h, int j) {
  return h->win_ws + h->guard + (size_t)j * ((size_t)h->n + h->guard);
}

// every cached graph of the iterations (their kernel arguments changed, or their key did)
void drop_graphs(bltt_ctx* h) {
  if (h->gexec) { cudaGraphExecDestroy(h->gexec); h->gexec = nullptr; }
  for (auto& p : h->graph_prof) { cudaEventDestroy(p.a); cudaEventDestroy(p.b); }
  h->graph_prof.clear();
  for (auto& w : h->win_graphs) {
    if (w.exec) cudaGraphExecDestroy(w.exec);
    for (auto& p : w.prof) { cudaEventDestroy(p.a); cudaEventDestroy(p.b); }
  }
  h->win_graphs.clear();
}

// the deferred-update window's z slots beyond the workspace's two: S - 1 vectors, allocated once
// for the largest window asked for
bltt_status ensure_window(bltt_ctx* h, int S) {
  if (S - 1 <= h->win_vectors) return BLTT_OK;
  if (h->win_ws) {
    cudaStreamSynchronize(h->stream);
    h->release(h->win_ws);
    h->win_ws = nullptr;
    h->win_vectors = 0;
  }
  drop_graphs(h);
  const size_t g = guard_of(h);
  CK(h, h->alloc(&h->win_ws, (size_t)(S - 1) * ((size_t)h->n + g) + g), "deferred-update slots");
  CK(h, fill_guards(h, h->win_ws, (size_t)(S - 1)), "guard bands");
  h->win_vectors = S - 1;
  return BLTT_OK;
}

// General commuting blocks: per mode i the eigenvalues of the block alpha-circulant,
// lambda_i^(k,alpha) = FFT_N(D_alpha lam_i)_k (eq. hatcalphaieigvaldef), and the tables
// lambda^{-1/2}/(2N) (principal branch, Def. 2) over (k <= N/2, mode i) in FP64, double-float and
// FP32, built on the host for every precision at once (one FFT of length N per mode).
bltt_status prepare_spectra_tables(bltt_ctx* h, double alpha) {
  if (h->pc_has64 && h->pc_hasdf && h->pc_has32) return BLTT_OK;
  const int N = h->N, half = N / 2;
  const long long M = h->M;
  const size_t count = (size_t)(half + 1) * (size_t)M;
  std::vector<double2> g64(count);
  std::vector<float4> gdf(count);
  std::vector<float2> g32(count);
  std::vector<double> dj(N);
  for (int j = 0; j < N; ++j) dj[j] = std::pow(alpha, (double)j / N);
  const double sc = 0.5 / N;
  std::vector<cd> x(N);
  for (long long i = 0; i < M; ++i) {
    for (int j = 0; j < N; ++j) x[j] = cd(dj[j] * h->lam[(size_t)j * M + i], 0.0);
    host_fft(x);
    for (int k = 0; k <= half; ++k) {
      const cd g = sc / std::sqrt(x[k]);          // std::sqrt: the principal branch
      const size_t e = (size_t)k * M + i;
      g64[e] = make_double2(g.real(), g.imag());
      gdf[e] = split_df(g.real(), g.imag());
      g32[e] = make_float2((float)g.real(), (float)g.imag());
    }
  }
  if (!h->pc_g64) CK(h, h->alloc(&h->pc_g64, count), "alloc g64 table");
  if (!h->pc_gdf) CK(h, h->alloc(&h->pc_gdf, count), "alloc gdf table");
  if (!h->pc_g32) CK(h, h->alloc(&h->pc_g32, count), "alloc g32 table");
  CK(h, cudaMemcpyAsync(h->pc_g64, g64.data(), count * sizeof(double2), cudaMemcpyHostToDevice, h->stream), "copy g64");
  CK(h, cudaMemcpyAsync(h->pc_gdf, gdf.data(), count * sizeof(float4), cudaMemcpyHostToDevice, h->stream), "copy gdf");
  CK(h, cudaMemcpyAsync(h->pc_g32, g32.data(), count * sizeof(float2), cudaMemcpyHostToDevice, h->stream), "copy g32");
  CK(h, cudaStreamSynchronize(h->stream), "sync after table upload");   // host vectors die here
  h->pc_has64 = h->pc_hasdf = h->pc_has32 = true;
  return BLTT_OK;
}

// per-alpha tables: D_alpha scalings, ahat = FFT_N(D a), bhat = FFT_N(D b) and, for the FP64
// preconditioner, the table lambda^{-1/2}/(2N) over (k <= N/2, mode i)
bltt_status prepare_precond(bltt_ctx* h, double alpha, int prec) {
  const int N = h->N;
  if (h->pc_alpha != alpha) {
    h->pc_has64 = h->pc_has32 = h->pc_hasdf = false;
    std::vector<double> dinv(N), d2(N);
    std::vector<cd> ah(N), bh(N);
    for (int j = 0; j < N; ++j) {
      double dj = std::pow(alpha, (double)j / N);
      dinv[j] = 1.0 / dj;
      d2[j] = dj * dj;
      ah[j] = cd(dj * h->a[j], 0.0);
      bh[j] = cd(dj * h->b[j] * h->pc_bscale, 0.0);
    }
    host_fft(ah);
    host_fft(bh);
    if (!h->pc_dinv) {
      CK(h, h->alloc(&h->pc_dinv, N), "alloc dinv");
      CK(h, h->alloc(&h->pc_d2, N), "alloc d2");
      CK(h, h->alloc(&h->pc_dinv32, N), "alloc dinv32");
      CK(h, h->alloc(&h->pc_d232, N), "alloc d232");
      CK(h, h->alloc(&h->pc_dinv_df, N), "alloc dinv_df");
      CK(h, h->alloc(&h->pc_d2_df, N), "alloc d2_df");
      CK(h, h->alloc(&h->pc_ahat64, N / 2 + 1), "alloc ahat");
      CK(h, h->alloc(&h->pc_bhat64, N / 2 + 1), "alloc bhat");
      CK(h, h->alloc(&h->pc_ahat32, N / 2 + 1), "alloc ahat32");
      CK(h, h->alloc(&h->pc_bhat32, N / 2 + 1), "alloc bhat32");
      CK(h, h->alloc(&h->pc_ahatdf, N / 2 + 1), "alloc ahatdf");
      CK(h, h->alloc(&h->pc_bhatdf, N / 2 + 1), "alloc bhatdf");
    }
    std::vector<double2> a64(N / 2 + 1), b64(N / 2 + 1);
    std::vector<float2> a32(N / 2 + 1), b32(N / 2 + 1);
    std::vector<float4> adf(N / 2 + 1), bdf(N / 2 + 1);
    for (int k = 0; k <= N / 2; ++k) {
      a64[k] = make_double2(ah[k].real(), ah[k].imag());
      b64[k] = make_double2(bh[k].real(), bh[k].imag());
      a32[k] = make_float2((float)ah[k].real(), (float)ah[k].imag());
      b32[k] = make_float2((float)bh[k].real(), (float)bh[k].imag());
      adf[k] = split_df(ah[k].real(), ah[k].imag());
      bdf[k] = split_df(bh[k].real(), bh[k].imag());
    }
    CK(h, cudaMemcpyAsync(h->pc_ahatdf, adf.data(), adf.size() * sizeof(float4), cudaMemcpyHostToDevice, h->stream), "copy ahatdf");
    CK(h, cudaMemcpyAsync(h->pc_bhatdf, bdf.data(), bdf.size() * sizeof(float4), cudaMemcpyHostToDevice, h->stream), "copy bhatdf");
    std::vector<float> dinv32(N), d232(N);
    std::vector<float2> dinvdf(N), d2df(N);
    for (int j = 0; j < N; ++j) {
      dinv32[j] = (float)dinv[j];
      d232[j] = (float)d2[j];
      dinvdf[j] = make_float2(dinv32[j], (float)(dinv[j] - (double)dinv32[j]));
      d2df[j] = make_float2(d232[j], (float)(d2[j] - (double)d232[j]));
    }
    CK(h, cudaMemcpyAsync(h->pc_dinv_df, dinvdf.data(), N * sizeof(float2), cudaMemcpyHostToDevice, h->stream), "copy dinv_df");
    CK(h, cudaMemcpyAsync(h->pc_d2_df, d2df.data(), N * sizeof(float2), cudaMemcpyHostToDevice, h->stream), "copy d2_df");
    CK(h, cudaMemcpyAsync(h->pc_dinv32, dinv32.data(), N * sizeof(float), cudaMemcpyHostToDevice, h->stream), "copy dinv32");
    CK(h, cudaMemcpyAsync(h->pc_d232, d232.data(), N * sizeof(float), cudaMemcpyHostToDevice, h->stream), "copy d232");
    CK(h, cudaMemcpyAsync(h->pc_dinv, dinv.data(), N * sizeof(double), cudaMemcpyHostToDevice, h->stream), "copy dinv");
    CK(h, cudaMemcpyAsync(h->pc_d2, d2.data(), N * sizeof(double), cudaMemcpyHostToDevice, h->stream), "copy d2");
    CK(h, cudaMemcpyAsync(h->pc_ahat64, a64.data(), a64.size() * sizeof(double2), cudaMemcpyHostToDevice, h->stream), "copy ahat");
    CK(h, cudaMemcpyAsync(h->pc_bhat64, b64.data(), b64.size() * sizeof(double2), cudaMemcpyHostToDevice, h->stream), "copy bhat");
    CK(h, cudaMemcpyAsync(h->pc_ahat32, a32.data(), a32.size() * sizeof(float2), cudaMemcpyHostToDevice, h->stream), "copy ahat32");
    CK(h, cudaMemcpyAsync(h->pc_bhat32, b32.data(), b32.size() * sizeof(float2), cudaMemcpyHostToDevice, h->stream), "copy bhat32");
    // the host vectors die at return: wait for the copies
    CK(h, cudaStreamSynchronize(h->stream), "sync after table upload");
    h->pc_alpha = alpha;
  }
  if (h->spectra) return prepare_spectra_tables(h, alpha);
  // the FP32 time pass evaluates lambda^{-1/2} from ahat32 and bhat32 where it needs it: no table
  if (prec == PREC_F32) h->pc_has32 = true;
  if (prec == PREC_F64 && !h->pc_has64) {
    if (!h->pc_g64) CK(h, h->alloc(&h->pc_g64, (size_t)(N / 2 + 1) * h->M), "alloc g64 table");
    cudaEvent_t pa = prof_begin(h);
    CK(h, launch_setup_g64(h->op, h->pc_ahat64, h->pc_bhat64, h->pc_g64, nullptr, h->stream), "setup g64");
    prof_end(h, "setup_g", pa);
    h->launches++;
    h->pc_has64 = true;
  }
  if (prec == PREC_DF && !h->pc_hasdf) {
    if (!h->pc_gdf) CK(h, h->alloc(&h->pc_gdf, (size_t)(N / 2 + 1) * h->M), "alloc gdf table");
    cudaEvent_t pa = prof_begin(h);
    CK(h, launch_setup_gdf(h->op, h->pc_ahat32, h->pc_bhat32, h->pc_ahatdf, h->pc_bhatdf,
                           h->pc_gdf, h->stream), "setup gdf");
    prof_end(h, "setup_g", pa);
    h->launches++;
    h->pc_hasdf = true;
  }
  return BLTT_OK;
}

PrecTables prec_tables(bltt_ctx* h, int none) {
  PrecTables pt{};
  pt.alpha = h->pc_alpha;
  pt.dinv = h->pc_dinv;
  pt.d2 = h->pc_d2;
  pt.dinv32 = h->pc_dinv32;
  pt.d232 = h->pc_d232;
  pt.dinv_df = h->pc_dinv_df;
  pt.d2_df = h->pc_d2_df;
  pt.gdf = h->pc_gdf;
  pt.g64 = h->pc_g64;
  pt.ahat32 = h->pc_ahat32;
  pt.bhat32 = h->pc_bhat32;
  pt.g32 = h->spectra ? h->pc_g32 : nullptr;
  pt.none = none;
  return pt;
}

// z = P^{-1} (combined input), in the spectral basis (time pass only) or the physical basis
// (DST-I of every slice, time pass, inverse DST-I); fused dot with `dot_with` into partials.
bltt_status precond_chain(bltt_ctx* h, int spectral, int prec, const PrecTables& pt,
                          const Combine& in, double* out, const double* dot_with,
                          double* partials, int* nparts, const int* phase) {
  const OpTables& op = h->op;
  const char* tp_name = pt.none ? "identity" : (prec == PREC_F64 ? "timepass64" : prec == PREC_DF ? "timepass_df" : "timepass32");
  const char* dst_name = prec == PREC_F64 ? "dst64" : prec == PREC_DF ? "dst_df" : "dst32";
  if (pt.none || spectral) {
    cudaEvent_t pa = prof_begin(h);
    CK(h, launch_timepass(op, pt, prec, in, out, dot_with, partials, nparts, phase, h->stream), "time pass");
    prof_end(h, tp_name, pa);
    h->launches++;
    return BLTT_OK;
  }
  if (h->dense) {
    // Steps 1 and 3 as FP64 GEMMs with the eigenvectors (a plain input vector: bltt_precond_apply)
    if (in.in1 || in.in2 || in.vout || dot_with || partials)
      return fail(h, BLTT_ERR_UNSUPPORTED, "a dense operator solves in its eigenbasis");
    double* t1 = vec(h, 8);
    double* t2 = vec(h, 9);
    const bool df = (h->op.mv_arith == 1);
    bltt_status s = eigen_transform(h, in.in0, t1, true, df);
    if (s != BLTT_OK) return s;
    Combine c{};
    c.in0 = t1;
    cudaEvent_t pa = prof_begin(h);
    CK(h, launch_timepass(op, pt, prec, c, t2, nullptr, nullptr, nullptr, phase, h->stream), "time pass");
    prof_end(h, tp_name, pa);
    h->launches++;
    return eigen_transform(h, t2, out, false, df);
  }
  for (int ax = 0; ax < op.d; ++ax) {
    Combine c{};
    if (ax == 0) c = in; else c.in0 = out;
    cudaEvent_t pa = prof_begin(h);
    CK(h, launch_dst(op, ax, prec, c, out, 0, nullptr, nullptr, nullptr, phase, h->stream), "dst");
    prof_end(h, dst_name, pa);
    h->launches++;
  }
  Combine c{};
  c.in0 = out;
  cudaEvent_t pt0 = prof_begin(h);
  CK(h, launch_timepass(op, pt, prec, c, out, nullptr, nullptr, nullptr, phase, h->stream), "time pass");
  prof_end(h, tp_name, pt0);
  h->launches++;
  for (int ax = 0; ax < op.d; ++ax) {
    Combine c2{};
    c2.in0 = out;
    const bool last = (ax == op.d - 1);
    cudaEvent_t pa = prof_begin(h);
    CK(h, launch_dst(op, ax, prec, c2, out, 0, last ? dot_with : nullptr, last ? partials : nullptr,
                     last ? nparts : nullptr, phase, h->stream), "dst");
    prof_end(h, dst_name, pa);
    h->launches++;
  }
  return BLTT_OK;
}

// out = (I (x) U) in, optionally time-reversed (first pass out of place), with ||out||^2 partials
bltt_status dst_all(bltt_ctx* h, const OpTables& op, const double* in, double* out, int flip,
                    double* partials, int* nparts) {
  const int arith = op.mv_arith ? PREC_DF : PREC_F64;
  for (int ax = 0; ax < op.d; ++ax) {
    Combine c{};
    c.in0 = (ax == 0) ? in : out;
    const bool last = (ax == op.d - 1);
    cudaEvent_t pa = prof_begin(h);
    CK(h, launch_dst(op, ax, arith, c, out, ax == 0 ? flip : 0, last && partials ? out : nullptr,
                     last ? partials : nullptr, last ? nparts : nullptr, nullptr, h->stream), "dst");
    prof_end(h, arith == PREC_DF ? "dst_df" : "dst64", pa);
    h->launches++;
  }
  return BLTT_OK;
}

const char* mv_name(const OpTables& op, int mode = MV_STORE) {
  if (op.ntaps > 0) return mode == MV_RESID ? "direct_resid" : "direct";
  if (op.mv_arith == 2 && mode == MV_STORE) return "conv_tc";
  return op.mv_arith ? "conv_df" : "conv";
}

cudaEvent_t prof_event(bltt_ctx* h) {
  if (h->capturing) {
    cudaEvent_t e;
    return cudaEventCreate(&e) == cudaSuccess ? e : nullptr;
  }
  if (h->ev_used == h->ev_pool.size()) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    h->ev_pool.push_back(e);
  }
  return h->ev_pool[h->ev_used++];
}

// record an event before a launch when profiling (returns null otherwise)
// during stream capture an event must be recorded as an external node to be timed at replay
void prof_record(bltt_ctx* h, cudaEvent_t e) {
  if (h->capturing) cudaEventRecordWithFlags(e, h->stream, cudaEventRecordExternal);
  else cudaEventRecord(e, h->stream);
}
cudaEvent_t prof_begin(bltt_ctx* h) {
  if (!h->prof) return nullptr;
  cudaEvent_t a = prof_event(h);
  if (a) prof_record(h, a);
  return a;
}
void prof_end(bltt_ctx* h, const char* name, cudaEvent_t a) {
  if (!h->prof || !a) return;
  cudaEvent_t b = prof_event(h);
  if (!b) return;
  prof_record(h, b);
  h->pending.push_back({name, a, b});
}
// accumulate the event pairs of the last graph replay (the caller has synchronised)
void prof_harvest_graph(bltt_ctx* h, const std::vector<bltt_ctx::Pending>& gp) {
  std::vector<float> ms(gp.size(), -1.f);
  for (size_t i = 0; i < gp.size(); ++i)
    if (cudaEventElapsedTime(&ms[i], gp[i].a, gp[i].b) != cudaSuccess) ms[i] = -1.f;
  for (size_t i = 0; i < gp.size(); ++i) {
    if (ms[i] < 0.f) continue;
    auto& st = h->stats[gp[i].name];
    st.launches += 1;
    st.ms += ms[i];
    st.max_ms = std::max(st.max_ms, (double)ms[i]);
    st.each.push_back(ms[i]);
  }
  (void)cudaGetLastError();   // a failed timing query must not surface at the next launch check
}

void prof_harvest(bltt_ctx* h) {
  if (h->pending.empty()) { h->ev_used = 0; return; }
  cudaStreamSynchronize(h->stream);
  std::vector<float> ms(h->pending.size(), 0.f);
  for (size_t i = 0; i < h->pending.size(); ++i)
    if (cudaEventElapsedTime(&ms[i], h->pending[i].a, h->pending[i].b) != cudaSuccess) ms[i] = -1.f;
  for (size_t i = 0; i < h->pending.size(); ++i) {
    if (ms[i] < 0.f) continue;
    auto& st = h->stats[h->pending[i].name];
    st.launches += 1;
    st.ms += ms[i];
    st.max_ms = std::max(st.max_ms, (double)ms[i]);
    st.each.push_back(ms[i]);
  }
  h->pending.clear();
  h->ev_used = 0;
  (void)cudaGetLastError();
}

}  // namespace

namespace bltt {
const OpTables& ctx_op(bltt_handle h) { return h->op; }
bltt_status ctx_prepare(bltt_handle h, double alpha, int prec) { return prepare_precond(h, alpha, prec); }
PrecTables ctx_prec_tables(bltt_handle h) { return prec_tables(h, 0); }
long long ctx_n(bltt_handle h) { return h->n; }
}  // namespace bltt

// =============================================================================================
extern "C" {

const char* bltt_version(void) { return "bltt-gb300 0.1 (sm_103a)"; }

const char* bltt_last_error(bltt_handle h) {
  return h ? h->err.c_str() : g_create_error.c_str();
}

bltt_status bltt_create(const bltt_blocks* blocks, int N, long long M, bltt_handle* out) {
  if (out) *out = nullptr;
  if (!blocks || !out || !blocks->a || !blocks->b)
    return fail(nullptr, BLTT_ERR_INVALID_ARG, "null argument");
  if (blocks->N != N || N < 2)
    return fail(nullptr, BLTT_ERR_INVALID_ARG, "N mismatch or N < 2");
  const bltt_space& sp = blocks->space;
  if (sp.ndim < 1 || sp.ndim > 3) return fail(nullptr, BLTT_ERR_INVALID_ARG, "ndim must be 1, 2 or 3");
  long long prodm = 1;
  for (int ax = 0; ax < sp.ndim; ++ax) {
    if (sp.m[ax] < 1 || !(sp.h[ax] > 0.0) || !std::isfinite(sp.h[ax]))
      return fail(nullptr, BLTT_ERR_INVALID_ARG, "bad m or h");
    prodm *= sp.m[ax];
  }
  if (prodm != M) return fail(nullptr, BLTT_ERR_INVALID_ARG, "M != prod(m)");
  // every FFT must fit one tile: 2N (matvec) and 2(m+1) (DST) <= kCap points
  if (!is_pow2(N) || 2 * N > kCap) return fail(nullptr, BLTT_ERR_UNSUPPORTED, "N must be a power of two <= 2048");
  for (int ax = 0; ax < sp.ndim; ++ax)
    if (!is_pow2(sp.m[ax] + 1) || 2 * (sp.m[ax] + 1) > kCap)
      return fail(nullptr, BLTT_ERR_UNSUPPORTED, "m+1 must be a power of two <= 2048");
  for (int k = 0; k < N; ++k)
    if (!std::isfinite(blocks->a[k]) || !std::isfinite(blocks->b[k]))
      return fail(nullptr, BLTT_ERR_NUMERIC, "non-finite block coefficient");

  bltt_ctx* h = new bltt_ctx();
  h->N = N; h->d = sp.ndim; h->M = M; h->n = (long long)N * M;
  for (int ax = 0; ax < 3; ++ax) { h->m[ax] = ax < sp.ndim ? sp.m[ax] : 1; h->h[ax] = ax < sp.ndim ? sp.h[ax] : 1.0; }
  h->a.assign(blocks->a, blocks->a + N);
  h->b.assign(blocks->b, blocks->b + N);

  // per-axis eigenvalues of L: (4/h^2) sin^2(pi (k+1) / (2(m+1)))
  std::vector<std::vector<double>> mu(3);
  double mu_min = 0.0, mu_max = 0.0;
  for (int ax = 0; ax < sp.ndim; ++ax) {
    mu[ax].resize(h->m[ax]);
    for (int k = 0; k < h->m[ax]; ++k) {
      long double s = sinl(3.141592653589793238462643383279502884L * (k + 1) / (2.0L * (h->m[ax] + 1)));
      mu[ax][k] = (double)(4.0L / ((long double)h->h[ax] * h->h[ax]) * s * s);
    }
    mu_min += mu[ax].front();
    mu_max += mu[ax].back();
  }
  // Assumption 1 (ii): c0(mu) = a0 + b0 mu - sum_k |a_k + b_k mu| is concave in mu, so its minimum
  // over [mu_min, mu_max] sits at an end point.
  auto c0_at = [&](double muv) {
    double v = h->a[0] + h->b[0] * muv;
    for (int k = 1; k < N; ++k) v -= std::fabs(h->a[k] + h->b[k] * muv);
    return v;
  };
  const double c0 = std::min(c0_at(mu_min), c0_at(mu_max));
  if (!(c0 > 0.0)) {
    char buf[160];
    snprintf(buf, sizeof buf, "Assumption 1 (ii) fails: c0 = %.6g <= 0", c0);
    delete h;
    return fail(nullptr, BLTT_ERR_ASSUMPTION, buf);
  }

  OpTables& op = h->op;
  op.N = N; op.log2N = ilog2i(N); op.d = h->d; op.M = M;
  for (int ax = 0; ax < 3; ++ax) { op.m[ax] = h->m[ax]; op.h2inv[ax] = 1.0 / (h->h[ax] * h->h[ax]); }
  cudaError_t e = cudaSuccess;
  for (int ax = 0; ax < h->d && e == cudaSuccess; ++ax) {
    double* p;
    e = upload(h, &p, mu[ax].data(), mu[ax].size());
    op.mu_axis[ax] = p;
    std::vector<float> m32(mu[ax].begin(), mu[ax].end());
    float* q;
    if (e == cudaSuccess) e = upload(h, &q, m32.data(), m32.size());
    op.mu_axis32[ax] = q;
  }
  // matvec spectra FFT_2N([a;0]) / (2N), FFT_2N([b;0]) / (2N), k = 0..N
  std::vector<cd> A2(2 * N, cd(0, 0)), B2(2 * N, cd(0, 0));
  for (int k = 0; k < N; ++k) { A2[k] = cd(h->a[k], 0); B2[k] = cd(h->b[k], 0); }
  host_fft(A2);
  host_fft(B2);
  std::vector<double2> Ah(N + 1), Bh(N + 1);
  for (int k = 0; k <= N; ++k) {
    Ah[k] = make_double2(A2[k].real() / (2.0 * N), A2[k].imag() / (2.0 * N));
    Bh[k] = make_double2(B2[k].real() / (2.0 * N), B2[k].imag() / (2.0 * N));
  }
  double2 *pA = nullptr, *pB = nullptr;
  if (e == cudaSuccess) e = upload(h, &pA, Ah.data(), Ah.size());
  if (e == cudaSuccess) e = upload(h, &pB, Bh.data(), Bh.size());
  op.Ahat = pA; op.Bhat = pB;
  // b = b0 e_0 ?
  bool b_e0 = true;
  for (int k = 1; k < N; ++k) if (h->b[k] != 0.0) b_e0 = false;
  op.b_kind = b_e0 ? 0 : 1;
  op.b0 = h->b[0];
  int last_nz = 0;
  for (int k = 0; k < N; ++k) if (h->a[k] != 0.0 || h->b[k] != 0.0) last_nz = k;
  op.ntaps = (last_nz < 4) ? last_nz + 1 : 0;
  double *pa = nullptr, *pb = nullptr;
  if (e == cudaSuccess) e = upload(h, &pa, h->a.data(), N);
  if (e == cudaSuccess) e = upload(h, &pb, h->b.data(), N);
  op.a_dev = pa; op.b_dev = pb;
  if (e == cudaSuccess) e = upload_twiddles(h, 2 * N, &op.tw_2N, nullptr);
  if (e == cudaSuccess) e = upload_df(h, Ah, &op.Ahat_df);
  if (e == cudaSuccess) e = upload_df(h, Bh, &op.Bhat_df);
  if (e == cudaSuccess) {
    const std::vector<double2>& tw = twiddles(2 * N);
    e = upload_df(h, tw, &op.tw_2N_df);
  }
  op.mv_arith = 0;
  // tensor-core time product: digit planes of the time-flipped a (when the problem qualifies)
  if (e == cudaSuccess && tc_eligible(op)) {
    int eT = 0, nc = 0;
    std::vector<uint16_t> hank((size_t)kTcDigits * (16 * (N / 128) + 15) * 64);
    tc_hankel_digits(h->a.data(), N, hank.data(), &eT, &nc);
    if (eT >= -60 && eT <= 60) {
      uint16_t* ph = nullptr;
      e = upload(h, &ph, hank.data(), hank.size());
      op.tc_hank = ph;
      op.tc_eT = eT;
      op.tc_ncores = nc;
    }
  }
  if (e == cudaSuccess) e = upload_twiddles(h, N, &op.tw_N, &op.tw_N32);
  if (e == cudaSuccess) {
    const std::vector<double2>& tw = twiddles(N);
    e = upload_df(h, tw, &op.tw_N_df);
  }
  for (int ax = 0; ax < h->d && e == cudaSuccess; ++ax) {
    e = upload_twiddles(h, 2 * (h->m[ax] + 1), &op.tw_dst[ax], &op.tw_dst32[ax]);
    if (e == cudaSuccess) {
      e = upload_df(h, twiddles(2 * (h->m[ax] + 1)), &op.tw_dst_df[ax]);
    }
  }
  for (int i = 0; i < 4 && e == cudaSuccess; ++i) e = cudaEventCreate(&h->ev[i]);
  if (e == cudaSuccess) e = prepare_kernel_attributes();
  if (e != cudaSuccess) {
    bltt_status s = (e == cudaErrorMemoryAllocation) ? BLTT_ERR_OOM : BLTT_ERR_CUDA;
    std::string msg = std::string("bltt_create: ") + cudaGetErrorString(e);
    h->stream_sync_ok = false;
    delete h;
    return fail(nullptr, s, msg);
  }
  *out = h;
  return BLTT_OK;
}

bltt_status bltt_destroy(bltt_handle h) {
  if (!h) return BLTT_OK;
  delete h;
  return BLTT_OK;
}

namespace {
// release the handle's eigenbasis and its tables (a dense operator's or general blocks'), so
// that a new one can take their place; the blocks then read a, b again
void drop_eigenbasis(bltt_ctx* h) {
  if (!h->dense) return;
  h->release(h->dU);
  h->dU = nullptr;
  h->release(const_cast<double*>(h->op.mu_tab));
  h->release(const_cast<float*>(h->op.mu_tab32));
  h->op.mu_tab = nullptr;
  h->op.mu_tab32 = nullptr;
  for (float*& q : h->dUp) { h->release(q); q = nullptr; }
  if (h->spectra) {
    h->release(const_cast<double2*>(h->op.Hm64));
    h->release(const_cast<float4*>(h->op.Hmdf));
    h->op.Hm64 = nullptr;
    h->op.Hmdf = nullptr;
    h->op.b_kind = h->spectra_b_kind;
    h->op.ntaps = h->spectra_ntaps;
    h->lam.clear();
    h->spectra = false;
  }
  h->dense = false;
}
}  // namespace

bltt_status bltt_set_dense_operator(bltt_handle h, const double* K) {
  if (!h) return BLTT_ERR_INVALID_ARG;
  if (!K) return fail(h, BLTT_ERR_INVALID_ARG, "null operator");
  if (h->var_coef) return fail(h, BLTT_ERR_UNSUPPORTED, "a variable coefficient is set on this handle");
  if (h->op.mv_arith == 2) return fail(h, BLTT_ERR_UNSUPPORTED, "the tensor-core matvec has no dense operator");
  const long long M = h->M;
  if (M > 8192) return fail(h, BLTT_ERR_UNSUPPORTED, "a dense operator needs M <= 8192");
  double kmax = 0.0;
  for (long long e = 0; e < M * M; ++e) {
    if (!std::isfinite(K[e])) return fail(h, BLTT_ERR_INVALID_ARG, "the operator must be finite");
    kmax = std::max(kmax, std::fabs(K[e]));
  }
  for (long long i = 0; i < M; ++i)
    for (long long j = 0; j < i; ++j)
      if (std::fabs(K[i * M + j] - K[j * M + i]) > 1e-12 * kmax)
        return fail(h, BLTT_ERR_INVALID_ARG, "the operator must be symmetric");
  // eigendecomposition on the device: K = U diag(mu) U^T (cuSOLVER, set-up only)
  double* dU = nullptr;
  double* dmu = nullptr;
  CK(h, h->alloc(&dU, (size_t)(M * M)), "eigenvectors");
  CK(h, h->alloc(&dmu, (size_t)M), "eigenvalues");
  CK(h, cudaMemcpy(dU, K, sizeof(double) * M * M, cudaMemcpyHostToDevice), "copy operator");
  cusolverDnHandle_t sol = nullptr;
  if (cusolverDnCreate(&sol) != CUSOLVER_STATUS_SUCCESS)
    return fail(h, BLTT_ERR_CUDA, "cuSOLVER handle");
  int lwork = 0;
  cusolverStatus_t cs = cusolverDnDsyevd_bufferSize(sol, CUSOLVER_EIG_MODE_VECTOR,
                                                    CUBLAS_FILL_MODE_LOWER, (int)M, dU, (int)M,
                                                    dmu, &lwork);
  double* work = nullptr;
  int* dinfo = nullptr;
  cudaError_t ce = cudaSuccess;
  if (cs == CUSOLVER_STATUS_SUCCESS) ce = cudaMalloc(&work, sizeof(double) * (size_t)std::max(lwork, 1));
  if (cs == CUSOLVER_STATUS_SUCCESS && ce == cudaSuccess) ce = cudaMalloc(&dinfo, sizeof(int));
  if (cs == CUSOLVER_STATUS_SUCCESS && ce == cudaSuccess)
    cs = cusolverDnDsyevd(sol, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, (int)M, dU,
                          (int)M, dmu, work, lwork, dinfo);
  int info = -1;
  if (cs == CUSOLVER_STATUS_SUCCESS && ce == cudaSuccess)
    ce = cudaMemcpy(&info, dinfo, sizeof(int), cudaMemcpyDeviceToHost);
  cudaFree(work);
  cudaFree(dinfo);
  cusolverDnDestroy(sol);
  // on any failure below the handle keeps its previous operator
  struct Drop {
    bltt_ctx* hh; void* p[7]; bool keep = false;
    ~Drop() { if (!keep) for (void* q : p) hh->release(q); }
  } drop{h, {dU, dmu, nullptr, nullptr, nullptr, nullptr, nullptr}};
  if (cs != CUSOLVER_STATUS_SUCCESS || ce != cudaSuccess || info != 0)
    return fail(h, BLTT_ERR_CUDA, "cuSOLVER eigendecomposition failed");
  std::vector<double> mu(M);
  CK(h, cudaMemcpy(mu.data(), dmu, sizeof(double) * M, cudaMemcpyDeviceToHost), "eigenvalues");
  // Assumption 1 (ii) on the new eigenvalues
  double c0 = 1e300;
  for (long long i = 0; i < M; ++i) {
    double v = h->a[0] + h->b[0] * mu[i];
    for (int k = 1; k < h->N; ++k) v -= std::fabs(h->a[k] + h->b[k] * mu[i]);
    c0 = std::min(c0, v);
  }
  if (!(c0 > 0.0)) return fail(h, BLTT_ERR_ASSUMPTION, "Assumption 1 (ii) fails for the operator's eigenvalues");
  std::vector<float> mu32(mu.begin(), mu.end());
  float* dmu32 = nullptr;
  CK(h, upload(h, &dmu32, mu32.data(), (size_t)M), "eigenvalues");
  drop.p[2] = dmu32;
  // double-float planes of U and U^T for the FP32-pipe basis changes
  float* planes[4] = {nullptr, nullptr, nullptr, nullptr};
  for (int k = 0; k < 4; ++k) {
    CK(h, h->alloc(&planes[k], (size_t)(M * M)), "eigenvector planes");
    drop.p[3 + k] = planes[k];
  }
  CK(h, launch_df_planes(dU, M, planes[0], planes[1], planes[2], planes[3], nullptr), "planes");
  CK(h, cudaDeviceSynchronize(), "planes");
  if (!h->blas && cublasCreate(&h->blas) != CUBLAS_STATUS_SUCCESS)
    return fail(h, BLTT_ERR_CUDA, "cuBLAS handle");
  drop.keep = true;
  drop_eigenbasis(h);
  for (int k = 0; k < 4; ++k) h->dUp[k] = planes[k];
  h->dU = dU;
  h->op.mu_tab = dmu;
  h->op.mu_tab32 = dmu32;
  h->dense = true;
  h->pc_alpha = -1.0;
  drop_graphs(h);
  return BLTT_OK;
}

bltt_status bltt_set_block_spectra(bltt_handle h, const double* U, const double* lam) {
  if (!h) return BLTT_ERR_INVALID_ARG;
  if (!U || !lam) return fail(h, BLTT_ERR_INVALID_ARG, "null eigenvectors or eigenvalues");
  if (h->var_coef) return fail(h, BLTT_ERR_UNSUPPORTED, "a variable coefficient is set on this handle");
  if (h->op.mv_arith == 2) return fail(h, BLTT_ERR_UNSUPPORTED, "the tensor-core matvec has no general blocks");
  const long long M = h->M;
  const int N = h->N;
  if (M > 8192) return fail(h, BLTT_ERR_UNSUPPORTED, "general commuting blocks need M <= 8192");
  for (long long e = 0; e < M * M; ++e)
    if (!std::isfinite(U[e])) return fail(h, BLTT_ERR_INVALID_ARG, "U must be finite");
  for (long long e = 0; e < (long long)N * M; ++e)
    if (!std::isfinite(lam[e])) return fail(h, BLTT_ERR_INVALID_ARG, "the eigenvalues must be finite");
  // orthonormal columns, probed with two fixed vectors: ||U^T (U x) - x|| <= 1e-10 ||x||
  {
    std::vector<double> x(M), y(M), z(M);
    uint64_t st = 0x9E3779B97F4A7C15ull;
    for (int probe = 0; probe < 2; ++probe) {
      double nx = 0.0;
      for (long long i = 0; i < M; ++i) {
        st = st * 6364136223846793005ull + 1442695040888963407ull;
        x[i] = (double)(st >> 11) * 0x1.0p-53 - 0.5;
        nx += x[i] * x[i];
      }
      for (long long r = 0; r < M; ++r) {
        double acc = 0.0;
        for (long long c = 0; c < M; ++c) acc += U[r * M + c] * x[c];
        y[r] = acc;
      }
      double err = 0.0;
      for (long long c = 0; c < M; ++c) {
        double acc = 0.0;
        for (long long r = 0; r < M; ++r) acc += U[r * M + c] * y[r];
        err += (acc - x[c]) * (acc - x[c]);
      }
      if (!(std::sqrt(err) <= 1e-10 * std::sqrt(nx)))
        return fail(h, BLTT_ERR_INVALID_ARG, "U must have orthonormal columns");
    }
  }
  // Assumption 1 (ii) on the blocks' eigenvalues (Proposition after Lemma 3.1)
  double c0 = 1e300;
  for (long long i = 0; i < M; ++i) {
    double v = lam[i];
    for (int k = 1; k < N; ++k) v -= std::fabs(lam[(size_t)k * M + i]);
    c0 = std::min(c0, v);
  }
  if (!(c0 > 0.0)) return fail(h, BLTT_ERR_ASSUMPTION, "Assumption 1 (ii) fails for the blocks' eigenvalues");
  // per-mode matvec spectra FFT_2N([lam_i; 0]) / (2N), k = 0..N (Sec. 5.1, the 2N embedding)
  const size_t cnt = (size_t)(N + 1) * (size_t)M;
  std::vector<double2> H64(cnt);
  std::vector<float4> Hdf(cnt);
  {
    std::vector<cd> x(2 * N);
    const double inv = 1.0 / (2.0 * N);
    for (long long i = 0; i < M; ++i) {
      for (int j = 0; j < 2 * N; ++j) x[j] = cd(j < N ? lam[(size_t)j * M + i] : 0.0, 0.0);
      host_fft(x);
      for (int k = 0; k <= N; ++k) {
        const size_t e = (size_t)k * M + i;
        H64[e] = make_double2(x[k].real() * inv, x[k].imag() * inv);
        Hdf[e] = split_df(H64[e].x, H64[e].y);
      }
    }
  }
  // U on the device, column-major (column i = mode i), and its double-float planes
  std::vector<double> Ucm((size_t)M * M);
  for (long long r = 0; r < M; ++r)
    for (long long c = 0; c < M; ++c) Ucm[(size_t)c * M + r] = U[r * M + c];
  double* dU = nullptr;
  double2* dH64 = nullptr;
  float4* dHdf = nullptr;
  float* planes[4] = {nullptr, nullptr, nullptr, nullptr};
  struct Drop {
    bltt_ctx* hh; void* p[7]; bool keep = false;
    ~Drop() { if (!keep) for (void* q : p) hh->release(q); }
  } drop{h, {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr}};
  CK(h, upload(h, &dU, Ucm.data(), Ucm.size()), "eigenvectors");
  drop.p[0] = dU;
  CK(h, upload(h, &dH64, H64.data(), cnt), "matvec spectra");
  drop.p[1] = dH64;
  CK(h, upload(h, &dHdf, Hdf.data(), cnt), "matvec spectra");
  drop.p[2] = dHdf;
  for (int k = 0; k < 4; ++k) {
    CK(h, h->alloc(&planes[k], (size_t)(M * M)), "eigenvector planes");
    drop.p[3 + k] = planes[k];
  }
  CK(h, launch_df_planes(dU, M, planes[0], planes[1], planes[2], planes[3], nullptr), "planes");
  CK(h, cudaDeviceSynchronize(), "planes");
  if (!h->blas && cublasCreate(&h->blas) != CUBLAS_STATUS_SUCCESS)
    return fail(h, BLTT_ERR_CUDA, "cuBLAS handle");
  drop.keep = true;
  drop_eigenbasis(h);
  h->spectra_b_kind = h->op.b_kind;
  h->spectra_ntaps = h->op.ntaps;
  for (int k = 0; k < 4; ++k) h->dUp[k] = planes[k];
  h->dU = dU;
  h->op.Hm64 = dH64;
  h->op.Hmdf = dHdf;
  h->op.b_kind = 1;          // no common spectrum: every mode has its own
  h->op.ntaps = 0;           // always the FFT product
  h->lam.assign(lam, lam + (size_t)N * M);
  h->dense = true;           // the solve runs in U's basis, as for a dense operator
  h->spectra = true;
  h->pc_alpha = -1.0;
  drop_graphs(h);
  return BLTT_OK;
}

bltt_status bltt_set_variable_coefficient(bltt_handle h, const double* const* face, double abar) {
  if (!h) return BLTT_ERR_INVALID_ARG;
  if (h->dense) return fail(h, BLTT_ERR_UNSUPPORTED, "a dense operator is set on this handle");
  if (!face) return fail(h, BLTT_ERR_INVALID_ARG, "null face array");
  if (!(abar > 0.0) || !std::isfinite(abar)) return fail(h, BLTT_ERR_INVALID_ARG, "abar must be positive");
  if (h->op.mv_arith == 2) return fail(h, BLTT_ERR_UNSUPPORTED, "the tensor-core matvec has no variable coefficient");
  double* dev[3] = {nullptr, nullptr, nullptr};
  for (int ax = 0; ax < h->d; ++ax) {
    if (!face[ax]) return fail(h, BLTT_ERR_INVALID_ARG, "null face array");
    const size_t cnt = (size_t)(h->M / h->m[ax]) * (size_t)(h->m[ax] + 1);
    for (size_t k = 0; k < cnt; ++k)
      if (!(face[ax][k] > 0.0) || !std::isfinite(face[ax][k]))
        return fail(h, BLTT_ERR_INVALID_ARG, "face coefficients must be positive and finite");
    CK(h, upload(h, &dev[ax], face[ax], cnt), "face coefficients");
  }
  for (int ax = 0; ax < 3; ++ax) h->op.kf[ax] = dev[ax];
  h->var_coef = true;
  h->pc_bscale = abar;
  h->pc_alpha = -1.0;                        // the preconditioner tables are rebuilt
  drop_graphs(h);                           // kernel arguments changed
  return BLTT_OK;
}

bltt_status bltt_set_stream(bltt_handle h, void* s) {
  if (!h) return BLTT_ERR_INVALID_ARG;
  h->stream = reinterpret_cast<cudaStream_t>(s);
  return BLTT_OK;
}

bltt_status bltt_set_matvec_arith(bltt_handle h, int arith) {
  if (!h) return BLTT_ERR_INVALID_ARG;
  if (arith != BLTT_ARITH_F64 && arith != BLTT_ARITH_F32X2 && arith != BLTT_ARITH_TC)
    return fail(h, BLTT_ERR_INVALID_ARG, "arith must be BLTT_ARITH_F64, _F32X2 or _TC");
  if (arith == BLTT_ARITH_TC) {
    bltt_status s = ensure_tc(h);
    if (s != BLTT_OK) return s;
  }
  h->op.mv_arith = (arith == BLTT_ARITH_TC) ? 2 : (arith == BLTT_ARITH_F32X2) ? 1 : 0;
  return BLTT_OK;
}

bltt_status bltt_matvec(bltt_handle h, const double* x, double* y, int flip) {
  if (!h) return BLTT_ERR_INVALID_ARG;
  if (!x || !y) return fail(h, BLTT_ERR_INVALID_ARG, "null vector");
  if (x == y) return fail(h, BLTT_ERR_INVALID_ARG, "x and y must not overlap");
  double* tmp = nullptr;
  if (h->op.b_kind == 1 && h->op.ntaps == 0) {
    bltt_status s = ensure_workspace(h);
    if (s != BLTT_OK) return s;
    tmp = vec(h, 9);
  }
  if (h->dense) {
    // y = (I (x) U) [Y] A_hat (I (x) U^T) x: the eigenbasis product between two GEMMs
    bltt_status s = ensure_workspace(h);
    if (s != BLTT_OK) return s;
    const bool df = (h->op.mv_arith == 1);
    s = eigen_transform(h, x, vec(h, 8), true, df);
    if (s != BLTT_OK) return s;
    PCK(h, mv_name(h->op), launch_matvec(h->op, 1, vec(h, 8), nullptr, vec(h, 9), flip ? 1 : 0,
                                         MV_STORE, nullptr, nullptr, nullptr, nullptr, nullptr,
                                         h->stream), "matvec");
    return eigen_transform(h, vec(h, 9), y, false, df);
  }
  PCK(h, mv_name(h->op), launch_matvec(h->op, 0, x, nullptr, y, flip ? 1 : 0, MV_STORE, nullptr, nullptr, nullptr,
                      nullptr, tmp, h->stream), "matvec");
  return BLTT_OK;
}

bltt_status bltt_precond_apply(bltt_handle h, double alpha, const double* v, double* z,
                               int precision) {
  if (!h) return BLTT_ERR_INVALID_ARG;
  if (!v || !z) return fail(h, BLTT_ERR_INVALID_ARG, "null vector");
  if (!(alpha > 0.0 && alpha <= 1.0)) return fail(h, BLTT_ERR_INVALID_ARG, "alpha must lie in (0, 1]");
  if (precision != 64 && precision != 32 && precision != 96) return fail(h, BLTT_ERR_INVALID_ARG, "precision must be 64, 32 or 96");
  bltt_status s = prepare_precond(h, alpha, precision);
  if (s != BLTT_OK) return s;
  if (h->dense) {
    s = ensure_workspace(h);
    if (s != BLTT_OK) return s;
  }
  PrecTables pt = prec_tables(h, 0);
  Combine c{};
  c.in0 = v;
  return precond_chain(h, 0, precision, pt, c, z, nullptr, nullptr, nullptr, nullptr);
}

}  // extern "C"

namespace {
// where a host-buffer solve copies u back: on h->io_stream, as soon as u is final, so that the
// copy overlaps the rest of the solve (the physical-basis residual check)
struct HostOut {
  double* u_host;
};
// a host-buffer solve's right-hand side: copied into the staging vector f in chunks of time
// slices on the copy stream, each chunk's entry DST starting as soon as it has landed
struct HostIn {
  const double* f_host;
};

bltt_status solve_impl(bltt_handle h, const double* f, double alpha, double tol, int maxit,
                       const bltt_solve_opts* opts, double* u, bltt_solve_info* info,
                       const HostOut* hout, const HostIn* hin = nullptr, bool inner = false);
bltt_status refine_solve(bltt_handle h, const double* f, double alpha, double tol, int maxit,
                         const bltt_solve_opts* opts, double* u, bltt_solve_info* info);
}  // namespace

extern "C" {

bltt_status bltt_minres_solve_ex(bltt_handle h, const double* f, double alpha, double tol,
                                 int maxit, const bltt_solve_opts* opts, double* u,
                                 bltt_solve_info* info) {
  if (opts && opts->refine > 0) return refine_solve(h, f, alpha, tol, maxit, opts, u, info);
  return solve_impl(h, f, alpha, tol, maxit, opts, u, info, nullptr);
}

}  // extern "C"

namespace {
// entry transform b = Y (I (x) U) f of a host-buffer solve: f arrives in C chunks of N/C time
// slices (copy stream); the DSTs of a chunk run on the compute stream once it has landed.  Lines
// of every axis stay inside a time slice, so a chunk is transformed as a problem of N/C slices
// whose output (flipped inside the chunk) is placed at the mirrored chunk of b.
bltt_status dst_entry_chunked(bltt_ctx* h, const OpTables& op, const double* f_host, double* f,
                              double* b, double* partials, int* nparts) {
  const int N = h->N;
  const long long M = h->M;
  const int C = (N >= 8 && h->n >= (1LL << 22)) ? 4 : 1;
  const int cN = N / C;
  const int arith = op.mv_arith ? PREC_DF : PREC_F64;
  cudaStream_t st = h->stream;
  int total = 0;
  for (int c = 0; c < C; ++c) {
    if (!h->io_chunk_ev[c])
      CK(h, cudaEventCreateWithFlags(&h->io_chunk_ev[c], cudaEventDisableTiming), "chunk event");
    const long long t0 = (long long)c * cN;
    CK(h, cudaMemcpyAsync(f + t0 * M, f_host + t0 * M, (size_t)cN * M * sizeof(double),
                          cudaMemcpyHostToDevice, h->io_stream), "copy f to the device");
    CK(h, cudaEventRecord(h->io_chunk_ev[c], h->io_stream), "event");
    CK(h, cudaStreamWaitEvent(st, h->io_chunk_ev[c], 0), "wait");
    OpTables oc = op;
    oc.N = cN;
    double* bc = b + (N - t0 - cN) * M;
    for (int ax = 0; ax < op.d; ++ax) {
      Combine cb{};
      cb.in0 = (ax == 0) ? f + t0 * M : bc;
      const bool last = (ax == op.d - 1);
      int np = 0;
      cudaEvent_t pa = prof_begin(h);
      CK(h, launch_dst(oc, ax, arith, cb, bc, ax == 0 ? 1 : 0, last ? bc : nullptr,
                       last ? partials + total : nullptr, last ? &np : nullptr, nullptr, st),
         "dst");
      prof_end(h, arith == PREC_DF ? "dst_df" : "dst64", pa);
      h->launches++;
      if (last) total += np;
    }
  }
  *nparts = total;
  return BLTT_OK;
}

bltt_status solve_impl(bltt_handle h, const double* f, double alpha, double tol, int maxit,
                       const bltt_solve_opts* opts, double* u, bltt_solve_info* info,
                       const HostOut* hout, const HostIn* hin, bool inner) {
  NvtxSpan span_solve(inner ? "bltt inner solve" : "bltt_minres_solve");
  NvtxSpan span;
  if (!h) return BLTT_ERR_INVALID_ARG;
  if (info) { std::memset(info, 0, sizeof *info); info->status = BLTT_ERR_INVALID_ARG; }
  if (!f || !u) return fail(h, BLTT_ERR_INVALID_ARG, "null vector");
  if (f == u) return fail(h, BLTT_ERR_INVALID_ARG, "u must not alias f");
  bltt_solve_opts o{};
  if (opts) o = *opts;
  if (o.precision == 0) o.precision = 64;
  if (o.precision != 64 && o.precision != 32 && o.precision != 96) return fail(h, BLTT_ERR_INVALID_ARG, "precision must be 64, 32 or 96");
  if (o.precond != BLTT_PRECOND_ABAC && o.precond != BLTT_PRECOND_NONE) return fail(h, BLTT_ERR_INVALID_ARG, "bad precond");
  const bool none = (o.precond == BLTT_PRECOND_NONE);
  if (!none && !(alpha > 0.0 && alpha <= 1.0)) return fail(h, BLTT_ERR_INVALID_ARG, "alpha must lie in (0, 1]");
  if (!(tol >= 0.0) || maxit < 1) return fail(h, BLTT_ERR_INVALID_ARG, "tol must be >= 0 and maxit >= 1");
  int basis = o.basis;
  // a variable coefficient leaves L undiagonalised by the DST: only the physical basis applies
  if (h->var_coef && basis == BLTT_BASIS_SPECTRAL)
    return fail(h, BLTT_ERR_UNSUPPORTED, "a variable coefficient needs the physical basis");
  // a dense operator: the solve runs in its eigenbasis (the physical basis would need K per slice)
  if (h->dense && basis == BLTT_BASIS_PHYSICAL)
    return fail(h, BLTT_ERR_UNSUPPORTED, "a dense operator solves in its eigenbasis");
  if (basis == BLTT_BASIS_AUTO) basis = h->var_coef ? BLTT_BASIS_PHYSICAL : BLTT_BASIS_SPECTRAL;
  if (basis != BLTT_BASIS_SPECTRAL && basis != BLTT_BASIS_PHYSICAL) return fail(h, BLTT_ERR_INVALID_ARG, "bad basis");
  const int spectral = (basis == BLTT_BASIS_SPECTRAL) ? 1 : 0;
  const int sync_every = o.sync_every > 0 ? o.sync_every : 2;

  if (o.matvec_arith < 0 || o.matvec_arith > 3) return fail(h, BLTT_ERR_INVALID_ARG, "bad matvec_arith");
  bltt_status s = ensure_workspace(h);
  if (s != BLTT_OK) return s;
  if (o.matvec_arith == BLTT_ARITH_TC) {
    s = ensure_tc(h);
    if (s != BLTT_OK) return s;
  }
  h->launches = 0;
  OpTables op = h->op;
  if (o.matvec_arith == BLTT_ARITH_F64) op.mv_arith = 0;
  if (o.matvec_arith == BLTT_ARITH_F32X2) op.mv_arith = 1;
  if (o.matvec_arith == BLTT_ARITH_TC) op.mv_arith = 2;
  const bool tc = (op.mv_arith == 2);
  cudaStream_t st = h->stream;
  CK(h, cudaEventRecord(h->ev[0], st), "event");
  if (o.rebuild) h->pc_alpha = -1.0;
  span.start("preconditioner set-up");
  if (!none) {
    s = prepare_precond(h, alpha, o.precision);
    if (s != BLTT_OK) return s;
  }
  CK(h, cudaEventRecord(h->ev[1], st), "event");
  PrecTables pt = prec_tables(h, none ? 1 : 0);

  double* bvec = vec(h, 0);
  double* vbuf[2] = {vec(h, 1), vec(h, 2)};
  double* q = vec(h, 7);
  double* x = spectral ? vec(h, 8) : u;
  double* tmp = vec(h, 9);
  const long long n = h->n;

  // state: tol, maxit
  // deferred solution update: the first S iterations store their z vectors and keep x and w as
  // coefficients over them (no per-iteration (w, x) update); S is a multiple of the graph block
  const int G = (sync_every + 1) & ~1;
  int S = 0;
  if (!o.single_block && o.defer_window >= 0 && G <= kMaxWin) {
    const int want = o.defer_window > 0 ? std::min(o.defer_window, kMaxWin) : 8;
    S = std::max(G, (want / G) * G);
    if (ensure_window(h, S) != BLTT_OK) { S = 0; (void)cudaGetLastError(); }
  }
  MinresDev* sh = h->state_host;
  std::memset(sh, 0, sizeof *sh);
  sh->tol = tol;
  sh->maxit = maxit;
  sh->phase = PH_RUN;
  sh->win = S;
  sh->stopfail = inner ? 1 : 0;
  CK(h, cudaMemcpyAsync(h->state, sh, sizeof *sh, cudaMemcpyHostToDevice, st), "state upload");
  int* phase = &h->state->phase;
  // the end of every solve: timings, status and statistics
  auto finish = [&](double relres_phys) -> bltt_status {
    h->ahead_blocks = (sh->iter + G - 1) / G;   // the next solve's first burst
    CK(h, cudaEventRecord(h->ev[2], st), "event");
    CK(h, cudaStreamSynchronize(st), "sync");
    prof_harvest(h);
    float t_all = 0.f, t_setup = 0.f;
    cudaEventElapsedTime(&t_all, h->ev[0], h->ev[2]);
    cudaEventElapsedTime(&t_setup, h->ev[0], h->ev[1]);
    bltt_status result;
    if (sh->phase == PH_DONE) result = (sh->status == 0) ? BLTT_OK : BLTT_ERR_NOT_CONVERGED;
    else if (sh->phase == PH_FAIL) result = BLTT_ERR_NUMERIC;
    else result = BLTT_ERR_NOT_CONVERGED;
    if (info) {
      info->iters = sh->iter;
      info->relres_est = sh->relres_est;
      info->relres_true = relres_phys;
      info->alpha_used = none ? 0.0 : alpha;
      info->alpha_source = 0;
      info->precision = o.precision;
      info->basis = basis;
      info->t_setup_ms = t_setup;
      info->t_solve_ms = t_all;
      info->kernel_launches = h->launches;
      info->status = result;
    }
    if (tc) {
      // a bounded wait of the tensor-core kernel that gave up shows as NaN partials; name it
      int flag = 0;
      CK(h, cudaMemcpy(&flag, op.tc_err, sizeof(int), cudaMemcpyDeviceToHost), "error flag");
      if (flag) {
        CK(h, cudaMemset(op.tc_err, 0, sizeof(int)), "error flag");
        if (info) info->status = BLTT_ERR_TIMEOUT;
        return fail(h, BLTT_ERR_TIMEOUT, "a bounded wait of the tensor-core matvec gave up");
      }
    }
    if (result == BLTT_ERR_NUMERIC) h->err = "MINRES breakdown: <z, v> negative or non-finite";
    else if (result == BLTT_ERR_NOT_CONVERGED) h->err = "maxit reached before the stopping rule held";
    return result;
  };

  if (o.single_block) {
    // the whole solve by one block (problems whose every phase is one FFT tile): DST basis, the
    // residual checked inside the loop; one launch.  Forms: FP64 throughout, or the chosen one
    // (FP32 preconditioner with the double-float product and DSTs)
    const bool f64 = (o.precision == 64 && op.mv_arith == 0);
    const bool chosen = (o.precision == 32 && op.mv_arith == 1);
    if (!spectral || !(f64 || chosen) || none || op.ntaps > 0 || h->dense || h->var_coef || hin ||
        hout)
      return fail(h, BLTT_ERR_UNSUPPORTED,
                  "single_block needs the DST basis, FP64 or the FP32 preconditioner with the "
                  "double-float product, the FFT product and device buffers");
    OneSolve os{};
    const int ncc = one_tile_columns(h->M, 2 * h->N);
    const int nct = one_tile_columns(h->M, h->N, chosen ? 2 * kCap : kCap);
    bool fits = ncc > 0 && nct > 0 && 2 * h->N <= kCap;
    for (int ax = 0; ax < h->d && fits; ++ax) {
      const int ncd = one_tile_columns((long long)h->N * h->M / h->m[ax], h->m[ax] + 1);
      fits = ncd > 0;
      if (fits) os.log2NC_dst[ax] = ilog2i(ncd);
    }
    if (!fits) return fail(h, BLTT_ERR_UNSUPPORTED, "single_block: a phase needs more than one tile");
    os.log2NC_conv = ilog2i(ncc);
    os.log2NC_tp = ilog2i(nct);
    os.op = op;
    os.pt = pt;
    os.st = h->state;
    os.f = f;
    os.u = u;
    os.b = vec(h, 0);
    for (int i = 0; i < 2; ++i) { os.v[i] = vec(h, 1 + i); os.z[i] = vec(h, 3 + i); os.w[i] = vec(h, 5 + i); }
    os.q = vec(h, 7);
    os.x = vec(h, 8);
    os.part = h->partials[0];
    os.maxit = maxit;
    cudaEvent_t pa = prof_begin(h);
    CK(h, launch_solve_one(os, chosen, st), "single-block solve");
    prof_end(h, "solve_one", pa);
    h->launches++;
    CK(h, cudaMemcpyAsync(sh, h->state, sizeof *sh, cudaMemcpyDeviceToHost, st), "state download");
    CK(h, cudaStreamSynchronize(st), "sync");
    return finish(sh->relres_true);
  }

  // b = Y f (spectral: Y (I (x) U) f) with ||b||^2
  span.start("entry transform");
  int nb = 0, nzv = 0, np = 0;
  if (spectral && h->dense) {
    // b = Y (I (x) U^T) f: one FP64 GEMM into the scratch vector, then the flip with ||b||^2
    if (hin)
      CK(h, cudaMemcpyAsync(const_cast<double*>(f), hin->f_host, (size_t)h->n * sizeof(double),
                            cudaMemcpyHostToDevice, st), "copy f to the device");
    s = eigen_transform(h, f, tmp, true, op.mv_arith == 1);
    if (s != BLTT_OK) return s;
    PCK(h, "flip", launch_flip_copy(tmp, bvec, h->N, h->M, h->partials[1], &nb, st), "flip");
    h->launches++;
  } else if (spectral && hin) {
    s = dst_entry_chunked(h, op, hin->f_host, const_cast<double*>(f), bvec, h->partials[1], &nb);
    if (s != BLTT_OK) return s;
  } else if (spectral) {
    s = dst_all(h, op, f, bvec, 1, h->partials[1], &nb);
    if (s != BLTT_OK) return s;
  } else {
    if (hin)
      CK(h, cudaMemcpyAsync(const_cast<double*>(f), hin->f_host, (size_t)h->n * sizeof(double),
                            cudaMemcpyHostToDevice, st), "copy f to the device");
    PCK(h, "flip", launch_flip_copy(f, bvec, h->N, h->M, h->partials[1], &nb, st), "flip");
    h->launches++;
  }
  // buffer roles by iteration t: v_t and v_{t-1} alternate between two vectors; inside the window
  // (t < S) iteration t reads z_t from slot t and writes z_{t+1} into slot t + 1; after it, z and w
  // alternate between two vectors each, starting from slot S (z_S) and the w vectors the fold
  // formed (wc = w_{S-1}, wo = w_{S-2})
  double* Zs[kMaxWin + 1] = {vec(h, 3), vec(h, 4)};
  for (int k = 2; k <= S; ++k) Zs[k] = win_vec(h, k - 2);
  double* const Zc[2] = {S ? Zs[S] : vec(h, 3), S ? Zs[S - 1] : vec(h, 4)};
  double* const Wc[2] = {vec(h, 5), vec(h, 6)};
  double* const V0[2] = {vbuf[0], vbuf[1]};
  struct Roles { double *vc, *vp, *zc, *zp, *wc, *wp; };
  auto roles = [&](int t) -> Roles {
    Roles r;
    r.vc = V0[t & 1];
    r.vp = V0[(t + 1) & 1];
    if (t < S) {
      r.zc = Zs[t]; r.zp = Zs[t + 1]; r.wc = r.wp = nullptr;
    } else {
      const int k = (t - S) & 1;
      r.zc = Zc[k]; r.zp = Zc[1 - k]; r.wc = Wc[k]; r.wp = Wc[1 - k];
    }
    return r;
  };
  FoldArgs fa{};
  for (int k = 0; k < S; ++k) fa.z[k] = Zs[k];
  fa.x = x; fa.wo = Wc[1]; fa.wc = Wc[0]; fa.n = n; fa.S = S;
  // v_1 = b (copied into V0[0]), z_0 = P^{-1} v_1 (into slot 0), <z_0, v_1>
  {
    Combine c{};
    c.in0 = bvec;
    c.vout = V0[0];
    s = precond_chain(h, spectral, o.precision, pt, c, Zs[0], V0[0], h->partials[0], &nzv, nullptr);
    if (s != BLTT_OK) return s;
  }
  CK(h, cudaMemsetAsync(V0[1], 0, n * sizeof(double), st), "memset v0");
  if (S == 0) {
    CK(h, cudaMemsetAsync(x, 0, n * sizeof(double), st), "memset x");
    CK(h, cudaMemsetAsync(Wc[0], 0, n * sizeof(double), st), "memset w0");
    CK(h, cudaMemsetAsync(Wc[1], 0, n * sizeof(double), st), "memset w1");
  }
  PCK(h, "scalar", launch_scalar_init(h->state, h->partials[0], nzv, h->partials[1], nb, st), "scalar init");
  h->launches++;

  // one MINRES iteration (A1..A4 of the hot loop)
  // DST basis with the FFT product: the true residual is checked by the host in the physical
  // basis once the estimate has met the stopping rule (the iterations halt in PH_VERIFY and
  // resume if the check fails), so the iterations carry no residual product of their own.  With
  // the direct product (a few taps) the physical residual would need the FP64 stencil of every
  // tap, several times the cost of the product itself: there the iterations check the residual
  // in the DST basis, where (I (x) U) is orthogonal and the norm is the same.
  const bool defer = (spectral != 0) && !h->dense && op.ntaps == 0;
  const long long per_iter = 5 + ((op.b_kind == 1 && op.ntaps == 0 && !spectral) ? 4 : 2) +
                             (spectral || none ? 0 : 2 * op.d) + (tc ? 1 : 0) - (defer ? 1 : 0);
  // kernels of iteration t: the last window iteration of a solve that checks its residual on the
  // device folds a second time (the w vectors, if the check sends the iterations on)
  auto launches_of = [&](int t) -> long long { return per_iter + ((!defer && t == S - 1) ? 1 : 0); };
  auto issue_iteration = [&](int t) -> bltt_status {
    const long long saved = h->launches;   // counted per iteration by the caller (launches_of)
    struct Restore { bltt_ctx* hh; long long v; ~Restore() { hh->launches = v; } } restore{h, saved};
    const Roles r = roles(t);
    // q = Y A z_t  (z_t = z_u / gamma_t), delta_t = <q, z_t>
    if (tc) {
      // the two kernels of the tensor-core product, profiled apart
      PCK(h, "tc_digits", launch_tc_digits(op, r.zc, &h->state->inv_gamma, phase, st),
          "digit planes");
      PCK(h, "conv_tc", launch_tc_product(op, spectral, r.zc, &h->state->inv_gamma, q, 1,
                                          h->partials[0], &np, phase, st), "matvec");
    } else {
      PCK(h, mv_name(op), launch_matvec(op, spectral, r.zc, &h->state->inv_gamma, q, 1,
                                        MV_STORE, nullptr, h->partials[0], &np, phase, tmp, st),
          "matvec");
    }
    PCK(h, "scalar", launch_scalar_delta(h->state, h->partials[0], np, st), "scalar delta");
    // v_{t+1} = q - (delta/gamma) v_t - (gamma/gamma_prev) v_{t-1} (over v_{t-1});
    // z_{t+1} = P^{-1} v_{t+1}; <z_{t+1}, v_{t+1}>
    Combine c{};
    c.in0 = q; c.in1 = r.vc; c.in2 = r.vp;
    c.coef = h->state->coef; c.vout = r.vp;
    bltt_status rs = precond_chain(h, spectral, o.precision, pt, c, r.zp, r.vp, h->partials[1],
                                   &np, phase);
    if (rs != BLTT_OK) return rs;
    PCK(h, "scalar", launch_scalar_gamma(h->state, h->partials[1], np, st), "scalar gamma");
    if (t < S) PCK(h, "fold", launch_fold(h->state, fa, st), "fold");
    else PCK(h, "w_update", launch_w_update(h->state, r.zc, r.wp, r.wc, x, n, st), "w update");
    if (defer) {
      PCK(h, "scalar", launch_scalar_defer(h->state, st), "scalar check");
      return BLTT_OK;
    }
    // true residual when the estimate says so
    PCK(h, mv_name(op, MV_RESID), launch_matvec(op, spectral, x, nullptr, nullptr, 1, MV_RESID, bvec,
                                      h->partials[0], &np, phase, tmp, st), "residual");
    PCK(h, "scalar", launch_scalar_check(h->state, h->partials[0], np, st), "scalar check");
    if (t == S - 1) PCK(h, "fold", launch_fold(h->state, fa, st), "fold");
    return BLTT_OK;
  };
  // A5: blocks of G iterations captured once in a CUDA graph and replayed (G even, so that the
  // alternating roles return to the same vectors; the window's blocks have a graph each); the
  // legacy stream cannot be captured
  const bool graph_mode = (st != nullptr) && !o.no_graph;
  const int nwin = S / G;
  int issued = 0;
  bool resumed = false;
  double relres_phys = 0.0;
  // host-buffer solve: u goes back on the copy stream once final
  auto copy_out = [&]() -> bltt_status {
    if (!hout) return BLTT_OK;
    CK(h, cudaEventRecord(h->io_ev, st), "event");
    CK(h, cudaStreamWaitEvent(h->io_stream, h->io_ev, 0), "wait");
    CK(h, cudaMemcpyAsync(hout->u_host, u, (size_t)h->n * sizeof(double), cudaMemcpyDeviceToHost,
                          h->io_stream), "copy u to the host");
    return BLTT_OK;
  };
  for (;;) {
    span.start("MINRES iterations");
    if (graph_mode && !resumed) {
      const void* key[14] = {(const void*)(intptr_t)spectral, (const void*)(intptr_t)o.precision,
                             (const void*)(intptr_t)op.mv_arith, (const void*)(intptr_t)none,
                             (const void*)(intptr_t)G, x, pt.g64, pt.ahat32, pt.gdf, pt.dinv, st,
                             (const void*)(intptr_t)op.ntaps, (const void*)(intptr_t)h->prof,
                             (const void*)(intptr_t)S};
      if (std::memcmp(key, h->gkey, sizeof key) != 0) {
        drop_graphs(h);
        std::memcpy(h->gkey, key, sizeof key);
      }
      if ((int)h->win_graphs.size() != nwin) h->win_graphs.resize(nwin);
      prof_harvest(h);   // nothing of a capture may mix with earlier events
      // capture (once) the graph of the block that starts at iteration t0
      auto graph_for = [&](int t0, cudaGraphExec_t& ex, std::vector<bltt_ctx::Pending>& gp) -> bltt_status {
        if (ex) return BLTT_OK;
        for (auto& p : gp) { cudaEventDestroy(p.a); cudaEventDestroy(p.b); }
        gp.clear();
        cudaGraph_t g = nullptr;
        CK(h, cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal), "begin capture");
        h->capturing = true;
        bltt_status cap = BLTT_OK;
        for (int i = 0; i < G && cap == BLTT_OK; ++i) cap = issue_iteration(t0 + i);
        h->capturing = false;
        gp.swap(h->pending);                 // the event-record nodes of this graph
        h->pending.clear();
        cudaError_t ce = cudaStreamEndCapture(st, &g);
        if (cap != BLTT_OK) { if (g) cudaGraphDestroy(g); return cap; }
        CK(h, ce, "end capture");
        ce = cudaGraphInstantiate(&ex, g, 0);
        cudaGraphDestroy(g);
        CK(h, ce, "graph instantiate");
        return BLTT_OK;
      };
      // the first look at the device state comes after as many blocks as the last solve on this
      // handle needed (at most 8; blocks past the stop return at once on the device), later ones
      // after every block; with profiling on, after every block (a graph's event nodes hold
      // its last replay only)
      int burst = h->prof ? 1 : std::max(1, std::min(8, h->ahead_blocks));
      for (;;) {
        std::vector<bltt_ctx::Pending>* gp_last = nullptr;
        for (int bb = 0; bb < burst && issued < maxit; ++bb) {
          const bool in_win = issued < S;
          const int b = issued / G;
          cudaGraphExec_t& ex = in_win ? h->win_graphs[b].exec : h->gexec;
          std::vector<bltt_ctx::Pending>& gp = in_win ? h->win_graphs[b].prof : h->graph_prof;
          s = graph_for(in_win ? issued : S, ex, gp);
          if (s != BLTT_OK) return s;
          CK(h, cudaGraphLaunch(ex, st), "graph launch");
          for (int i = 0; i < G; ++i) h->launches += launches_of(issued + i);
          issued += G;
          gp_last = &gp;
        }
        burst = 1;
        CK(h, cudaMemcpyAsync(sh, h->state, sizeof *sh, cudaMemcpyDeviceToHost, st), "state download");
        CK(h, cudaStreamSynchronize(st), "sync");
        if (h->prof && gp_last) prof_harvest_graph(h, *gp_last);
        if (sh->phase != PH_RUN || issued >= maxit) break;
      }
    } else {
      for (;;) {
        s = issue_iteration(issued);
        if (s != BLTT_OK) return s;
        h->launches += launches_of(issued);
        ++issued;
        if (issued % sync_every == 0 || issued >= maxit) {
          CK(h, cudaMemcpyAsync(sh, h->state, sizeof *sh, cudaMemcpyDeviceToHost, st), "state download");
          CK(h, cudaStreamSynchronize(st), "sync");
          if (sh->phase != PH_RUN || issued >= maxit) break;
        }
      }
    }
    span.start("exit transform and true residual");
    // a window solve forms x at every stop on the device; not when it failed before its fold,
    // nor when it took no iteration (x = 0)
    if (S > 0 && sh->iter == 0) {
      CK(h, cudaMemsetAsync(x, 0, n * sizeof(double), st), "memset x");
    } else if (S > 0 && sh->phase == PH_FAIL && sh->iter <= S) {
      FoldArgs fx = fa;
      fx.req = 1;
      PCK(h, "fold", launch_fold(h->state, fx, st), "fold");
      h->launches++;
    }
    relres_phys = sh->relres_true;
    if (!spectral) {
      s = copy_out();
      if (s != BLTT_OK) return s;
      break;
    }
    if (h->dense) {
      // u = (I (x) U) x_hat by one FP64 GEMM; the true residual was checked in the eigenbasis
      // (U orthogonal: the same norm) by the iterations
      s = eigen_transform(h, x, u, false, op.mv_arith == 1);
      if (s != BLTT_OK) return s;
      s = copy_out();
      if (s != BLTT_OK) return s;
      break;
    }
    if (!defer) {
      // the direct product's iterations checked the residual in the DST basis: u = (I (x) U) x_hat
      s = dst_all(h, op, x, u, 0, nullptr, nullptr);
      if (s != BLTT_OK) return s;
      s = copy_out();
      if (s != BLTT_OK) return s;
      break;
    }
    // u = (I (x) U) x_hat, then ||f - A u|| / ||f|| in the physical basis (while u is copied out)
    s = dst_all(h, op, x, u, 0, nullptr, nullptr);
    if (s != BLTT_OK) return s;
    s = copy_out();
    if (s != BLTT_OK) return s;
    int nr = 0;
    PCK(h, mv_name(op, MV_RESID), launch_matvec(op, 0, u, nullptr, nullptr, 0, MV_RESID, f, h->partials[0], &nr, nullptr,
                        tmp, st), "final residual");
    h->launches += (op.b_kind == 1 && op.ntaps == 0) ? 2 : 1;
    PCK(h, "scalar", launch_sum_partials(h->partials[0], nr, h->scal, st), "sum");
    h->launches++;
    CK(h, cudaMemcpyAsync(h->scal_host, h->scal, sizeof(double), cudaMemcpyDeviceToHost, st), "copy");
    CK(h, cudaStreamSynchronize(st), "sync");
    if (sh->normb > 0) relres_phys = std::sqrt(h->scal_host[0]) / sh->normb;
    if (sh->phase != PH_VERIFY) break;
    // the check the iterations left to the host
    sh->relres_true = relres_phys;
    if (!std::isfinite(relres_phys)) { sh->phase = PH_FAIL; sh->status = 5; break; }
    if (relres_phys <= tol || sh->gamma_new == 0.0) {
      sh->phase = PH_DONE;
      sh->status = (relres_phys <= tol) ? 0 : 6;
      break;
    }
    // an inner solve of refinement ends at a failed check: the outer loop corrects from the
    // true residual instead
    if (sh->iter >= maxit || inner) { sh->phase = PH_MAXIT; sh->status = 6; break; }
    // resume: direct launches from iteration sh->iter (a replayed graph could be stopped
    // mid-block); u may still be on its way to the host.  At the window's end the iterations
    // after it need the w vectors, which the fold at the stop left out
    if (hout) CK(h, cudaStreamSynchronize(h->io_stream), "sync copy stream");
    issued = sh->iter;
    resumed = true;
    sh->phase = PH_RUN;
    CK(h, cudaMemcpyAsync(phase, &sh->phase, sizeof(int), cudaMemcpyHostToDevice, st), "resume");
    if (S > 0 && issued == S) {
      FoldArgs fw = fa;
      fw.req = 2;
      PCK(h, "fold", launch_fold(h->state, fw, st), "fold");
      h->launches++;
    }
  }
  return finish(relres_phys);
}

// Mixed-precision iterative refinement around MINRES (the fallback of the precision forms): an
// inner solve that fails a true-residual check ends there; the outer loop forms r = f - A u by a
// fresh FP64-accurate product in the physical basis, solves A d = r in the same form to the
// tolerance that brings ||f - A u|| / ||f|| to tol, and adds d to u.
bltt_status refine_solve(bltt_handle h, const double* f, double alpha, double tol, int maxit,
                         const bltt_solve_opts* opts, double* u, bltt_solve_info* info) {
  NvtxSpan span_refine("bltt_minres_solve (refinement)");
  if (!h) return BLTT_ERR_INVALID_ARG;
  if (info) { std::memset(info, 0, sizeof *info); info->status = BLTT_ERR_INVALID_ARG; }
  if (h->dense) return fail(h, BLTT_ERR_UNSUPPORTED, "refinement needs the blocks' physical product");
  if (!f || !u || f == u) return fail(h, BLTT_ERR_INVALID_ARG, "null or aliased vector");
  bltt_solve_opts o = *opts;
  const int R = o.refine;
  o.refine = 0;
  // every inner solve gets at most an equal share of the budget: a MINRES run whose recurrences
  // have drifted stagnates rather than failing a check, and the share ends it
  const int cap = std::max(1, (maxit + R) / (R + 1));
  bltt_solve_info in{};
  bltt_status s = solve_impl(h, f, alpha, tol, std::min(cap, maxit), &o, u, &in, nullptr, nullptr,
                             true);
  bltt_solve_info tot = in;
  tot.refinements = 0;
  auto out = [&](bltt_status r) {
    tot.status = r;
    if (info) *info = tot;
    return r;
  };
  // a first solve that broke down (a P^{-1} that is no longer positive definite in the reduced
  // precision) restarts from u = 0 in the corrections' precision
  if (s == BLTT_ERR_NUMERIC && o.precision == 32)
    CK(h, cudaMemsetAsync(u, 0, (size_t)h->n * sizeof(double), h->stream), "restart");
  else if (s != BLTT_ERR_NOT_CONVERGED)
    return out(s);
  if (!h->ir_r) {
    CK(h, h->alloc(&h->ir_r, (size_t)h->n), "refinement residual");
    CK(h, h->alloc(&h->ir_d, (size_t)h->n), "refinement correction");
  }
  OpTables op = h->op;
  if (o.matvec_arith == BLTT_ARITH_F64) op.mv_arith = 0;
  if (o.matvec_arith == BLTT_ARITH_F32X2 || o.matvec_arith == BLTT_ARITH_TC) op.mv_arith = 1;
  cudaStream_t st = h->stream;
  const long long n = h->n;
  double* tmp = vec(h, 9);
  // ||x||^2 of a vector, and r = f - A u with ||r||^2, synchronously
  auto sum_to_host = [&](int np) -> double {
    if (launch_sum_partials(h->partials[0], np, h->scal, st) != cudaSuccess) return NAN;
    if (cudaMemcpyAsync(h->scal_host, h->scal, sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return NAN;
    return h->scal_host[0];
  };
  int np = 0;
  CK(h, launch_norm2(f, n, h->partials[0], &np, st), "norm");
  const double nf = std::sqrt(sum_to_host(np));
  tot.kernel_launches += 2;
  auto residual = [&]() -> double {
    int nr = 0;
    if (launch_matvec(op, 0, u, nullptr, h->ir_r, 0, MV_RESID, f, h->partials[0], &nr, nullptr,
                      tmp, st) != cudaSuccess)
      return NAN;
    tot.kernel_launches += (op.b_kind == 1 && op.ntaps == 0) ? 3 : 2;
    return std::sqrt(sum_to_host(nr));
  };
  double rel = residual() / nf;
  bltt_status res = BLTT_ERR_NOT_CONVERGED;
  // the corrections run with the FP32 preconditioner raised to double-float: a correction is only
  // needed where the FP32 rounding, amplified by kappa(D_alpha), has stalled the first solve
  if (o.precision == 32) o.precision = 96;
  for (int k = 0; k < R; ++k) {
    tot.relres_true = rel;
    if (!std::isfinite(rel)) return out(fail(h, BLTT_ERR_NUMERIC, "non-finite residual in refinement"));
    if (rel <= tol) { res = BLTT_OK; break; }
    if (tot.iters >= maxit) break;
    // A d = r to ||r - A d|| <= tol ||f||
    bltt_solve_info ik{};
    s = solve_impl(h, h->ir_r, alpha, tol / rel, std::min(cap, maxit - tot.iters), &o, h->ir_d,
                   &ik, nullptr, nullptr, true);
    if (s != BLTT_OK && s != BLTT_ERR_NOT_CONVERGED) return out(s);   // u as before this step
    CK(h, launch_axpy(u, h->ir_d, n, st), "refinement update");
    tot.iters += ik.iters;
    tot.kernel_launches += ik.kernel_launches + 1;
    tot.t_setup_ms += ik.t_setup_ms;
    tot.t_solve_ms += ik.t_solve_ms;
    tot.relres_est = ik.relres_est;
    tot.refinements = k + 1;
    rel = residual() / nf;
  }
  if (rel <= tol) res = BLTT_OK;
  tot.relres_true = rel;
  if (res != BLTT_OK) h->err = "refinement ended before the residual reached tol";
  return out(res);
}
}  // namespace

extern "C" {

bltt_status bltt_minres_solve_host(bltt_handle h, const double* f_host, double alpha, double tol,
                                   int maxit, const bltt_solve_opts* opts, double* u_host,
                                   bltt_solve_info* info) {
  if (!h) return BLTT_ERR_INVALID_ARG;
  if (info) { std::memset(info, 0, sizeof *info); info->status = BLTT_ERR_INVALID_ARG; }
  if (!f_host || !u_host) return fail(h, BLTT_ERR_INVALID_ARG, "null vector");
  if (f_host == u_host) return fail(h, BLTT_ERR_INVALID_ARG, "u must not alias f");
  if (!h->io_f) {
    CK(h, h->alloc(&h->io_f, (size_t)h->n), "staging of f");
    CK(h, h->alloc(&h->io_u, (size_t)h->n), "staging of u");
    CK(h, cudaStreamCreateWithFlags(&h->io_stream, cudaStreamNonBlocking), "copy stream");
    CK(h, cudaEventCreateWithFlags(&h->io_ev, cudaEventDisableTiming), "copy event");
  }
  if (opts && opts->refine > 0) {
    // refinement: f in, the device-buffer solve with its outer corrections, u out
    const size_t bytes = (size_t)h->n * sizeof(double);
    CK(h, cudaMemcpyAsync(h->io_f, f_host, bytes, cudaMemcpyHostToDevice, h->stream), "copy f to the device");
    const bltt_status sr = refine_solve(h, h->io_f, alpha, tol, maxit, opts, h->io_u, info);
    CK(h, cudaMemcpyAsync(u_host, h->io_u, bytes, cudaMemcpyDeviceToHost, h->stream), "copy u to the host");
    CK(h, cudaStreamSynchronize(h->stream), "sync");
    return sr;
  }
  const HostOut hout{u_host};
  const HostIn hin{f_host};
  const bltt_status st = solve_impl(h, h->io_f, alpha, tol, maxit, opts, h->io_u, info, &hout,
                                    &hin);
  // whatever the status, no copy into u_host is still in flight when the call returns
  const cudaError_t ce = cudaStreamSynchronize(h->io_stream);
  if (st == BLTT_OK && ce != cudaSuccess) return fail(h, BLTT_ERR_CUDA, cudaGetErrorString(ce));
  return st;
}

bltt_status bltt_profile_enable(bltt_handle h, int enable) {
  if (!h) return BLTT_ERR_INVALID_ARG;
  prof_harvest(h);
  h->stats.clear();
  h->prof = enable != 0;
  return BLTT_OK;
}

int bltt_profile_read(bltt_handle h, bltt_kernel_stat* out, int max_entries) {
  if (!h) return -1;
  prof_harvest(h);
  int k = 0;
  for (auto& kv : h->stats) {
    if (out && k < max_entries) {
      std::memset(&out[k], 0, sizeof out[k]);
      std::strncpy(out[k].name, kv.first.c_str(), sizeof out[k].name - 1);
      out[k].launches = kv.second.launches;
      out[k].total_ms = kv.second.ms;
      // a launch is active when it took more than 1/4 of its family's longest launch
      for (float m : kv.second.each)
        if (m > 0.25 * kv.second.max_ms) { out[k].active_launches += 1; out[k].active_ms += m; }
    }
    ++k;
  }
  return k;
}

bltt_status bltt_check_guards(bltt_handle h, int* bands_checked) {
  if (!h) return BLTT_ERR_INVALID_ARG;
  if (bands_checked) *bands_checked = 0;
  if (!h->guard) return BLTT_OK;
  CK(h, cudaStreamSynchronize(h->stream), "sync");
  std::vector<uint64_t> got(h->guard);
  auto check = [&](double* base, size_t nvec, const char* what) -> bltt_status {
    for (size_t k = 0; base && k <= nvec; ++k) {
      CK(h, cudaMemcpy(got.data(), base + k * (h->n + h->guard), h->guard * 8,
                       cudaMemcpyDeviceToHost), "guard band read");
      for (size_t i = 0; i < h->guard; ++i)
        if (got[i] != kGuardBits)
          return fail(h, BLTT_ERR_CUDA, std::string("guard band ") + std::to_string(k) + " of the " +
                                            what + " was overwritten (element " + std::to_string(i) + ")");
      if (bands_checked) ++*bands_checked;
    }
    return BLTT_OK;
  };
  bltt_status s = check(h->ws, h->ws ? h->ws_vectors : 0, "workspace");
  if (s == BLTT_OK) s = check(h->win_ws, h->win_ws ? (size_t)h->win_vectors : 0, "window slots");
  return s;
}

bltt_status bltt_guard_poke(bltt_handle h, int band) {
  if (!h) return BLTT_ERR_INVALID_ARG;
  if (!h->guard || !h->ws || band < 0 || (size_t)band > h->ws_vectors)
    return fail(h, BLTT_ERR_INVALID_ARG, "no such guard band");
  const double v = 1.0;
  CK(h, cudaMemcpy(h->ws + (size_t)band * (h->n + h->guard) + h->guard / 2, &v, sizeof v,
                   cudaMemcpyHostToDevice), "guard band write");
  return BLTT_OK;
}

bltt_status bltt_minres_solve(bltt_handle h, const double* f, double alpha, double tol, int maxit,
                              int precision, double* u, bltt_solve_info* info) {
  bltt_solve_opts o{};
  o.precision = precision;
  return bltt_minres_solve_ex(h, f, alpha, tol, maxit, &o, u, info);
}

}  // extern "C"
