// batched.cu - bltt_solve_batched: many BLTT systems of uneven N and M, each with several
// right-hand sides, solved together.
//
// Every (system, right-hand side) pair is an item with its own MINRES state; items of one system
// share that system's operator and preconditioner tables.  Items run in lockstep phases: one
// launch per phase covers the tiles of every item of a wave (persistent blocks stride over the
// concatenated tile list; items that have converged skip their tiles).  The phase sequence of two
// MINRES iterations is captured once per wave in a CUDA graph and replayed until every item has
// stopped; the first S iterations defer their (w, x) update as a single solve does (one graph
// per two of them, their z slots differ).  Waves are sized so that their workspace fits the device memory that is free.
// Items of at least kBigItem unknowns fill the GPU on their own: their FFT phases use the
// single-item kernels (operator tables as kernel parameters, two blocks per SM) inside the same
// graph, and only the smaller items share the multi-item launches, whose tile width for each
// (kernel, N, M, d) shape is chosen by a small autotuner that times the candidate widths on the
// first batch that meets the shape and caches the choice.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "internal.h"

using namespace bltt;

namespace {

// unknowns from which an item runs its FFT phases as single-item launches (at least 512 tiles)
constexpr long long kBigItem = 1LL << 21;

struct Item {
  bool big;
  int sys, rhs;
  long long n, M;
  int N, d, m[3];
  const double* f;
  double* u;
  // workspace (device)
  double *b, *v[2], *z[2], *w[2], *q, *x, *p0, *p1;
  double* zs[kMaxWin + 1];   // deferred-update window: z slots (zs[0], zs[1] are z[0], z[1])
  MinresDev* st;
  long long tiles_conv, tiles_tp, tiles_dst[3], maxtiles;
  int l2nc_conv, l2nc_tp, l2nc_dst[3];
};

int ilog2ll(long long v) { int l = 0; while ((1LL << l) < v) ++l; return l; }

// ---------------------------------------------------------------------------------------------
// tile-width autotuner: key (kind, N, M, d, prec) -> log2 of the complex columns per tile
std::mutex g_tune_mu;
std::map<std::tuple<int, int, long long, int, int>, int> g_tune;

template <class F>
float time_launch(cudaStream_t st, F&& launch) {
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  launch();                       // warm
  cudaEventRecord(a, st);
  launch();
  cudaEventRecord(b, st);
  cudaEventSynchronize(b);
  float ms = 1e30f;
  if (cudaGetLastError() == cudaSuccess) cudaEventElapsedTime(&ms, a, b);
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return ms;
}

// Pick log2NC for the conv / time-pass kernels of one item shape among the default width and
// one and two halvings, timing single-item multi launches on the item's own buffers.
int tune(int kind, const Item& it, const OpTables& op, const PrecTables& pt, int prec, int arith,
         bool enable, cudaStream_t st, const double* scratch_in, double* scratch_out) {
  const int L = (kind == 0) ? 2 * it.N : it.N;
  const int nc0 = tile_columns(it.M, L);
  const int l0 = ilog2ll(nc0);
  auto key = std::make_tuple(kind, it.N, it.M, it.d, kind == 0 ? arith : prec);
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto f = g_tune.find(key);
    if (f != g_tune.end()) return f->second;
  }
  int best = l0;
  if (enable && l0 > 0) {
    float best_ms = 1e30f;
    for (int l = l0; l >= std::max(0, l0 - 2); --l) {
      const long long tiles = (it.M + (2LL << l) - 1) / (2LL << l);
      long long prefix0 = 0;
      long long* dpre = nullptr;
      cudaMalloc(&dpre, sizeof(long long));
      cudaMemcpy(dpre, &prefix0, sizeof prefix0, cudaMemcpyHostToDevice);
      float ms;
      if (kind == 0) {
        ConvItem ci{};
        ci.op = op; ci.x = scratch_in; ci.y = scratch_out; ci.flip = 1; ci.mode = MV_STORE;
        ci.spectral = 1; ci.log2NC = l; ci.partials = nullptr;
        ConvItem* d = nullptr;
        cudaMalloc(&d, sizeof ci);
        cudaMemcpy(d, &ci, sizeof ci, cudaMemcpyHostToDevice);
        ms = time_launch(st, [&] { launch_conv_multi(arith, d, dpre, 1, tiles, st); });
        cudaFree(d);
      } else {
        TpItem ti{};
        ti.op = op; ti.pt = pt; ti.cb.in0 = scratch_in; ti.out = scratch_out; ti.log2NC = l;
        ti.partials = nullptr;
        TpItem* d = nullptr;
        cudaMalloc(&d, sizeof ti);
        cudaMemcpy(d, &ti, sizeof ti, cudaMemcpyHostToDevice);
        ms = time_launch(st, [&] { launch_timepass_multi(prec, d, dpre, 1, tiles, st); });
        cudaFree(d);
      }
      cudaFree(dpre);
      if (ms < best_ms) { best_ms = ms; best = l; }
    }
  }
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune[key] = best;
  return best;
}

template <typename T>
cudaError_t upload_vec(const std::vector<T>& v, T** d) {
  *d = nullptr;
  if (v.empty()) return cudaSuccess;
  cudaError_t e = cudaMalloc(d, v.size() * sizeof(T));
  if (e != cudaSuccess) return e;
  return cudaMemcpy(*d, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
}

}  // namespace

extern "C" bltt_status bltt_solve_batched(int nsys, const bltt_blocks* sys, const int* nrhs,
                                          const double* const* f_dev, double* const* u_dev,
                                          const double* alpha, double tol, int maxit,
                                          const bltt_solve_opts* opts, bltt_solve_info* info) {
  if (nsys <= 0 || !sys || !nrhs || !f_dev || !u_dev) return BLTT_ERR_INVALID_ARG;
  if (!(tol >= 0.0) || maxit < 1) return BLTT_ERR_INVALID_ARG;
  bltt_solve_opts o{};
  if (opts) o = *opts;
  if (o.precision == 0) o.precision = 64;
  if (o.precision != 64 && o.precision != 32 && o.precision != 96) return BLTT_ERR_INVALID_ARG;
  const int prec = o.precision;
  // the batched driver has no tensor-core product: BLTT_ARITH_TC runs as double-float
  const int arith = (o.matvec_arith == BLTT_ARITH_F32X2 || o.matvec_arith == BLTT_ARITH_TC) ? 1 : 0;
  int total_items = 0;
  for (int s = 0; s < nsys; ++s) {
    if (nrhs[s] < 1) return BLTT_ERR_INVALID_ARG;
    total_items += nrhs[s];
  }
  if (info) std::memset(info, 0, sizeof(bltt_solve_info) * total_items);
  cudaStream_t st = nullptr;
  if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return BLTT_ERR_CUDA;
  cudaEvent_t ev0, ev1;
  cudaEventCreate(&ev0);
  cudaEventCreate(&ev1);
  cudaEventRecord(ev0, st);

  // handles and per-system preconditioner tables
  std::vector<bltt_handle> H(nsys, nullptr);
  std::vector<double> alph(nsys);
  bltt_status result = BLTT_OK;
  auto cleanup = [&]() {
    for (auto h : H) if (h) bltt_destroy(h);
    cudaEventDestroy(ev0);
    cudaEventDestroy(ev1);
    cudaStreamDestroy(st);
  };
  for (int s = 0; s < nsys; ++s) {
    long long M = 1;
    for (int ax = 0; ax < sys[s].space.ndim && ax < 3; ++ax) M *= sys[s].space.m[ax];
    bltt_status r = bltt_create(&sys[s], sys[s].N, M, &H[s]);
    if (r != BLTT_OK) { cleanup(); return r; }
    bltt_set_stream(H[s], st);
    bltt_set_matvec_arith(H[s], arith ? BLTT_ARITH_F32X2 : BLTT_ARITH_F64);
    // default alpha per preconditioner arithmetic: the paper's 1e-8 in FP64; raised where the
    // rounding, amplified by kappa(D_alpha) = alpha^{-(N-1)/N}, would cost iterations (1e-2 for
    // FP32, 1e-6 for double-float)
    alph[s] = alpha ? alpha[s] : (prec == PREC_F32 ? 1e-2 : prec == PREC_DF ? 1e-6 : 1e-8);
    if (!(alph[s] > 0.0 && alph[s] <= 1.0)) { cleanup(); return BLTT_ERR_INVALID_ARG; }
    r = ctx_prepare(H[s], alph[s], prec);
    if (r != BLTT_OK) { cleanup(); return r; }
  }

  // items and their tile counts
  std::vector<Item> items;
  items.reserve(total_items);
  int k = 0;
  for (int s = 0; s < nsys; ++s) {
    const OpTables& op = ctx_op(H[s]);
    if (op.ntaps > 0) { cleanup(); return BLTT_ERR_UNSUPPORTED; }   // FFT-matvec systems only
    for (int r = 0; r < nrhs[s]; ++r, ++k) {
      Item it{};
      it.sys = s; it.rhs = r; it.N = op.N; it.M = op.M; it.n = (long long)op.N * op.M; it.d = op.d;
      it.big = it.n >= kBigItem;
      for (int ax = 0; ax < 3; ++ax) it.m[ax] = op.m[ax];
      it.f = f_dev[k]; it.u = u_dev[k];
      if (!it.f || !it.u || it.f == it.u) { cleanup(); return BLTT_ERR_INVALID_ARG; }
      const int ncc = tile_columns(it.M, 2 * it.N), nct = tile_columns(it.M, it.N);
      it.l2nc_conv = ilog2ll(ncc);
      it.l2nc_tp = ilog2ll(nct);
      it.tiles_conv = (it.M + 2 * ncc - 1) / (2 * ncc);
      it.tiles_tp = (it.M + 2 * nct - 1) / (2 * nct);
      // a large item's time pass is a single-item launch, whose tile may differ (its partial
      // sums are what the scalar kernels read)
      if (it.big) it.tiles_tp = timepass_tiles(op, prec);
      // the autotuner may narrow tiles up to 4x: size the partial sums for that
      it.maxtiles = 4 * std::max(it.tiles_conv, it.tiles_tp) + 4;
      long long inner = 1;
      for (int ax = 0; ax < 3; ++ax) {
        if (ax < it.d) {
          const long long nl = it.n / it.m[ax];
          const int nc = tile_columns(nl, it.m[ax] + 1);
          it.l2nc_dst[ax] = ilog2ll(nc);
          it.tiles_dst[ax] = (nl + 2 * nc - 1) / (2 * nc);
          it.maxtiles = std::max(it.maxtiles, it.tiles_dst[ax]);
          inner *= it.m[ax];
        } else {
          it.tiles_dst[ax] = 0;
          it.l2nc_dst[ax] = 0;
        }
      }
      (void)inner;
      items.push_back(it);
    }
  }

  // waves under the free-memory budget: 9 vectors + 2 partial buffers + state per item
  size_t free_b = 0, tot_b = 0;
  cudaMemGetInfo(&free_b, &tot_b);
  size_t budget = (size_t)(0.85 * (double)free_b);
  // BLTT_BATCH_MAX_BYTES caps the per-wave workspace (used to exercise the wave split)
  if (const char* cap = std::getenv("BLTT_BATCH_MAX_BYTES")) {
    const double v = std::atof(cap);
    if (v > 0 && v < (double)budget) budget = (size_t)v;
  }
  // deferred solution update over the first S iterations (as in a single solve): S - 1 more z
  // slots per item; S = 0 with a negative defer_window
  const int S = (o.defer_window < 0) ? 0 : (o.defer_window > 0 ? std::max(2, (std::min(o.defer_window, kMaxWin) / 2) * 2) : 8);
  auto item_bytes = [S](const Item& it) {
    return (size_t)((9 + (S ? S - 1 : 0)) * it.n + 2 * it.maxtiles) * sizeof(double) +
           sizeof(MinresDev) + 4096 + (size_t)(S ? S - 1 : 0) * 256;
  };
  std::vector<std::vector<int>> waves;
  {
    std::vector<int> order(items.size());
    for (size_t i = 0; i < order.size(); ++i) order[i] = (int)i;
    std::stable_sort(order.begin(), order.end(),
                     [&](int a, int b) { return items[a].n > items[b].n; });
    std::vector<int> cur;
    size_t used = 0;
    for (int i : order) {
      const size_t b = item_bytes(items[i]);
      if (b > budget) { cleanup(); return BLTT_ERR_OOM; }
      if (used + b > budget && !cur.empty()) { waves.push_back(cur); cur.clear(); used = 0; }
      cur.push_back(i);
      used += b;
    }
    if (!cur.empty()) waves.push_back(cur);
  }

  int* run_count = nullptr;
  int* run_count_h = nullptr;
  cudaMalloc(&run_count, sizeof(int));
  cudaMallocHost(&run_count_h, sizeof(int));

  // one arena sized for the largest wave, reused by every wave
  size_t arena_bytes = 0;
  int max_ni = 0;
  for (const auto& wave : waves) {
    size_t bytes = 0;
    for (int i : wave) bytes += item_bytes(items[i]);
    arena_bytes = std::max(arena_bytes, bytes);
    max_ni = std::max(max_ni, (int)wave.size());
  }
  unsigned char* arena = nullptr;
  MinresDev* states = nullptr;
  if (cudaMalloc(&arena, arena_bytes) != cudaSuccess ||
      cudaMalloc(&states, sizeof(MinresDev) * max_ni) != cudaSuccess) {
    if (arena) cudaFree(arena);
    cudaFree(run_count);
    cudaFreeHost(run_count_h);
    cleanup();
    return BLTT_ERR_OOM;
  }

  const nvtxRangeId_t span_all = nvtxRangeStartA("bltt_solve_batched");
  for (const auto& wave : waves) {
    const nvtxRangeId_t span_wave = nvtxRangeStartA("batched wave");
    struct EndSpan { nvtxRangeId_t id; ~EndSpan() { nvtxRangeEnd(id); } } end_wave{span_wave};
    const int ni = (int)wave.size();
    size_t off = 0;
    auto carve = [&](size_t nbytes) {
      unsigned char* p = arena + off;
      off += (nbytes + 255) & ~size_t(255);
      return reinterpret_cast<double*>(p);
    };
    for (int j = 0; j < ni; ++j) {
      Item& it = items[wave[j]];
      it.b = carve(it.n * 8);
      it.v[0] = carve(it.n * 8); it.v[1] = carve(it.n * 8);
      it.z[0] = carve(it.n * 8); it.z[1] = carve(it.n * 8);
      it.w[0] = carve(it.n * 8); it.w[1] = carve(it.n * 8);
      it.q = carve(it.n * 8);
      it.x = carve(it.n * 8);
      it.zs[0] = it.z[0]; it.zs[1] = it.z[1];
      for (int k = 2; k <= S; ++k) it.zs[k] = carve(it.n * 8);
      it.p0 = carve(it.maxtiles * 8);
      it.p1 = carve(it.maxtiles * 8);
      it.st = states + j;
    }
    // states: tol, maxit, phase
    {
      std::vector<MinresDev> sh(ni);
      for (auto& s0 : sh) {
        std::memset(&s0, 0, sizeof s0);
        s0.tol = tol; s0.maxit = maxit; s0.phase = PH_RUN; s0.win = S;
      }
      cudaMemcpyAsync(states, sh.data(), sizeof(MinresDev) * ni, cudaMemcpyHostToDevice, st);
      cudaStreamSynchronize(st);
    }
    // autotune the tile widths of this wave's shapes (uses q and z[0] as scratch)
    for (int j = 0; j < ni; ++j) {
      Item& it = items[wave[j]];
      const OpTables& op = ctx_op(H[it.sys]);
      PrecTables pt = ctx_prec_tables(H[it.sys]);
      const bool en = (o.sync_every >= 0);
      if (it.big) continue;   // single-item launches keep the default widths
      it.l2nc_conv = tune(0, it, op, pt, prec, arith, en, st, it.f, it.q);
      it.l2nc_tp = tune(1, it, op, pt, prec, arith, en, st, it.f, it.z[0]);
      it.tiles_conv = (it.M + (2LL << it.l2nc_conv) - 1) / (2LL << it.l2nc_conv);
      it.tiles_tp = (it.M + (2LL << it.l2nc_tp) - 1) / (2LL << it.l2nc_tp);
    }

    // descriptors
    std::vector<DstItem> dst_in[3], dst_out[3];
    std::vector<long long> pre_dst[3];
    std::vector<long long> pre_conv, pre_tp;
    // iteration roles j = 0 .. S-1 (the window's iterations) and j = S, S+1 (the alternating roles
    // after it; without a window, j = 0, 1)
    const int nj = S + 2;
    auto zc_of = [&](const Item& it, int t) -> double* {
      if (S == 0) return it.zs[t & 1];
      return t < S ? it.zs[t] : it.zs[((t - S) & 1) ? S - 1 : S];
    };
    auto zp_of = [&](const Item& it, int t) -> double* {
      if (S == 0) return it.zs[(t + 1) & 1];
      return t < S ? it.zs[t + 1] : it.zs[((t - S) & 1) ? S : S - 1];
    };
    std::vector<TpItem> tp_init, tp_it[kMaxWin + 2];
    std::vector<ConvItem> cv_it[kMaxWin + 2], cv_res;
    std::vector<VecItem> w_loop[2];
    std::vector<FoldItem> folds;
    std::vector<ScalItem> sc_init, sc_delta, sc_gamma, sc_check;
    long long tot_conv = 0, tot_tp = 0, tot_dst[3] = {0, 0, 0};
    std::vector<int> bigs;   // wave positions of the items with single-item launches
    int ns = 0;              // items in the multi-item descriptors
    for (int j = 0; j < ni; ++j) {
      Item& it = items[wave[j]];
      const OpTables& op = ctx_op(H[it.sys]);
      PrecTables pt = ctx_prec_tables(H[it.sys]);
      const int dprec = arith ? PREC_DF : PREC_F64;
      if (it.big) bigs.push_back(j);
      else ++ns;
      // entry (f -> b = Y (I x U) f, ||b||^2 in the last pass) and exit (x -> u) DSTs
      long long inner = 1;
      for (int ax = 0; ax < 3; ++ax) {
        DstItem di{}, dq{};
        di.N = it.N; di.M = it.M;
        if (ax < it.d) {
          di.m = it.m[ax]; di.P = it.m[ax] + 1; di.log2P = ilog2ll(di.P);
          di.nlines = it.n / it.m[ax]; di.inner = inner; di.log2NC = it.l2nc_dst[ax];
          di.tw = dprec == PREC_DF ? (const void*)op.tw_dst_df[ax] : (const void*)op.tw_dst[ax];
          inner *= it.m[ax];
        } else {
          di.nlines = 0; di.inner = 1; di.m = 1; di.P = 2; di.log2P = 1;
        }
        dq = di;
        di.cb.in0 = (ax == 0) ? it.f : it.b;
        di.out = it.b;
        di.flip = (ax == 0) ? 1 : 0;
        if (ax == it.d - 1) { di.dot_with = it.b; di.partials = it.p1; }
        dq.cb.in0 = (ax == 0) ? it.x : it.u;
        dq.out = it.u;
        dq.flip = 0;
        if (!it.big) {
          pre_dst[ax].push_back(tot_dst[ax]);
          tot_dst[ax] += it.tiles_dst[ax];
          dst_in[ax].push_back(di);
          dst_out[ax].push_back(dq);
        }
      }
      if (!it.big) {
        pre_conv.push_back(tot_conv);
        tot_conv += it.tiles_conv;
        pre_tp.push_back(tot_tp);
        tot_tp += it.tiles_tp;
      }
      TpItem ti{};
      ti.op = op; ti.pt = pt; ti.log2NC = it.l2nc_tp;
      ti.cb.in0 = it.b; ti.cb.vout = it.v[0];
      ti.out = it.z[0]; ti.dot_with = it.v[0]; ti.partials = it.p0;
      if (!it.big) tp_init.push_back(ti);
      ScalItem si{};
      si.st = it.st; si.p0 = it.p0; si.n0 = (int)it.tiles_tp; si.p1 = it.p1;
      si.n1 = (int)it.tiles_dst[it.d - 1];
      sc_init.push_back(si);
      for (int j = 0; j < nj; ++j) {
        const int cur = j & 1, prv = 1 - cur;
        ConvItem ci{};
        ci.op = op; ci.x = zc_of(it, j); ci.xscale = &it.st->inv_gamma; ci.y = it.q; ci.flip = 1;
        ci.mode = MV_STORE; ci.spectral = 1; ci.log2NC = it.l2nc_conv; ci.partials = it.p0;
        ci.phase = &it.st->phase; ci.want = PH_RUN;
        if (!it.big) cv_it[j].push_back(ci);
        TpItem tl{};
        tl.op = op; tl.pt = pt; tl.log2NC = it.l2nc_tp;
        tl.cb.in0 = it.q; tl.cb.in1 = it.v[cur]; tl.cb.in2 = it.v[prv]; tl.cb.coef = it.st->coef;
        tl.cb.vout = it.v[prv]; tl.out = zp_of(it, j); tl.dot_with = it.v[prv]; tl.partials = it.p1;
        tl.phase = &it.st->phase; tl.want = PH_RUN;
        if (!it.big) tp_it[j].push_back(tl);
        if (j >= S) {
          const int k = (j - S) & 1;
          VecItem vi{};
          vi.st = it.st; vi.z = zc_of(it, j); vi.w_prev = it.w[1 - k]; vi.w = it.w[k];
          vi.x = it.x; vi.n = it.n;
          w_loop[k].push_back(vi);
        }
      }
      if (S > 0) {
        FoldItem fi{};
        fi.st = it.st;
        for (int k = 0; k < S; ++k) fi.a.z[k] = it.zs[k];
        fi.a.x = it.x; fi.a.wo = it.w[1]; fi.a.wc = it.w[0]; fi.a.n = it.n; fi.a.S = S;
        folds.push_back(fi);
      }
      ConvItem cr{};
      cr.op = op; cr.x = it.x; cr.y = nullptr; cr.rhs = it.b; cr.flip = 1; cr.mode = MV_RESID;
      cr.spectral = 1; cr.log2NC = it.l2nc_conv; cr.partials = it.p0; cr.phase = &it.st->phase;
      cr.want = PH_CHECK;
      if (!it.big) cv_res.push_back(cr);
      ScalItem sd{};
      sd.st = it.st; sd.p0 = it.p0; sd.n0 = (int)it.tiles_conv;
      sc_delta.push_back(sd);
      sc_check.push_back(sd);
      ScalItem sg{};
      sg.st = it.st; sg.p0 = it.p1; sg.n0 = (int)it.tiles_tp;
      sc_gamma.push_back(sg);
    }
    // device copies
    std::vector<void*> dev_allocs;
    cudaError_t e = cudaSuccess;
    auto up = [&](auto& v) {
      using T = typename std::remove_reference<decltype(v)>::type::value_type;
      T* d = nullptr;
      if (e == cudaSuccess) e = upload_vec(v, &d);
      if (d) dev_allocs.push_back(d);
      return d;
    };
    DstItem* d_dst_in[3]; DstItem* d_dst_out[3]; long long* d_pre_dst[3];
    for (int ax = 0; ax < 3; ++ax) { d_dst_in[ax] = up(dst_in[ax]); d_dst_out[ax] = up(dst_out[ax]); d_pre_dst[ax] = up(pre_dst[ax]); }
    long long* d_pre_conv = up(pre_conv);
    long long* d_pre_tp = up(pre_tp);
    TpItem* d_tp_init = up(tp_init);
    TpItem* d_tp_it[kMaxWin + 2];
    ConvItem* d_cv_it[kMaxWin + 2];
    for (int j = 0; j < nj; ++j) { d_tp_it[j] = up(tp_it[j]); d_cv_it[j] = up(cv_it[j]); }
    FoldItem* d_folds = up(folds);
    ConvItem* d_cv_res = up(cv_res);
    VecItem* d_w_loop[2] = {up(w_loop[0]), up(w_loop[1])};
    ScalItem* d_sc_init = up(sc_init);
    ScalItem* d_sc_delta = up(sc_delta);
    ScalItem* d_sc_gamma = up(sc_gamma);
    ScalItem* d_sc_check = up(sc_check);
    const int dprec = arith ? PREC_DF : PREC_F64;
    // single-item launches of the big items (same operands as their descriptors above)
    auto big_dst = [&](bool entry) {
      cudaError_t r = cudaSuccess;
      for (int j : bigs) {
        const Item& it = items[wave[j]];
        const OpTables& op = ctx_op(H[it.sys]);
        for (int ax = 0; ax < it.d && r == cudaSuccess; ++ax) {
          Combine c{};
          const bool last = (ax == it.d - 1);
          if (entry) {
            c.in0 = (ax == 0) ? it.f : it.b;
            r = launch_dst(op, ax, dprec, c, it.b, ax == 0 ? 1 : 0, last ? it.b : nullptr,
                           last ? it.p1 : nullptr, nullptr, nullptr, st);
          } else {
            c.in0 = (ax == 0) ? it.x : it.u;
            r = launch_dst(op, ax, dprec, c, it.u, 0, nullptr, nullptr, nullptr, nullptr, st);
          }
        }
      }
      return r;
    };
    // iteration role t of the big items: t < S the window's iteration t; S, S+1 after it
    auto big_tp = [&](int t, bool init) {
      cudaError_t r = cudaSuccess;
      for (int j : bigs) {
        if (r != cudaSuccess) break;
        const Item& it = items[wave[j]];
        const OpTables& op = ctx_op(H[it.sys]);
        PrecTables pt = ctx_prec_tables(H[it.sys]);
        Combine c{};
        if (init) {
          c.in0 = it.b; c.vout = it.v[0];
          r = launch_timepass(op, pt, prec, c, it.z[0], it.v[0], it.p0, nullptr, nullptr, st);
        } else {
          const int cur = t & 1, prv = 1 - cur;
          c.in0 = it.q; c.in1 = it.v[cur]; c.in2 = it.v[prv]; c.coef = it.st->coef;
          c.vout = it.v[prv];
          r = launch_timepass(op, pt, prec, c, zp_of(it, t), it.v[prv], it.p1, nullptr,
                              &it.st->phase, st);
        }
      }
      return r;
    };
    auto big_conv = [&](int t, bool resid) {
      cudaError_t r = cudaSuccess;
      for (int j : bigs) {
        if (r != cudaSuccess) break;
        const Item& it = items[wave[j]];
        const OpTables& op = ctx_op(H[it.sys]);
        if (resid)
          r = launch_matvec(op, 1, it.x, nullptr, nullptr, 1, MV_RESID, it.b, it.p0, nullptr,
                            &it.st->phase, nullptr, st);
        else
          r = launch_matvec(op, 1, zc_of(it, t), &it.st->inv_gamma, it.q, 1, MV_STORE, nullptr,
                            it.p0, nullptr, &it.st->phase, nullptr, st);
      }
      return r;
    };
    // entry: DSTs, first preconditioner apply, zero vectors, scalar init
    if (e == cudaSuccess) e = big_dst(true);
    for (int ax = 0; ax < 3 && e == cudaSuccess && ns > 0; ++ax)
      e = launch_dst_multi(dprec, d_dst_in[ax], d_pre_dst[ax], ns, tot_dst[ax], st);
    if (e == cudaSuccess) e = big_tp(0, true);
    if (e == cudaSuccess && ns > 0) e = launch_timepass_multi(prec, d_tp_init, d_pre_tp, ns, tot_tp, st);
    for (int j = 0; j < ni && e == cudaSuccess; ++j) {
      Item& it = items[wave[j]];
      e = cudaMemsetAsync(it.x, 0, it.n * 8, st);
      if (e == cudaSuccess) e = cudaMemsetAsync(it.v[1], 0, it.n * 8, st);
      if (S == 0 && e == cudaSuccess) e = cudaMemsetAsync(it.w[0], 0, it.n * 8, st);
      if (S == 0 && e == cudaSuccess) e = cudaMemsetAsync(it.w[1], 0, it.n * 8, st);
    }
    if (e == cudaSuccess) e = launch_scalar_multi(0, d_sc_init, ni, st);
    // warm the persistent-grid queries outside the capture
    persistent_grid(0, dprec); persistent_grid(1, prec); persistent_grid(2, dprec);
    // one MINRES iteration of every item of the wave, in role j
    auto iteration = [&](int j) -> cudaError_t {
      cudaError_t ce = big_conv(j, false);
      if (ce == cudaSuccess && ns > 0) ce = launch_conv_multi(arith, d_cv_it[j], d_pre_conv, ns, tot_conv, st);
      if (ce == cudaSuccess) ce = launch_scalar_multi(1, d_sc_delta, ni, st);
      if (ce == cudaSuccess) ce = big_tp(j, false);
      if (ce == cudaSuccess && ns > 0) ce = launch_timepass_multi(prec, d_tp_it[j], d_pre_tp, ns, tot_tp, st);
      if (ce == cudaSuccess) ce = launch_scalar_multi(2, d_sc_gamma, ni, st);
      if (ce == cudaSuccess)
        ce = (j < S) ? launch_fold_multi(d_folds, ni, S, st)
                     : launch_w_update_multi(d_w_loop[(j - S) & 1], ni, st);
      if (ce == cudaSuccess) ce = big_conv(j, true);
      if (ce == cudaSuccess && ns > 0) ce = launch_conv_multi(arith, d_cv_res, d_pre_conv, ns, tot_conv, st);
      if (ce == cudaSuccess) ce = launch_scalar_multi(3, d_sc_check, ni, st);
      // a check that failed at the window's last iteration: the w vectors for the iterations after
      if (ce == cudaSuccess && j == S - 1) ce = launch_fold_multi(d_folds, ni, S, st);
      return ce;
    };
    // graphs of two iterations: one per block of the window, one for the iterations after it
    const int nblk = S / 2 + 1;
    std::vector<cudaGraphExec_t> gexec(nblk, nullptr);
    for (int g = 0; g < nblk && e == cudaSuccess; ++g) {
      const int j0 = (g < nblk - 1) ? 2 * g : S;
      cudaGraph_t graph = nullptr;
      e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
      if (e != cudaSuccess) break;
      cudaError_t ce = iteration(j0);
      if (ce == cudaSuccess) ce = iteration(j0 + 1);
      e = cudaStreamEndCapture(st, &graph);
      if (e == cudaSuccess) e = ce;
      if (e == cudaSuccess) e = cudaGraphInstantiate(&gexec[g], graph, 0);
      if (graph) cudaGraphDestroy(graph);
    }
    int issued = 0;
    while (e == cudaSuccess) {
      e = cudaGraphLaunch(gexec[issued < S ? issued / 2 : nblk - 1], st);
      issued += 2;
      if (e == cudaSuccess) e = launch_count_running(d_sc_check, ni, run_count, st);
      if (e == cudaSuccess) e = cudaMemcpyAsync(run_count_h, run_count, sizeof(int), cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(st);
      if (e != cudaSuccess || *run_count_h == 0 || issued >= maxit) break;
    }
    // exit DSTs: u = (I x U) x_hat
    if (e == cudaSuccess) e = big_dst(false);
    for (int ax = 0; ax < 3 && e == cudaSuccess && ns > 0; ++ax)
      e = launch_dst_multi(dprec, d_dst_out[ax], d_pre_dst[ax], ns, tot_dst[ax], st);
    std::vector<MinresDev> sh(ni);
    if (e == cudaSuccess) e = cudaMemcpyAsync(sh.data(), states, sizeof(MinresDev) * ni, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    for (auto g : gexec)
      if (g) cudaGraphExecDestroy(g);
    for (void* p : dev_allocs) cudaFree(p);
    if (e != cudaSuccess) { result = BLTT_ERR_CUDA; break; }
    for (int j = 0; j < ni; ++j) {
      const Item& it = items[wave[j]];
      int idx = 0;
      for (int s = 0; s < it.sys; ++s) idx += nrhs[s];
      idx += it.rhs;
      bltt_status stt;
      if (sh[j].phase == PH_DONE) stt = (sh[j].status == 0) ? BLTT_OK : BLTT_ERR_NOT_CONVERGED;
      else if (sh[j].phase == PH_FAIL) stt = BLTT_ERR_NUMERIC;
      else stt = BLTT_ERR_NOT_CONVERGED;
      if (stt != BLTT_OK && result == BLTT_OK) result = stt;
      if (info) {
        info[idx].iters = sh[j].iter;
        info[idx].relres_est = sh[j].relres_est;
        info[idx].relres_true = sh[j].relres_true;
        info[idx].alpha_used = alph[it.sys];
        info[idx].alpha_source = alpha ? 0 : 2;
        info[idx].precision = prec;
        info[idx].basis = BLTT_BASIS_SPECTRAL;
        info[idx].status = stt;
      }
    }
  }
  nvtxRangeEnd(span_all);
  cudaEventRecord(ev1, st);
  cudaEventSynchronize(ev1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, ev0, ev1);
  if (info)
    for (int i = 0; i < total_items; ++i) info[i].t_solve_ms = ms;
  cudaFree(states);
  cudaFree(arena);
  cudaFree(run_count);
  cudaFreeHost(run_count_h);
  cleanup();
  return result;
}
