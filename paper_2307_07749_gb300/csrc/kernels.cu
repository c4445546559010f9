// kernels.cu - sm_103a kernels of libbltt: DST-I along a spatial axis, the alpha-scaled time pass
// of the ABAC preconditioner, the BLTT matvec (2N circulant embedding or direct taps), the
// preconditioner set-up and the MINRES vector/scalar kernels.
#include <atomic>
#include <math.h>
#include <stdlib.h>
#include <algorithm>
#include <type_traits>
#include "tiles.cuh"
#include "launch_util.h"
#include "spec.h"

namespace bltt {

// ============================================================================================
// host helpers
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

constexpr int kDirectChunk = 32;   // time steps of one work unit (two walks of half as many)

// One work unit: a group of kDirectThreads x P consecutive points (P per thread, kDirectThreads
// apart) over two walks of kDirectChunk/2 time steps: t = t0, t0+1, ... in the first half of the
// time axis and its mirror tau = N-1-t downwards.  The fused dot product delta = <Y A x, x>
// multiplies the output of step t, stored at row N-1-t = tau, by x_tau, which the mirror walk has
// in a register at the same step (and the other way round), so x is read once and y written once:
// 16 B per unknown.  Each walk keeps the K-1 neighbouring values (and their L x in the physical
// basis) in registers; they are loaded at the walk's start.  Units run point groups fastest, so
// that the blocks in flight read neighbouring runs of the same rows.
template <int K, bool SPECTRAL>
__global__ void __launch_bounds__(kDirectThreads)
k_direct(OpTables op, const double* __restrict__ x, const double* xscale, double* y, int flip,
         int mode, const double* rhs, double* partials, const int* phase, int want) {
  if (skip_phase(phase, want)) return;
  constexpr bool spectral = SPECTRAL;
  constexpr int P = SPECTRAL ? kDirectPts : 1;
  constexpr int D2 = SPECTRAL ? 1 : 6;          // stencil neighbours kept per point
  constexpr int HALF = kDirectChunk / 2;
  __shared__ double red[32];
  const int N = op.N, Nh = op.N / 2;            // N is even (a power of two >= 2)
  const long long M = op.M;
  const double s = xscale ? *xscale : 1.0;
  bool any_b = false;
#pragma unroll
  for (int k = 0; k < K; ++k) any_b |= (op.b_dev[k] != 0.0);
  const bool lap = !spectral && any_b;
  const long long groups = (M + P * kDirectThreads - 1) / (P * kDirectThreads);
  const long long units = groups * ((Nh + HALF - 1) / HALF);
  double acc = 0.0;
  for (long long u = blockIdx.x; u < units; u += gridDim.x) {
    const int chunk = (int)(u / groups);
    const long long c0 = (u - (long long)chunk * groups) * (P * kDirectThreads);
    const int t0 = chunk * HALF, t1 = min(Nh, t0 + HALF);
    const int tau0 = N - 1 - t0;
    long long ip[P];
    // xf[k] = x_{t-k} (forward walk), xb[k] = x_{tau-k} (mirror walk); lf, lb: their L x
    double ca[P][K], cb[P][K], xf[P][K], lf[P][K], xb[P][K], lb[P][K];
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
        xf[q][k] = 0.0; lf[q][k] = 0.0; xb[q][k] = 0.0; lb[q][k] = 0.0;
      }
#pragma unroll
      for (int k = 1; k < K; ++k) {
        // the forward walk's earlier steps t0 - k (zero before the first step), stored one slot
        // ahead: the step loop shifts before it uses them
        const int tk = t0 - k;
        if (tk >= 0) {
          const double* xt = x + (long long)tk * M + i;
          xf[q][k - 1] = xt[0];
          if (!spectral && lap) lf[q][k - 1] = apply_stencil<D2>(pst[q], xt);
        }
        // the mirror walk's first K-1 values tau0 - (k-1); its step loop loads the K-th
        const int tb = tau0 - (k - 1);
        if (tb >= 0) {
          const double* xt = x + (long long)tb * M + i;
          xb[q][k - 1] = xt[0];
          if (!spectral && lap) lb[q][k - 1] = apply_stencil<D2>(pst[q], xt);
        }
      }
    }
    for (int t = t0; t < t1; ++t) {
      const int tau = N - 1 - t;
      const int tn = tau - (K - 1);                // the mirror walk's new value: x_{tau-K+1}
      const long long rf = (long long)(flip ? tau : t) * M;   // where the outputs of t and tau go
      const long long rb = (long long)(flip ? t : tau) * M;
      double xsf[P], xsb[P], prf[P], prb[P];
#pragma unroll
      for (int q = 0; q < P; ++q) {
        const long long i = ip[q] < M ? ip[q] : M - 1;
        xsf[q] = x[(long long)t * M + i];
        xsb[q] = tn >= 0 ? x[(long long)tn * M + i] : 0.0;
        prf[q] = 0.0; prb[q] = 0.0;
        if (mode != MV_STORE) { prf[q] = rhs[rf + i]; prb[q] = rhs[rb + i]; }
      }
#pragma unroll
      for (int q = 0; q < P; ++q) {
        const long long i = ip[q] < M ? ip[q] : M - 1;
#pragma unroll
        for (int k = K - 1; k > 0; --k) { xf[q][k] = xf[q][k - 1]; lf[q][k] = lf[q][k - 1]; }
        xf[q][0] = xsf[q];
        xb[q][K - 1] = xsb[q];
        if (!spectral && lap) {
          lf[q][0] = apply_stencil<D2>(pst[q], x + (long long)t * M + i);
          lb[q][K - 1] = tn >= 0 ? apply_stencil<D2>(pst[q], x + (long long)tn * M + i) : 0.0;
        }
        double vf = 0.0, vb = 0.0;
#pragma unroll
        for (int k = 0; k < K; ++k) {
          vf = fma(ca[q][k], xf[q][k], vf);
          vb = fma(ca[q][k], xb[q][k], vb);
          if (!spectral) { vf = fma(cb[q][k], lf[q][k], vf); vb = fma(cb[q][k], lb[q][k], vb); }
        }
        if (ip[q] < M) {
          if (mode == MV_STORE) {
            y[rf + i] = vf;
            y[rb + i] = vb;
            // partner of each output: x at the row it is stored in (times s once per block)
            if (partials) acc = fma(vb, flip ? xf[q][0] : xb[q][0], fma(vf, flip ? xb[q][0] : xf[q][0], acc));
          } else {
            const double r1 = prf[q] - vf, r2 = prb[q] - vb;
            if (y) { y[rf + i] = r1; y[rb + i] = r2; }
            acc = fma(r2, r2, fma(r1, r1, acc));
          }
        }
#pragma unroll
        for (int k = 0; k < K - 1; ++k) { xb[q][k] = xb[q][k + 1]; lb[q][k] = lb[q][k + 1]; }
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
  st->fold_req = 0;
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
  const int t = st->iter;   // this iteration's index
  st->iter += 1;
  st->relres_est = fabs(st->eta) / st->eta0;
  if (gn == 0.0 || st->relres_est <= st->tol || st->iter >= st->maxit) st->phase = PH_CHECK;
  if (t >= st->win) {
    st->wpending = 1;
    st->fold_req = 0;
    return;
  }
  // deferred update: w_t = w_cz z_t + w_cwp w_{t-2} + w_cw w_{t-1} and x += w_ceta w_t, applied to
  // the coefficients over z_0 .. z_t (w_{-1} = w_{-2} = 0, x_0 = 0)
  st->wpending = 0;
  for (int k = 0; k <= t; ++k) {
    double wn = fma(st->w_cwp, st->cwo[k], st->w_cw * st->cwc[k]);
    if (k == t) wn += st->w_cz;
    st->xi[k] = fma(st->w_ceta, wn, st->xi[k]);
    st->cwo[k] = st->cwc[k];
    st->cwc[k] = wn;
  }
  // a stop or a true-residual check needs x now; the window's last iteration hands the two latest
  // w vectors (and x) to the per-iteration update of the iterations after it
  int req = (st->phase != PH_RUN) ? 1 : 0;
  if (st->iter == st->win && st->phase == PH_RUN) req = 3;
  st->fold_req = req;
}

__device__ __forceinline__ void scalar_check(MinresDev* st, const double* p, int np) {
  __shared__ double red[32];
  const bool check = (st->phase == PH_CHECK);
  double r2 = check ? reduce_partials(p, np, red) : 0.0;
  if (threadIdx.x != 0) return;
  st->wpending = 0;
  st->fold_req = 0;
  if (!check) return;
  const double rr = sqrt(r2) / st->normb;
  st->relres_true = rr;
  if (!isfinite(rr)) { st->phase = PH_FAIL; st->status = 5; return; }
  if (rr <= st->tol || st->gamma_new == 0.0) {
    st->phase = PH_DONE; st->status = (rr <= st->tol) ? 0 : 6;
  } else if (st->iter >= st->maxit) {
    st->phase = PH_MAXIT; st->status = 6;
  } else if (st->stopfail) {
    st->phase = PH_MAXIT; st->status = 6;   // an inner solve of refinement ends here
  } else {
    st->phase = PH_RUN;
    // the check failed at the last deferred iteration: the iterations after it need the w vectors
    if (st->win > 0 && st->iter == st->win) st->fold_req = 2;
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
  st->fold_req = 0;
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

// Deferred-update fold: x = sum_s xi_s z_s (bit 0 of the request) and the two latest w vectors
// wo = sum_s cwo_s z_s, wc = sum_s cwc_s z_s (bit 1) over the k = min(iter, S) stored z's, in FP64,
// summed in slot order.  Pairs of elements as 16-byte accesses.  The loop is latency-bound unless
// each thread keeps several loads in flight: a thread takes U = 8 / KB pairs per step (KB >= k, a
// power of two picked on the device from k) and issues all their loads before the first
// multiply-add, so that about eight loads are in flight per thread whatever k is (with one pair
// per step the fold took the same 0.9 ms on the 66.6 M-unknown workload for k = 1 and k = 8).
template <int R, int KB>
__device__ __forceinline__ void fold_pairs(const FoldArgs& a, int k, const double* cx,
                                           const double* co, const double* cc, long long e,
                                           long long stride) {
  constexpr int U = KB >= 8 ? 1 : 8 / KB;
  const long long n2 = a.n >> 1;
  auto one = [&](const double2* zv, long long i) {
    double2 x = make_double2(0.0, 0.0), wo = x, wc = x;
#pragma unroll
    for (int s = 0; s < KB; ++s) {
      if (s < k) {
        if (R & 1) { x.x = fma(cx[s], zv[s].x, x.x); x.y = fma(cx[s], zv[s].y, x.y); }
        if (R & 2) {
          wo.x = fma(co[s], zv[s].x, wo.x); wo.y = fma(co[s], zv[s].y, wo.y);
          wc.x = fma(cc[s], zv[s].x, wc.x); wc.y = fma(cc[s], zv[s].y, wc.y);
        }
      }
    }
    if (R & 1) __stcs(reinterpret_cast<double2*>(a.x) + i, x);
    if (R & 2) {
      __stcs(reinterpret_cast<double2*>(a.wo) + i, wo);
      __stcs(reinterpret_cast<double2*>(a.wc) + i, wc);
    }
  };
  for (; e + (U - 1) * stride < n2; e += U * stride) {
    double2 zv[U][KB];
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
      for (int s = 0; s < KB; ++s)
        if (s < k) zv[u][s] = __ldcs(reinterpret_cast<const double2*>(a.z[s]) + e + u * stride);
#pragma unroll
    for (int u = 0; u < U; ++u) one(zv[u], e + u * stride);
  }
  for (; e < n2; e += stride) {
    double2 zv[KB];
#pragma unroll
    for (int s = 0; s < KB; ++s)
      if (s < k) zv[s] = __ldcs(reinterpret_cast<const double2*>(a.z[s]) + e);
    one(zv, e);
  }
}

template <int R, int KMAX>
__device__ __forceinline__ void fold_dispatch(const FoldArgs& a, int k, const double* cx,
                                              const double* co, const double* cc, long long e,
                                              long long stride) {
  if (k <= 1) fold_pairs<R, 1>(a, k, cx, co, cc, e, stride);
  else if (k <= 2) fold_pairs<R, 2>(a, k, cx, co, cc, e, stride);
  else if (KMAX >= 4 && k <= 4) fold_pairs<R, (KMAX >= 4 ? 4 : 2)>(a, k, cx, co, cc, e, stride);
  else if (KMAX >= 8 && k <= 8) fold_pairs<R, (KMAX >= 8 ? 8 : 2)>(a, k, cx, co, cc, e, stride);
  else if (KMAX >= 16) fold_pairs<R, (KMAX >= 16 ? 16 : 2)>(a, k, cx, co, cc, e, stride);
}

template <int KMAX>
__global__ void __launch_bounds__(256, 2) k_fold(const MinresDev* st, FoldArgs a) {
  const int req = a.req ? a.req : st->fold_req;
  if (!req) return;
  const int k = min(st->iter, a.S);
  __shared__ double cx[kMaxWin], co[kMaxWin], cc[kMaxWin];
  if (threadIdx.x < kMaxWin) {
    cx[threadIdx.x] = st->xi[threadIdx.x];
    co[threadIdx.x] = st->cwo[threadIdx.x];
    cc[threadIdx.x] = st->cwc[threadIdx.x];
  }
  __syncthreads();
  if (k < 1 || k > KMAX) return;   // the launcher picks KMAX >= the window, so k > KMAX never
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long stride = (long long)gridDim.x * blockDim.x;
  if (req == 1) fold_dispatch<1, KMAX>(a, k, cx, co, cc, e, stride);
  else if (req == 2) fold_dispatch<2, KMAX>(a, k, cx, co, cc, e, stride);
  else fold_dispatch<3, KMAX>(a, k, cx, co, cc, e, stride);
}

// the fold of every item of a batched wave, one item after the other, each over the whole grid
template <int KMAX>
__global__ void __launch_bounds__(256, 2) k_fold_multi(const FoldItem* __restrict__ items, int ni) {
  __shared__ double cx[kMaxWin], co[kMaxWin], cc[kMaxWin];
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (int i = 0; i < ni; ++i) {
    const MinresDev* st = items[i].st;
    const int req = st->fold_req;
    const int k = min(st->iter, items[i].a.S);
    if (!req || k < 1 || k > KMAX) continue;   // the same for every thread of the block
    __syncthreads();                           // the previous item's coefficients are read
    if (threadIdx.x < kMaxWin) {
      cx[threadIdx.x] = st->xi[threadIdx.x];
      co[threadIdx.x] = st->cwo[threadIdx.x];
      cc[threadIdx.x] = st->cwc[threadIdx.x];
    }
    __syncthreads();
    const FoldArgs a = items[i].a;
    if (req == 1) fold_dispatch<1, KMAX>(a, k, cx, co, cc, e, stride);
    else if (req == 2) fold_dispatch<2, KMAX>(a, k, cx, co, cc, e, stride);
    else fold_dispatch<3, KMAX>(a, k, cx, co, cc, e, stride);
  }
}

__global__ void __launch_bounds__(256) k_axpy(double* u, const double* d, long long n) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x)
    u[e] += d[e];
}
__global__ void __launch_bounds__(256) k_norm2(const double* x, long long n, double* partials) {
  __shared__ double red[32];
  double acc = 0.0;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x)
    acc = fma(x[e], x[e], acc);
  const double s = block_sum<256>(acc, red);
  if (threadIdx.x == 0) partials[blockIdx.x] = s;
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

template <class A> static cudaError_t ensure_smem_dst() {
  static std::atomic<unsigned long long> done{0};
  return once_per_device(done, [] {
    const size_t smem = TileCfg<A>::CAP * sizeof(typename A::V);
    cudaError_t e = set_smem(k_dst<A, false>, smem);
    if (e == cudaSuccess) e = set_smem(k_dst<A, true>, smem);
    return e;
  });
}

template <class A>
static cudaError_t run_dst(const OpTables& op, long long grid, long long nlines, int m,
                           long long inner, int P, int log2NC, const Combine& in, double* out,
                           int flip, const double* dot_with, double* partials,
                           const typename A::V* tw, const int* phase, cudaStream_t st, int prec) {
  const size_t smem = TileCfg<A>::CAP * sizeof(typename A::V);
  cudaError_t e = cudaSuccess;
  if (spec_dst(prec, inner == 1, ilog2(P), log2NC, (unsigned)grid, smem, st, nlines, m, inner, in,
               out, flip, op.N, op.M, dot_with, partials, tw, phase, PH_RUN, &e))
    return e;
  if ((e = ensure_smem_dst<A>()) != cudaSuccess) return e;
  auto kern = (inner == 1) ? k_dst<A, true> : k_dst<A, false>;
  kern<<<(unsigned)grid, TileCfg<A>::NT, smem, st>>>(nlines, m, inner, P, ilog2(P), log2NC, in,
                                                     out, flip, op.N, op.M, dot_with, partials,
                                                     tw, phase, PH_RUN);
  return cudaGetLastError();
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
  if (e == cudaSuccess) e = spec_prepare_conv_attributes();
  if (e == cudaSuccess) e = spec_prepare_tp_attributes();
  if (e == cudaSuccess) e = spec_prepare_dst_attributes();
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
  if (prec == PREC_F64)
    return run_dst<ArithD>(op, grid, nlines, m, inner, P, log2NC, in, out, flip, dot_with,
                           partials, op.tw_dst[axis], phase, st, prec);
  if (prec == PREC_DF)
    return run_dst<ArithDF>(op, grid, nlines, m, inner, P, log2NC, in, out, flip, dot_with,
                            partials, op.tw_dst_df[axis], phase, st, prec);
  return run_dst<ArithF>(op, grid, nlines, m, inner, P, log2NC, in, out, flip, dot_with,
                         partials, op.tw_dst32[axis], phase, st, PREC_F32);
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
    if (spec_timepass(prec, std::is_same<Cfg, WideTileF>::value, op.log2N, log2NC,
                      (unsigned)grid, smem, st, op, pt, in, out, dot_with, partials, phase,
                      PH_RUN, tw, &e))
      return e;
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
  const int prec = std::is_same<A, ArithDF>::value ? PREC_DF : PREC_F64;
  auto launch = [&](int spec_, int which, double* out, int flip_, int mode_, const double* rhs_,
                    double* partials_, const double* st_src_) -> cudaError_t {
    cudaError_t el = cudaSuccess;
    if (spec_conv(prec, op.log2N, log2NC, (unsigned)grid, smem, st, op, spec_, which, x, xscale,
                  out, flip_, mode_, rhs_, partials_, phase, want, st_src_, &el))
      return el;
    k_conv<A><<<(unsigned)grid, TileCfg<A>::NT, smem, st>>>(op, spec_, which, x, xscale, out, flip_,
                                                           mode_, rhs_, partials_, phase, want,
                                                           st_src_, log2NC);
    return cudaGetLastError();
  };
  const double* st_src = x;
  if (!spectral && op.b_kind == 1) {
    // conv_b(x) first (scaled like x), then y = conv_a(x) + L conv_b(x)
    if ((e = launch(0, 1, tmp, 0, MV_STORE, nullptr, nullptr, nullptr)) != cudaSuccess) return e;
    st_src = tmp;
  }
  return launch(spectral, 0, y, flip, mode, rhs, partials, st_src);
}

cudaError_t launch_matvec(const OpTables& op, int spectral, const double* x, const double* xscale,
                          double* y, int flip, int mode, const double* rhs, double* partials,
                          int* nparts, const int* phase, double* tmp, cudaStream_t st) {
  const int want = (mode == MV_RESID) ? PH_CHECK : PH_RUN;
  if (op.ntaps > 0) {
    const long long per = (long long)(spectral ? kDirectPts : 1) * kDirectThreads;
    const int half = kDirectChunk / 2;
    long long g = (op.M + per - 1) / per * ((op.N / 2 + half - 1) / half);
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
// the fold of a window of S slots (the vectors' element count is even: N >= 2 is a power of two)
cudaError_t launch_fold(const MinresDev* s, const FoldArgs& a, cudaStream_t st) {
  for (int i = 0; i < a.S; ++i)
    if (!a.z[i] || (((uintptr_t)a.z[i]) & 15)) return cudaErrorInvalidValue;
  if ((((uintptr_t)a.x | (uintptr_t)a.wo | (uintptr_t)a.wc) & 15) || a.S > kMaxWin || a.S < 1 ||
      (a.n & 1))
    return cudaErrorInvalidValue;
  const int g = grid_stream(a.n / 2, 256);
  if (a.S <= 2) k_fold<2><<<g, 256, 0, st>>>(s, a);
  else if (a.S <= 4) k_fold<4><<<g, 256, 0, st>>>(s, a);
  else if (a.S <= 8) k_fold<8><<<g, 256, 0, st>>>(s, a);
  else k_fold<16><<<g, 256, 0, st>>>(s, a);
  return cudaGetLastError();
}

cudaError_t launch_fold_multi(const FoldItem* items, int nitems, int kmax, cudaStream_t st) {
  if (nitems <= 0) return cudaSuccess;
  const int g = 152 * 2;
  if (kmax <= 2) k_fold_multi<2><<<g, 256, 0, st>>>(items, nitems);
  else if (kmax <= 4) k_fold_multi<4><<<g, 256, 0, st>>>(items, nitems);
  else if (kmax <= 8) k_fold_multi<8><<<g, 256, 0, st>>>(items, nitems);
  else k_fold_multi<16><<<g, 256, 0, st>>>(items, nitems);
  return cudaGetLastError();
}

cudaError_t launch_axpy(double* u, const double* d, long long n, cudaStream_t st) {
  k_axpy<<<grid_stream(n, 256), 256, 0, st>>>(u, d, n);
  return cudaGetLastError();
}
cudaError_t launch_norm2(const double* x, long long n, double* partials, int* nparts,
                         cudaStream_t st) {
  const int g = grid_stream(n, 256);
  if (nparts) *nparts = g;
  k_norm2<<<g, 256, 0, st>>>(x, n, partials);
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
