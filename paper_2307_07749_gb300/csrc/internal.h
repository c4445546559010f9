// internal.h - declarations shared by the libbltt translation units (host side).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/bltt.h"

namespace bltt {

constexpr int kThreads = 256;      // threads of an FFT tile kernel (double-float: twice as many)
constexpr int kCap = 4096;         // complex points per FFT tile (64 KB of FP64 smem)
constexpr int kMaxPartials = 1 << 20;
constexpr int kMaxCols = 256;     // real lines per FFT tile (column info kept in shared memory)
constexpr int kMaxWin = 16;       // iterations whose solution update a solve may defer

// MINRES scalar state, resident on the device for the whole solve.
// PH_VERIFY: the recurrence estimate met the stopping rule in a solve whose true residual the
// host checks (DST basis: the physical-basis residual after the exit transform), iterations halted
enum Phase { PH_RUN = 0, PH_CHECK = 1, PH_DONE = 2, PH_FAIL = 3, PH_MAXIT = 4, PH_VERIFY = 5 };

struct MinresDev {
  double gamma, gamma_prev, delta, eta, eta0;
  double s, s_prev, c, c_prev;
  double inv_gamma;      // 1/gamma_j: normalises z_j where the matvec reads it
  double coef[3];        // v_{j+1} = coef0 q + coef1 v_j + coef2 v_{j-1}
  double w_inv_gamma;    // 1/gamma_j for the w update of iteration j
  double w_a1inv, w_a2, w_a3, w_ceta;
  double w_cz, w_cwp, w_cw;   // w_{j+1} = w_cz z_j + w_cwp w_{j-1} + w_cw w_j (folded coefficients)
  double normb, relres_est, relres_true, tol;
  double gamma_new;
  int iter, maxit, phase, status, wpending;
  int stopfail;          // a failed true-residual check ends the solve (inner solves of refinement)
  // deferred solution update over the first `win` iterations: their w vectors and x are kept as
  // coefficients over the stored z_0 .. z_{win-1} (xi: x, cwo / cwc: the two latest w), and
  // k_fold forms the vectors only when needed.  fold_req: bit 0 x, bit 1 the two w vectors.
  int win, fold_req;
  double xi[kMaxWin], cwo[kMaxWin], cwc[kMaxWin];
};

// the vectors of a deferred-update fold: x = sum_s xi_s z_s, wo = sum_s cwo_s z_s,
// wc = sum_s cwc_s z_s over the first min(iter, S) window slots
struct FoldArgs {
  const double* z[kMaxWin];
  double* x;
  double* wo;
  double* wc;
  long long n;
  int S;
  int req;       // 0: the device's fold_req decides; else this request
};

// Operator data handed to the kernels (device pointers).
struct OpTables {
  int N, log2N, d, m[3];
  long long M;
  double h2inv[3];            // 1/h^2 per axis
  const double* mu_axis[3];   // per-axis eigenvalues of L (device, length m[ax])
  const float* mu_axis32[3];
  // matvec: Ahat, Bhat = FFT_2N([a;0]), FFT_2N([b;0]) scaled by 1/(2N), k = 0..N (device)
  const double2* Ahat;
  const double2* Bhat;
  int b_kind;                 // 0: b = b0 e_0; 1: general b
  double b0;
  int ntaps;                  // >0: a and b vanish beyond ntaps (direct matvec), else FFT matvec
  const double* a_dev;        // a, b (device, length N) for the direct matvec
  const double* b_dev;
  const double2* tw_2N;       // twiddles for length 2N
  const double2* tw_N;
  const float2* tw_N32;
  const double2* tw_dst[3];   // twiddles for length 2(m_ax+1)
  const float2* tw_dst32[3];
  // double-float copies for the FP32-pipe matvec (complex as {re.hi, re.lo, im.hi, im.lo})
  const float4* Ahat_df;
  const float4* Bhat_df;
  const float4* tw_2N_df;
  const float4* tw_dst_df[3];
  const float4* tw_N_df;
  // dense operator K (commuting blocks a_k I + b_k K): its eigenvalues per mode, in the order of
  // the eigenvector columns (null: the Laplacian's, from the per-axis tables)
  const double* mu_tab;
  const float* mu_tab32;
  // general commuting blocks (given by their eigenvalues per mode): the matvec spectrum of each
  // mode, FFT_2N([lam_i; 0]) / (2N) for k = 0..N, frequency-major [k][i] (null: a + mu_i b)
  const double2* Hm64;
  const float4* Hmdf;
  // variable coefficient (null: L = -Delta_h): a at the cell faces along each axis, arrays of the
  // grid's shape with that axis one longer (x fastest); L becomes L_a = -Delta_{a,h}
  const double* kf[3];
  int mv_arith;               // 0: FP64, 1: double-float (matvec and the FP64-accurate DSTs),
                              // 2: tensor-core time product in MV_STORE matvecs, else as 1
  // tensor-core time product (kernels in tcmv.cu): bf16 digit planes of the time-flipped
  // coefficients as 8x8 Hankel core matrices, their power-of-two scale, and the workspace that
  // receives the digit planes and column exponents of each matvec input
  const uint16_t* tc_hank;    // [kTcDigits][tc_ncores][64] bf16 bit patterns (device)
  int tc_ncores, tc_eT;
  uint16_t* tc_xd;            // [strips][N/16][kTcDigits][2048] bf16 bit patterns (device)
  int* tc_xe;                 // [strips * 128] column exponents (device)
  int* tc_err;                // device flag: a bounded wait of the tensor-core kernel gave up
};

// Per-alpha preconditioner data.
struct PrecTables {
  double alpha;
  const double* dinv;    // 1/d_j, d_j = alpha^{j/N}
  const double* d2;      // d_j^2
  const float* dinv32;   // the same in FP32
  const float* d232;
  const float2* dinv_df; // the same as double-float (hi, lo)
  const float2* d2_df;
  const float4* gdf;     // [(N/2+1)][M]: the g64 table as double-float, f32x2 form
  const double2* g64;    // [(N/2+1)][M]: lambda^{-1/2}/(2N), FP64 form
  const float2* ahat32;  // [N/2+1]: FFT_N(D a); the FP32 form evaluates lambda^{-1/2}/(2N) from
  const float2* bhat32;  // these two where it uses it
  const float2* g32;     // [(N/2+1)][M]: the table in FP32 for general commuting blocks (else null)
  int none;              // 1: identity preconditioner (MINRES-I)
};

// A fused "v = in0 + c1*in1 + c2*in2" load in FP64 (c1, c2 = coef[1], coef[2] from device
// memory; coef[0] is not used).
struct Combine {
  const double* in0;
  const double* in1;     // may be null
  const double* in2;     // may be null
  const double* coef;    // device, 3 doubles; null when in1 and in2 are null
  double* vout;          // if set, the combined value is stored here
};

// a whole DST-basis MINRES solve by one block (problems whose every phase is one FFT tile): the
// operator tables, the solve's vectors and the tile shapes of each phase
struct OneSolve {
  OpTables op;
  PrecTables pt;
  MinresDev* st;
  const double* f;       // right-hand side (physical basis)
  double* u;             // solution (physical basis)
  double* b;             // Y (I (x) U) f
  double* v[2];
  double* z[2];
  double* w[2];
  double* q;
  double* x;             // solution in the DST basis
  double* part;          // 8 partial-sum slots (one per reduction)
  int maxit;
  int log2NC_conv, log2NC_tp;
  int log2NC_dst[3];     // per axis
};

// preconditioner / transform arithmetic codes
enum { PREC_F32 = 32, PREC_F64 = 64, PREC_DF = 96 };

// launchers (kernels.cu); all return cudaGetLastError()
cudaError_t launch_dst(const OpTables& op, int axis, int prec, const Combine& in, double* out,
                       int flip, const double* dot_with, double* partials, int* nparts,
                       const int* phase, cudaStream_t st);
// blocks (= partial sums) of a single-item launch_timepass of this problem and precision
long long timepass_tiles(const OpTables& op, int prec);
cudaError_t launch_timepass(const OpTables& op, const PrecTables& pt, int prec, const Combine& in,
                            double* out, const double* dot_with, double* partials, int* nparts,
                            const int* phase, cudaStream_t st);
// matvec modes
enum MvMode { MV_STORE = 0, MV_RESID = 1 };
cudaError_t launch_matvec(const OpTables& op, int spectral, const double* x, const double* xscale,
                          double* y, int flip, int mode, const double* rhs, double* partials,
                          int* nparts, const int* phase, double* tmp, cudaStream_t st);
// tensor-core time product (tcmv.cu)
constexpr int kTcDigits = 5;          // bf16 digit planes per operand
bool tc_eligible(const OpTables& op); // b = b0 e_0, FFT-class a, N in {128, 256, 512, 1024}
int tc_strips(long long M);           // 128-line strips of the spatial index
size_t tc_workspace_bytes(int N, long long M);
// digit planes of the time-flipped a (host), eT with max|a| < 2^eT, ncores = 16 N/128 + 15
void tc_hankel_digits(const double* a, int N, uint16_t* out, int* eT, int* ncores);
// y = Y A (s x) or A (s x) (flip 0) with the time product on the tensor cores; partials (if not
// null) receive <y, s x> per block, *nparts their count.  launch_tc_matvec = launch_tc_digits
// (digit planes and line exponents of s x into the workspace) then launch_tc_product.
cudaError_t launch_tc_digits(const OpTables& op, const double* x, const double* xscale,
                             const int* phase, cudaStream_t st);
cudaError_t launch_tc_product(const OpTables& op, int spectral, const double* x,
                              const double* xscale, double* y, int flip, double* partials,
                              int* nparts, const int* phase, cudaStream_t st);
cudaError_t launch_tc_matvec(const OpTables& op, int spectral, const double* x,
                             const double* xscale, double* y, int flip, double* partials,
                             int* nparts, const int* phase, cudaStream_t st);
cudaError_t launch_setup_g64(const OpTables& op, const double2* ahat, const double2* bhat,
                             double2* g64, float4* gdf, cudaStream_t st);
cudaError_t launch_setup_gdf(const OpTables& op, const float2* ahat32, const float2* bhat32,
                             const float4* ahatdf, const float4* bhatdf, float4* gdf,
                             cudaStream_t st);
// dense-operator basis changes in double-float (dfgemm.cu): hi/lo planes of U and U^T
// (column-major), and C = A X for A given by its planes (M x M) and X, C time-major (M x N)
cudaError_t launch_df_planes(const double* U, long long M, float* Uh, float* Ul, float* Th,
                             float* Tl, cudaStream_t st);
cudaError_t launch_df_gemm(const float* Ah, const float* Al, const double* X, double* C, int M,
                           int N, cudaStream_t st);
cudaError_t launch_flip_copy(const double* f, double* b, int N, long long M, double* partials,
                             int* nparts, cudaStream_t st);
cudaError_t launch_scalar_init(MinresDev* s, const double* partials_zv, int nzv,
                               const double* partials_b, int nb, cudaStream_t st);
cudaError_t launch_scalar_delta(MinresDev* s, const double* partials, int np, cudaStream_t st);
cudaError_t launch_scalar_gamma(MinresDev* s, const double* partials, int np, cudaStream_t st);
cudaError_t launch_scalar_check(MinresDev* s, const double* partials, int np, cudaStream_t st);
cudaError_t launch_scalar_defer(MinresDev* s, cudaStream_t st);   // PH_CHECK -> PH_VERIFY
// the whole-solve block: nc of a phase's single tile (0 if it needs more than one tile), and the launch
int one_tile_columns(long long nlines, int Lfft, int cap_points = kCap);
// chosen: double-float product and DSTs with the FP32 time pass (else FP64 throughout)
cudaError_t launch_solve_one(const OneSolve& s, bool chosen, cudaStream_t st);
cudaError_t launch_w_update(MinresDev* s, const double* z, double* w_prev, const double* w,
                            double* x, long long n, cudaStream_t st);
cudaError_t launch_fold(const MinresDev* s, const FoldArgs& a, cudaStream_t st);
// u += d (FP64) and partial sums of ||x||^2 (iterative refinement)
cudaError_t launch_axpy(double* u, const double* d, long long n, cudaStream_t st);
cudaError_t launch_norm2(const double* x, long long n, double* partials, int* nparts,
                         cudaStream_t st);
cudaError_t launch_copy_scaled_check(const double* src, double* dst, long long n, cudaStream_t st);
cudaError_t launch_sum_partials(const double* partials, int np, double* out, cudaStream_t st);

// complex columns per tile for a line batch (tiles of `cap` complex points)
int tile_columns(long long nlines, int Lfft, int cap = kCap);
cudaError_t prepare_kernel_attributes();         // shared-memory limits of every tile kernel

// ---------------------------------------------------------------------------------------------
// Multi-item ("wave") launches for batched solves: one launch covers the tiles of many items
// (a system with one right-hand side each); persistent blocks stride over the concatenated tile
// list, find their item by binary search in `prefix` (prefix[i] = tiles of items < i), skip items
// whose phase differs from `want`, and run the same per-tile code as the single-item kernels.
struct ConvItem {
  OpTables op;
  const double* x;
  const double* xscale;   // device scalar or null
  double* y;
  const double* rhs;
  double* partials;
  const int* phase;
  int want, flip, mode, spectral, log2NC, pad;
};
struct TpItem {
  OpTables op;
  PrecTables pt;
  Combine cb;
  double* out;
  const double* dot_with;
  double* partials;
  const int* phase;
  int want, log2NC;
};
struct DstItem {
  long long nlines, inner, N, M;
  int m, P, log2P, log2NC, flip, pad;   // DST-I length m, FFT length P = m + 1
  Combine cb;
  double* out;
  const double* dot_with;
  double* partials;
  const void* tw;
};
struct VecItem {            // element-wise MINRES update (w, x) of one item
  const MinresDev* st;
  const double* z;
  double* w_prev;
  const double* w;
  double* x;
  long long n;
};
struct ScalItem {           // scalar recurrence of one item
  MinresDev* st;
  const double* p0;         // partials for the first reduction
  const double* p1;         // partials for the second (init only)
  int n0, n1;
};

int persistent_grid(int kind, int prec);   // resident blocks for a multi-item launch

// handle internals used by the batched driver (defined in bltt_api.cu)
const OpTables& ctx_op(bltt_handle h);
bltt_status ctx_prepare(bltt_handle h, double alpha, int prec);
PrecTables ctx_prec_tables(bltt_handle h);
long long ctx_n(bltt_handle h);
cudaError_t launch_conv_multi(int arith, const ConvItem* items, const long long* prefix,
                              int nitems, long long total, cudaStream_t st);
cudaError_t launch_timepass_multi(int prec, const TpItem* items, const long long* prefix,
                                  int nitems, long long total, cudaStream_t st);
cudaError_t launch_dst_multi(int prec, const DstItem* items, const long long* prefix, int nitems,
                             long long total, cudaStream_t st);
cudaError_t launch_w_update_multi(const VecItem* items, int nitems, cudaStream_t st);
struct FoldItem {           // deferred-update fold of one item (its state decides the request)
  const MinresDev* st;
  FoldArgs a;
};
// kmax: the largest window among the items
cudaError_t launch_fold_multi(const FoldItem* items, int nitems, int kmax, cudaStream_t st);
// which: 0 init, 1 delta, 2 gamma, 3 check
cudaError_t launch_scalar_multi(int which, const ScalItem* items, int nitems, cudaStream_t st);
cudaError_t launch_count_running(const ScalItem* items, int nitems, int* out, cudaStream_t st);

}  // namespace bltt
