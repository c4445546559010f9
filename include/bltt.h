/*
 * bltt.h - C ABI of libbltt: preconditioned MINRES for block lower triangular Toeplitz (BLTT)
 * all-at-once systems A u = f, on one GB300 GPU (sm_103a).
 *
 * Method (arXiv 2307.07749): time-reverse the system to the symmetric indefinite form
 * Y A u = Y f (Sec. 2, eq. symmetrizedblttsys) and solve it by preconditioned MINRES with the
 * absolute-value block alpha-circulant preconditioner P_alpha = |C_alpha| (Sec. 3, eqs.
 * tensordef2calpha, calphaabsdef, precdef), applied as in Sec. 5.1.
 *
 * Problem class: blocks A_(k) = a_k I + b_k L, k = 0..N-1 (eq. amatdef), L = -Delta_h the
 * central-difference Dirichlet Laplacian on a uniform d-dimensional grid (d = 1, 2, 3), which the
 * normalised DST-I diagonalises (Sec. 5.1).  The blocks commute (Assumption 1 (i)) by construction.
 *
 * Vector layout everywhere: time-major, u[n*M + i], n = 0..N-1 the time step, i the lexicographic
 * spatial index with x fastest; M = m[0]*...*m[d-1].  Vectors are contiguous FP64.
 *
 * Conventions shared by every entry point:
 *  - Memory: vector arguments named *_dev are caller-owned device pointers (e.g. torch tensors),
 *    8-byte aligned, length N*M; the library never frees them.  All other pointers are host memory.
 *    The library owns its tables and workspace (allocated in bltt_create / on first use).
 *  - Streams: work is issued on the handle's stream (bltt_set_stream; default: the legacy
 *    stream).  bltt_matvec and bltt_precond_apply are asynchronous; bltt_minres_solve synchronises
 *    on that stream to fill its info struct.
 *  - Errors: every call returns a bltt_status; nothing aborts, exits or traps.  A failed call
 *    leaves outputs unspecified; bltt_last_error(h) returns a message for the last failure on h.
 *  - Threads: a handle is not thread-safe; distinct handles may be used from distinct threads.
 *  - Sizes: N and every m[ax]+1 must be powers of two with 2 <= N <= 2048 and
 *    2 <= m[ax]+1 <= 2048 (each FFT, of length 2N or 2(m+1), must fit one 4096-point tile);
 *    other sizes return BLTT_ERR_UNSUPPORTED.
 */
#ifndef BLTT_H
#define BLTT_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct bltt_ctx* bltt_handle;

typedef enum {
  BLTT_OK = 0,
  BLTT_ERR_INVALID_ARG = 1,   /* null pointer, alpha outside (0,1], bad sizes or flags        */
  BLTT_ERR_ASSUMPTION = 2,    /* Assumption 1 (ii) fails: c0 = min_i(l_i^(0) - sum|l_i^(k)|) <= 0 */
  BLTT_ERR_OOM = 3,           /* device allocation failed                                      */
  BLTT_ERR_CUDA = 4,          /* a CUDA runtime call failed                                    */
  BLTT_ERR_NUMERIC = 5,       /* NaN/Inf in the data or <z, v> < 0 (MINRES breakdown)           */
  BLTT_ERR_NOT_CONVERGED = 6, /* maxit reached before the stopping rule held                   */
  BLTT_ERR_TIMEOUT = 7,       /* a bounded device-side wait gave up                            */
  BLTT_ERR_UNSUPPORTED = 8    /* sizes outside the supported set                               */
} bltt_status;

/* Spatial grid: ndim in {1,2,3}, m[ax] interior points and spacing h[ax] per axis (x first).
 * L = -Delta_h with zero Dirichlet values (Sec. 5.2). Unused axes are ignored. */
typedef struct {
  int ndim;
  int m[3];
  double h[3];
} bltt_space;

/* The BLTT matrix: N blocks A_(k) = a[k] I + b[k] L (eq. amatdef).  a, b: host arrays of length N,
 * copied by bltt_create. */
typedef struct {
  int N;
  const double* a;
  const double* b;
  bltt_space space;
} bltt_blocks;

/* Arithmetic of the preconditioner apply: FP64, FP32, or double-float (F32X2: FP64-accurate to
 * about 1e-14 relative, computed on the FP32 pipes).  The matvec, the Lanczos recurrences and the
 * true residual stay FP64-accurate whatever this is; vectors are FP64 in memory throughout. */
enum { BLTT_PREC_F64 = 64, BLTT_PREC_F32 = 32, BLTT_PREC_F32X2 = 96 };

/* Basis the MINRES vectors live in during the iteration.  SPECTRAL: the DST-I basis of the
 * blocks (U is orthogonal and symmetric, Sec. 3), so the loop needs no DST; the iterates are the
 * physical ones multiplied by I (x) U.  PHYSICAL: the textbook form, DSTs inside P_alpha^{-1}.
 * AUTO picks SPECTRAL. */
enum { BLTT_BASIS_AUTO = 0, BLTT_BASIS_SPECTRAL = 1, BLTT_BASIS_PHYSICAL = 2 };

/* Preconditioner kind: ABAC P_alpha (alpha = 1 gives the absolute-value block circulant P_1),
 * or none (MINRES-I, the paper's unpreconditioned comparison solver, Sec. 5.2). */
enum { BLTT_PRECOND_ABAC = 0, BLTT_PRECOND_NONE = 1 };

/* Arithmetic of the FFT matvec (the 2N circulant-embedding time convolution).  F64: native FP64.
 * F32X2: every value carried as an unevaluated sum of two FP32 numbers (double-float, about 48
 * significant bits) and computed on the FP32 pipes, which GB300 runs at 58x its FP64 rate; the
 * product stays FP64 in memory and agrees with the FP64 result to about 1e-14 relative.
 * TC: the time convolution of the in-loop products y = Y A z (not the residual checks, which stay
 * F32X2) runs on the tensor cores as a dense product with the time-flipped Toeplitz (Hankel)
 * matrix of a: x and a are split into five balanced 8-bit digits relative to a power-of-two
 * bound of each spatial line (of a), the digit products are exact bf16 x bf16 -> FP32 tensor-core
 * sums, and the b_0 term and the scale are double-float.  Relative error about 2^-40 of
 * sum_k |a_k| |x_k| per element.  Requires b = b_0 e_0, an FFT-class a (more than 4 nonzeros)
 * and N in {128, 256, 512, 1024}; elsewhere it is BLTT_ERR_UNSUPPORTED.  Uses a workspace of
 * N * 128 * ceil(M/128) * 8 bytes, allocated on first use.  Every wait of its kernel is bounded:
 * a wait for progress gives up after about a second (BLTT_TC_WAIT_CYCLES in the environment, in
 * SM cycles, shortens it), the block then drains its own copies and MMAs and frees its tensor
 * memory, and the solve returns BLTT_ERR_TIMEOUT with the context still usable.
 * DEFAULT: the handle's setting (F64 unless bltt_set_matvec_arith changed it). */
enum { BLTT_ARITH_DEFAULT = 0, BLTT_ARITH_F64 = 1, BLTT_ARITH_F32X2 = 2, BLTT_ARITH_TC = 3 };

typedef struct {
  int precision;     /* BLTT_PREC_F64 (default when 0) or BLTT_PREC_F32                        */
  int basis;         /* BLTT_BASIS_*                                                            */
  int precond;       /* BLTT_PRECOND_*                                                          */
  int sync_every;    /* iterations issued between host checks of the device state (0: 2); in
                        graph replay the first check of a solve comes after as many blocks of
                        them as the previous solve on the handle needed (at most 8): iterations
                        past the stop return at once on the device                              */
  int rebuild;       /* 1: rebuild the per-alpha preconditioner tables even if cached            */
  int matvec_arith;  /* BLTT_ARITH_*                                                             */
  int no_graph;      /* 1: launch every kernel directly; 0: capture sync_every (rounded up to even)
                        iterations in a CUDA graph, cached per handle, and replay it whenever the
                        handle's stream is not the legacy stream (which cannot be captured); with
                        profiling on, the graph carries event-record nodes around each kernel    */
  int single_block;  /* 1: run the whole solve (entry transform, every iteration, exit transform)
                        in one kernel launch of one thread block, for problems whose every phase
                        is one FFT tile (e.g. N = 64, m = 63); DST basis, the FFT product, device
                        buffers, ABAC, and either FP64 throughout (precision 64, matvec F64) or
                        the FP32 preconditioner with the double-float product and DSTs (precision
                        32, matvec F32X2); the true residual is checked in the DST basis inside the
                        loop.  Else BLTT_ERR_UNSUPPORTED.                                          */
  int defer_window;  /* deferred solution update.  MINRES updates its direction vectors w and the
                        iterate x every iteration (Sec. 4: three vectors read, two written).  With a
                        window of S iterations the first S iterations instead keep their
                        preconditioned vectors z_0 .. z_{S-1} in S - 1 extra workspace vectors and
                        track x and w as coefficients over them; x is formed by one pass over the
                        stored z's when a stop or a true-residual check needs it, and the two w
                        vectors once, if the iterations go past the window.  Same iterates up to
                        rounding.  0: S = 8; 1..16: S (rounded down to a multiple of the graph
                        block, at least one block); -1: off (an update every iteration).  If the
                        extra vectors cannot be allocated the solve runs without the window.      */
  int refine;        /* mixed-precision iterative refinement, the fallback of the precision forms
                        (a reduced-precision preconditioner can make MINRES's recurrences drift
                        from the true residual and stall): 0 off.  k > 0: every MINRES solve runs
                        at most ceil(maxit / (k + 1)) iterations and ends at a failed
                        true-residual check instead of resuming; then, up to k times, the
                        residual r = f - A u is formed by a fresh FP64-accurate product in the
                        physical basis, A d = r is solved by MINRES to the tolerance that brings
                        ||f - A u|| / ||f|| to tol, and u += d.  The corrections raise an FP32
                        preconditioner to double-float; a first FP32 solve that broke down
                        restarts from u = 0.  maxit covers all solves, info->iters sums them,
                        info->refinements counts the corrections and info->relres_true is the
                        final fresh residual.  A solve that converges within its share is
                        unchanged.  Not for a dense operator or block spectra (the physical
                        product needs the blocks themselves): BLTT_ERR_UNSUPPORTED there.      */
} bltt_solve_opts;

typedef struct {
  int iters;              /* MINRES iterations (one matvec + one preconditioner apply each)    */
  double relres_est;      /* |eta_j| / eta_0: P^{-1}-norm residual estimate of the recurrence  */
  double relres_true;     /* ||Y f - Y A u||_2 / ||Y f||_2, recomputed in FP64 at the end      */
  double alpha_used;
  int alpha_source;       /* 0: caller, 1: learned predictor, 2: fallback rule alpha = 1e-8    */
  int precision;          /* preconditioner precision used (64 or 32)                          */
  int basis;              /* basis used (BLTT_BASIS_SPECTRAL or BLTT_BASIS_PHYSICAL)           */
  double t_setup_ms;      /* per-alpha preconditioner set-up (device time)                     */
  double t_solve_ms;      /* whole solve incl. set-up, device time on the handle's stream      */
  long long kernel_launches; /* kernels issued by the solve                                    */
  int status;             /* bltt_status of the solve                                          */
  int refinements;        /* outer corrections of bltt_solve_opts.refine that ran (else 0)     */
} bltt_solve_info;

/* Create a handle for the BLTT matrix `blocks` with N time steps and M spatial unknowns
 * (M must equal prod(m)).  Checks Assumption 1 (ii) (Proposition after Lemma 3.1): with
 * mu_i the eigenvalues of L, c0 = min_i (a_0 + b_0 mu_i - sum_{k>=1} |a_k + b_k mu_i|) must be
 * > 0, else BLTT_ERR_ASSUMPTION.  Builds the matvec spectra FFT_{2N}([a;0]), FFT_{2N}([b;0])
 * (Sec. 5.1, the FFT matvec) and the per-axis eigenvalue tables; allocates no vector workspace.
 * *out receives the handle (NULL on failure). */
bltt_status bltt_create(const bltt_blocks* blocks, int N, long long M, bltt_handle* out);

/* Release the handle, its tables and workspace.  NULL is accepted. */
bltt_status bltt_destroy(bltt_handle h);

/* Variable coefficient (Sec. 5.2, Example heateqvarcoeff): the blocks become A_(k) = a_k I + b_k L_a
 * with L_a = -Delta_{a,h}, the central-difference discretisation of -div(a grad) with zero
 * Dirichlet values: per axis, (L_a u)_c = [a_{c-1/2} (u_c - u_{c-1}) + a_{c+1/2} (u_c - u_{c+1})]/h^2.
 *   face[ax] (host, ax < d): a at the faces along axis ax, an array of the grid's shape with that
 *     axis one longer, x fastest; entry f along the axis sits between points f-1 and f of its line
 *     (f = 0 and f = m_ax are the boundary faces).  (m_ax + 1) * M / m_ax positive finite values.
 *   abar: the preconditioner is built for the blocks a_k I + abar b_k L (eq. meancoeffheateqtsmat;
 *     the paper takes the mean of a over the grid points); > 0.
 * Matvecs and solves then use L_a.  Solves run in the physical basis (AUTO picks it; SPECTRAL
 * gives BLTT_ERR_UNSUPPORTED: the DST does not diagonalise L_a), and the tensor-core product is
 * unsupported.  The face arrays are copied to the device; a later call replaces them. */
bltt_status bltt_set_variable_coefficient(bltt_handle h, const double* const* face, double abar);

/* Dense commuting blocks (Sec. 3: the blocks A_(k) = a_k I + b_k K share the eigenvectors of one
 * symmetric K, so the preconditioner of Sec. 5.1 applies with K's eigenbasis in place of the
 * DST-I).  K (host): M x M, row-major (symmetric, so either order), finite, symmetric to 1e-12 of
 * its largest entry; M <= 8192.  The handle computes K = U diag(mu) U^T once on the device (a
 * cuSOLVER symmetric eigensolver: set-up, not the hot path) and re-checks Assumption 1 (ii) with
 * mu (BLTT_ERR_ASSUMPTION if it fails; the handle then keeps its previous operator).  Matvecs,
 * preconditioner applies and solves then use K: the solve runs in the eigenbasis (AUTO and
 * SPECTRAL; PHYSICAL gives BLTT_ERR_UNSUPPORTED), entering and leaving it by one GEMM each, with
 * the true residual checked there (U orthogonal: the same norm as in the physical basis).  The
 * GEMMs follow the matvec arithmetic: FP64 (cuBLAS) with BLTT_ARITH_F64, double-float on the
 * FP32 pipes (about 2^-47 relative per multiply-add) with BLTT_ARITH_F32X2.  The handle keeps U
 * in FP64 (M^2 doubles) and as double-float planes of U and U^T (4 M^2 floats).  bltt_matvec
 * and bltt_precond_apply take and return physical-basis vectors (a GEMM on each side).  Exclusive with bltt_set_variable_coefficient and the tensor-core matvec
 * (BLTT_ERR_UNSUPPORTED).  A later call replaces K. */
bltt_status bltt_set_dense_operator(bltt_handle h, const double* K);

/* General commuting symmetric blocks (Assumption 1 (i); Sec. 3): the blocks share one
 * orthonormal eigenbasis U, A_(k) = U diag(lam_k) U^T, and need not be a_k I + b_k L or
 * functions of one operator.  The preconditioner of Sec. 5.1 then applies with U in place of the
 * DST-I and each mode's own eigenvalue sequence lam_i^(k) in place of a_k + b_k mu_i.
 *   U (host): M x M, row-major, column i the eigenvector of mode i; its columns must be
 *     orthonormal (probed with two fixed vectors: ||U^T U x - x|| <= 1e-10 ||x||, else
 *     BLTT_ERR_INVALID_ARG).  lam (host): N*M values, lam[k*M + i] the eigenvalue of A_(k) on
 *     column i of U.  Both finite; M <= 8192.
 * Assumption 1 (ii) is checked on lam: min_i (lam_i^(0) - sum_{k>=1} |lam_i^(k)|) > 0, else
 * BLTT_ERR_ASSUMPTION (the handle then keeps its previous operator).  From then on the handle's
 * blocks are these: the a, b given to bltt_create are no longer used (any that pass its check
 * will do, e.g. a = e_0, b = 0), but M = prod(m) and N still hold.
 * Arithmetic: the matvec is the 2N-embedding FFT product with a per-mode spectrum
 * FFT_2N([lam_i; 0]) (tables of (N+1) M complex values, FP64 and double-float, built on the
 * host here); the preconditioner's per-(frequency, mode) tables lambda^{-1/2}/(2N) of
 * eq. hatcalphaieigvaldef are built on the host for each new alpha (one FFT of length N per
 * mode, FP64, double-float and FP32 copies of (N/2+1) M entries).  Solves run in U's basis
 * (AUTO and SPECTRAL; PHYSICAL gives BLTT_ERR_UNSUPPORTED) with one GEMM in and one out and the
 * true residual checked there, as after bltt_set_dense_operator; bltt_matvec and
 * bltt_precond_apply take and return physical vectors.  Not with bltt_set_variable_coefficient,
 * the tensor-core product or the single-block solve (BLTT_ERR_UNSUPPORTED).  A later call, or
 * bltt_set_dense_operator, replaces the blocks. */
bltt_status bltt_set_block_spectra(bltt_handle h, const double* U, const double* lam);

/* Issue all later work of h on `cuda_stream` (a cudaStream_t; NULL = legacy default stream). */
bltt_status bltt_set_stream(bltt_handle h, void* cuda_stream);

/* Set the handle's matvec arithmetic (BLTT_ARITH_F64, _F32X2 or _TC); used by bltt_matvec
 * and by solves whose opts leave matvec_arith at DEFAULT.  Blocks with at most 4 nonzero
 * coefficients use the direct shifted sum in FP64 whatever this setting. */
bltt_status bltt_set_matvec_arith(bltt_handle h, int arith);

/* y = A x (flip = 0) or y = Y A x (flip = 1), A the BLTT matrix (eq. amatdef), Y = Y_N (x) I_M
 * the time reversal (Sec. 2).  The time convolution runs as a 2N zero-padded circulant
 * product with FFTs along time, or as a direct shifted sum when a and b have at most 4 leading
 * nonzeros (Sec. 5.1, the O(MN log N) matvec); L acts as the 2d+1 point stencil.  FP64.
 * x_dev and y_dev must not overlap. */
bltt_status bltt_matvec(bltt_handle h, const double* x_dev, double* y_dev, int flip);

/* z = P_alpha^{-1} v = C_alpha^{-1/2} (C_alpha^{-1/2})^* v (Sec. 5.1): DST-I of every time slice,
 * per spatial mode the alpha-scaled time pass D F conj(Lambda)^{-1/2} F^* D^{-1} followed by
 * D^{-1} F Lambda^{-1/2} F^* D (eqs. hatcalphaidiagform, sqrtcalphabdiagform), inverse DST-I.
 * 0 < alpha <= 1.  precision: BLTT_PREC_* (arithmetic of the whole apply; v and z stay FP64).
 * v_dev and z_dev may be equal (in place). */
bltt_status bltt_precond_apply(bltt_handle h, double alpha, const double* v_dev, double* z_dev,
                               int precision);

/* Solve A u = f through MINRES on Y A u = Y f with P_alpha (Sec. 2-3, Sec. 5).  Zero initial
 * guess (Sec. 5.2).  Stops when the recurrence estimate |eta_j|/eta_0 <= tol and then the true
 * relative residual ||Yf - YAu||/||Yf|| <= tol (both FP64-accurate); otherwise iterates on, up
 * to maxit.  In the DST basis the true residual is the physical-basis one of the returned u,
 * computed after the exit transform (the iterations resume if it misses tol).
 * f_dev: the unflipped right-hand side; u_dev: the solution (may not alias f_dev).
 * opts may be NULL (FP64, AUTO basis, ABAC).  info (host, may be NULL) receives the statistics.
 * Returns BLTT_OK, BLTT_ERR_NOT_CONVERGED (u holds the last iterate), BLTT_ERR_NUMERIC, ... */
bltt_status bltt_minres_solve_ex(bltt_handle h, const double* f_dev, double alpha, double tol,
                                 int maxit, const bltt_solve_opts* opts, double* u_dev,
                                 bltt_solve_info* info);

/* Same as bltt_minres_solve_ex with opts = {precision, AUTO, ABAC, 0}. */
bltt_status bltt_minres_solve(bltt_handle h, const double* f_dev, double alpha, double tol,
                              int maxit, int precision, double* u_dev, bltt_solve_info* info);

/* The solve of bltt_minres_solve_ex (Sec. 2-3, Sec. 5) with f and u in HOST memory: f_host (N*M
 * doubles) is copied into a device staging buffer on the handle's stream, and u goes back into
 * u_host on a second stream of the handle as soon as it is final, overlapping the physical-basis
 * residual check that ends the solve; above 2^22 unknowns in the DST basis, f arrives in four
 * chunks of time slices whose entry transforms start as each lands.  Pinned host buffers (cudaHostAlloc / cudaHostRegister)
 * make both copies asynchronous DMA; pageable ones work but are staged by the driver.  The first
 * call allocates the two staging vectors and the copy stream; they live until bltt_destroy.
 * Returns when u_host holds the result (same statuses as bltt_minres_solve_ex; u_host may not
 * alias f_host; a status raised before the iterations end leaves u_host untouched).  The paper has no host-memory variant: it is the end-to-end form of its solve. */
bltt_status bltt_minres_solve_host(bltt_handle h, const double* f_host, double alpha, double tol,
                                   int maxit, const bltt_solve_opts* opts, double* u_host,
                                   bltt_solve_info* info);

/* Solve many BLTT systems with several right-hand sides each, together (batching: one launch per
 * MINRES phase covers every (system, right-hand side) item of a wave below 2^21 unknowns, and each
 * larger item, which fills the GPU by itself, gets its own launch of that phase; the phase
 * sequence of two iterations is captured in a CUDA graph and replayed until every item has
 * stopped).  Each item
 * is the solve of bltt_minres_solve_ex in the DST basis (Sec. 2-3, Sec. 5) with its own MINRES
 * state; the items of one system share its tables.  Waves are sized to 85% of the free device
 * memory (or to the byte count in the environment variable BLTT_BATCH_MAX_BYTES, if smaller);
 * the tile widths of the shared launches come from a built-in autotuner (opts->sync_every < 0
 * disables it).
 *   nsys systems sys[s] (host structs as for bltt_create; N and m[ax]+1 powers of two) with
 *   nrhs[s] >= 1 right-hand sides each; f_dev / u_dev: host arrays of sum(nrhs) device pointers
 *   (system-major), each a vector of that system's N*M doubles, u not aliasing f.
 *   alpha: host array of nsys values in (0,1], or NULL for the default rule (1e-8; 1e-2 for the
 *   FP32 preconditioner and 1e-6 for the double-float one, where their rounding costs no
 *   iteration against FP64 at the same alpha).  opts: precision, matvec_arith and defer_window
 *   as for bltt_minres_solve_ex (basis is always the DST basis; refine is not applied); may be
 *   NULL.  info: host array of sum(nrhs) entries or NULL;
 *   relres_true is the true residual of the DST-basis system (equal to the physical one up to
 *   the rounding of the exit DST).
 * Returns BLTT_OK when every item converged, else the first failing item's status.  Systems whose
 * blocks have at most 4 nonzero coefficients (the direct matvec) give BLTT_ERR_UNSUPPORTED. */
bltt_status bltt_solve_batched(int nsys, const bltt_blocks* sys, const int* nrhs,
                               const double* const* f_dev, double* const* u_dev,
                               const double* alpha, double tol, int maxit,
                               const bltt_solve_opts* opts, bltt_solve_info* info);

/* ---- learned alpha --------------------------------------------------------------------------
 * A small MLP predicts the alpha that minimises the MINRES iterations of a problem from four
 * features (log N, log M, gamma, log(tau/h^2)); the paper fixes alpha = 1e-8 (Sec. 5.2) and its
 * Theorem 1 only bounds alpha from above, so the network is an addition of this library, trained
 * on alpha sweeps run by this solver.  Network: 4 -> 32 -> 32 -> 1, tanh hidden layers, FP32.
 * Model: a host array of BLTT_ALPHA_MODEL_FLOATS floats laid out as W1[32][4], b1[32], W2[32][32],
 * b2[32], w3[32], b3 (the 1249 trainable parameters), then mean[4], std[4] of the features and
 * y_mean, y_std of the label log10(alpha): the network maps (x - mean)/std to
 * (log10(alpha) - y_mean)/y_std.  The caller initialises the parameters (no random draws inside).
 * Loss: mean squared error over the n samples.  All three calls allocate device memory for their
 * inputs and scratch and synchronise the legacy stream.  std and y_std must be > 0, else
 * BLTT_ERR_INVALID_ARG. */
#define BLTT_ALPHA_MODEL_FLOATS 1259
#define BLTT_ALPHA_NPARAM 1249

/* Gradient of the loss w.r.t. the 1249 parameters (grad_out, host) and the loss (loss_out, host,
 * may be NULL), by one forward and one backward pass over the n samples (feats: [n][4] host,
 * labels: n values of log10(alpha), host). */
bltt_status bltt_alpha_grad(const float* model, const float* feats, const float* labels, int n,
                            float* grad_out, float* loss_out);

/* Train `model` in place: `epochs` full-batch Adam steps (learning rate lr, beta1 0.9, beta2
 * 0.999, eps 1e-8) on the n samples.  loss_hist (host, may be NULL) receives the loss before each
 * step.  One CUDA block runs the whole training; sums over samples run in a fixed order. */
bltt_status bltt_alpha_train(float* model, const float* feats, const float* labels, int n,
                             int epochs, float lr, float* loss_hist);

/* alpha_out[s] = 10^(network(feats[s])) for n feature rows (host arrays). */
bltt_status bltt_alpha_predict(const float* model, const float* feats, int n, float* alpha_out);

/* Per-kernel device time, collected with CUDA events around every launch on the handle's
 * stream while profiling is enabled (tracing aid; adds two event records per launch). */
typedef struct {
  char name[24];          /* kernel family: conv, conv_df, direct, dst64, dst32, timepass64, ... */
  long long launches;     /* all launches, including ones that returned at once because the   */
  double total_ms;        /* solve had already converged (device-side early exit)            */
  long long active_launches;  /* launches that took more than 1/4 of the family's longest one */
  double active_ms;
} bltt_kernel_stat;

/* Enable (1) or disable (0) per-launch timing on h; either way the counters are reset. */
bltt_status bltt_profile_enable(bltt_handle h, int enable);

/* Synchronise h's stream and copy up to max_entries statistics to out (host array).  Returns the
 * number of kernel families recorded (may exceed max_entries), or -1 for a NULL handle. */
int bltt_profile_read(bltt_handle h, bltt_kernel_stat* out, int max_entries);

/* Guard bands, a substitute for a memory checker (no counterpart in the paper).  With
 * BLTT_GUARD_BANDS=1 in the environment when h first allocates its solve workspace, every
 * workspace vector and every deferred-update slot sits between bands of 256 doubles that hold a
 * fixed NaN bit pattern no kernel writes.  bltt_check_guards synchronises h's stream, reads every
 * band back and returns BLTT_ERR_CUDA (with the band and element in bltt_last_error) if one was
 * overwritten, else BLTT_OK; *bands_checked (may be NULL) receives the number of bands read (0
 * without guard bands).  bltt_guard_poke writes one element of workspace band `band` from the
 * host (0 <= band <= 10): a hook for the tests of the check itself; BLTT_ERR_INVALID_ARG without
 * guard bands or for another band. */
bltt_status bltt_check_guards(bltt_handle h, int* bands_checked);
bltt_status bltt_guard_poke(bltt_handle h, int band);

/* Relative true residual ||f - A u||_2 / ||f||_2 of a candidate solution u of A u = f (and, if
 * r_dev is not NULL, the residual vector r = f - A u), with neither a handle nor any allocation.
 * The paper has no counterpart: this entry point exists for callers that cannot allocate memory
 * at all, e.g. code running under an allocator or memory pool that forbids new device
 * allocations, or a host process with a fixed device-memory budget, which therefore cannot call
 * bltt_create (it allocates tables and workspace).  It calls no cudaMalloc, cudaFree,
 * cudaMallocHost or allocating library routine.
 *   blocks, N, M: as for bltt_create (the Assumption 1 check is not made).  u_dev, f_dev,
 *   r_dev: caller-owned device vectors of N*M doubles; r_dev may be NULL and must not alias u or
 *   f.  cuda_stream: the stream to run on (NULL: legacy stream).  The call copies its operator
 *   tables from host memory on that stream and synchronises the stream before it returns, to
 *   hand the residual to the host.  relres_out: host double receiving the relative residual (the
 *   absolute norm when f = 0).  Arithmetic: FP64, with the same kernels as bltt_matvec.
 * Scratch: one file-scope device array of 2 MiB, loaded with the operator tables and the partial
 * sums on every call.  It is shared by every call in the process and keeps the last call's
 * contents; calls whose work overlaps on the GPU (other threads, other streams) race on it and
 * must be serialised by the caller.  Every value a call reads from it is written earlier in the
 * same call, so nothing needs clearing.  Set-up: the first call on each device (with that device
 * current) looks up the array's device address with cudaGetSymbolAddress; make that first call
 * before any stream capture.
 * Limits (else BLTT_ERR_UNSUPPORTED): the sizes of bltt_create (N and every m[ax]+1 powers of
 * two, at most 2048); at most 131072 FFT tiles (spatial modes / tile width); and blocks with more
 * than 4 nonzero coefficients need b = b0 e_0 (otherwise an N*M temporary would be needed).
 * Other errors: BLTT_ERR_INVALID_ARG, BLTT_ERR_CUDA, BLTT_ERR_NUMERIC (a non-finite block
 * coefficient or residual). */
bltt_status bltt_residual_noalloc(const bltt_blocks* blocks, int N, long long M,
                                  const double* u_dev, const double* f_dev, double* r_dev,
                                  void* cuda_stream, double* relres_out);

/* Message for the last failed call on h ("" if none); for h == NULL, the last failure of
 * bltt_create on this thread.  The string stays valid until the next call on h. */
const char* bltt_last_error(bltt_handle h);

/* Library version string. */
const char* bltt_version(void);

#ifdef __cplusplus
}
#endif
#endif /* BLTT_H */
