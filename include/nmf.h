/*
 * nmf.h -- C ABI of libnmf: compressed NeNMF on one GB300 GPU (sm_103a).
 *
 * The problem (eq. 1): X ~= G F with X (n x m) nonnegative, G (n x p) >= 0,
 * F (p x m) >= 0. NeNMF alternately solves eq. (2) for G and eq. (3) for F by
 * an inner Nesterov loop (Sec. 2). Compressed NeNMF (Alg. 1) runs the same
 * loop on X_L = L X and X_R = X R, where L (nu x n) and R (m x nu) come from
 * the randomized subspace iteration of Alg. 2.
 *
 * Conventions shared by every call
 *  - Matrices are dense, row-major, float32 (float64 in the *_f64 twins), with
 *    the leading dimension equal to the number of columns (no padding): X is n x m, G is n x p, F is p x m,
 *    L is nu x n, R is m x nu, X_L is nu x m, X_R is n x nu.
 *  - Every matrix pointer is DEVICE memory owned by the caller, unless a
 *    parameter says "host". The library keeps no pointer after a call returns.
 *  - The library allocates no device memory. Each call that needs scratch space
 *    has a *_workspace_size() query; the caller passes that many bytes of
 *    device memory, 256-byte aligned. Workspace contents need no initialisation
 *    and are not meaningful after the call.
 *  - Calls are asynchronous and stream ordered on `stream` (a cudaStream_t;
 *    NULL is the legacy default stream). They return after enqueueing work.
 *    Argument errors are detected on the host, before anything is enqueued.
 *  - Errors found on the device (non-finite values, a Cholesky breakdown the
 *    shifted retry could not repair, a bounded wait that ran out) are written
 *    to a status word in the workspace; nmf_workspace_status() reads it after
 *    the stream has reached that point. A later kernel of the same call turns
 *    into a no-op once that word is nonzero.
 *  - Sizes: 1 <= p <= NMF_MAX_RANK, p <= nu <= NMF_MAX_SKETCH, nu <= min(n, m).
 */
#ifndef NMF_H
#define NMF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* nmf_stream_t; /* identical to cudaStream_t */

typedef enum nmf_status {
  NMF_OK = 0,
  NMF_ERR_INVALID_ARG = 1,    /* bad size, null pointer, unsupported combination */
  NMF_ERR_WORKSPACE = 2,      /* workspace null, too small or misaligned */
  NMF_ERR_CUDA = 3,           /* a CUDA runtime call failed (launch, config) */
  NMF_ERR_NOT_SPD = 4,        /* Gram matrix not positive definite even after the shift */
  NMF_ERR_NONFINITE = 5,      /* NaN or Inf met on the device */
  NMF_ERR_DEVICE_TIMEOUT = 6, /* a bounded device-side wait gave up */
  NMF_ERR_UNSUPPORTED = 7     /* device is not sm_103 or feature not built */
} nmf_status_t;

typedef enum nmf_prec {
  NMF_PREC_FP32 = 0, /* X products in float32 on CUDA cores */
  NMF_PREC_BF16 = 1  /* X rounded once to bfloat16; products on tcgen05 tensor cores, float32 accumulate */
} nmf_prec_t;

enum { NMF_MAX_RANK = 32, NMF_MAX_SKETCH = 64 };

/* Human-readable name of a status code (static storage). */
const char* nmf_status_string(nmf_status_t status);

/* Library ABI version: 100 * major + minor. */
int nmf_version(void);

/*
 * Reads the device status word of a workspace used by an earlier call.
 * Blocks until `stream` has drained. *status receives an nmf_status_t value.
 */
nmf_status_t nmf_workspace_status(nmf_stream_t stream, const void* workspace, int* status);

/* ------------------------------------------------------------------------ */
/* Gaussian sketches (Alg. 2: the two Gaussian test matrices)                */
/* ------------------------------------------------------------------------ */
/*
 * out (rows x cols, device, row-major) <- iid N(0, 1) values, counter-based:
 * element e uses Philox4x32-10 (Salmon et al. 2011) at counter
 * (e/4 mod 2^32, (e/4) >> 32, stream_id, 0) with key (seed mod 2^32, seed >> 32);
 * the four words x0..x3 map to u_j = ((x_j >> 9) + 0.5) / 2^23 and Box-Muller
 * pairs (u0, u1) -> elements 4g, 4g+1 and (u2, u3) -> 4g+2, 4g+3 (cos, sin).
 * nmf_compress uses stream_id 0 for Omega_L (m x nu) and 1 for Omega_R (nu x n).
 */
nmf_status_t nmf_gaussian_sketch(nmf_stream_t stream, int rows, int cols, uint64_t seed,
                                 uint32_t stream_id, float* out);

/* ------------------------------------------------------------------------ */
/* Compression: randomized subspace iteration (Alg. 2) and X_L, X_R (Alg. 1) */
/* ------------------------------------------------------------------------ */
size_t nmf_compress_workspace_size(int n, int m, int nu, nmf_prec_t prec);

/*
 * Alg. 2 with q power steps, each orthonormalisation a CholeskyQR2 whose Gram
 * matrix is accumulated, factorised and inverted in extended (float-float)
 * precision; then X_L = L X and X_R = X R (the compression step of Alg. 1).
 *
 *  X        n x m input, nonnegative (not checked).
 *  omega_L  m x nu Gaussian sketch, or NULL to draw it from `seed` (stream 0).
 *  omega_R  nu x n Gaussian sketch, or NULL to draw it from `seed` (stream 1).
 *           Both NULL or both non-NULL.
 *  L        out, nu x n, orthonormal rows: L = (Q_L^(q))^T.
 *  R        out, m x nu, orthonormal columns: R = (Q_R^(q))^T.
 *  XL       out, nu x m, X_L = L X.
 *  XR       out, n x nu, X_R = X R.
 * Alg. 2's output step names the half-step bases Q~^(q), which have the
 * wrong shapes; the full-step bases Q^(q) are used. prec selects how the
 * 2q+2 passes over X compute: NMF_PREC_BF16: X rounded to bfloat16 once,
 * tensor cores; NMF_PREC_FP32: float32 accuracy, on the tensor cores with X
 * and the operands split into three bfloat16 parts each (widths nu <= 32),
 * else float32 CUDA cores.
 */
nmf_status_t nmf_compress(nmf_stream_t stream, int n, int m, int nu, int q, nmf_prec_t prec,
                          const float* X, const float* omega_L, const float* omega_R, uint64_t seed,
                          float* L, float* R, float* XL, float* XR, void* workspace,
                          size_t workspace_bytes);

/*
 * Compression variants (the paper's Sec. 3 names the alternatives; Alg. 2 is
 * the one it studies):
 *  NMF_VARIANT_SUBSPACE      Alg. 2 as nmf_compress reads it (the default).
 *  NMF_VARIANT_SWAPPED       Alg. 2's output step with the tildes swapped, the
 *                            other dimensionally valid reading: L = Q~_R^(q),
 *                            R = Q~_L^(q), the half-step bases (q >= 1).
 *  NMF_VARIANT_SINGLE_CHAIN  one chain (omega_L only): L = Q_L^(q)^T and R the
 *                            next half-step basis orth(X^T Q_L^(q)); 2q + 3
 *                            passes of one product each.
 *  NMF_VARIANT_POWER         randomized power iteration ("structured random
 *                            projection"): Alg. 2's products with no
 *                            orthonormalisation between them (columns only
 *                            rescaled to unit norm) and one at the end.
 *  NMF_VARIANT_GAUSSIAN      plain random projection (Sec. 3 footnote):
 *                            L = Omega_R / sqrt(nu), R = Omega_L / sqrt(nu);
 *                            L, R are not orthonormal; one pass over X.
 * Same arguments, workspace and outputs as nmf_compress.
 */
typedef enum nmf_compress_variant {
  NMF_VARIANT_SUBSPACE = 0,
  NMF_VARIANT_SWAPPED = 1,
  NMF_VARIANT_SINGLE_CHAIN = 2,
  NMF_VARIANT_POWER = 3,
  NMF_VARIANT_GAUSSIAN = 4
} nmf_compress_variant_t;

nmf_status_t nmf_compress_variant(nmf_stream_t stream, int n, int m, int nu, int q, nmf_prec_t prec, int variant,
                                  const float* X, const float* omega_L, const float* omega_R, uint64_t seed,
                                  float* L, float* R, float* XL, float* XR, void* workspace,
                                  size_t workspace_bytes);

/*
 * Many independent compressions (Alg. 2 and X_L, X_R for each): the items run
 * on up to 8 library-owned streams forked from `stream` (an event fork and
 * join, so the call is stream-ordered and capturable); each item draws its
 * sketches from its own seed. Each item's X passes are planned for one
 * stream's share of the SMs (a quarter more than the device's SMs /
 * min(count, 8)), so that the streams' passes run side by side: an item
 * whose tile grid fits that share
 * gets nmf_compress_variant's plan and results bit for bit; a larger one
 * gets a split-K partition with fewer parts (the same products summed in
 * another order: equal to rounding).
 * The library creates its streams and events once per device and keeps
 * them; concurrent enqueues on one device are serialised by a mutex.
 * Workspace: min(count, 8) slots of the largest item's compression workspace.
 */
typedef struct nmf_compress_item {
  int n, m, nu, q;
  const float* X;   /* n x m, device */
  uint64_t seed;    /* sketch seed (streams 0 and 1 of nmf_gaussian_sketch) */
  float* L;         /* out: nu x n */
  float* R;         /* out: m x nu */
  float* XL;        /* out: nu x m */
  float* XR;        /* out: n x nu */
} nmf_compress_item_t;

size_t nmf_compress_batched_workspace_size(int count, const nmf_compress_item_t* items, nmf_prec_t prec);

nmf_status_t nmf_compress_batched(nmf_stream_t stream, int count, const nmf_compress_item_t* items, nmf_prec_t prec,
                                  int variant, void* workspace, size_t workspace_bytes);

/* ------------------------------------------------------------------------ */
/* NeNMF solve: plain (eq. 2-3) or compressed (Alg. 1)                        */
/* ------------------------------------------------------------------------ */
typedef enum nenmf_mode { NENMF_PLAIN = 0, NENMF_COMPRESSED = 1 } nenmf_mode_t;
typedef enum nenmf_tol_mode { NENMF_TOL_REL = 0, NENMF_TOL_ABS = 1 } nenmf_tol_mode_t;

typedef struct nenmf_problem {
  int mode;          /* nenmf_mode_t */
  int n, m, p, nu;   /* nu is ignored in plain mode */
  int prec;          /* plain mode: nmf_prec_t of the two X products per outer iteration */
  const float* X;    /* plain mode: n x m; ignored in compressed mode */
  const float* L;    /* compressed: nu x n */
  const float* R;    /* compressed: m x nu */
  const float* XL;   /* compressed: nu x m */
  const float* XR;   /* compressed: n x nu */
} nenmf_problem_t;

typedef struct nenmf_params {
  int max_outer;       /* outer iterations T (>= 0) */
  int max_inner;       /* Max_iter of the inner loop, per factor (>= 1) */
  int min_inner;       /* the stop test is not applied before this many iterations (>= 1) */
  int tol_mode;        /* nenmf_tol_mode_t */
  double tol;          /* <= 0 disables the projected-gradient stop test */
  float* record_G;     /* optional device [max_outer][n][p]: G after each outer iteration */
  float* record_F;     /* optional device [max_outer][p][m]: F after each outer iteration */
  long long* record_time_ns; /* optional device [max_outer + 1]: %globaltimer at the start and after each outer iteration */
  int restart;         /* 1: adaptive restart of the inner loop (per vector, when its objective
                          1/2 y^T H y - b^T y rises by more than 1e-5 of sum |y| (|grad| + |b|),
                          that extrapolation uses beta_0 = 0 and the vector's weights start
                          again from beta_1); 0: off */
} nenmf_params_t;

typedef struct nenmf_stats {
  int status;             /* device-detected nmf_status_t */
  int outer_done;         /* outer iterations completed */
  int last_inner[2];      /* inner iterations of the last G and F solves */
  long long total_inner[2]; /* inner iterations summed over the run (G, F) */
  double eps;             /* absolute stop threshold used (0 when disabled) */
  double pg_norm[2];      /* ||P grad||_F of the last G and F solves at their returned iterates */
  double lipschitz[2];    /* L_c of the last G and F solves */
} nenmf_stats_t;

size_t nenmf_solve_workspace_size(const nenmf_problem_t* problem);

/*
 * Runs max_outer outer iterations from (G, F), updating both in place.
 * The inner loop (Sec. 2): Y_0 = current factor, alpha_0 = 1; per k:
 * F_k = max(0, Y_k - (H Y_k - B) / L_c), Y_{k+1} = F_k + beta_k (F_k - F_{k-1}),
 * beta_k = (alpha_k - 1) / alpha_{k+1}, with L_c = lambda_max(H) and the
 * projected-gradient test ||P grad(F_k)||_F <= eps from min_inner on
 * (eps = tol * initial joint projected-gradient norm for NENMF_TOL_REL).
 * The returned factor is the projected iterate F_k.
 *  problem  host pointer; its matrix pointers are device memory.
 *  params   host pointer.
 *  stats    device pointer to one nenmf_stats_t (may be NULL).
 * Compressed mode runs all outer iterations in one persistent cooperative
 * launch when its CTAs (one per 128 columns of the larger side) fit on the
 * device at once and their shares of the p x nu products stay small
 * (ceil(max(n, m) / 128) * p * nu <= 16384); otherwise one launch per factor
 * update. The stop test of the per-update kernels needs all their CTAs
 * resident at once; a compressed problem with more vectors than that (about
 * 150 x 128 at p = 32) runs on the batched kernel instead (one problem, one
 * cluster; no snapshots there: NMF_ERR_UNSUPPORTED if record_* is set),
 * plain mode returns NMF_ERR_UNSUPPORTED. The workspace query covers all.
 */
nmf_status_t nenmf_solve(nmf_stream_t stream, const nenmf_problem_t* problem, float* G, float* F,
                         const nenmf_params_t* params, nenmf_stats_t* stats, void* workspace,
                         size_t workspace_bytes);

/* ------------------------------------------------------------------------ */
/* float64 twins (Alg. 2, Alg. 1, plain NeNMF, the inner loop of Sec. 2)     */
/* ------------------------------------------------------------------------ */
/*
 * The same computations as nmf_compress and nenmf_solve, every step in
 * float64 on the GPU, for parity at tight tolerances on small problems. They
 * are not a fast path (float64 runs at 1/64 of the float32 rate on this GPU):
 * products are one-output-per-thread loops, the small factorisations run in
 * one thread, each inner solve in one CTA. Results are deterministic.
 */
typedef struct nenmf_problem_f64 {
  int mode;          /* nenmf_mode_t */
  int n, m, p, nu;   /* 1 <= p <= min(32, n, m); compressed: p <= nu <= min(NMF_MAX_SKETCH, n, m) */
  const double* X;   /* plain mode: n x m; ignored in compressed mode */
  const double* L;   /* compressed: nu x n */
  const double* R;   /* compressed: m x nu */
  const double* XL;  /* compressed: nu x m */
  const double* XR;  /* compressed: n x nu */
} nenmf_problem_f64_t;

size_t nmf_compress_f64_workspace_size(int n, int m, int nu);

/*
 * Alg. 2 with q power steps and X_L = L X, X_R = X R, in float64. Layouts,
 * sketches and outputs as nmf_compress (omega_L m x nu, omega_R nu x n, both
 * device or both NULL: NULL draws the float32 sketches of nmf_gaussian_sketch
 * from `seed`, streams 0 and 1, and widens them). Each orthonormalisation is
 * CholeskyQR in three float64 passes, the first shifted (S + 1e-14 tr(S) I)
 * when a pivot is below 1e-24 of the largest diagonal entry: the Q of the QR
 * with a positive diagonal for a well-conditioned basis.
 * Errors: NMF_ERR_INVALID_ARG (sizes: 1 <= nu <= min(NMF_MAX_SKETCH, n, m),
 * 0 <= q <= 64; null outputs; one sketch NULL and the other not),
 * NMF_ERR_WORKSPACE; device: NMF_ERR_NOT_SPD, NMF_ERR_NONFINITE.
 */
nmf_status_t nmf_compress_f64(nmf_stream_t stream, int n, int m, int nu, int q, const double* X,
                              const double* omega_L, const double* omega_R, uint64_t seed, double* L, double* R,
                              double* XL, double* XR, void* workspace, size_t workspace_bytes);

size_t nenmf_solve_f64_workspace_size(const nenmf_problem_f64_t* problem);

/*
 * nenmf_solve in float64 (both modes): max_outer outer iterations from
 * (G, F) (device, n x p and p x m, updated in place), the inner loop, stop
 * test, eps rule and adaptive restart of nenmf_solve; L_c = lambda_max(H) by
 * cyclic Jacobi. record_G, record_F and record_time_ns must be NULL
 * (NMF_ERR_UNSUPPORTED otherwise). stats as nenmf_solve (device, may be NULL).
 */
nmf_status_t nenmf_solve_f64(nmf_stream_t stream, const nenmf_problem_f64_t* problem, double* G, double* F,
                             const nenmf_params_t* params, nenmf_stats_t* stats, void* workspace,
                             size_t workspace_bytes);

size_t nenmf_backward_f64_workspace_size(const nenmf_problem_f64_t* problem, const nenmf_params_t* params);

/*
 * nenmf_backward in float64 (compressed mode; NMF_ERR_UNSUPPORTED in plain
 * mode): the cotangents of X_L, X_R, G0, F0 (and optionally of X through
 * X_L = L X, X_R = X R: dX = L^T dXL + dXR R^T, n x m) given those of the
 * returned G_T (n x p) and F_T (p x m), for max_outer T outer iterations of
 * exactly max_inner K inner iterations (tol <= 0, restart 0, T <= 4096,
 * K <= 1024; NMF_ERR_INVALID_ARG otherwise). The forward is recomputed from
 * (G0, F0), so no snapshots are passed. Readings as nenmf_backward: the
 * projection's derivative 1[z > 0], d lambda_max = v v^T for the unit top
 * eigenvector v (cyclic Jacobi).
 */
nmf_status_t nenmf_backward_f64(nmf_stream_t stream, const nenmf_problem_f64_t* problem,
                                const nenmf_params_t* params, const double* G0, const double* F0,
                                const double* dG_T, const double* dF_T, double* dXL, double* dXR, double* dG0,
                                double* dF0, double* dX, void* workspace, size_t workspace_bytes);

/* ------------------------------------------------------------------------ */
/* Many independent compressed problems of different sizes (Alg. 1)          */
/* ------------------------------------------------------------------------ */
/*
 * The same method as nenmf_solve in compressed mode, applied to `count`
 * unrelated problems (each its own n, m, p, nu and L, R, X_L, X_R from
 * nmf_compress) in one persistent launch: thread-block clusters of
 * `cluster` CTAs each take a list of problems (assigned on the host,
 * longest first, by an estimate of each problem's device time) and run all
 * of a problem's outer iterations before the next. Results per problem are
 * those of nenmf_solve with the same arguments up to float32 summation order.
 */
typedef struct nenmf_batch_config {
  int cluster; /* CTAs per problem: 0 = chosen by the planner, else 1, 2, 4 or 8 */
  int threads; /* threads per CTA: 0 = 256, else 128 or 256 (128: two CTAs per SM,
                  so twice the clusters in flight, each with half the lanes) */
} nenmf_batch_config_t;

/* Workspace bytes for nenmf_solve_batched with these arguments (0 on invalid
 * arguments). problems, params and config (may be NULL) are host pointers. */
size_t nenmf_solve_batched_workspace_size(int count, const nenmf_problem_t* problems,
                                          const nenmf_params_t* params, const nenmf_batch_config_t* config);

/* The plan nenmf_solve_batched would use: chosen->cluster, chosen->threads and
 * the number of clusters launched. Host-only; needs the device current for
 * occupancy. */
nmf_status_t nenmf_batch_plan_info(int count, const nenmf_problem_t* problems, const nenmf_params_t* params,
                                   const nenmf_batch_config_t* config, nenmf_batch_config_t* chosen,
                                   int* clusters);

/*
 *  problems  host array of `count` problems, all NENMF_COMPRESSED (plain
 *            mode: NMF_ERR_UNSUPPORTED); 1 <= p <= nu <= NMF_MAX_SKETCH.
 *  G, F      host arrays of `count` device pointers: G[i] n_i x p_i and
 *            F[i] p_i x m_i, row-major, updated in place.
 *  params    host pointer, shared by all problems; record_* must be NULL.
 *            tol_mode NENMF_TOL_REL takes eps per problem from that
 *            problem's initial projected gradient.
 *  stats     device array of `count` entries (may be NULL).
 * Stream-ordered; capturable in a CUDA graph (descriptors travel as kernel
 * parameters). count == 0 returns NMF_OK without launching.
 */
nmf_status_t nenmf_solve_batched(nmf_stream_t stream, int count, const nenmf_problem_t* problems,
                                 float* const* G, float* const* F, const nenmf_params_t* params,
                                 const nenmf_batch_config_t* config, nenmf_stats_t* stats, void* workspace,
                                 size_t workspace_bytes);

/*
 * Measured choice of the cluster size (CTAs per problem) and of the threads
 * per CTA for nenmf_solve_batched: each candidate (cluster 1, 2, 4, 8) x
 * (threads 256, 128) with a valid plan runs trial_outer outer iterations of
 * these problems (params otherwise as given; record_* ignored) from scratch
 * copies of G and F, once untimed and once timed with CUDA events;
 * best->cluster and best->threads receive the fastest. trial_ms (host, 8
 * floats, may be NULL) receives each candidate's time in ms, index
 * 2 * (cluster index) + (threads == 128), -1 where a candidate has no valid
 * plan. The caller's G and F are not modified.
 * Synchronous: returns after the trials ran (it reads their times).
 * Errors: as nenmf_solve_batched; NMF_ERR_INVALID_ARG if trial_outer < 1,
 * count < 1 or best is NULL; the first device error of a trial.
 */
size_t nenmf_batch_autotune_workspace_size(int count, const nenmf_problem_t* problems,
                                           const nenmf_params_t* params, int trial_outer);
nmf_status_t nenmf_batch_autotune(nmf_stream_t stream, int count, const nenmf_problem_t* problems,
                                  float* const* G, float* const* F, const nenmf_params_t* params, int trial_outer,
                                  nenmf_batch_config_t* best, float* trial_ms, void* workspace,
                                  size_t workspace_bytes);

/* ------------------------------------------------------------------------ */
/* Reverse-mode derivative of the compressed solve (Alg. 1, Sec. 2)          */
/* ------------------------------------------------------------------------ */
/*
 * The paper defines no derivative; this differentiates the map
 * (X_L, X_R, G0, F0) -> (G_T, F_T) of nenmf_solve in compressed mode with
 * the stop test off (every inner solve runs max_inner iterations), holding
 * L and R fixed. Conventions: max(0, z) has derivative 1[z > 0];
 * L_c = lambda_max(H) has derivative v v^T (v its unit eigenvector). The
 * forward's inner iterations are recomputed from the per-outer snapshots.
 *
 * Workspace bytes for nenmf_backward (0 on invalid arguments).
 */
size_t nenmf_backward_workspace_size(const nenmf_problem_t* problem, const nenmf_params_t* params);

/*
 *  problem             host pointer, NENMF_COMPRESSED (else NMF_ERR_UNSUPPORTED).
 *  params              host pointer: max_outer T and max_inner K of the forward;
 *                      tol must be <= 0 (NMF_ERR_INVALID_ARG otherwise).
 *  G0, F0              the forward's initial factors (n x p, p x m).
 *  record_G, record_F  the forward's snapshots [T][n][p] and [T][p][m]
 *                      (nenmf_solve with params->record_G / record_F set).
 *  dG_T, dF_T          cotangents of the returned G_T and F_T.
 *  dXL, dXR            out: cotangents of X_L (nu x m) and X_R (n x nu).
 *  dG0, dF0            out: cotangents of G0 and F0.
 *  dX                  optional out (may be NULL): n x m, L^T dXL + dXR R^T,
 *                      the cotangent of X through X_L = L X and X_R = X R.
 * All device pointers, row-major, distinct buffers; stream-ordered.
 */
nmf_status_t nenmf_backward(nmf_stream_t stream, const nenmf_problem_t* problem, const nenmf_params_t* params,
                            const float* G0, const float* F0, const float* record_G, const float* record_F,
                            const float* dG_T, const float* dF_T, float* dXL, float* dXR, float* dG0,
                            float* dF0, float* dX, void* workspace, size_t workspace_bytes);

/* ------------------------------------------------------------------------ */
/* One pass over X, two products (the building block of Alg. 2)              */
/* ------------------------------------------------------------------------ */
size_t nmf_dual_product_workspace_size(int n, int m, int k, nmf_prec_t prec);

/*
 * YN = X A (n x k) and YT = X^T B (m x k) from a single read of X, the two
 * products every pass of Alg. 2 needs (X Q~_L and X^T Q_L^T for one chain,
 * the transposed pair for the other; Alg. 1's X R and L X likewise).
 *  A   m x k (or NULL together with YN), B  n x k (or NULL together with YT);
 *  1 <= k <= NMF_MAX_SKETCH. Partial sums are combined in a fixed order, so
 *  results are bitwise reproducible. prec as for nmf_compress (NMF_PREC_BF16
 *  rounds X, A and B to bfloat16 and accumulates in float32).
 */
nmf_status_t nmf_dual_product(nmf_stream_t stream, int n, int m, int k, nmf_prec_t prec, const float* X,
                              const float* A, const float* B, float* YN, float* YT, void* workspace,
                              size_t workspace_bytes);

size_t nmf_project_workspace_size(int n, int m, int nu, nmf_prec_t prec);

/*
 * The compression step of Alg. 1 for given bases: X_L = L X (nu x m) and
 * X_R = X R (n x nu) from one pass over X (as nmf_compress ends). L is
 * nu x n, R is m x nu (device, row-major); prec as nmf_compress. Used where
 * the bases stay fixed while X changes (the differentiated map of
 * nenmf_backward). Errors: NMF_ERR_INVALID_ARG (1 <= nu <= min(NMF_MAX_SKETCH,
 * n, m), null pointers), NMF_ERR_WORKSPACE.
 */
nmf_status_t nmf_project(nmf_stream_t stream, int n, int m, int nu, nmf_prec_t prec, const float* X, const float* L,
                         const float* R, float* XL, float* XR, void* workspace, size_t workspace_bytes);

/*
 * Selects kernels, for cross-checks between paths (flags, OR-ed; 0 is the
 * default, the fastest path):
 *  NMF_PATH_XPASS_CUDA_CORES  NMF_PREC_BF16 X passes on float32 CUDA cores
 *                             instead of tcgen05 tensor cores (same input
 *                             rounding, different summation order);
 *  NMF_PATH_SOLVE_PER_UPDATE  nenmf_solve in compressed mode as one launch
 *                             per factor update instead of one persistent
 *                             launch for all outer iterations (same
 *                             arithmetic in the same order: identical results).
 * Process-wide; not thread-safe against concurrent calls. Workspace sizes
 * depend on it: query after setting.
 */
enum { NMF_PATH_XPASS_CUDA_CORES = 1, NMF_PATH_SOLVE_PER_UPDATE = 2 };
void nmf_set_kernel_path(int flags);

/*
 * Number of kernel launches this library has enqueued in the process so far
 * (all calls, all threads; memsets and copies are not counted). Benchmarks
 * take the difference around a timed region.
 */
long long nmf_kernel_launches(void);

/* ------------------------------------------------------------------------ */
/* Failure-path testing                                                       */
/* ------------------------------------------------------------------------ */
/*
 * Makes later kernels fail one of their bounded device waits on purpose, so
 * that a test can exercise the NMF_ERR_DEVICE_TIMEOUT path (status word set,
 * every CTA leaving its waits, the call's later kernels turning into no-ops)
 * without hanging or faulting the GPU. Not for production use.
 *  NMF_FAULT_NONE        normal operation (the default).
 *  NMF_FAULT_STOP_TEST   in the solve kernels, CTA 0 never publishes its
 *                        stop-test partials, so every CTA that needs the
 *                        global sum waits until the limit runs out.
 *  NMF_FAULT_XPASS_COPY  in the tensor-core X pass, CTA 0 arms its first
 *                        pipeline stage but issues none of its copies, so the
 *                        MMA issuer's wait for that stage runs out.
 * wait_limit_ns > 0 replaces the 2-second limit of every bounded device wait
 * (stop test, grid barrier, pipeline stages); 0 restores it.
 * Process-wide; a kernel takes the setting when it is enqueued; not
 * thread-safe against concurrent calls. Errors: NMF_ERR_INVALID_ARG for an
 * unknown fault or a negative limit.
 */
typedef enum nmf_fault { NMF_FAULT_NONE = 0, NMF_FAULT_STOP_TEST = 1, NMF_FAULT_XPASS_COPY = 2 } nmf_fault_t;

nmf_status_t nmf_inject_fault(int fault, long long wait_limit_ns);

/* ------------------------------------------------------------------------ */
/* Relative reconstruction error, eq. (4)                                     */
/* ------------------------------------------------------------------------ */
size_t nmf_rre_workspace_size(int n, int m, int p);

/*
 * out (device, 2 doubles) <- { ||X - G F||_F^2, ||X||_F^2 } in one pass over X,
 * products in float32 and sums in float64 (fixed reduction order). Any n >= 1
 * is accepted: beyond 64 x 65535 rows each block walks several row blocks.
 */
nmf_status_t nmf_rre(nmf_stream_t stream, int n, int m, int p, const float* X, const float* G,
                     const float* F, double* out, void* workspace, size_t workspace_bytes);

/* ------------------------------------------------------------------------ */
/* Relative reconstruction error without a caller workspace                   */
/* ------------------------------------------------------------------------ */
/*
 * The paper has no counterpart to this call; it exists for callers that
 * cannot allocate device memory. Examples: a hook that evaluates the fit
 * between solver calls inside a framework that owns all device memory
 * through its own pool and hands out no buffers to plug-ins, or a
 * monitoring loop that must not call cudaMalloc because cudaMalloc can
 * synchronise the device and stall the work it watches. Such callers still
 * pass X, G, F and `out`, but no workspace.
 *
 * Same result as nmf_rre (same kernels, same fixed summation order). The
 * per-block partial sums live in one fixed array inside the library
 * (2 x NMF_RRE_STATIC_MAX_PARTS doubles, 1 MiB), which every GPU that loads
 * the library keeps until the process exits.
 *  - The first call on a device looks up that array's device address
 *    (cudaGetSymbolAddress) with the device current; make that first call
 *    before starting any stream capture. A cudaDeviceReset replaces the
 *    device's context and the array with it: the next call notices the new
 *    context and looks the address up again, so make that call before any
 *    capture too.
 *  - All calls share the array: calls that can overlap on the GPU (other
 *    streams, other host threads) race and must be serialised by the caller.
 *  - Every partial is written before it is read, so nothing has to start at
 *    zero; the array keeps the last call's contents.
 *  - Sizes needing more than NMF_RRE_STATIC_MAX_PARTS blocks, where blocks =
 *    ceil(m / 256) * min(ceil(n / 64), 65535), return NMF_ERR_WORKSPACE
 *    before anything is enqueued.
 */
#define NMF_RRE_STATIC_MAX_PARTS 65536
nmf_status_t nmf_rre_static(nmf_stream_t stream, int n, int m, int p, const float* X, const float* G,
                            const float* F, double* out);

/* ------------------------------------------------------------------------ */
/* Row-sharded runs (X split by row blocks across GPUs)                      */
/* ------------------------------------------------------------------------ */
/*
 * With X split by row blocks, every product X A of a pass is local, every
 * X^T B is a partial sum to all-reduce, and the orthonormal bases of Alg. 2
 * (CholeskyQR) need their Gram matrix summed over the row blocks. In the
 * outer loop of Alg. 1 the rows of G are local (X_R = X R has the rows of X),
 * G_L = L G is a partial sum, and the stop test of the inner loop (Sec. 2)
 * sums ||P grad||^2 over all row blocks. The three calls below are the
 * per-GPU steps between those collectives; the Python module
 * paper_1812_04315_gb300.sharded drives them.
 *
 * nmf_gram: S = Y^T Y (nu x nu, float64, both triangles written) of this
 * GPU's N x nu rows Y (device, row-major), summed in float-float (products
 * exact, ~48-bit sums) in a fixed order, so that the partial Grams of all
 * row blocks can be added by an all-reduce. 1 <= nu <= NMF_MAX_SKETCH.
 */
size_t nmf_gram_workspace_size(int N, int nu);
nmf_status_t nmf_gram(nmf_stream_t stream, int N, int nu, const float* Y, double* S, void* workspace,
                      size_t workspace_bytes);

/*
 * nmf_orth_apply: one CholeskyQR pass over this GPU's rows: Q = Y R^{-1}
 * (N x nu, device, row-major; may alias Y) with R^T R = S the given
 * (summed) Gram, S factorised in float-float; when a pivot is not safely
 * positive, S + 1e-10 tr(S) I is factorised instead (shifted CholeskyQR), and
 * a second pass is then still needed. Every row block applies the same R.
 * A Gram whose diagonal is not positive sets NMF_ERR_NOT_SPD in the
 * workspace status.
 */
size_t nmf_orth_apply_workspace_size(int N, int nu);
nmf_status_t nmf_orth_apply(nmf_stream_t stream, int N, int nu, const float* Y, const double* S, float* Q,
                            void* workspace, size_t workspace_bytes);

/*
 * nenmf_nnls_block: iterations k0 .. k0 + kb - 1 of the Nesterov inner loop
 * of Sec. 2 on the N columns of a p x N unknown (this GPU's columns),
 * min_{F >= 0} 1/2 tr(F^T H F) - tr(B^T F):
 *   f_k = max(0, y_k - (H y_k - b) / L_c),  y_{k+1} = f_k + beta_k (f_k - f_{k-1}),
 * L_c = lambda_max(H) (computed here from H; written to *Lc), beta_k from the
 * alpha recurrence (beta_0 = 0), as nenmf_solve without restart.
 *  H       p x p, symmetric (device, row-major).
 *  B       p x N (device, row-major).
 *  Y       p x N in/out: y_{k0} on entry (y_0 = F^t), y_{k0+kb} on return.
 *  Fprev   p x N in/out: f_{k0-1} (any value when k0 = 0), f_{k0+kb-1} on return.
 *  keep    [kb][p][N] out: f_k of every iteration of the block.
 *  pg2     [max(kb, 1)] out (device, float64): this GPU's share of
 *          ||P grad(f_k)||_F^2, P grad = grad where f > 0, min(0, grad) where
 *          f = 0 (summed over its columns in a fixed order).
 * kb = 0 evaluates pg2[0] at Y (no step); with L_c = 0 no step is taken
 * either and every pg2 entry holds the value at Y. The caller sums pg2 over
 * the row blocks and stops at the first k (k + 1 >= min_inner) whose total
 * is <= eps^2, taking keep[k - k0]. 1 <= p <= NMF_MAX_RANK,
 * 0 <= k0, k0 + kb <= max_inner.
 */
size_t nenmf_nnls_block_workspace_size(int N, int p, int kb, int max_inner);
nmf_status_t nenmf_nnls_block(nmf_stream_t stream, int N, int p, const float* H, const float* B, float* Y,
                              float* Fprev, int k0, int kb, int max_inner, float* keep, double* pg2, double* Lc,
                              void* workspace, size_t workspace_bytes);

#ifdef __cplusplus
}
#endif

#endif /* NMF_H */
