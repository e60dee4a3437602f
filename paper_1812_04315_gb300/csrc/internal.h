// internal.h -- launchers shared between libnmf translation units (host side).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "common.cuh"

// Returns NMF_ERR_CUDA from the enclosing entry point when a runtime call fails.
#define NMF_CU(call)                                   \
  do {                                                 \
    cudaError_t e_ = (call);                           \
    if (e_ != cudaSuccess) return NMF_ERR_CUDA;        \
  } while (0)

namespace nmf {

// ---------------------------------------------------------------------------
// Workspace carving: a bump allocator over the caller's workspace. With a
// null base it only measures (used by the *_workspace_size queries).
// ---------------------------------------------------------------------------
struct Carver {
  char* base;
  size_t off = 0;
  explicit Carver(void* b) : base(static_cast<char*>(b)) {}
  template <typename T>
  T* take(size_t count) {
    off = round_up_sz(off, 256);
    T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
    off += count * sizeof(T);
    return p;
  }
  size_t size() const { return round_up_sz(off, 256); }
};

// ---------------------------------------------------------------------------
// X passes: Y_N = X * A (n x nu) and Y_T = X^T * B (m x nu) in one read of X,
// as per-region partial sums (deterministic split-K).
// Operands are stored transposed and zero padded: opA is NV x lda holding
// A^T (row c = column c of A), opB is NV x ldb holding B^T.
// Partials: partN[S_c][n][NV], partT[S_r][m][NV] (float32).
// ---------------------------------------------------------------------------
struct XPassPlan {
  int tile_r, tile_c;   // tile size in rows / columns of X
  int tiles_r, tiles_c;
  int S_r, S_c;         // region grid: S_r row groups x S_c column groups
  int NV;               // padded operand / partial width
  int ctas;
  int tiled;            // bfloat16 X held tile by tile (the tensor-core path's layout)
  int parts;            // tiled: 1 (bfloat16 X, bfloat16 operands) or 3 (float32 X and
                        // operands as three bfloat16 parts each, OP_BF16X3)
};

struct XPassArgs {
  int n, m;
  const void* X;        // float (prec FP32) or __nv_bfloat16 (prec BF16)
  int ldx;              // elements
  const void* opA;      // NV x lda, same element type as X
  int lda;
  const void* opB;      // NV x ldb
  int ldb;
  float* partN;         // may be null when !doN
  float* partT;         // may be null when !doT
  int nu;               // meaningful columns (<= NV)
  bool doN, doT;
  Control* ctrl;
};

// Plans (tile sizes, region grid) for a pass at the given width. A float32
// pass runs on the tensor cores as three bfloat16 parts when split_ok and the
// width allows it (NV <= kSplitMaxNV), else on CUDA cores.
constexpr int kSplitMaxNV = 32;
XPassPlan xpass_plan(int n, int m, int nu, nmf_prec_t prec, int num_sms, bool split_ok = true);
// Operand format and bytes of one operand buffer (NV rows of ld elements per part).
inline int op_format(const XPassPlan& pl, nmf_prec_t prec) {
  return pl.tiled && pl.parts == 3 ? OP_BF16X3 : prec == NMF_PREC_BF16 ? OP_BF16 : OP_F32;
}
inline size_t op_bytes(const XPassPlan& pl, nmf_prec_t prec, int ld) {
  const int f = op_format(pl, prec);
  return (size_t)pl.NV * ld * (f == OP_F32 ? 4 : f == OP_BF16 ? 2 : 6);
}
// Whether the pass reads a converted copy of X (bfloat16 rows, or tiles).
inline bool x_converted(const XPassPlan& pl, nmf_prec_t prec) { return pl.tiled || prec == NMF_PREC_BF16; }
cudaError_t xpass_launch(const XPassPlan& plan, const XPassArgs& a, nmf_prec_t prec, cudaStream_t s);
// bfloat16 copy of a float32 X in the layout the plan's kernel reads:
// row-major with ldxb columns, or (plan.tiled) tile by tile.
size_t xb_elems(const XPassPlan& plan, int n, int ldxb);
cudaError_t xb_convert(const XPassPlan& plan, const float* X, int n, int m, __nv_bfloat16* Xb, int ldxb,
                       Control* ctrl, cudaStream_t s);
cudaError_t xpass_tc_convert(const XPassPlan& plan, const float* X, int n, int m, void* Xt, Control* ctrl,
                             cudaStream_t s);
// Float32 CUDA-core path for bfloat16 X (same rounding of inputs as the
// tensor-core path, different summation order); used as an independent check.
cudaError_t xpass_simt_launch(const XPassPlan& plan, const XPassArgs& a, bool bf16, cudaStream_t s);
XPassPlan xpass_simt_plan(int n, int m, int nu, int num_sms);
// Tensor-core (tcgen05) path for bfloat16 X.
XPassPlan xpass_tc_plan(int n, int m, int nu, int num_sms, int parts);
cudaError_t xpass_tc_launch(const XPassPlan& plan, const XPassArgs& a, cudaStream_t s);
bool xpass_tc_available();

// ---------------------------------------------------------------------------
// Row kernels of the orthonormalisation (CholeskyQR2, float-float Gram and
// Cholesky). A "job" is one tall matrix of N rows and nu columns.
// ---------------------------------------------------------------------------
constexpr int kOrthRows = 256;  // rows per CTA in the row kernels (one per thread)

struct RowJob {
  // source: X pass partials (reduce step) or a dense N x nu matrix whose Gram
  // partials are given (apply step: factor the Gram, q R = y row by row)
  const float* part;    // S x N x ldp (reduce step)
  int S, ldp;
  const float* src;     // N x nu (apply step)
  const float2* gram_in;  // apply step: [gram_parts][nu*(nu+1)/2] float-float partials of src^T src
  int gram_parts;
  int N, nu;
  // outputs (each optional)
  float* Y;             // N x nu row-major (may alias src: rows are read before written)
  float* Yt;            // nu x N row-major (transpose)
  void* op;             // NV x ldop transposed operand (OpFormat op_fmt; OP_BF16X3: parts NV * ldop apart)
  int ldop, op_fmt;
  size_t op_part;       // elements between the parts of an OP_BF16X3 operand
  float2* gram_part;    // [ctas][nu*(nu+1)/2] float-float partial Gram of the output rows
  int gram_always;      // form gram_part unconditionally
  int gram_on_shift;    // form gram_part when *shift_flag (as read) or this factorisation shifted
  int* shift_flag;      // apply step: raised (by CTA 0) when the factorisation needed the shift
  const int* run_flag;  // optional: skip the job unless *run_flag != 0
  const int* skip_flag; // optional: skip the job when *skip_flag != 0
  int diag_only;        // apply step: R = diag(sqrt(S_cc)) (columns rescaled to unit norm, span kept)
  int gram_only;        // src given: no factorisation, src's rows kept as they are (Gram partial only)
  float skip_tol;       // apply step: keep src as it is when its Gram is within this of I (0: never)
  // apply step, one pass enough: when the factorisation did not shift and the
  // ratio of its largest to smallest pivot is below single_ratio, the rows
  // go to the final outputs below (not Y, Yt, op, no Gram partial) and
  // *single_flag is raised (so the next pass can skip); 0: never
  float single_ratio;
  int* single_flag;
  float* Y_final;
  float* Yt_final;
  void* op_final;
};

cudaError_t rows_launch(const RowJob* jobs, int njobs, Control* ctrl, cudaStream_t s);
inline int rows_ctas(int N) { return ceil_div(N, kOrthRows); }

// ---------------------------------------------------------------------------
// Nesterov inner solve (Sec. 2) over the columns of a p x N unknown.
// ---------------------------------------------------------------------------
enum BSource { B_FROM_ROWS = 0, B_FROM_COLS = 1, B_FROM_PARTIALS = 2 };
enum Epilogue { EPI_NONE = 0, EPI_W_ROWS = 1, EPI_W_COLS = 2, EPI_GRAM = 3 };
constexpr int kSolveThreads = 128;
constexpr int kSolveWarps = kSolveThreads / 32;
constexpr int kMaxStopCtas = 320;  // CTAs one stop test spans at most
constexpr int kMaxInnerIters = 4096;  // largest max_inner accepted

constexpr int kMaxReduceFloats = 16384;  // per-CTA shared-memory budget for reducing the predecessor's partials

// Group size of the epilogue partials: 1 (each CTA's partial is read by the
// next kernel directly) unless ctas * P floats exceed the reduce budget, in
// which case the last CTA of each group of `group` CTAs sums its group.
inline int partial_group_size(int ctas, int P) {
  const long total = (long)ctas * P;
  return total <= kMaxReduceFloats ? 1 : (int)((total + kMaxReduceFloats - 1) / kMaxReduceFloats);
}
__host__ __device__ inline int group_count(int ctas, int group) { return ceil_div(ctas, group); }
// Floats between consecutive per-CTA partials: P rounded up to a multiple of
// four, so every partial starts on a 16-byte boundary (bulk copies, float4).
__host__ __device__ inline int partial_stride(int P) { return (P + 3) & ~3; }

struct SolveArgs {
  int p, N, nu;
  float* Y;              // p x N, in/out (unchanged unless MODE_SOLVE)
  // B of the subproblem
  int bsrc;              // BSource
  const float* D;        // B_FROM_ROWS: N x nu; B_FROM_COLS: nu x N
  const float* Bpart;    // B_FROM_PARTIALS: [Bparts][N][Bld]
  int Bparts, Bld;
  // the predecessor's partials of W (compressed: p x nu) or H (plain: p x p)
  const float* part_in;  // [groups_in][partial_stride(P)]
  int groups_in;
  // iteration
  int max_inner, min_inner;
  bool stop_test;
  int restart;           // adaptive restart of the inner loop (per vector)
  int side;              // 0 = G, 1 = F (stats slot)
  double* pg2_init;      // MODE_EVAL: per-CTA ||P grad(Y0)||^2
  double* pg2_part;      // [ctas]: ||P grad||^2 of the returned iterate, per CTA
  unsigned long long* stop_slots;  // [max_inner][ctas]: tagged stop-test partials, one row per test (zeroed per call)
  int epoch;             // distinct for every solve launch of one call (tags of stop_slots)
  // epilogue: the next phase's W or Gram matrix, per CTA (and per group)
  int epi;               // Epilogue
  const float* E;        // EPI_W_ROWS: N x nu; EPI_W_COLS: nu x N
  float* part_out;       // [ctas][partial_stride(P)], padding zero
  int group;             // partial_group_size(ctas, partial_stride(P))
  float* group_out;      // [group_count(ctas, group)][partial_stride(P)] when group > 1
  unsigned int* tail_ctr;  // [group_count(ctas, group)], zero, left zero (group > 1)
  void* op_out;          // optional transposed operand NV x op_ld (float or bf16)
  int op_ld, op_bf16;
  float* record;         // optional snapshot: Y^T as N x p (G) or Y as p x N (F)
  int record_transposed;
  unsigned long long* time_out;  // optional: atomicMax of %globaltimer at exit
  nenmf_stats_t* stats;  // optional
  Control* ctrl;
};

enum SolveMode { MODE_EPI_ONLY = 0, MODE_EVAL = 1, MODE_SOLVE = 2 };
int solve_ctas(int N);
// MODE_EPI_ONLY: only the epilogue on Y as given; MODE_EVAL: the projected-
// gradient norm of Y0 into pg2_init, then the epilogue on Y0; MODE_SOLVE:
// the inner loop. `beta` holds beta_k for k < max_inner.
cudaError_t solve_launch_mode(const SolveArgs& a, const float* beta, int mode, cudaStream_t s);
cudaError_t beta_launch(float* beta, int K, cudaStream_t s);
// CTAs of the solve kernel that fit on the device at once (the stop test
// needs every CTA of a launch resident).
int solve_max_coresident(int p, int nu, int epi, int groups_in);
// Persistent compressed solve (all outer iterations in one cooperative
// launch; persist.cu). ok: the problem fits (every CTA resident at once,
// the shares small enough for every CTA to read them all).
struct PersistPlan {
  bool ok;
  int ctas, PM;
  int PL;  // rows of the inner loop's register arithmetic (<= PM; see persist.cu)
  size_t smem;
  bool keep_shared;  // pending stop-test iterates in shared memory (else in the workspace)
};
struct PersistLaunch {
  int n, m, p, nu;
  const float *L, *R, *XL, *XR;
  float *G, *F;
  int max_outer, max_inner, min_inner, restart;
  const float* beta;
  float *partG, *partF;
  double *pg2G, *pg2F, *initG, *initF;
  unsigned long long* slots;  // [kMaxInnerIters][ctas]
  unsigned int* bar;          // zero
  float* keep;                // persist_keep_floats(plan) floats
  float *record_G, *record_F;
  unsigned long long* times;
  double tol;
  int tol_mode;
  nenmf_stats_t* stats;
  Control* ctrl;
};
PersistPlan persist_plan(int n, int m, int p, int nu, bool test, bool restart);
// Workspace floats for the pending iterates when they do not fit in shared
// memory (0 when they do, or when the problem is not run persistently).
size_t persist_keep_floats(int n, int m, int p, int nu);
cudaError_t persist_launch(const PersistPlan& pl, const PersistLaunch& L, cudaStream_t s);

// Sums final per-CTA partials into the stats struct (one thread).
cudaError_t stats_launch(nenmf_stats_t* stats, const double* pg2_final_G, int ctasG,
                         const double* pg2_final_F, int ctasF, Control* ctrl, int outer, cudaStream_t s);
// eps2 = tol^2 * (sum of init partials) (REL) or tol^2 (ABS), or -1 when off.
cudaError_t eps_launch(Control* ctrl, const double* pg2_G, int ctasG, const double* pg2_F, int ctasF,
                       double tol, int tol_mode, nenmf_stats_t* stats, cudaStream_t s);

// ---------------------------------------------------------------------------
// Auxiliary kernels.
// ---------------------------------------------------------------------------
cudaError_t sketch_launch(int rows, int cols, uint64_t seed, uint32_t stream_id, float* out, cudaStream_t s);
// X (n x m float, ld m) -> Xb (n x ldb bfloat16), padding columns zero.
cudaError_t to_bf16_launch(const float* X, int n, int m, __nv_bfloat16* Xb, int ldb, Control* ctrl,
                           cudaStream_t s);
// out[c][r] = in[r][c] for an R x C float matrix; `out` has leading dim ldo and
// OpFormat fmt (OP_BF16X3: parts part_stride elements apart). Padding (rows
// >= C, cols >= R) is untouched.
cudaError_t transpose_launch(const float* in, int R, int C, void* out, int ldo, int fmt, Control* ctrl,
                             cudaStream_t s, size_t part_stride = 0);
// Copies a rows x cols float matrix into an operand (OpFormat fmt) with leading dim ldo.
cudaError_t copy_rows_launch(const float* in, int rows, int cols, void* out, int ldo, int fmt,
                             Control* ctrl, cudaStream_t s, size_t part_stride = 0);
cudaError_t timestamp_launch(unsigned long long* t, cudaStream_t s);
// out[i] = alpha * in[i] (may alias)
cudaError_t scale_launch(const float* in, float* out, long long count, float alpha, cudaStream_t s);
cudaError_t rre_launch(int n, int m, int p, const float* X, const float* G, const float* F, double* out,
                       double* part, int parts, cudaStream_t s);
int rre_parts(int n, int m);

int device_sm_count();
bool device_is_sm103();

// Host-side count of kernel launches enqueued by the library (all threads).
void count_launches(int k);

// Failure-path testing (nmf_inject_fault): the fault the next launches carry
// and the limit of every bounded device wait (2 s unless a test lowers it).
int injected_fault();
// Whether the compression kernels may be launched as programmatic dependents
// (on by default; a PdlOff object turns it off for this host thread while it lives).
bool pdl_allowed();
struct PdlOff {
  PdlOff();
  ~PdlOff();
};
unsigned long long wait_limit_ns();

// Raises a kernel's dynamic shared-memory limit to `bytes` once per device
// (cached: the attribute call is not repeated on the launch path).
cudaError_t allow_dynamic_smem(const void* kernel, int bytes);

}  // namespace nmf
