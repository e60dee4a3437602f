// capi.cu -- the extern "C" entry points of include/nmf.h: argument checks,
// workspace carving and the stream-ordered schedules of Alg. 2 (nmf_compress)
// and of Alg. 1 / plain NeNMF (nenmf_solve).
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <mutex>
#include <utility>
#include <vector>

#include "internal.h"

using namespace nmf;

namespace {


int g_force_simt = 0;     // nmf_set_kernel_path bit 0
int g_per_update = 0;     // nmf_set_kernel_path bit 1

int sm_count() {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 152;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) return 152;
  return sms;
}

bool ws_ok(const void* ws, size_t bytes, size_t need) {
  return ws != nullptr && (reinterpret_cast<uintptr_t>(ws) & 255u) == 0 && bytes >= need;
}

bool use_tc(nmf_prec_t prec) { return prec == NMF_PREC_BF16 && !g_force_simt && xpass_tc_available(); }
// float32 passes as three bfloat16 parts on the tensor cores (widths up to kSplitMaxNV)
bool use_split(nmf_prec_t prec, int nu) {
  return prec == NMF_PREC_FP32 && !g_force_simt && round_up(nu, 16) <= nmf::kSplitMaxNV && xpass_tc_available();
}

}  // namespace

namespace nmf {

static std::atomic<long long> g_launches{0};
void count_launches(int k) { g_launches.fetch_add(k, std::memory_order_relaxed); }

constexpr unsigned long long kDefaultWaitNs = 2000000000ull;  // 2 s
// Programmatic dependent launch of the compression kernels, per host thread.
static thread_local int t_pdl_off = 0;
bool pdl_allowed() { return t_pdl_off == 0; }
PdlOff::PdlOff() { ++t_pdl_off; }
PdlOff::~PdlOff() { --t_pdl_off; }

static std::atomic<int> g_fault{NMF_FAULT_NONE};
static std::atomic<unsigned long long> g_wait_ns{kDefaultWaitNs};
int injected_fault() { return g_fault.load(std::memory_order_relaxed); }
unsigned long long wait_limit_ns() { return g_wait_ns.load(std::memory_order_relaxed); }

cudaError_t allow_dynamic_smem(const void* kernel, int bytes) {
  static std::mutex mu;
  static std::vector<std::pair<std::pair<const void*, int>, int>> done;  // (kernel, device) -> bytes
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(mu);
  for (auto& d : done)
    if (d.first.first == kernel && d.first.second == dev) {
      if (d.second >= bytes) return cudaSuccess;
      e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
      if (e == cudaSuccess) d.second = bytes;
      return e;
    }
  e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess) done.push_back({{kernel, dev}, bytes});
  return e;
}

int device_sm_count() { return sm_count(); }

XPassPlan xpass_plan(int n, int m, int nu, nmf_prec_t prec, int num_sms, bool split_ok) {
  if (use_tc(prec)) return xpass_tc_plan(n, m, nu, num_sms, 1);
  if (split_ok && use_split(prec, nu)) return xpass_tc_plan(n, m, nu, num_sms, 3);
  return xpass_simt_plan(n, m, nu, num_sms);
}

cudaError_t xpass_launch(const XPassPlan& plan, const XPassArgs& a, nmf_prec_t prec, cudaStream_t s) {
  if (plan.tiled) return xpass_tc_launch(plan, a, s);
  return xpass_simt_launch(plan, a, prec == NMF_PREC_BF16, s);
}

size_t xb_elems(const XPassPlan& plan, int n, int ldxb) {
  return plan.tiled ? (size_t)plan.tiles_r * plan.tiles_c * plan.tile_r * plan.tile_c * plan.parts
                    : (size_t)n * ldxb;
}

cudaError_t xb_convert(const XPassPlan& plan, const float* X, int n, int m, __nv_bfloat16* Xb, int ldxb,
                       Control* ctrl, cudaStream_t s) {
  if (plan.tiled) return xpass_tc_convert(plan, X, n, m, Xb, ctrl, s);
  return to_bf16_launch(X, n, m, Xb, ldxb, ctrl, s);
}

}  // namespace nmf

namespace {

// The second CholeskyQR pass is skipped when the first pass's basis has a
// Gram matrix within this of I (every entry, float-float value).
constexpr float kSecondPassSkip = 1e-6f;
// One CholeskyQR pass is taken when the first factorisation did not shift and
// its pivots span less than this ratio: kappa(Y)^2 of about that size, so the
// float-float Gram leaves Q orthonormal to ~3e7 x 2^-48 ~ 1e-7, below the
// 1e-6 at which the second pass would keep Q anyway.
constexpr float kSinglePassPivotRatio = 3e7f;

// ----------------------------------------------------------------------------
// nmf_compress workspace
// ----------------------------------------------------------------------------
struct CompressWs {
  Control* ctrl;
  __nv_bfloat16* Xb;
  int ldxb;
  void* opA;   // NV x lda
  int lda;
  void* opB;   // NV x ldb
  int ldb;
  float* partN;
  float* partT;
  float* YN[2];
  float* YT[2];
  float2* gramN[2];  // ping-pong Gram partials of the N job
  float2* gramT[2];
  float* omega;
  XPassPlan plan;
  size_t bytes;
};

// SMs an X pass of the compression is planned for: all of them, or the
// share of one lane while a batched compression (or its workspace query)
// sets a budget on this host thread. A pass planned for fewer SMs leaves
// the others to the other lanes' passes, which then run side by side.
static thread_local int t_xpass_sms = 0;
struct XPassSmBudget {
  int prev;
  explicit XPassSmBudget(int sms) : prev(t_xpass_sms) { t_xpass_sms = sms; }
  ~XPassSmBudget() { t_xpass_sms = prev; }
};

CompressWs carve_compress(void* base, int n, int m, int nu, nmf_prec_t prec) {
  CompressWs w{};
  Carver cv(base);
  w.plan = xpass_plan(n, m, nu, prec, t_xpass_sms > 0 ? t_xpass_sms : sm_count());
  const int NV = w.plan.NV;
  w.ctrl = cv.take<Control>(1);
  if (x_converted(w.plan, prec)) {
    w.ldxb = round_up(m, 64);
    w.Xb = cv.take<__nv_bfloat16>(xb_elems(w.plan, n, w.ldxb));
  }
  w.lda = round_up(m, 128);
  w.ldb = round_up(n, 128);
  w.opA = cv.take<char>(op_bytes(w.plan, prec, w.lda));
  w.opB = cv.take<char>(op_bytes(w.plan, prec, w.ldb));
  w.partN = cv.take<float>((size_t)w.plan.S_c * n * NV);
  w.partT = cv.take<float>((size_t)w.plan.S_r * m * NV);
  for (int i = 0; i < 2; ++i) {
    w.YN[i] = cv.take<float>((size_t)n * nu);
    w.YT[i] = cv.take<float>((size_t)m * nu);
  }
  const int E = nu * (nu + 1) / 2;
  const int E2 = (E + 1) & ~1;  // Gram partials use an even float2 stride
  for (int i = 0; i < 2; ++i) {
    w.gramN[i] = cv.take<float2>((size_t)rows_ctas(n) * E2);
    w.gramT[i] = cv.take<float2>((size_t)rows_ctas(m) * E2);
  }
  w.omega = cv.take<float>((size_t)(n > m ? n : m) * nu);
  w.bytes = cv.size();
  return w;
}

// Which products of a pass a step works on (N: X A, n rows; T: X^T B, m rows).
struct Jobs {
  bool N, T;
};

// One CholeskyQR2 (+ conditional third pass) of the present products of a
// pass. Outputs: the next operands (N job -> opB, T job -> opA); with Lout
// and Rout set, L = Q_N^T and R = Q_T; with XLout set, the T product itself
// (before orthonormalisation) transposed into XLout.
nmf_status_t orthonormalize(const CompressWs& w, int n, int m, int nu, int ofmt, Jobs jb, float* Lout, float* Rout,
                            float* XLout, cudaStream_t s) {
  Control* ctrl = w.ctrl;
  const int NV = w.plan.NV;
  NMF_CU(cudaMemsetAsync(ctrl->flags, 0, 4 * sizeof(int), s));  // shift flags, single-pass flags
  RowJob r1[2] = {}, r2[2] = {}, r3[2] = {}, r4[2] = {};
  int k = 0;
  for (int t = 0; t < 2; ++t) {
    const bool isN = t == 0;
    if (isN ? !jb.N : !jb.T) continue;
    const int N = isN ? n : m;
    float* Y0 = isN ? w.YN[0] : w.YT[0];
    float* Y1 = isN ? w.YN[1] : w.YT[1];
    float2* g0 = isN ? w.gramN[0] : w.gramT[0];
    float2* g1 = isN ? w.gramN[1] : w.gramT[1];
    int* flag = &ctrl->flags[t];
    // reduce: Y = sum of the X pass partials, Gram 1
    RowJob& a = r1[k];
    a.part = isN ? w.partN : w.partT; a.S = isN ? w.plan.S_c : w.plan.S_r; a.ldp = NV; a.N = N; a.nu = nu;
    a.Y = Y0; a.gram_part = g0; a.gram_always = 1;
    if (!isN) a.Yt = XLout;
    // apply 1: factor Gram 1 (shift if needed), Q1 = Y R1^-1, Gram 2
    RowJob& b = r2[k];
    b.src = Y0; b.gram_in = g0; b.gram_parts = rows_ctas(N); b.N = N; b.nu = nu;
    b.Y = Y1; b.gram_part = g1; b.gram_always = 1; b.shift_flag = flag;
    // apply 2: Q2 = Q1 R2^-1 -> outputs; Gram 3 only if some factorisation shifted
    float* Q = isN ? Y0 : (Rout ? Rout : Y0);
    RowJob& c = r3[k];
    c.src = Y1; c.gram_in = g1; c.gram_parts = rows_ctas(N); c.N = N; c.nu = nu;
    c.Y = Q; c.op = isN ? w.opB : w.opA; c.ldop = isN ? w.ldb : w.lda; c.op_fmt = ofmt;
    c.op_part = (size_t)NV * c.ldop;
    if (isN) c.Yt = Lout;
    c.gram_part = g0; c.gram_on_shift = 1; c.shift_flag = flag;
    // the first pass's float-float Gram and factor leave Q1 orthonormal to
    // about float32 rounding unless Y is ill conditioned: then the second
    // pass would change Q1 by as little, and is skipped
    c.skip_tol = kSecondPassSkip;
    // apply 1 may find one pass enough: it then writes apply 2's outputs and
    // apply 2 (and the third pass, whose shift flag stays down) do nothing
    b.single_ratio = kSinglePassPivotRatio;
    b.single_flag = &ctrl->flags[2 + t];
    b.Y_final = c.Y; b.Yt_final = c.Yt; b.op_final = c.op; b.ldop = c.ldop; b.op_fmt = c.op_fmt;
    b.op_part = c.op_part;
    c.skip_flag = &ctrl->flags[2 + t];
    // apply 3, in place, only where a shift was taken
    RowJob& d = r4[k];
    d = c;
    d.src = Q; d.gram_in = g0; d.gram_part = nullptr; d.gram_on_shift = 0; d.shift_flag = nullptr; d.run_flag = flag;
    ++k;
  }
  NMF_CU(rows_launch(r1, k, ctrl, s));
  NMF_CU(rows_launch(r2, k, ctrl, s));
  NMF_CU(rows_launch(r3, k, ctrl, s));
  NMF_CU(rows_launch(r4, k, ctrl, s));
  return NMF_OK;
}

// The power-iteration variant's step between products: every column of the
// present products rescaled to unit norm (span unchanged, no
// orthonormalisation), written as the next operands.
nmf_status_t normalize_columns(const CompressWs& w, int n, int m, int nu, int ofmt, Jobs jb, cudaStream_t s) {
  Control* ctrl = w.ctrl;
  const int NV = w.plan.NV;
  RowJob r1[2] = {}, r2[2] = {};
  int k = 0;
  for (int t = 0; t < 2; ++t) {
    const bool isN = t == 0;
    if (isN ? !jb.N : !jb.T) continue;
    const int N = isN ? n : m;
    float* Y0 = isN ? w.YN[0] : w.YT[0];
    float2* g0 = isN ? w.gramN[0] : w.gramT[0];
    RowJob& a = r1[k];
    a.part = isN ? w.partN : w.partT; a.S = isN ? w.plan.S_c : w.plan.S_r; a.ldp = NV; a.N = N; a.nu = nu;
    a.Y = Y0; a.gram_part = g0; a.gram_always = 1;
    RowJob& b = r2[k];
    b.src = Y0; b.gram_in = g0; b.gram_parts = rows_ctas(N); b.N = N; b.nu = nu; b.diag_only = 1;
    b.op = isN ? w.opB : w.opA; b.ldop = isN ? w.ldb : w.lda; b.op_fmt = ofmt; b.op_part = (size_t)NV * b.ldop;
    ++k;
  }
  NMF_CU(rows_launch(r1, k, ctrl, s));
  NMF_CU(rows_launch(r2, k, ctrl, s));
  return NMF_OK;
}

}  // namespace

namespace {

// ----------------------------------------------------------------------------
// nenmf_solve workspace
// ----------------------------------------------------------------------------
constexpr int kMaxInner = kMaxInnerIters;

struct SolveWs {
  Control* ctrl;
  float* beta;
  float* Gt;       // p x n
  int ctasG, ctasF;
  int P;           // floats between partials: p * nu (compressed) or p * p (plain), padded to 4
  int groupG, groupF;  // partial group sizes (1: the successor reads per-CTA partials)
  float* partG;    // [ctasG][P]: the G side's share of the F update's W (or Gram)
  float* partF;    // [ctasF][P]: the F side's share of the G update's W (or Gram)
  float* groupOutG;  // [group_count(ctasG, groupG)][P] when groupG > 1
  float* groupOutF;
  unsigned int* ctr;  // group tickets: G side, then F side
  int nctr;
  double* pg2G;    // [ctasG]
  double* pg2F;
  unsigned long long* slots;  // stop-test words: G side [kMaxInnerIters][ctasG], then F side
  double* initG;   // [ctasG]
  double* initF;   // [ctasF]
  unsigned int* bar;  // persistent solve: grid barrier arrivals
  float* keep;     // persistent solve: pending stop-test iterates, when they are not in shared memory
  __nv_bfloat16* Xb;
  int ldxb;
  void* opF;       // NV x ldF: F as the N-product operand (A^T = F)
  int ldF;
  void* opG;       // NV x ldG: G^T as the T-product operand (B^T = G^T)
  int ldG;
  float* partN;
  float* partT;
  XPassPlan plan;
  size_t bytes;
};

SolveWs carve_solve(void* base, const nenmf_problem_t& pr) {
  SolveWs w{};
  Carver cv(base);
  const int n = pr.n, m = pr.m, p = pr.p;
  const bool plain = pr.mode == NENMF_PLAIN;
  const int nu = plain ? 0 : pr.nu;
  const int P = partial_stride(plain ? p * p : p * nu);
  w.P = P;
  w.ctrl = cv.take<Control>(1);
  w.beta = cv.take<float>(kMaxInner);
  w.Gt = cv.take<float>((size_t)p * n);
  w.ctasG = solve_ctas(n);
  w.ctasF = solve_ctas(m);
  w.groupG = partial_group_size(w.ctasG, P);
  w.groupF = partial_group_size(w.ctasF, P);
  w.partG = cv.take<float>((size_t)w.ctasG * P);
  w.partF = cv.take<float>((size_t)w.ctasF * P);
  w.groupOutG = cv.take<float>((size_t)group_count(w.ctasG, w.groupG) * P);
  w.groupOutF = cv.take<float>((size_t)group_count(w.ctasF, w.groupF) * P);
  w.nctr = group_count(w.ctasG, w.groupG) + group_count(w.ctasF, w.groupF);
  w.ctr = cv.take<unsigned int>(w.nctr);
  w.pg2G = cv.take<double>(w.ctasG);
  w.pg2F = cv.take<double>(w.ctasF);
  w.slots = cv.take<unsigned long long>((size_t)kMaxInnerIters * (w.ctasG + w.ctasF));
  w.initG = cv.take<double>(w.ctasG);
  w.initF = cv.take<double>(w.ctasF);
  w.bar = cv.take<unsigned int>(1);
  if (!plain) w.keep = cv.take<float>(persist_keep_floats(n, m, p, nu));
  if (plain) {
    const nmf_prec_t prec = (nmf_prec_t)pr.prec;
    // plain NeNMF's float32 passes stay on CUDA cores: the solve kernels write
    // their operands as float32 or one bfloat16 part
    w.plan = xpass_plan(n, m, p, prec, sm_count(), false);
    const size_t es = prec == NMF_PREC_BF16 ? 2 : 4;
    if (prec == NMF_PREC_BF16) {
      w.ldxb = round_up(m, 64);
      w.Xb = cv.take<__nv_bfloat16>(xb_elems(w.plan, n, w.ldxb));
    }
    w.ldF = round_up(m, 128);
    w.ldG = round_up(n, 128);
    w.opF = cv.take<char>((size_t)w.plan.NV * w.ldF * es);
    w.opG = cv.take<char>((size_t)w.plan.NV * w.ldG * es);
    w.partN = cv.take<float>((size_t)w.plan.S_c * n * w.plan.NV);
    w.partT = cv.take<float>((size_t)w.plan.S_r * m * w.plan.NV);
  }
  w.bytes = cv.size();
  return w;
}

bool problem_ok(const nenmf_problem_t* pr) {
  if (!pr) return false;
  if (pr->n < 1 || pr->m < 1 || pr->p < 1 || pr->p > NMF_MAX_RANK) return false;
  if (pr->mode == NENMF_PLAIN) {
    if (!pr->X) return false;
    if (pr->prec != NMF_PREC_FP32 && pr->prec != NMF_PREC_BF16) return false;
    return true;
  }
  if (pr->mode != NENMF_COMPRESSED) return false;
  if (pr->nu < pr->p || pr->nu > NMF_MAX_SKETCH) return false;
  return pr->L && pr->R && pr->XL && pr->XR;
}

// ----------------------------------------------------------------------------
// nmf_dual_product workspace
// ----------------------------------------------------------------------------
struct DualWs {
  Control* ctrl;
  __nv_bfloat16* Xb;
  int ldxb;
  void* opA;
  int lda;
  void* opB;
  int ldb;
  float* partN;
  float* partT;
  XPassPlan plan;
  size_t bytes;
};

DualWs carve_dual(void* base, int n, int m, int k, nmf_prec_t prec) {
  DualWs w{};
  Carver cv(base);
  w.plan = xpass_plan(n, m, k, prec, sm_count());
  w.ctrl = cv.take<Control>(1);
  if (x_converted(w.plan, prec)) {
    w.ldxb = round_up(m, 64);
    w.Xb = cv.take<__nv_bfloat16>(xb_elems(w.plan, n, w.ldxb));
  }
  w.lda = round_up(m, 128);
  w.ldb = round_up(n, 128);
  w.opA = cv.take<char>(op_bytes(w.plan, prec, w.lda));
  w.opB = cv.take<char>(op_bytes(w.plan, prec, w.ldb));
  w.partN = cv.take<float>((size_t)w.plan.S_c * n * w.plan.NV);
  w.partT = cv.take<float>((size_t)w.plan.S_r * m * w.plan.NV);
  w.bytes = cv.size();
  return w;
}

}  // namespace

extern "C" {

const char* nmf_status_string(nmf_status_t st) {
  switch (st) {
    case NMF_OK: return "ok";
    case NMF_ERR_INVALID_ARG: return "invalid argument";
    case NMF_ERR_WORKSPACE: return "workspace missing, misaligned or too small";
    case NMF_ERR_CUDA: return "CUDA runtime error";
    case NMF_ERR_NOT_SPD: return "Gram matrix not positive definite";
    case NMF_ERR_NONFINITE: return "non-finite value";
    case NMF_ERR_DEVICE_TIMEOUT: return "bounded device wait timed out";
    case NMF_ERR_UNSUPPORTED: return "unsupported device or configuration";
  }
  return "unknown status";
}

int nmf_version(void) { return 100; }

nmf_status_t nmf_workspace_status(nmf_stream_t stream, const void* workspace, int* status) {
  if (!workspace || !status) return NMF_ERR_INVALID_ARG;
  int v = 0;
  NMF_CU(cudaMemcpyAsync(&v, workspace, sizeof(int), cudaMemcpyDeviceToHost, (cudaStream_t)stream));
  NMF_CU(cudaStreamSynchronize((cudaStream_t)stream));
  *status = v;
  return NMF_OK;
}

void nmf_set_kernel_path(int flags) {
  g_force_simt = (flags & NMF_PATH_XPASS_CUDA_CORES) ? 1 : 0;
  g_per_update = (flags & NMF_PATH_SOLVE_PER_UPDATE) ? 1 : 0;
}

long long nmf_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

nmf_status_t nmf_inject_fault(int fault, long long wait_limit_ns) {
  if (fault != NMF_FAULT_NONE && fault != NMF_FAULT_STOP_TEST && fault != NMF_FAULT_XPASS_COPY)
    return NMF_ERR_INVALID_ARG;
  if (wait_limit_ns < 0) return NMF_ERR_INVALID_ARG;
  g_fault.store(fault, std::memory_order_relaxed);
  g_wait_ns.store(wait_limit_ns > 0 ? (unsigned long long)wait_limit_ns : kDefaultWaitNs, std::memory_order_relaxed);
  return NMF_OK;
}

nmf_status_t nmf_gaussian_sketch(nmf_stream_t stream, int rows, int cols, uint64_t seed, uint32_t stream_id,
                                 float* out) {
  if (rows < 0 || cols < 0 || (!out && rows * (long long)cols > 0)) return NMF_ERR_INVALID_ARG;
  if (rows == 0 || cols == 0) return NMF_OK;
  NMF_CU(sketch_launch(rows, cols, seed, stream_id, out, (cudaStream_t)stream));
  return NMF_OK;
}

size_t nmf_compress_workspace_size(int n, int m, int nu, nmf_prec_t prec) {
  if (n < 1 || m < 1 || nu < 1 || nu > NMF_MAX_SKETCH) return 0;
  return carve_compress(nullptr, n, m, nu, prec).bytes;
}

nmf_status_t nmf_compress_variant(nmf_stream_t stream, int n, int m, int nu, int q, nmf_prec_t prec, int variant,
                                  const float* X, const float* omega_L, const float* omega_R, uint64_t seed,
                                  float* L, float* R, float* XL, float* XR, void* workspace,
                                  size_t workspace_bytes) {
  if (n < 1 || m < 1 || nu < 1 || nu > NMF_MAX_SKETCH || nu > n || nu > m || q < 0) return NMF_ERR_INVALID_ARG;
  if (prec != NMF_PREC_FP32 && prec != NMF_PREC_BF16) return NMF_ERR_INVALID_ARG;
  if (variant < NMF_VARIANT_SUBSPACE || variant > NMF_VARIANT_GAUSSIAN) return NMF_ERR_INVALID_ARG;
  if (variant == NMF_VARIANT_SWAPPED && q < 1) return NMF_ERR_INVALID_ARG;
  if (!X || !L || !R || !XL || !XR) return NMF_ERR_INVALID_ARG;
  if ((omega_L == nullptr) != (omega_R == nullptr)) return NMF_ERR_INVALID_ARG;
  const CompressWs w = carve_compress(workspace, n, m, nu, prec);
  if (!ws_ok(workspace, workspace_bytes, w.bytes)) return NMF_ERR_WORKSPACE;
  cudaStream_t s = (cudaStream_t)stream;
  const bool xconv = x_converted(w.plan, prec);
  const int ofmt = op_format(w.plan, prec);
  const int NV = w.plan.NV;
  const size_t partA = (size_t)NV * w.lda, partB = (size_t)NV * w.ldb;  // OP_BF16X3 part strides

  NMF_CU(cudaMemsetAsync(w.ctrl, 0, sizeof(Control), s));
  NMF_CU(cudaMemsetAsync(w.opA, 0, op_bytes(w.plan, prec, w.lda), s));
  NMF_CU(cudaMemsetAsync(w.opB, 0, op_bytes(w.plan, prec, w.ldb), s));
  if (xconv) NMF_CU(xb_convert(w.plan, X, n, m, w.Xb, w.ldxb, w.ctrl, s));

  XPassArgs xa{};
  xa.n = n;
  xa.m = m;
  xa.X = xconv ? (const void*)w.Xb : (const void*)X;
  xa.ldx = xconv ? w.ldxb : m;
  xa.opA = w.opA;
  xa.lda = w.lda;
  xa.opB = w.opB;
  xa.ldb = w.ldb;
  xa.partN = w.partN;
  xa.partT = w.partT;
  xa.nu = nu;
  xa.doN = xa.doT = true;
  xa.ctrl = w.ctrl;
  XPassArgs xN = xa, xT = xa;
  xN.doT = false;
  xT.doN = false;
  const Jobs both{true, true}, onlyN{true, false}, onlyT{false, true};
  // the closing pass: X_R = X R (N product) and/or X_L = (X^T L^T)^T (T product)
  auto closing = [&](Jobs jb) -> nmf_status_t {
    NMF_CU(xpass_launch(w.plan, jb.T ? xa : xN, prec, s));
    RowJob r[2] = {};
    int k = 0;
    r[k].part = w.partN; r[k].S = w.plan.S_c; r[k].ldp = NV; r[k].N = n; r[k].nu = nu; r[k].Y = XR;
    ++k;
    if (jb.T) {
      r[k].part = w.partT; r[k].S = w.plan.S_r; r[k].ldp = NV; r[k].N = m; r[k].nu = nu; r[k].Yt = XL;
      ++k;
    }
    NMF_CU(rows_launch(r, k, w.ctrl, s));
    return NMF_OK;
  };

  if (variant == NMF_VARIANT_GAUSSIAN) {
    // L = Omega_R / sqrt(nu) (nu x n), R = Omega_L / sqrt(nu) (m x nu); one pass for X_L, X_R
    const float sc = 1.f / sqrtf((float)nu);
    if (omega_L) {
      NMF_CU(scale_launch(omega_L, R, (long long)m * nu, sc, s));
      NMF_CU(scale_launch(omega_R, L, (long long)nu * n, sc, s));
    } else {
      NMF_CU(sketch_launch(m, nu, seed, 0u, R, s));
      NMF_CU(scale_launch(R, R, (long long)m * nu, sc, s));
      NMF_CU(sketch_launch(nu, n, seed, 1u, L, s));
      NMF_CU(scale_launch(L, L, (long long)nu * n, sc, s));
    }
    NMF_CU(transpose_launch(R, m, nu, w.opA, w.lda, ofmt, w.ctrl, s, partA));
    NMF_CU(copy_rows_launch(L, nu, n, w.opB, w.ldb, ofmt, w.ctrl, s, partB));
    return closing(both);
  }

  // Omega_L (m x nu) -> opA rows (A^T), Omega_R (nu x n) -> opB rows (B^T = Omega_R).
  const float* oL = omega_L;
  if (!oL) {
    NMF_CU(sketch_launch(m, nu, seed, 0u, w.omega, s));
    oL = w.omega;
  }
  NMF_CU(transpose_launch(oL, m, nu, w.opA, w.lda, ofmt, w.ctrl, s, partA));
  const float* oR = omega_R;
  if (!oR) {
    NMF_CU(sketch_launch(nu, n, seed, 1u, w.omega, s));
    oR = w.omega;
  }
  NMF_CU(copy_rows_launch(oR, nu, n, w.opB, w.ldb, ofmt, w.ctrl, s, partB));

  nmf_status_t st = NMF_OK;
  if (variant == NMF_VARIANT_SINGLE_CHAIN) {
    // one chain: Q_L^(0) = orth(X Omega_L); Q~ = orth(X^T Q_L), Q_L = orth(X Q~) q times;
    // L = Q_L^(q)^T; X_L^T = X^T Q_L^(q) and R = orth(X^T Q_L^(q)); X_R = X R
    NMF_CU(xpass_launch(w.plan, xN, prec, s));
    if ((st = orthonormalize(w, n, m, nu, ofmt, onlyN, q == 0 ? L : nullptr, nullptr, nullptr, s)) != NMF_OK) return st;
    for (int k = 1; k <= q; ++k) {
      NMF_CU(xpass_launch(w.plan, xT, prec, s));
      if ((st = orthonormalize(w, n, m, nu, ofmt, onlyT, nullptr, nullptr, nullptr, s)) != NMF_OK) return st;
      NMF_CU(xpass_launch(w.plan, xN, prec, s));
      if ((st = orthonormalize(w, n, m, nu, ofmt, onlyN, k == q ? L : nullptr, nullptr, nullptr, s)) != NMF_OK)
        return st;
    }
    NMF_CU(xpass_launch(w.plan, xT, prec, s));
    if ((st = orthonormalize(w, n, m, nu, ofmt, onlyT, nullptr, R, XL, s)) != NMF_OK) return st;
    return closing(onlyN);
  }

  // two chains, both products of every pass: the chains trade N and T roles
  // each pass (see the file header). Subspace iteration orthonormalises after
  // passes 0 .. 2q (L, R after the last); the swapped reading stops one pass
  // earlier, where the half-step bases Q~_R^(q), Q~_L^(q) sit in the N and T
  // jobs; power iteration only rescales columns until the last pass.
  const int steps = variant == NMF_VARIANT_SWAPPED ? 2 * q : 2 * q + 1;
  for (int pass = 0; pass < steps; ++pass) {
    NMF_CU(xpass_launch(w.plan, xa, prec, s));
    const bool last = pass == steps - 1;
    if (variant == NMF_VARIANT_POWER && !last) st = normalize_columns(w, n, m, nu, ofmt, both, s);
    else st = orthonormalize(w, n, m, nu, ofmt, both, last ? L : nullptr, last ? R : nullptr, nullptr, s);
    if (st != NMF_OK) return st;
  }
  return closing(both);
}

namespace {

// Lanes of a batched compression: library-owned streams of one device,
// created on first use and kept for the process; calls that enqueue on
// them are serialised by a mutex (the enqueue only, not the GPU work).
constexpr int kLanes = 8;
struct LaneSet {
  int dev = -1;
  cudaStream_t s[kLanes] = {};
  cudaEvent_t fork = nullptr;
  cudaEvent_t join[kLanes] = {};
};
std::mutex g_lane_mu;
std::vector<LaneSet> g_lanes;

cudaError_t lanes_for_device(LaneSet** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  for (auto& l : g_lanes)
    if (l.dev == dev) {
      *out = &l;
      return cudaSuccess;
    }
  LaneSet l;
  l.dev = dev;
  for (int i = 0; i < kLanes; ++i) {
    if ((e = cudaStreamCreateWithFlags(&l.s[i], cudaStreamNonBlocking)) != cudaSuccess) return e;
    if ((e = cudaEventCreateWithFlags(&l.join[i], cudaEventDisableTiming)) != cudaSuccess) return e;
  }
  if ((e = cudaEventCreateWithFlags(&l.fork, cudaEventDisableTiming)) != cudaSuccess) return e;
  g_lanes.push_back(l);
  *out = &g_lanes.back();
  return cudaSuccess;
}

size_t batch_slot_bytes(int count, const nmf_compress_item_t* items, nmf_prec_t prec) {
  size_t slot = 0;
  for (int i = 0; i < count; ++i) {
    const size_t b = nmf_compress_workspace_size(items[i].n, items[i].m, items[i].nu, prec);
    if (b == 0) return 0;
    slot = std::max(slot, round_up_sz(b, 256));
  }
  return slot;
}

}  // namespace

// The SMs one lane's X passes are planned for: a quarter more than an even
// share (the lanes' passes seldom coincide all at once; at 8 lanes on 152
// SMs the batched compression measured 24.2 ms with 24 SMs a lane, 24.8
// with 19, 25.7 with 16 and 27.2 with 12).
static int lane_sms(int lanes) {
  lanes = std::max(1, lanes);
  const int sms = sm_count();
  return std::min(sms, std::max(1, (5 * sms + 4 * lanes - 1) / (4 * lanes)));
}

size_t nmf_compress_batched_workspace_size(int count, const nmf_compress_item_t* items, nmf_prec_t prec) {
  if (count < 1 || !items) return 0;
  XPassSmBudget budget(lane_sms(std::min(count, kLanes)));
  const size_t slot = batch_slot_bytes(count, items, prec);
  return slot * (size_t)std::min(count, kLanes);
}

nmf_status_t nmf_compress_batched(nmf_stream_t stream, int count, const nmf_compress_item_t* items, nmf_prec_t prec,
                                  int variant, void* workspace, size_t workspace_bytes) {
  if (count < 0 || (count > 0 && !items)) return NMF_ERR_INVALID_ARG;
  if (count == 0) return NMF_OK;
  for (int i = 0; i < count; ++i) {
    const nmf_compress_item_t& it = items[i];
    if (it.n < 1 || it.m < 1 || it.nu < 1 || it.nu > NMF_MAX_SKETCH || it.nu > it.n || it.nu > it.m || it.q < 0)
      return NMF_ERR_INVALID_ARG;
    if (!it.X || !it.L || !it.R || !it.XL || !it.XR) return NMF_ERR_INVALID_ARG;
    if (variant == NMF_VARIANT_SWAPPED && it.q < 1) return NMF_ERR_INVALID_ARG;
  }
  if (prec != NMF_PREC_FP32 && prec != NMF_PREC_BF16) return NMF_ERR_INVALID_ARG;
  if (variant < NMF_VARIANT_SUBSPACE || variant > NMF_VARIANT_GAUSSIAN) return NMF_ERR_INVALID_ARG;
  const int lanes = std::min(count, kLanes);
  // each item's X passes planned for one lane's share of the SMs
  XPassSmBudget budget(lane_sms(lanes));
  const size_t slot = batch_slot_bytes(count, items, prec);
  if (!ws_ok(workspace, workspace_bytes, slot * lanes)) return NMF_ERR_WORKSPACE;
  std::lock_guard<std::mutex> g(g_lane_mu);
  LaneSet* L = nullptr;
  NMF_CU(lanes_for_device(&L));
  cudaStream_t s = (cudaStream_t)stream;
  // fork: every lane starts after what the caller's stream holds
  NMF_CU(cudaEventRecord(L->fork, s));
  for (int k = 0; k < lanes; ++k) NMF_CU(cudaStreamWaitEvent(L->s[k], L->fork, 0));
  // Programmatic dependent launch stays off on the lanes: a dependent X pass
  // whose CTAs start early would hold SMs (and their shared memory) while it
  // waits, away from the other lanes' kernels.
  PdlOff pdl_off;
  for (int i = 0; i < count; ++i) {
    const int k = i % lanes;
    const nmf_compress_item_t& it = items[i];
    char* ws = static_cast<char*>(workspace) + (size_t)k * slot;
    const nmf_status_t st =
        nmf_compress_variant((nmf_stream_t)L->s[k], it.n, it.m, it.nu, it.q, prec, variant, it.X, nullptr, nullptr,
                             it.seed, it.L, it.R, it.XL, it.XR, ws, slot);
    if (st != NMF_OK) return st;
  }
  // join: the caller's stream continues after every lane
  for (int k = 0; k < lanes; ++k) {
    NMF_CU(cudaEventRecord(L->join[k], L->s[k]));
    NMF_CU(cudaStreamWaitEvent(s, L->join[k], 0));
  }
  return NMF_OK;
}

nmf_status_t nmf_compress(nmf_stream_t stream, int n, int m, int nu, int q, nmf_prec_t prec, const float* X,
                          const float* omega_L, const float* omega_R, uint64_t seed, float* L, float* R, float* XL,
                          float* XR, void* workspace, size_t workspace_bytes) {
  return nmf_compress_variant(stream, n, m, nu, q, prec, NMF_VARIANT_SUBSPACE, X, omega_L, omega_R, seed, L, R, XL,
                              XR, workspace, workspace_bytes);
}

// The stop test needs every CTA of a solve launch resident at once. A
// compressed problem with more vectors than that runs on the batched kernel
// instead (one problem, one cluster of CTAs: its stop test is block-wise and
// needs no co-residency).
bool too_many_ctas(const nenmf_problem_t& pr) {
  const bool plain = pr.mode == NENMF_PLAIN;
  const int nu = plain ? 0 : pr.nu;
  const int epiG = plain ? EPI_GRAM : EPI_W_COLS;
  const int epiF = plain ? EPI_GRAM : EPI_W_ROWS;
  const int P = partial_stride(plain ? pr.p * pr.p : pr.p * nu);
  const int ctasG = solve_ctas(pr.n), ctasF = solve_ctas(pr.m);
  const int gG = partial_group_size(ctasG, P), gF = partial_group_size(ctasF, P);
  const int inG = gF > 1 ? group_count(ctasF, gF) : ctasF;
  const int inF = gG > 1 ? group_count(ctasG, gG) : ctasG;
  return ctasG > kMaxStopCtas || ctasF > kMaxStopCtas || ctasG > solve_max_coresident(pr.p, nu, epiG, inG) ||
         ctasF > solve_max_coresident(pr.p, nu, epiF, inF);
}

constexpr int kLargeCluster = 8;

size_t large_workspace(const nenmf_problem_t& pr) {
  nenmf_params_t worst{};
  worst.max_outer = 1;
  worst.max_inner = kMaxInnerIters;
  worst.min_inner = 1;
  worst.tol = 1.0;
  worst.tol_mode = NENMF_TOL_REL;
  const nenmf_batch_config_t cfg{kLargeCluster, 0};
  return nenmf_solve_batched_workspace_size(1, &pr, &worst, &cfg);
}

size_t nenmf_solve_workspace_size(const nenmf_problem_t* problem) {
  if (!problem_ok(problem)) return 0;
  size_t b = carve_solve(nullptr, *problem).bytes;
  if (problem->mode == NENMF_COMPRESSED && too_many_ctas(*problem)) b = std::max(b, large_workspace(*problem));
  return b;
}

nmf_status_t nenmf_solve(nmf_stream_t stream, const nenmf_problem_t* problem, float* G, float* F,
                         const nenmf_params_t* params, nenmf_stats_t* stats, void* workspace, size_t workspace_bytes) {
  if (!problem_ok(problem) || !params || !G || !F) return NMF_ERR_INVALID_ARG;
  const nenmf_problem_t pr = *problem;
  const nenmf_params_t pa = *params;
  if (pa.max_outer < 0 || pa.max_outer > 32000 || pa.max_inner < 1 || pa.max_inner > kMaxInner || pa.min_inner < 1)
    return NMF_ERR_INVALID_ARG;
  if (pa.tol_mode != NENMF_TOL_REL && pa.tol_mode != NENMF_TOL_ABS) return NMF_ERR_INVALID_ARG;
  const SolveWs w = carve_solve(workspace, pr);
  if (!ws_ok(workspace, workspace_bytes, w.bytes)) return NMF_ERR_WORKSPACE;
  const bool plain = pr.mode == NENMF_PLAIN;
  const int n = pr.n, m = pr.m, p = pr.p, nu = plain ? 0 : pr.nu;
  const bool test = pa.tol > 0.0;
  const int epiG = plain ? EPI_GRAM : EPI_W_COLS;
  const int epiF = plain ? EPI_GRAM : EPI_W_ROWS;
  const int groupsInG = w.groupF > 1 ? group_count(w.ctasF, w.groupF) : w.ctasF;  // read by the G update
  const int groupsInF = w.groupG > 1 ? group_count(w.ctasG, w.groupG) : w.ctasG;  // read by the F update
  if (test && (w.ctasG > kMaxStopCtas || w.ctasF > kMaxStopCtas || w.ctasG > solve_max_coresident(p, nu, epiG, groupsInG) ||
               w.ctasF > solve_max_coresident(p, nu, epiF, groupsInF))) {
    // more vectors than one co-resident grid: compressed problems go to the
    // batched kernel (snapshots are single-kernel only)
    if (plain || pa.record_G || pa.record_F || pa.record_time_ns) return NMF_ERR_UNSUPPORTED;
    const nenmf_batch_config_t cfg{kLargeCluster, 0};
    return nenmf_solve_batched(stream, 1, &pr, &G, &F, &pa, &cfg, stats, workspace, workspace_bytes);
  }
  cudaStream_t s = (cudaStream_t)stream;
  Control* ctrl = w.ctrl;
  const nmf_prec_t prec = (nmf_prec_t)pr.prec;
  const bool bf16 = plain && prec == NMF_PREC_BF16;
  unsigned long long* times = reinterpret_cast<unsigned long long*>(pa.record_time_ns);

  if (!plain && !g_per_update) {
    // Alg. 1 in one persistent launch when every CTA fits at once
    const PersistPlan pp = persist_plan(n, m, p, nu, test, pa.restart != 0);
    // (pending iterates outside shared memory need the workspace's keep buffer)
    if (pp.ok && (pp.keep_shared || persist_keep_floats(n, m, p, nu) > 0)) {
      NMF_CU(cudaMemsetAsync(ctrl, 0, sizeof(Control), s));
      NMF_CU(cudaMemsetAsync(w.bar, 0, sizeof(unsigned int), s));
      if (test)
        NMF_CU(cudaMemsetAsync(w.slots, 0, sizeof(unsigned long long) * pa.max_inner * pp.ctas, s));
      if (stats) NMF_CU(cudaMemsetAsync(stats, 0, sizeof(nenmf_stats_t), s));
      if (times) {
        NMF_CU(cudaMemsetAsync(times, 0, sizeof(long long) * ((size_t)pa.max_outer + 1), s));
        NMF_CU(timestamp_launch(times, s));
      }
      NMF_CU(beta_launch(w.beta, pa.max_inner, s));
      PersistLaunch L{};
      L.n = n; L.m = m; L.p = p; L.nu = nu;
      L.L = pr.L; L.R = pr.R; L.XL = pr.XL; L.XR = pr.XR;
      L.G = G; L.F = F;
      L.max_outer = pa.max_outer; L.max_inner = pa.max_inner; L.min_inner = pa.min_inner;
      L.restart = pa.restart ? 1 : 0;
      L.beta = w.beta;
      L.partG = w.partG; L.partF = w.partF;
      L.pg2G = w.pg2G; L.pg2F = w.pg2F; L.initG = w.initG; L.initF = w.initF;
      L.slots = w.slots; L.bar = w.bar; L.keep = w.keep;
      L.record_G = pa.record_G; L.record_F = pa.record_F; L.times = times;
      L.tol = pa.tol; L.tol_mode = pa.tol_mode;
      L.stats = stats; L.ctrl = ctrl;
      NMF_CU(persist_launch(pp, L, s));
      if (stats || pa.max_outer > 0)
        NMF_CU(stats_launch(stats, pa.max_outer > 0 ? w.pg2G : nullptr, w.ctasG, pa.max_outer > 0 ? w.pg2F : nullptr,
                            w.ctasF, ctrl, pa.max_outer, s));
      return NMF_OK;
    }
  }

  NMF_CU(cudaMemsetAsync(ctrl, 0, sizeof(Control), s));
  NMF_CU(cudaMemsetAsync(w.ctr, 0, sizeof(unsigned int) * w.nctr, s));
  if (test) {
    // one row of words per test and side; tags from an earlier call could match, so clear the rows used
    NMF_CU(cudaMemsetAsync(w.slots, 0, sizeof(unsigned long long) * pa.max_inner * w.ctasG, s));
    NMF_CU(cudaMemsetAsync(w.slots + (size_t)kMaxInnerIters * w.ctasG, 0,
                           sizeof(unsigned long long) * pa.max_inner * w.ctasF, s));
  }
  if (stats) NMF_CU(cudaMemsetAsync(stats, 0, sizeof(nenmf_stats_t), s));
  if (times) {
    NMF_CU(cudaMemsetAsync(times, 0, sizeof(long long) * ((size_t)pa.max_outer + 1), s));
    NMF_CU(timestamp_launch(times, s));
  }
  NMF_CU(beta_launch(w.beta, pa.max_inner, s));
  NMF_CU(transpose_launch(G, n, p, w.Gt, n, 0, ctrl, s));

  XPassArgs xa{};
  if (plain) {
    const size_t es = bf16 ? 2 : 4;
    NMF_CU(cudaMemsetAsync(w.opF, 0, (size_t)w.plan.NV * w.ldF * es, s));
    NMF_CU(cudaMemsetAsync(w.opG, 0, (size_t)w.plan.NV * w.ldG * es, s));
    if (bf16) NMF_CU(xb_convert(w.plan, pr.X, n, m, w.Xb, w.ldxb, ctrl, s));
    xa.n = n;
    xa.m = m;
    xa.X = bf16 ? (const void*)w.Xb : (const void*)pr.X;
    xa.ldx = bf16 ? w.ldxb : m;
    xa.opA = w.opF;
    xa.lda = w.ldF;
    xa.opB = w.opG;
    xa.ldb = w.ldG;
    xa.partN = w.partN;
    xa.partT = w.partT;
    xa.nu = p;
    xa.ctrl = ctrl;
  }
  XPassArgs xN = xa, xT = xa;
  xN.doN = true; xN.doT = false;
  xT.doN = false; xT.doT = true;

  SolveArgs g{};
  g.p = p; g.N = n; g.nu = nu; g.Y = w.Gt;
  g.max_inner = pa.max_inner; g.min_inner = pa.min_inner; g.stop_test = test; g.side = 0;
  g.restart = pa.restart ? 1 : 0;
  g.pg2_init = w.initG; g.pg2_part = w.pg2G; g.stats = stats; g.ctrl = ctrl;
  g.epi = epiG;
  g.part_in = w.groupF > 1 ? w.groupOutF : w.partF;
  g.groups_in = groupsInG;
  g.part_out = w.partG; g.group = w.groupG; g.group_out = w.groupOutG; g.tail_ctr = w.ctr;
  g.stop_slots = w.slots;
  SolveArgs f = g;
  f.N = m; f.Y = F; f.side = 1; f.pg2_init = w.initF; f.pg2_part = w.pg2F; f.epi = epiF;
  f.part_in = w.groupG > 1 ? w.groupOutG : w.partG;
  f.groups_in = groupsInF;
  f.part_out = w.partF; f.group = w.groupF; f.group_out = w.groupOutF;
  f.tail_ctr = w.ctr + group_count(w.ctasG, w.groupG);
  f.stop_slots = w.slots + (size_t)kMaxInnerIters * w.ctasG;
  if (plain) {
    g.bsrc = B_FROM_PARTIALS; g.Bpart = w.partN; g.Bparts = w.plan.S_c; g.Bld = w.plan.NV;
    g.op_out = w.opG; g.op_ld = w.ldG; g.op_bf16 = bf16;
    f.bsrc = B_FROM_PARTIALS; f.Bpart = w.partT; f.Bparts = w.plan.S_r; f.Bld = w.plan.NV;
    f.op_out = w.opF; f.op_ld = w.ldF; f.op_bf16 = bf16;
  } else {
    g.bsrc = B_FROM_ROWS; g.D = pr.XR; g.E = pr.L;
    f.bsrc = B_FROM_COLS; f.D = pr.XL; f.E = pr.R;
  }

  // Products of the initial F for the first G update (and its operand copy).
  {
    SolveArgs f0 = f;
    f0.stats = nullptr;
    NMF_CU(solve_launch_mode(f0, w.beta, MODE_EPI_ONLY, s));
  }
  if (test) {
    // eps from the projected gradients at (G0, F0) of the objective being solved.
    if (plain) NMF_CU(xpass_launch(w.plan, xN, prec, s));
    SolveArgs g0 = g;
    g0.stats = nullptr;
    NMF_CU(solve_launch_mode(g0, w.beta, MODE_EVAL, s));
    if (plain) NMF_CU(xpass_launch(w.plan, xT, prec, s));
    SolveArgs f0 = f;
    f0.stats = nullptr;
    f0.epi = EPI_NONE;
    f0.op_out = nullptr;
    NMF_CU(solve_launch_mode(f0, w.beta, MODE_EVAL, s));
  }
  NMF_CU(eps_launch(ctrl, w.initG, w.ctasG, w.initF, w.ctasF, pa.tol, pa.tol_mode, stats, s));

  for (int t = 0; t < pa.max_outer; ++t) {
    if (plain) NMF_CU(xpass_launch(w.plan, xN, prec, s));
    SolveArgs gt = g;
    gt.epoch = 2 * t + 1;
    if (pa.record_G) {
      gt.record = pa.record_G + (size_t)t * n * p;
      gt.record_transposed = 1;
    }
    NMF_CU(solve_launch_mode(gt, w.beta, MODE_SOLVE, s));
    if (plain) NMF_CU(xpass_launch(w.plan, xT, prec, s));
    SolveArgs ft = f;
    ft.epoch = 2 * t + 2;
    if (pa.record_F) ft.record = pa.record_F + (size_t)t * p * m;
    if (times) ft.time_out = times + t + 1;
    NMF_CU(solve_launch_mode(ft, w.beta, MODE_SOLVE, s));
  }
  if (stats || pa.max_outer > 0)
    NMF_CU(stats_launch(stats, pa.max_outer > 0 ? w.pg2G : nullptr, w.ctasG, pa.max_outer > 0 ? w.pg2F : nullptr,
                        w.ctasF, ctrl, pa.max_outer, s));
  NMF_CU(transpose_launch(w.Gt, p, n, G, p, 0, nullptr, s));
  return NMF_OK;
}

size_t nmf_rre_workspace_size(int n, int m, int p) {
  if (n < 1 || m < 1 || p < 1) return 0;
  return round_up_sz((size_t)rre_parts(n, m) * 2 * sizeof(double), 256);
}

nmf_status_t nmf_rre(nmf_stream_t stream, int n, int m, int p, const float* X, const float* G, const float* F,
                     double* out, void* workspace, size_t workspace_bytes) {
  if (n < 1 || m < 1 || p < 1 || p > NMF_MAX_RANK || !X || !G || !F || !out) return NMF_ERR_INVALID_ARG;
  if (!ws_ok(workspace, workspace_bytes, nmf_rre_workspace_size(n, m, p))) return NMF_ERR_WORKSPACE;
  NMF_CU(rre_launch(n, m, p, X, G, F, out, static_cast<double*>(workspace), rre_parts(n, m), (cudaStream_t)stream));
  return NMF_OK;
}

size_t nmf_dual_product_workspace_size(int n, int m, int k, nmf_prec_t prec) {
  if (n < 1 || m < 1 || k < 1 || k > NMF_MAX_SKETCH) return 0;
  return carve_dual(nullptr, n, m, k, prec).bytes;
}

nmf_status_t nmf_dual_product(nmf_stream_t stream, int n, int m, int k, nmf_prec_t prec, const float* X,
                              const float* A, const float* B, float* YN, float* YT, void* workspace,
                              size_t workspace_bytes) {
  if (n < 1 || m < 1 || k < 1 || k > NMF_MAX_SKETCH || !X) return NMF_ERR_INVALID_ARG;
  if (prec != NMF_PREC_FP32 && prec != NMF_PREC_BF16) return NMF_ERR_INVALID_ARG;
  if ((A == nullptr) != (YN == nullptr) || (B == nullptr) != (YT == nullptr) || (!A && !B))
    return NMF_ERR_INVALID_ARG;
  const DualWs w = carve_dual(workspace, n, m, k, prec);
  if (!ws_ok(workspace, workspace_bytes, w.bytes)) return NMF_ERR_WORKSPACE;
  cudaStream_t s = (cudaStream_t)stream;
  const bool xconv = x_converted(w.plan, prec);
  const int ofmt = op_format(w.plan, prec);
  NMF_CU(cudaMemsetAsync(w.ctrl, 0, sizeof(Control), s));
  NMF_CU(cudaMemsetAsync(w.opA, 0, op_bytes(w.plan, prec, w.lda), s));
  NMF_CU(cudaMemsetAsync(w.opB, 0, op_bytes(w.plan, prec, w.ldb), s));
  if (xconv) NMF_CU(xb_convert(w.plan, X, n, m, w.Xb, w.ldxb, w.ctrl, s));
  if (A) NMF_CU(transpose_launch(A, m, k, w.opA, w.lda, ofmt, w.ctrl, s, (size_t)w.plan.NV * w.lda));
  if (B) NMF_CU(transpose_launch(B, n, k, w.opB, w.ldb, ofmt, w.ctrl, s, (size_t)w.plan.NV * w.ldb));
  XPassArgs xa{};
  xa.n = n; xa.m = m;
  xa.X = xconv ? (const void*)w.Xb : (const void*)X;
  xa.ldx = xconv ? w.ldxb : m;
  xa.opA = w.opA; xa.lda = w.lda; xa.opB = w.opB; xa.ldb = w.ldb;
  xa.partN = w.partN; xa.partT = w.partT; xa.nu = k;
  xa.doN = A != nullptr; xa.doT = B != nullptr;
  xa.ctrl = w.ctrl;
  NMF_CU(xpass_launch(w.plan, xa, prec, s));
  RowJob r[2] = {};
  int nj = 0;
  if (A) {
    r[nj].part = w.partN; r[nj].S = w.plan.S_c; r[nj].ldp = w.plan.NV; r[nj].N = n; r[nj].nu = k; r[nj].Y = YN;
    ++nj;
  }
  if (B) {
    r[nj].part = w.partT; r[nj].S = w.plan.S_r; r[nj].ldp = w.plan.NV; r[nj].N = m; r[nj].nu = k; r[nj].Y = YT;
    ++nj;
  }
  NMF_CU(rows_launch(r, nj, w.ctrl, s));
  return NMF_OK;
}

size_t nmf_project_workspace_size(int n, int m, int nu, nmf_prec_t prec) {
  if (n < 1 || m < 1 || nu < 1 || nu > NMF_MAX_SKETCH || nu > n || nu > m) return 0;
  return carve_dual(nullptr, n, m, nu, prec).bytes;
}

nmf_status_t nmf_project(nmf_stream_t stream, int n, int m, int nu, nmf_prec_t prec, const float* X, const float* L,
                         const float* R, float* XL, float* XR, void* workspace, size_t workspace_bytes) {
  if (n < 1 || m < 1 || nu < 1 || nu > NMF_MAX_SKETCH || nu > n || nu > m || !X || !L || !R || !XL || !XR)
    return NMF_ERR_INVALID_ARG;
  if (prec != NMF_PREC_FP32 && prec != NMF_PREC_BF16) return NMF_ERR_INVALID_ARG;
  const DualWs w = carve_dual(workspace, n, m, nu, prec);
  if (!ws_ok(workspace, workspace_bytes, w.bytes)) return NMF_ERR_WORKSPACE;
  cudaStream_t s = (cudaStream_t)stream;
  const bool xconv = x_converted(w.plan, prec);
  const int ofmt = op_format(w.plan, prec);
  NMF_CU(cudaMemsetAsync(w.ctrl, 0, sizeof(Control), s));
  NMF_CU(cudaMemsetAsync(w.opA, 0, op_bytes(w.plan, prec, w.lda), s));
  NMF_CU(cudaMemsetAsync(w.opB, 0, op_bytes(w.plan, prec, w.ldb), s));
  if (xconv) NMF_CU(xb_convert(w.plan, X, n, m, w.Xb, w.ldxb, w.ctrl, s));
  // X_R = X R: R is the N-product operand (stored transposed); X_L^T = X^T L^T:
  // the T-product operand is (L^T)^T = L itself, copied row by row
  NMF_CU(transpose_launch(R, m, nu, w.opA, w.lda, ofmt, w.ctrl, s, (size_t)w.plan.NV * w.lda));
  NMF_CU(copy_rows_launch(L, nu, n, w.opB, w.ldb, ofmt, w.ctrl, s, (size_t)w.plan.NV * w.ldb));
  XPassArgs xa{};
  xa.n = n; xa.m = m;
  xa.X = xconv ? (const void*)w.Xb : (const void*)X;
  xa.ldx = xconv ? w.ldxb : m;
  xa.opA = w.opA; xa.lda = w.lda; xa.opB = w.opB; xa.ldb = w.ldb;
  xa.partN = w.partN; xa.partT = w.partT; xa.nu = nu;
  xa.doN = true; xa.doT = true;
  xa.ctrl = w.ctrl;
  NMF_CU(xpass_launch(w.plan, xa, prec, s));
  RowJob r[2] = {};
  r[0].part = w.partN; r[0].S = w.plan.S_c; r[0].ldp = w.plan.NV; r[0].N = n; r[0].nu = nu; r[0].Y = XR;
  r[1].part = w.partT; r[1].S = w.plan.S_r; r[1].ldp = w.plan.NV; r[1].N = m; r[1].nu = nu; r[1].Yt = XL;
  NMF_CU(rows_launch(r, 2, w.ctrl, s));
  return NMF_OK;
}

}  // extern "C"
