// shard.cu -- the pieces a row-sharded run of the method needs beyond the
// single-GPU calls (X split by row blocks across GPUs; the exchange steps
// are collectives between the calls below):
//
//   nmf_gram         S = Y^T Y of this GPU's rows of an N x nu basis, in
//                    float-float, returned in float64 so the partial Grams of
//                    all row blocks can be summed by an all-reduce (Alg. 2's
//                    orthonormal bases, CholeskyQR);
//   nmf_orth_apply   Q = Y R^{-1} with R^T R = S for a given (summed) Gram:
//                    one CholeskyQR pass over this GPU's rows;
//   nenmf_nnls_block a block of iterations of the Nesterov inner loop (Sec. 2)
//                    on this GPU's columns, recording each iteration's share
//                    of ||P grad||^2 and its iterate, so that the stop test
//                    over all row blocks is decided after one all-reduce per
//                    block, as the sequential rule decides it.
#include "internal.h"
#include "nnls_device.cuh"
#include "stop_test.cuh"

namespace nmf {
namespace {

constexpr int kNnlsThreads = 128;

__device__ __forceinline__ void tri_of(int e, int nu, int& a, int& b) {
  a = 0;
  while (e >= nu - a) {
    e -= nu - a;
    ++a;
  }
  b = a + e;
}

// S (nu x nu, float64, both triangles) = sum of the float-float partial Grams
// (upper triangle, stride E2), summed in the order of the partials.
__global__ void gram_sum_kernel(const float2* parts, int nparts, int nu, int E2, double* S, Control* ctrl) {
  if (call_failed(ctrl)) return;
  const int E = nu * (nu + 1) / 2;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < E; e += gridDim.x * blockDim.x) {
    DF s{0.f, 0.f};
    for (int q = 0; q < nparts; ++q) {
      const float2 v = parts[(size_t)q * E2 + e];
      df_add(s, v.x, v.y);
    }
    int a, b;
    tri_of(e, nu, a, b);
    const double v = (double)s.hi + (double)s.lo;
    S[a * nu + b] = v;
    S[b * nu + a] = v;
  }
}

// A float64 Gram (upper triangle read) as one float-float partial.
__global__ void gram_from_f64_kernel(const double* S, int nu, int E2, float2* g) {
  const int E = nu * (nu + 1) / 2;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < E2; e += gridDim.x * blockDim.x) {
    if (e >= E) {
      g[e] = make_float2(0.f, 0.f);
      continue;
    }
    int a, b;
    tri_of(e, nu, a, b);
    const double v = S[a * nu + b];
    const float hi = (float)v;
    g[e] = make_float2(hi, (float)(v - (double)hi));
  }
}

struct NnlsArgs {
  int N, p;
  const float* H;   // p x p
  const float* B;   // p x N
  float* Y;         // p x N: the point the next step starts from (in/out)
  float* Fp;        // p x N: the previous iterate (in/out)
  int k0, kb;       // iterations k0 .. k0 + kb - 1 (kb = 0: evaluate ||P grad||^2 at Y)
  const float* beta;  // beta_k, k < max_inner
  float* keep;      // [kb][p][N]: the iterate of every iteration of the block
  double* part;     // [ctas][max(kb, 1)]: per-CTA shares of ||P grad||^2
  double* lc;       // L_c (written by CTA 0)
  Control* ctrl;
};

// g = H y - b; from PM = 24 on with one row of H live at a time (registers).
template <int PM>
__device__ __forceinline__ void hmv(const float* Hs, const float* y, const float* b, float* g) {
  if constexpr (PM >= 24) hmatvec_rolled<PM>(Hs, y, b, g);
  else hmatvec<PM>(Hs, y, b, g);
}

// One thread per column, the symmetric H (zero padded to PM) in shared
// memory. Every CTA computes L_c = lambda_max(H) itself (the same value);
// the step is that of the single-GPU solve: f = max(0, y - g / L_c), then
// y = f + beta_k (f - f_prev).
template <int PM>
__global__ void __launch_bounds__(kNnlsThreads) nnls_block_kernel(NnlsArgs a) {
  if (call_failed(a.ctrl)) return;
  __shared__ __align__(16) float Hs[PM * PM];
  __shared__ __align__(16) float Ms[2 * PM * lam_stride<PM>()];
  __shared__ float2 red[kNnlsThreads / 32];
  __shared__ double lam_s;
  const int tid = threadIdx.x, p = a.p;
  for (int i = tid; i < PM * PM; i += blockDim.x) {
    const int r = i / PM, c = i % PM;
    Hs[i] = (r < p && c < p) ? a.H[r * p + c] : 0.f;
  }
  __syncthreads();
  if (tid < 32) {
    const double lam = lambda_max_warp<PM>(Hs, Ms, p);
    if (tid == 0) lam_s = lam;
  }
  __syncthreads();
  double Lc_d = lam_s;
  if (!isfinite(Lc_d)) {
    if (tid == 0) set_status(a.ctrl, NMF_ERR_NONFINITE);
    Lc_d = 0.0;
  }
  if (blockIdx.x == 0 && tid == 0) *a.lc = Lc_d;
  const float Lc = (float)Lc_d;
  const int j = blockIdx.x * blockDim.x + tid;
  const bool active = j < a.N;
  float y[PM], fp[PM], b[PM], f[PM], g[PM];
#pragma unroll
  for (int c = 0; c < PM; ++c) {
    const bool in = active && c < p;
    y[c] = in ? a.Y[(size_t)c * a.N + j] : 0.f;
    fp[c] = in ? a.Fp[(size_t)c * a.N + j] : 0.f;
    b[c] = in ? a.B[(size_t)c * a.N + j] : 0.f;
  }
  const int slots = a.kb > 0 ? a.kb : 1;
  if (a.kb == 0 || !(Lc > 0.f)) {
    // evaluate at Y (also the L_c = 0 case, where the loop takes no step)
    hmv<PM>(Hs, y, b, g);
    const double s = block_sum_df(active ? pg_sq<PM>(y, g) : 0.f, red);
    if (tid == 0)
      for (int i = 0; i < slots; ++i) a.part[(size_t)blockIdx.x * slots + i] = s;
    return;
  }
  const float inv_Lc = 1.f / Lc;
  for (int i = 0; i < a.kb; ++i) {
    const int k = a.k0 + i;
    hmv<PM>(Hs, y, b, g);
#pragma unroll
    for (int c = 0; c < PM; ++c) f[c] = fmaxf(0.f, fmaf(-g[c], inv_Lc, y[c]));
    hmv<PM>(Hs, f, b, g);
    const double s = block_sum_df(active ? pg_sq<PM>(f, g) : 0.f, red);
    if (tid == 0) a.part[(size_t)blockIdx.x * slots + i] = s;
    const float beta = a.beta[k];
#pragma unroll
    for (int c = 0; c < PM; ++c) {
      if (active && c < p) a.keep[((size_t)i * p + c) * a.N + j] = f[c];
      y[c] = fmaf(beta, f[c] - fp[c], f[c]);
      fp[c] = f[c];
    }
  }
  if (active)
#pragma unroll
    for (int c = 0; c < PM; ++c)
      if (c < p) {
        a.Y[(size_t)c * a.N + j] = y[c];
        a.Fp[(size_t)c * a.N + j] = fp[c];
      }
}

// pg2[i] = sum over CTAs (in order) of part[cta][i].
__global__ void part_sum_kernel(const double* part, int ctas, int slots, double* pg2) {
  const int i = threadIdx.x;
  if (i >= slots) return;
  double s = 0.0;
  for (int c = 0; c < ctas; ++c) s += part[(size_t)c * slots + i];
  pg2[i] = s;
}

template <int PM>
cudaError_t nnls_launch_pm(const NnlsArgs& a, int ctas, cudaStream_t s) {
  count_launches(1);
  nnls_block_kernel<PM><<<ctas, kNnlsThreads, 0, s>>>(a);
  return cudaGetLastError();
}

// Workspace layouts.
struct GramWs {
  Control* ctrl;
  float2* parts;
  size_t bytes;
};
GramWs carve_gram(void* base, int N, int nu) {
  GramWs w{};
  Carver cv(base);
  w.ctrl = cv.take<Control>(1);
  w.parts = cv.take<float2>((size_t)rows_ctas(N) * (((nu * (nu + 1) / 2) + 1) & ~1));
  w.bytes = cv.size();
  return w;
}
struct ApplyWs {
  Control* ctrl;
  float2* g;
  size_t bytes;
};
ApplyWs carve_apply(void* base, int nu) {
  ApplyWs w{};
  Carver cv(base);
  w.ctrl = cv.take<Control>(1);
  w.g = cv.take<float2>((size_t)(((nu * (nu + 1) / 2) + 1) & ~1));
  w.bytes = cv.size();
  return w;
}
struct NnlsWs {
  Control* ctrl;
  float* beta;
  double* part;
  size_t bytes;
};
NnlsWs carve_nnls(void* base, int N, int max_inner, int kb) {
  NnlsWs w{};
  Carver cv(base);
  w.ctrl = cv.take<Control>(1);
  w.beta = cv.take<float>(max_inner > 0 ? max_inner : 1);
  w.part = cv.take<double>((size_t)ceil_div(N, kNnlsThreads) * (kb > 0 ? kb : 1));
  w.bytes = cv.size();
  return w;
}

bool ws_fits(const void* ws, size_t bytes, size_t need) {
  return ws != nullptr && (reinterpret_cast<uintptr_t>(ws) & 255u) == 0 && bytes >= need;
}

}  // namespace
}  // namespace nmf

using namespace nmf;

extern "C" {

size_t nmf_gram_workspace_size(int N, int nu) {
  if (N < 1 || nu < 1 || nu > NMF_MAX_SKETCH) return 0;
  return carve_gram(nullptr, N, nu).bytes;
}

nmf_status_t nmf_gram(nmf_stream_t stream, int N, int nu, const float* Y, double* S, void* workspace,
                      size_t workspace_bytes) {
  if (N < 1 || nu < 1 || nu > NMF_MAX_SKETCH || !Y || !S) return NMF_ERR_INVALID_ARG;
  const GramWs w = carve_gram(workspace, N, nu);
  if (!ws_fits(workspace, workspace_bytes, w.bytes)) return NMF_ERR_WORKSPACE;
  cudaStream_t s = (cudaStream_t)stream;
  NMF_CU(cudaMemsetAsync(w.ctrl, 0, sizeof(Control), s));
  RowJob j{};
  j.src = Y;
  j.N = N;
  j.nu = nu;
  j.gram_only = 1;
  j.gram_part = w.parts;
  j.gram_always = 1;
  NMF_CU(rows_launch(&j, 1, w.ctrl, s));
  const int E = nu * (nu + 1) / 2, E2 = (E + 1) & ~1;
  count_launches(1);
  gram_sum_kernel<<<ceil_div(E, 256), 256, 0, s>>>(w.parts, rows_ctas(N), nu, E2, S, w.ctrl);
  NMF_CU(cudaGetLastError());
  return NMF_OK;
}

size_t nmf_orth_apply_workspace_size(int N, int nu) {
  if (N < 1 || nu < 1 || nu > NMF_MAX_SKETCH) return 0;
  return carve_apply(nullptr, nu).bytes;
}

nmf_status_t nmf_orth_apply(nmf_stream_t stream, int N, int nu, const float* Y, const double* S, float* Q,
                            void* workspace, size_t workspace_bytes) {
  if (N < 1 || nu < 1 || nu > NMF_MAX_SKETCH || !Y || !S || !Q) return NMF_ERR_INVALID_ARG;
  const ApplyWs w = carve_apply(workspace, nu);
  if (!ws_fits(workspace, workspace_bytes, w.bytes)) return NMF_ERR_WORKSPACE;
  cudaStream_t s = (cudaStream_t)stream;
  NMF_CU(cudaMemsetAsync(w.ctrl, 0, sizeof(Control), s));
  const int E = nu * (nu + 1) / 2, E2 = (E + 1) & ~1;
  count_launches(1);
  gram_from_f64_kernel<<<ceil_div(E2, 256), 256, 0, s>>>(S, nu, E2, w.g);
  NMF_CU(cudaGetLastError());
  RowJob j{};
  j.src = Y;
  j.gram_in = w.g;
  j.gram_parts = 1;
  j.N = N;
  j.nu = nu;
  j.Y = Q;
  NMF_CU(rows_launch(&j, 1, w.ctrl, s));
  return NMF_OK;
}

size_t nenmf_nnls_block_workspace_size(int N, int p, int kb, int max_inner) {
  if (N < 1 || p < 1 || p > NMF_MAX_RANK || kb < 0 || max_inner < 1) return 0;
  return carve_nnls(nullptr, N, max_inner, kb).bytes;
}

nmf_status_t nenmf_nnls_block(nmf_stream_t stream, int N, int p, const float* H, const float* B, float* Y,
                              float* Fprev, int k0, int kb, int max_inner, float* keep, double* pg2, double* Lc,
                              void* workspace, size_t workspace_bytes) {
  if (N < 1 || p < 1 || p > NMF_MAX_RANK || kb < 0 || max_inner < 1 || k0 < 0 || k0 + kb > max_inner)
    return NMF_ERR_INVALID_ARG;
  if (!H || !B || !Y || !Fprev || !pg2 || !Lc || (kb > 0 && !keep)) return NMF_ERR_INVALID_ARG;
  const NnlsWs w = carve_nnls(workspace, N, max_inner, kb);
  if (!ws_fits(workspace, workspace_bytes, w.bytes)) return NMF_ERR_WORKSPACE;
  cudaStream_t s = (cudaStream_t)stream;
  NMF_CU(cudaMemsetAsync(w.ctrl, 0, sizeof(Control), s));
  NMF_CU(beta_launch(w.beta, max_inner, s));
  NnlsArgs a{};
  a.N = N;
  a.p = p;
  a.H = H;
  a.B = B;
  a.Y = Y;
  a.Fp = Fprev;
  a.k0 = k0;
  a.kb = kb;
  a.beta = w.beta;
  a.keep = keep;
  a.part = w.part;
  a.lc = Lc;
  a.ctrl = w.ctrl;
  const int ctas = ceil_div(N, kNnlsThreads);
  const int PM = p <= 4 ? 4 : p <= 8 ? 8 : p <= 12 ? 12 : p <= 16 ? 16 : p <= 24 ? 24 : 32;
  switch (PM) {
    case 4: NMF_CU(nnls_launch_pm<4>(a, ctas, s)); break;
    case 8: NMF_CU(nnls_launch_pm<8>(a, ctas, s)); break;
    case 12: NMF_CU(nnls_launch_pm<12>(a, ctas, s)); break;
    case 16: NMF_CU(nnls_launch_pm<16>(a, ctas, s)); break;
    case 24: NMF_CU(nnls_launch_pm<24>(a, ctas, s)); break;
    default: NMF_CU(nnls_launch_pm<32>(a, ctas, s)); break;
  }
  const int slots = kb > 0 ? kb : 1;
  count_launches(1);
  part_sum_kernel<<<1, 32, 0, s>>>(w.part, ctas, slots, pg2);
  NMF_CU(cudaGetLastError());
  return NMF_OK;
}

}  // extern "C"
