// orth.cu -- orthonormal bases for Alg. 2 ("QR decomposition", "orthonormal
// bases"), computed as CholeskyQR2 with a shifted first step when needed:
//
//   S = Y^T Y      Gram matrix, products exact (fmaf split) and sums in
//                  float-float, partials per CTA summed in a fixed order;
//   S = R^T R      Cholesky in float64 (one CTA); if a pivot is not
//                  safely positive, S + s I with s = 1e-10 trace(S) is used
//                  instead (shifted CholeskyQR, Fukaya et al. 2020) and a
//                  third pass is scheduled;
//   Q = Y R^{-1}   row by row in float32.
//
// Every pass keeps span(Q) = span(Y) (R is invertible), and the product of the
// R factors is upper triangular with a positive diagonal, so for a full-rank Y
// the result is the Q of the QR factorisation with diag(R) > 0.
#include "internal.h"

namespace nmf {
namespace {

constexpr int kRowThreads = 256;
constexpr int kMaxJobs = 2;
constexpr int kYsStride = NMF_MAX_SKETCH + 1;

struct RowJobs {
  RowJob j[kMaxJobs];
  int start[kMaxJobs + 1];
  int njobs;
};
struct CholJobs {
  CholJob j[kMaxJobs];
  int njobs;
};

__device__ __forceinline__ void tri_index(int e, int nu, int& a, int& b) {
  a = 0;
  while (e >= nu - a) {
    e -= nu - a;
    ++a;
  }
  b = a + e;
}

__global__ void __launch_bounds__(kRowThreads) rows_kernel(RowJobs jobs, Control* ctrl) {
  if (call_failed(ctrl)) return;
  int jj = 0;
  while (jj + 1 < jobs.njobs && (int)blockIdx.x >= jobs.start[jj + 1]) ++jj;
  const RowJob& J = jobs.j[jj];
  if (J.run_flag && *((volatile const int*)J.run_flag) == 0) return;
  const int cta = blockIdx.x - jobs.start[jj];
  const int r0 = cta * kOrthRows;
  const int rows = min(kOrthRows, J.N - r0);
  const int nu = J.nu;
  const int tid = threadIdx.x;

  extern __shared__ float smem[];
  float* Ys = smem;                              // kOrthRows x kYsStride
  float* Rs = Ys + kOrthRows * kYsStride;        // nu x nu (apply only)

  if (J.part) {
    // Sum over the S partials with 4 independent accumulators (loads in
    // flight together), combined in a fixed order.
    for (int i = tid; i < rows * nu; i += kRowThreads) {
      const int r = i / nu, c = i % nu;
      const float* p = J.part + (size_t)(r0 + r) * J.ldp + c;
      const size_t stride = (size_t)J.N * J.ldp;
      float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
      int k = 0;
      for (; k + 4 <= J.S; k += 4) {
        s0 += __ldcg(p + (k + 0) * stride);
        s1 += __ldcg(p + (k + 1) * stride);
        s2 += __ldcg(p + (k + 2) * stride);
        s3 += __ldcg(p + (k + 3) * stride);
      }
      for (; k < J.S; ++k) s0 += __ldcg(p + k * stride);
      Ys[r * kYsStride + c] = (s0 + s1) + (s2 + s3);
    }
  } else {
    for (int i = tid; i < nu * nu; i += kRowThreads) Rs[i] = J.rinv[i];
    for (int i = tid; i < rows * nu; i += kRowThreads) {
      const int r = i / nu, c = i % nu;
      Ys[r * kYsStride + c] = J.src[(size_t)(r0 + r) * nu + c];
    }
    __syncthreads();
    // q_r = y_r * Rinv, Rinv upper triangular: q[c] = sum_{k <= c} y[k] Rinv[k][c].
    // Thread t owns row t (t < rows); results staged in registers, then stored.
    float q[NMF_MAX_SKETCH];
    if (tid < rows) {
      const float* y = Ys + tid * kYsStride;
#pragma unroll
      for (int c = 0; c < NMF_MAX_SKETCH; ++c) {
        if (c < nu) {
          float s = 0.f;
          for (int k = 0; k <= c; ++k) s = fmaf(y[k], Rs[k * nu + c], s);
          q[c] = s;
        }
      }
    }
    __syncthreads();
    if (tid < rows) {
#pragma unroll
      for (int c = 0; c < NMF_MAX_SKETCH; ++c)
        if (c < nu) Ys[tid * kYsStride + c] = q[c];
    }
  }
  __syncthreads();

  bool bad = false;
  if (J.Y)
    for (int i = tid; i < rows * nu; i += kRowThreads) {
      const int r = i / nu, c = i % nu;
      const float v = Ys[r * kYsStride + c];
      bad |= !isfinite(v);
      J.Y[(size_t)(r0 + r) * nu + c] = v;
    }
  if (J.Yt)
    for (int i = tid; i < rows * nu; i += kRowThreads) {
      const int c = i / rows, r = i % rows;
      J.Yt[(size_t)c * J.N + r0 + r] = Ys[r * kYsStride + c];
    }
  if (J.op)
    for (int i = tid; i < rows * nu; i += kRowThreads) {
      const int c = i / rows, r = i % rows;
      const float v = Ys[r * kYsStride + c];
      if (J.op_bf16)
        static_cast<__nv_bfloat16*>(J.op)[(size_t)c * J.ldop + r0 + r] = __float2bfloat16_rn(v);
      else
        static_cast<float*>(J.op)[(size_t)c * J.ldop + r0 + r] = v;
    }
  if (bad) set_status(ctrl, NMF_ERR_NONFINITE);
  if (J.gram_part && (!J.gram_flag || *((volatile const int*)J.gram_flag) != 0)) {
    const int E = nu * (nu + 1) / 2;
    for (int e = tid; e < E; e += kRowThreads) {
      int a, b;
      tri_index(e, nu, a, b);
      DF s{0.f, 0.f};
      for (int r = 0; r < rows; ++r) df_add_product(s, Ys[r * kYsStride + a], Ys[r * kYsStride + b]);
      df_norm(s);
      J.gram_part[(size_t)cta * E + e] = make_float2(s.hi, s.lo);
    }
  }
}

constexpr int kCholThreads = 256;
constexpr int kSS = NMF_MAX_SKETCH + 1;  // double stride

__global__ void __launch_bounds__(kCholThreads) chol_kernel(CholJobs jobs, Control* ctrl) {
  if (call_failed(ctrl)) return;
  const CholJob& J = jobs.j[blockIdx.x];
  if (J.run_flag && *((volatile const int*)J.run_flag) == 0) return;
  const int nu = J.nu;
  const int E = nu * (nu + 1) / 2;
  const int tid = threadIdx.x;
  extern __shared__ double dsm[];
  double* S = dsm;              // nu x kSS, the Gram matrix
  double* A = S + nu * kSS;     // work / factor
  __shared__ int fail;
  __shared__ double shift;

  // Sum of the per-CTA float-float partials: 8 independent accumulators per
  // entry (loads in flight together), combined in a fixed order.
  for (int e = tid; e < E; e += kCholThreads) {
    constexpr int kAcc = 8;
    DF s[kAcc];
#pragma unroll
    for (int i = 0; i < kAcc; ++i) s[i] = DF{0.f, 0.f};
    int p = 0;
    for (; p + kAcc <= J.parts; p += kAcc) {
#pragma unroll
      for (int i = 0; i < kAcc; ++i) {
        const float2 v = __ldcg(J.gram_part + (size_t)(p + i) * E + e);
        df_add(s[i], v.x, v.y);
      }
    }
    for (int i = 0; p < J.parts; ++p, ++i) {
      const float2 v = __ldcg(J.gram_part + (size_t)p * E + e);
      df_add(s[i], v.x, v.y);
    }
#pragma unroll
    for (int i = 1; i < kAcc; ++i) df_add(s[0], s[i].hi, s[i].lo);
    int a, b;
    tri_index(e, nu, a, b);
    const double v = (double)s[0].hi + (double)s[0].lo;
    S[a * kSS + b] = v;
    S[b * kSS + a] = v;
  }
  __syncthreads();
  if (tid == 0) {
    double tr = 0.0;
    bool finite = true;
    for (int j = 0; j < nu; ++j) {
      tr += S[j * kSS + j];
      finite &= isfinite(S[j * kSS + j]);
    }
    shift = finite ? tr : -1.0;
  }
  __syncthreads();
  const double trace = shift;
  if (!(trace > 0.0)) {
    if (tid == 0) set_status(ctrl, trace < 0.0 ? NMF_ERR_NONFINITE : NMF_ERR_NOT_SPD);
    return;
  }
  double maxdiag = 0.0;
  for (int j = 0; j < nu; ++j) maxdiag = fmax(maxdiag, S[j * kSS + j]);
  const double pivot_floor = 1e-14 * maxdiag;

  int shifted = 0;
  for (int attempt = 0; attempt < 2; ++attempt) {
    shifted = attempt;
    const double s_add = attempt == 0 ? 0.0 : 1e-10 * trace;
    for (int i = tid; i < nu * nu; i += kCholThreads) {
      const int a = i / nu, b = i % nu;
      A[a * kSS + b] = S[a * kSS + b] + (a == b ? s_add : 0.0);
    }
    if (tid == 0) fail = 0;
    __syncthreads();
    for (int j = 0; j < nu; ++j) {
      if (tid == 0) {
        const double d = A[j * kSS + j];
        if (!(d > pivot_floor) || !isfinite(d)) fail = 1;
        else A[j * kSS + j] = sqrt(d);
      }
      __syncthreads();
      if (fail) break;
      const double rjj = A[j * kSS + j];
      for (int i = j + 1 + tid; i < nu; i += kCholThreads) A[j * kSS + i] /= rjj;
      __syncthreads();
      const int w = nu - j - 1;
      for (int t = tid; t < w * w; t += kCholThreads) {
        const int i = j + 1 + t / w, k = j + 1 + t % w;
        if (k >= i) A[i * kSS + k] -= A[j * kSS + i] * A[j * kSS + k];
      }
      __syncthreads();
    }
    if (!fail) break;
    __syncthreads();
  }
  if (fail) {
    if (tid == 0) set_status(ctrl, NMF_ERR_NOT_SPD);
    return;
  }
  if (tid == 0 && J.shift_flag) {
    if (J.reset_flag) *J.shift_flag = shifted;
    else if (shifted) *J.shift_flag = 1;
  }
  // Inverse of the upper factor R (upper triangle of A), column c by thread c,
  // back substitution in float64; results into S (no longer needed).
  if (tid < nu) {
    const int c = tid;
    for (int i = nu - 1; i > c; --i) S[i * kSS + c] = 0.0;
    S[c * kSS + c] = 1.0 / A[c * kSS + c];
    for (int i = c - 1; i >= 0; --i) {
      double s = 0.0;
      for (int k = i + 1; k <= c; ++k) s = fma(A[i * kSS + k], S[k * kSS + c], s);
      S[i * kSS + c] = -s / A[i * kSS + i];
    }
  }
  __syncthreads();
  for (int i = tid; i < nu * nu; i += kCholThreads) {
    const int a = i / nu, b = i % nu;
    J.rinv[i] = (float)S[a * kSS + b];
  }
}

}  // namespace

cudaError_t rows_launch(const RowJob* jobs, int njobs, Control* ctrl, cudaStream_t s) {
  RowJobs rj{};
  rj.njobs = njobs;
  int total = 0;
  int max_nu = 0;
  for (int i = 0; i < njobs; ++i) {
    rj.j[i] = jobs[i];
    rj.start[i] = total;
    total += rows_ctas(jobs[i].N);
    if (jobs[i].nu > max_nu) max_nu = jobs[i].nu;
  }
  rj.start[njobs] = total;
  const size_t smem = (size_t)(kOrthRows * kYsStride + max_nu * max_nu) * sizeof(float);
  cudaError_t e = allow_dynamic_smem((const void*)rows_kernel, (int)smem);
  if (e != cudaSuccess) return e;
  count_launches(1);
  rows_kernel<<<total, kRowThreads, smem, s>>>(rj, ctrl);
  return cudaGetLastError();
}

cudaError_t chol_launch(const CholJob* jobs, int njobs, Control* ctrl, cudaStream_t s) {
  CholJobs cj{};
  cj.njobs = njobs;
  int max_nu = 0;
  for (int i = 0; i < njobs; ++i) {
    cj.j[i] = jobs[i];
    if (jobs[i].nu > max_nu) max_nu = jobs[i].nu;
  }
  const size_t smem = (size_t)2 * max_nu * kSS * sizeof(double);
  cudaError_t e = allow_dynamic_smem((const void*)chol_kernel, (int)smem);
  if (e != cudaSuccess) return e;
  count_launches(1);
  chol_kernel<<<njobs, kCholThreads, smem, s>>>(cj, ctrl);
  return cudaGetLastError();
}

}  // namespace nmf
