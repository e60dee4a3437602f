// orth.cu -- orthonormal bases for Alg. 2 ("QR decomposition", "orthonormal
// bases"), computed as CholeskyQR2 with a shifted first step when needed:
//
//   S = Y^T Y      Gram matrix: products exact (fmaf split), sums in
//                  float-float (~48 significant bits), one partial per CTA;
//   S = R^T R      Cholesky, also in float-float. GB300 runs float64 at 1/64
//                  of the float32 rate; float-float arithmetic runs on the
//                  float32 pipes with nearly the same precision, which is
//                  what CholeskyQR needs (kappa(Y)^2 * 2^-48 << 1). If a pivot
//                  is not safely positive, S + s I with s = 1e-10 trace(S) is
//                  factorised instead (shifted CholeskyQR, Fukaya et al.
//                  2020) and a third pass is scheduled;
//   Q = Y R^{-1}   R^{-1} in float-float (per CTA), then row by row with
//                  float-float dot products and one final rounding.
//
// Kernels: one "reduce" launch sums the X pass partials into Y and forms the
// first Gram partials; each "apply" launch sums the previous Gram partials
// (every CTA, in the same fixed order, so every CTA gets the same S), factors
// S redundantly per CTA, applies R^{-1} to its rows and forms the next Gram
// partials. Every pass keeps span(Q) = span(Y) (R is invertible), and the
// product of the R factors is upper triangular with a positive diagonal, so
// for a full-rank Y the result is the Q of the QR with diag(R) > 0.
#include "internal.h"

namespace nmf {
namespace {

constexpr int kRowThreads = kOrthRows;  // one row per thread in the apply step
constexpr int kMaxJobs = 2;
constexpr int kYsStride = NMF_MAX_SKETCH + 1;
constexpr int kAs = NMF_MAX_SKETCH + 1;           // stride of the factorisation arrays
constexpr int kStageFloat2 = 6 * 1024;            // Gram partial staging (48 KB)

struct RowJobs {
  RowJob j[kMaxJobs];
  int start[kMaxJobs + 1];
  int njobs;
};

// ---- float-float arithmetic (value = hi + lo, |lo| <= ulp(hi) / 2) --------
struct FF {
  float hi, lo;
};
__device__ __forceinline__ FF ff_quick(float a, float b) {  // |a| >= |b|
  const float s = a + b;
  return FF{s, b - (s - a)};
}
__device__ __forceinline__ FF ff_add(FF x, FF y) {
  const float s = x.hi + y.hi;
  const float bb = s - x.hi;
  float e = (x.hi - (s - bb)) + (y.hi - bb);
  e += x.lo + y.lo;
  return ff_quick(s, e);
}
__device__ __forceinline__ FF ff_neg(FF x) { return FF{-x.hi, -x.lo}; }
__device__ __forceinline__ FF ff_mul(FF x, FF y) {
  const float p = x.hi * y.hi;
  float e = fmaf(x.hi, y.hi, -p);
  e = fmaf(x.hi, y.lo, e);
  e = fmaf(x.lo, y.hi, e);
  return ff_quick(p, e);
}
__device__ __forceinline__ FF ff_div(FF x, FF y) {
  const float q1 = x.hi / y.hi;
  const FF r = ff_add(x, ff_neg(ff_mul(y, FF{q1, 0.f})));
  const float q2 = r.hi / y.hi;
  return ff_quick(q1, q2);
}
__device__ __forceinline__ FF ff_sqrt(FF x) {
  if (!(x.hi > 0.f)) return FF{0.f, 0.f};
  const float s = sqrtf(x.hi);
  const float p = s * s;
  const float e = fmaf(s, s, -p);
  const float r = ((x.hi - p) - e + x.lo) / (2.f * s);
  return ff_quick(s, r);
}

// Partials of a Gram matrix are stored with an even stride of float2
// (E rounded up to 2), so every partial starts on a 16-byte boundary.
__host__ __device__ __forceinline__ int gram_stride(int nu) { return (nu * (nu + 1) / 2 + 1) & ~1; }

__device__ __forceinline__ void tri_index(int e, int nu, int& a, int& b) {
  a = 0;
  while (e >= nu - a) {
    e -= nu - a;
    ++a;
  }
  b = a + e;
}

// Sum of the Gram partials (fixed order), float-float Cholesky S = R^T R and
// the float-float inverse R^{-1}, redundantly in every CTA. Leaves R^{-1}
// (upper, stride kAs) in (Ihi, Ilo). Returns 0 (ok), 1 (ok, shifted) or -1
// (failure: status set).
__device__ int factor_gram(const float2* gram, int parts, int nu, float* stage, float* Ahi, float* Alo, float* Ihi,
                           float* Ilo, Control* ctrl, bool diag_only) {
  __shared__ int fail;
  __shared__ float maxdiag_s, trace_s;
  __shared__ float Sdiag[NMF_MAX_SKETCH], Sdiag_lo[NMF_MAX_SKETCH];
  const int tid = threadIdx.x;
  const int E = nu * (nu + 1) / 2;
  const int E2 = gram_stride(nu);
  // (1) S = sum of partials, staged through shared memory in chunks of parts
  for (int e = tid; e < nu * kAs; e += blockDim.x) {
    Ahi[e] = 0.f;
    Alo[e] = 0.f;
  }
  __syncthreads();
  const int chunk = max(1, kStageFloat2 / E2);
  float2* st = reinterpret_cast<float2*>(stage);
  for (int p0 = 0; p0 < parts; p0 += chunk) {
    const int np = min(chunk, parts - p0);
    const float4* src = reinterpret_cast<const float4*>(gram + (size_t)p0 * E2);  // even offset: 16-byte aligned
    const int n4 = np * E2 / 2;
    for (int i = tid; i < n4; i += blockDim.x) reinterpret_cast<float4*>(st)[i] = __ldcg(src + i);
    __syncthreads();
    for (int e = tid; e < E; e += blockDim.x) {
      int a, b;
      tri_index(e, nu, a, b);
      FF s{Ahi[a * kAs + b], Alo[a * kAs + b]};
      for (int q = 0; q < np; ++q) {
        const float2 v = st[(size_t)q * E2 + e];
        s = ff_add(s, FF{v.x, v.y});
      }
      Ahi[a * kAs + b] = s.hi;
      Alo[a * kAs + b] = s.lo;
    }
    __syncthreads();
  }
  // S kept in the upper triangle; the diagonal bounds the pivots
  if (tid == 0) {
    float md = 0.f, tr = 0.f;
    bool finite = true;
    for (int j = 0; j < nu; ++j) {
      const float d = Ahi[j * kAs + j];
      finite &= isfinite(d);
      md = fmaxf(md, d);
      tr += d;
    }
    maxdiag_s = finite ? md : -1.f;
    trace_s = tr;
  }
  __syncthreads();
  if (!(maxdiag_s > 0.f)) {
    if (tid == 0) set_status(ctrl, maxdiag_s < 0.f ? NMF_ERR_NONFINITE : NMF_ERR_NOT_SPD);
    return -1;
  }
  if (diag_only) {
    // R^{-1} = diag(1 / sqrt(S_cc)): every column rescaled to unit norm; a
    // zero column stays zero
    for (int e = tid; e < nu * kAs; e += blockDim.x) {
      Ihi[e] = 0.f;
      Ilo[e] = 0.f;
    }
    __syncthreads();
    for (int c = tid; c < nu; c += blockDim.x) {
      const FF d{Ahi[c * kAs + c], Alo[c * kAs + c]};
      if (d.hi > 0.f) {
        const FF r = ff_div(FF{1.f, 0.f}, ff_sqrt(d));
        Ihi[c * kAs + c] = r.hi;
        Ilo[c * kAs + c] = r.lo;
      }
    }
    __syncthreads();
    return 0;
  }
  const float floor = 1e-13f * maxdiag_s;
  // The upper triangle of (Ahi, Alo) is factorised in place; S's off-diagonal
  // entries are kept, both parts, in the lower triangle and its diagonal in
  // Sdiag for a shifted retry. The shift is far below float32 resolution of
  // S, so the retry needs S to float-float accuracy.
  for (int e = tid; e < E; e += blockDim.x) {
    int a, b;
    tri_index(e, nu, a, b);
    if (a == b) {
      Sdiag[a] = Ahi[a * kAs + a];
      Sdiag_lo[a] = Alo[a * kAs + a];
    } else {
      Ahi[b * kAs + a] = Ahi[a * kAs + b];
      Alo[b * kAs + a] = Alo[a * kAs + b];
    }
  }
  __syncthreads();
  int shifted = 0;
  for (int attempt = 0; attempt < 2; ++attempt) {
    if (attempt == 1) {
      // restore S from the lower triangle and shift the diagonal
      const FF sh{1e-10f * trace_s, 0.f};
      for (int e = tid; e < E; e += blockDim.x) {
        int a, b;
        tri_index(e, nu, a, b);
        const FF v = a == b ? ff_add(FF{Sdiag[a], Sdiag_lo[a]}, sh) : FF{Ahi[b * kAs + a], Alo[b * kAs + a]};
        Ahi[a * kAs + b] = v.hi;
        Alo[a * kAs + b] = v.lo;
      }
      shifted = 1;
    }
    if (tid == 0) fail = 0;
    __syncthreads();
    for (int j = 0; j < nu; ++j) {
      if (tid == 0) {
        const FF d{Ahi[j * kAs + j], Alo[j * kAs + j]};
        if (!(d.hi > floor) || !isfinite(d.hi)) {
          fail = 1;
        } else {
          const FF r = ff_sqrt(d);
          Ahi[j * kAs + j] = r.hi;
          Alo[j * kAs + j] = r.lo;
        }
      }
      __syncthreads();
      if (fail) break;
      const FF rjj{Ahi[j * kAs + j], Alo[j * kAs + j]};
      for (int i = j + 1 + tid; i < nu; i += blockDim.x) {
        const FF v = ff_div(FF{Ahi[j * kAs + i], Alo[j * kAs + i]}, rjj);
        Ahi[j * kAs + i] = v.hi;
        Alo[j * kAs + i] = v.lo;
      }
      __syncthreads();
      const int w = nu - j - 1;
      for (int t = tid; t < w * w; t += blockDim.x) {
        const int i = j + 1 + t / w, k = j + 1 + t % w;
        if (k >= i) {
          const FF prod = ff_mul(FF{Ahi[j * kAs + i], Alo[j * kAs + i]}, FF{Ahi[j * kAs + k], Alo[j * kAs + k]});
          const FF v = ff_add(FF{Ahi[i * kAs + k], Alo[i * kAs + k]}, ff_neg(prod));
          Ahi[i * kAs + k] = v.hi;
          Alo[i * kAs + k] = v.lo;
        }
      }
      __syncthreads();
    }
    if (!fail) break;
    __syncthreads();
  }
  if (fail) {
    if (tid == 0) set_status(ctrl, NMF_ERR_NOT_SPD);
    return -1;
  }
  // R^{-1} column by column (thread c owns column c): back substitution
  // x_c = 1 / R_cc, x_i = -(sum_{k=i+1..c} R_ik x_k) / R_ii, in float-float.
  for (int c = tid; c < nu; c += blockDim.x) {
    for (int i = c + 1; i < nu; ++i) {
      Ihi[i * kAs + c] = 0.f;
      Ilo[i * kAs + c] = 0.f;
    }
    const FF xc = ff_div(FF{1.f, 0.f}, FF{Ahi[c * kAs + c], Alo[c * kAs + c]});
    Ihi[c * kAs + c] = xc.hi;
    Ilo[c * kAs + c] = xc.lo;
    for (int i = c - 1; i >= 0; --i) {
      FF s{0.f, 0.f};
      for (int k = i + 1; k <= c; ++k)
        s = ff_add(s, ff_mul(FF{Ahi[i * kAs + k], Alo[i * kAs + k]}, FF{Ihi[k * kAs + c], Ilo[k * kAs + c]}));
      const FF x = ff_neg(ff_div(s, FF{Ahi[i * kAs + i], Alo[i * kAs + i]}));
      Ihi[i * kAs + c] = x.hi;
      Ilo[i * kAs + c] = x.lo;
    }
  }
  __syncthreads();
  return shifted;
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

  extern __shared__ __align__(16) float smem[];
  float* Ys = smem;                                 // kOrthRows x kYsStride (also Gram staging)
  float* Ahi = Ys + kOrthRows * kYsStride;          // nu x kAs
  float* Alo = Ahi + NMF_MAX_SKETCH * kAs;
  float* Ihi = Alo + NMF_MAX_SKETCH * kAs;          // R^{-1}, float-float
  float* Ilo = Ihi + NMF_MAX_SKETCH * kAs;
  __shared__ int shifted_s;

  bool extra_gram = false;
  if (J.part) {
    // Y = sum over the S partials, 4 independent accumulators, fixed order.
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
    const int sh = factor_gram(J.gram_in, J.gram_parts, nu, Ys, Ahi, Alo, Ihi, Ilo, ctrl, J.diag_only != 0);
    if (sh < 0) return;
    if (tid == 0) shifted_s = sh;
    __syncthreads();
    if (J.shift_flag) {
      // pass 1 records its shift; later passes add theirs; a shift anywhere
      // schedules the conditional third pass (every CTA computes the same)
      const int before = *((volatile const int*)J.shift_flag);
      extra_gram = J.gram_on_shift && (before || shifted_s);
      __syncthreads();
      if (cta == 0 && tid == 0 && shifted_s && !before) *J.shift_flag = 1;
    }
    for (int i = tid; i < rows * nu; i += kRowThreads) {
      const int r = i / nu, c = i % nu;
      Ys[r * kYsStride + c] = J.src[(size_t)(r0 + r) * nu + c];
    }
    __syncthreads();
    // q = y R^{-1}: q_c = sum_{k<=c} y_k (R^{-1})_kc with exact float32 x
    // float-float products and float-float sums, one rounding at the end;
    // columns from the last to the first, so the row is overwritten in place.
    if (tid < rows) {
      float* y = Ys + tid * kYsStride;
      for (int c = nu - 1; c >= 0; --c) {
        FF acc{0.f, 0.f};
        for (int k = 0; k <= c; ++k) {
          const float yk = y[k];
          const float ph = yk * Ihi[k * kAs + c];
          const float pe = fmaf(yk, Ilo[k * kAs + c], fmaf(yk, Ihi[k * kAs + c], -ph));
          acc = ff_add(acc, ff_quick(ph, pe));
        }
        y[c] = acc.hi + acc.lo;
      }
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
  if (J.gram_part && (J.gram_always || extra_gram)) {
    const int E = nu * (nu + 1) / 2;
    const int E2 = gram_stride(nu);
    for (int e = tid; e < E2; e += kRowThreads) {
      if (e >= E) {
        J.gram_part[(size_t)cta * E2 + e] = make_float2(0.f, 0.f);
        continue;
      }
      int a, b;
      tri_index(e, nu, a, b);
      DF s{0.f, 0.f};
      for (int r = 0; r < rows; ++r) df_add_product(s, Ys[r * kYsStride + a], Ys[r * kYsStride + b]);
      df_norm(s);
      J.gram_part[(size_t)cta * E2 + e] = make_float2(s.hi, s.lo);
    }
  }
}

size_t rows_smem() {
  return (size_t)(kOrthRows * kYsStride + 4 * NMF_MAX_SKETCH * kAs) * sizeof(float);
}

}  // namespace

cudaError_t rows_launch(const RowJob* jobs, int njobs, Control* ctrl, cudaStream_t s) {
  RowJobs rj{};
  rj.njobs = njobs;
  int total = 0;
  for (int i = 0; i < njobs; ++i) {
    rj.j[i] = jobs[i];
    rj.start[i] = total;
    total += rows_ctas(jobs[i].N);
  }
  rj.start[njobs] = total;
  const size_t smem = rows_smem();
  cudaError_t e = allow_dynamic_smem((const void*)rows_kernel, (int)smem);
  if (e != cudaSuccess) return e;
  count_launches(1);
  rows_kernel<<<total, kRowThreads, smem, s>>>(rj, ctrl);
  return cudaGetLastError();
}

}  // namespace nmf
