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
// (upper, stride kAs) in (Ihi, Ilo). Returns 0 (ok), 1 (ok, shifted), 2 (S
// within skip_tol of I: R = I, nothing left in Ihi, Ilo), 3 (ok, not
// shifted, largest / smallest pivot below single_ratio) or -1 (failure:
// status set).
__device__ int factor_gram(const float2* gram, int parts, int nu, float* stage, float* Ahi, float* Alo, float* Ihi,
                           float* Ilo, Control* ctrl, bool diag_only, float skip_tol, float single_ratio) {
  __shared__ float maxdiag_s, trace_s;
  __shared__ float Sdiag[NMF_MAX_SKETCH], Sdiag_lo[NMF_MAX_SKETCH];
  __shared__ float Dinv_hi[NMF_MAX_SKETCH], Dinv_lo[NMF_MAX_SKETCH];
  __shared__ float Rs_hi[NMF_MAX_SKETCH], Rs_lo[NMF_MAX_SKETCH];
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
    // eight loads in flight per thread before any store
    for (int i0 = tid; i0 < n4; i0 += 8 * (int)blockDim.x) {
      float4 v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int i = i0 + u * (int)blockDim.x;
        if (i < n4) v[u] = __ldcg(src + i);
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int i = i0 + u * (int)blockDim.x;
        if (i < n4) reinterpret_cast<float4*>(st)[i] = v[u];
      }
    }
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
  // A basis already orthonormal to skip_tol (every entry of S - I within it,
  // the float-float value): nothing to factorise, the caller keeps its rows.
  // Every CTA sums the same partials in the same order, so all decide alike.
  if (skip_tol > 0.f) {
    __shared__ int off_s;
    if (tid == 0) off_s = 0;
    __syncthreads();
    for (int e = tid; e < E; e += blockDim.x) {
      int a, b;
      tri_index(e, nu, a, b);
      const float v = (Ahi[a * kAs + b] - (a == b ? 1.f : 0.f)) + Alo[a * kAs + b];
      if (!(fabsf(v) <= skip_tol)) off_s = 1;
    }
    __syncthreads();
    if (!off_s) return 2;
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
  bool fail = false;
  // this thread's first entry of the upper triangle (the common case nu <= 22
  // has at most one per thread)
  int pa = 0, pb = 0;
  if (tid < E) tri_index(tid, nu, pa, pb);
  for (int attempt = 0; attempt < 2; ++attempt) {
    if (attempt == 1) {
      // restore S from the lower triangle and shift the diagonal
      __syncthreads();
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
    __syncthreads();
    // S = U^T D U (LDL^T, right-looking): step j takes the pivot d_j and
    // subtracts (S_ji / d_j) S_jk from every trailing entry j < i <= k. All
    // threads read the same pivot and take the same decision, so a step needs
    // one barrier. Row j is read, never written, during step j.
    fail = false;
    for (int j = 0; j < nu; ++j) {
      const FF d{Ahi[j * kAs + j], Alo[j * kAs + j]};
      if (!(d.hi > floor) || !isfinite(d.hi)) {
        fail = true;
        break;
      }
      const FF inv = ff_div(FF{1.f, 0.f}, d);
      if (tid == 0) {
        Dinv_hi[j] = inv.hi;
        Dinv_lo[j] = inv.lo;
      }
      for (int e = tid; e < E; e += blockDim.x) {
        int i = pa, k = pb;
        if (e != tid) tri_index(e, nu, i, k);
        if (i <= j) continue;
        const FF l = ff_mul(FF{Ahi[j * kAs + i], Alo[j * kAs + i]}, inv);
        const FF v = ff_add(FF{Ahi[i * kAs + k], Alo[i * kAs + k]},
                            ff_neg(ff_mul(l, FF{Ahi[j * kAs + k], Alo[j * kAs + k]})));
        Ahi[i * kAs + k] = v.hi;
        Alo[i * kAs + k] = v.lo;
      }
      __syncthreads();
    }
    if (!fail) break;
  }
  if (fail) {
    if (tid == 0) set_status(ctrl, NMF_ERR_NOT_SPD);
    return -1;
  }
  // One pass suffices when S is well conditioned: the pivots of S = U^T D U
  // bound kappa(Y)^2 from below by max d / min d, and a float-float Gram and
  // factor leave Q orthonormal to about kappa(Y)^2 2^-48 beside the float32
  // rounding of its entries. Every thread reads the same pivots.
  bool single = false;
  if (!shifted && single_ratio > 0.f) {
    float dmax = 0.f, dmin = 3.4e38f;
    for (int j = 0; j < nu; ++j) {
      const float d = Ahi[j * kAs + j];
      dmax = fmaxf(dmax, d);
      dmin = fminf(dmin, d);
    }
    single = dmax < single_ratio * dmin;
  }
  // R = D^{1/2} U, so R^{-1} = U^{-1} D^{-1/2}. U_jk = S'_jk / d_j (strict
  // upper part), and X = U^{-1} starts as the identity.
  for (int e = tid; e < E; e += blockDim.x) {
    int i = pa, k = pb;
    if (e != tid) tri_index(e, nu, i, k);
    if (i < k) {
      const FF u = ff_mul(FF{Ahi[i * kAs + k], Alo[i * kAs + k]}, FF{Dinv_hi[i], Dinv_lo[i]});
      Ahi[i * kAs + k] = u.hi;
      Alo[i * kAs + k] = u.lo;
    }
  }
  for (int c = tid; c < nu; c += blockDim.x) {
    const FF r = ff_div(FF{1.f, 0.f}, ff_sqrt(FF{Ahi[c * kAs + c], Alo[c * kAs + c]}));
    Rs_hi[c] = r.hi;
    Rs_lo[c] = r.lo;
  }
  for (int e = tid; e < nu * kAs; e += blockDim.x) {
    Ihi[e] = (e / kAs == e % kAs) ? 1.f : 0.f;
    Ilo[e] = 0.f;
  }
  __syncthreads();
  // U X = I with a unit diagonal, column-oriented: once row k of X is final
  // (k from the last row to the second), X_ic -= U_ik X_kc for every i < k <= c.
  for (int k = nu - 1; k >= 1; --k) {
    const int w = nu - k;
    for (int t = tid; t < k * w; t += blockDim.x) {
      const int i = t / w, c = k + t % w;
      const FF v = ff_add(FF{Ihi[i * kAs + c], Ilo[i * kAs + c]},
                          ff_neg(ff_mul(FF{Ahi[i * kAs + k], Alo[i * kAs + k]}, FF{Ihi[k * kAs + c], Ilo[k * kAs + c]})));
      Ihi[i * kAs + c] = v.hi;
      Ilo[i * kAs + c] = v.lo;
    }
    __syncthreads();
  }
  // column c of R^{-1} = column c of U^{-1} times d_c^{-1/2}
  for (int e = tid; e < E; e += blockDim.x) {
    int i = pa, c = pb;
    if (e != tid) tri_index(e, nu, i, c);
    const FF v = ff_mul(FF{Ihi[i * kAs + c], Ilo[i * kAs + c]}, FF{Rs_hi[c], Rs_lo[c]});
    Ihi[i * kAs + c] = v.hi;
    Ilo[i * kAs + c] = v.lo;
  }
  __syncthreads();
  return single ? 3 : shifted;
}

__global__ void __launch_bounds__(kRowThreads) rows_kernel(RowJobs jobs, Control* ctrl) {
  // launched as a programmatic dependent: wait for the predecessor's writes
  // (its X pass partials, Gram partials, flags) before reading anything
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;");
  int jj = 0;
  while (jj + 1 < jobs.njobs && (int)blockIdx.x >= jobs.start[jj + 1]) ++jj;
  const RowJob& J = jobs.j[jj];
  {
    // the call's status and this job's flags, loaded together (one round trip)
    const int failed = *((volatile const int*)&ctrl->status);
    const int run = J.run_flag ? *((volatile const int*)J.run_flag) : 1;
    const int skip = J.skip_flag ? *((volatile const int*)J.skip_flag) : 0;
    if (failed != 0 || run == 0 || skip != 0) return;
  }
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
  bool single = false;  // one pass was enough: the rows go to the final outputs
  if (J.part) {
    // Y = sum over the S partials: four accumulators (partial k feeds
    // accumulator k mod 4, in increasing k), float4 over four columns. A
    // thread takes two (row, column block) items at a time with up to 8
    // partials of each in flight (16 loads). Rows of a partial are ldp floats,
    // ldp a multiple of 16, so the float4 loads are aligned.
    const int nu4 = (nu + 3) >> 2;
    const size_t stride4 = (size_t)J.N * J.ldp / 4;
    const int S4 = J.S & ~3;
    const int items = rows * nu4;
    for (int i0 = tid; i0 < items; i0 += 2 * kRowThreads) {
      const int ib = i0 + kRowThreads;
      const bool two = ib < items;
      const int ia_r = i0 / nu4, ia_c = i0 % nu4;
      const int ib_r = two ? ib / nu4 : ia_r, ib_c = two ? ib % nu4 : ia_c;
      const float4* pa = reinterpret_cast<const float4*>(J.part + (size_t)(r0 + ia_r) * J.ldp) + ia_c;
      const float4* pb = reinterpret_cast<const float4*>(J.part + (size_t)(r0 + ib_r) * J.ldp) + ib_c;
      float4 acc[2][4];
#pragma unroll
      for (int u = 0; u < 4; ++u) acc[0][u] = acc[1][u] = make_float4(0.f, 0.f, 0.f, 0.f);
      for (int k0 = 0; k0 < S4; k0 += 8) {
        float4 va[8], vb[8];
#pragma unroll
        for (int u = 0; u < 8; ++u)
          if (k0 + u < S4) {
            va[u] = __ldcg(pa + (k0 + u) * stride4);
            if (two) vb[u] = __ldcg(pb + (k0 + u) * stride4);
          }
#pragma unroll
        for (int u = 0; u < 8; ++u)
          if (k0 + u < S4) {
            acc[0][u & 3].x += va[u].x;
            acc[0][u & 3].y += va[u].y;
            acc[0][u & 3].z += va[u].z;
            acc[0][u & 3].w += va[u].w;
            if (two) {
              acc[1][u & 3].x += vb[u].x;
              acc[1][u & 3].y += vb[u].y;
              acc[1][u & 3].z += vb[u].z;
              acc[1][u & 3].w += vb[u].w;
            }
          }
      }
      for (int k = S4; k < J.S; ++k) {
        const float4 v = __ldcg(pa + k * stride4);
        acc[0][0].x += v.x;
        acc[0][0].y += v.y;
        acc[0][0].z += v.z;
        acc[0][0].w += v.w;
        if (two) {
          const float4 w = __ldcg(pb + k * stride4);
          acc[1][0].x += w.x;
          acc[1][0].y += w.y;
          acc[1][0].z += w.z;
          acc[1][0].w += w.w;
        }
      }
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        if (h == 1 && !two) break;
        const int r = h ? ib_r : ia_r, c4 = h ? ib_c : ia_c;
        const float4* A = acc[h];
        const float o[4] = {(A[0].x + A[1].x) + (A[2].x + A[3].x), (A[0].y + A[1].y) + (A[2].y + A[3].y),
                            (A[0].z + A[1].z) + (A[2].z + A[3].z), (A[0].w + A[1].w) + (A[2].w + A[3].w)};
#pragma unroll
        for (int t = 0; t < 4; ++t)
          if (4 * c4 + t < nu) Ys[r * kYsStride + 4 * c4 + t] = o[t];
      }
    }
  } else {
    // the skip is only taken while no factorisation of this basis has shifted
    const int shifted_before = J.shift_flag ? *((volatile const int*)J.shift_flag) : 0;
    const int sh = J.gram_only ? 2
                               : factor_gram(J.gram_in, J.gram_parts, nu, Ys, Ahi, Alo, Ihi, Ilo, ctrl,
                                             J.diag_only != 0, shifted_before ? 0.f : J.skip_tol,
                                             shifted_before ? 0.f : J.single_ratio);
    if (sh < 0) return;
    const bool keep_rows = sh == 2;
    single = sh == 3;
    if (single && cta == 0 && tid == 0) *J.single_flag = 1;  // every CTA decided alike
    if (tid == 0) shifted_s = (keep_rows || single) ? 0 : sh;
    __syncthreads();
    if (J.shift_flag) {
      // pass 1 records its shift; later passes add theirs; a shift anywhere
      // schedules the conditional third pass (every CTA computes the same)
      const int before = *((volatile const int*)J.shift_flag);
      extra_gram = J.gram_on_shift && (before || shifted_s);
      __syncthreads();
      if (cta == 0 && tid == 0 && shifted_s && !before) *J.shift_flag = 1;
    }
    // this CTA's rows of src: one contiguous block of rows * nu floats, read
    // as float4 with up to 8 loads in flight per thread when the block is
    // 16-byte aligned (it starts kOrthRows * nu floats after its
    // predecessor; src itself may be a caller's buffer), else as floats
    {
      const float* blk = J.src + (size_t)r0 * nu;
      const int total = rows * nu;
      const int n4 = (reinterpret_cast<uintptr_t>(blk) & 15u) == 0 ? total >> 2 : 0;
      const float4* b4 = reinterpret_cast<const float4*>(blk);
      for (int i0 = tid; i0 < n4; i0 += 8 * kRowThreads) {
        float4 v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u)
          if (i0 + u * kRowThreads < n4) v[u] = __ldcg(b4 + i0 + u * kRowThreads);
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int i = 4 * (i0 + u * kRowThreads);
          if (i0 + u * kRowThreads < n4) {
            const float e[4] = {v[u].x, v[u].y, v[u].z, v[u].w};
#pragma unroll
            for (int t = 0; t < 4; ++t) Ys[((i + t) / nu) * kYsStride + (i + t) % nu] = e[t];
          }
        }
      }
      for (int i = 4 * n4 + tid; i < total; i += kRowThreads) Ys[(i / nu) * kYsStride + i % nu] = blk[i];
    }
    __syncthreads();
    // q = y R^{-1}: q_c = sum_{k<=c} y_k (R^{-1})_kc, a compensated dot
    // product (Dot2 of Ogita, Rump and Oishi, 2005, with the float-float
    // R^{-1}): each product's exact error, the running sum's exact rounding
    // error (TwoSum) and the low part of R^{-1} are gathered in a float
    // correction added once at the end, so q_c is as accurate as if summed in
    // twice the precision, then rounded. Columns from the last to the first,
    // so the row is overwritten in place.
    if (tid < rows && !keep_rows) {
      float* y = Ys + tid * kYsStride;
      for (int c = nu - 1; c >= 0; --c) {
        float sum = 0.f, corr = 0.f;
        for (int k = 0; k <= c; ++k) {
          const float yk = y[k];
          const float ih = Ihi[k * kAs + c];
          const float ph = yk * ih;
          const float pe = fmaf(yk, Ilo[k * kAs + c], fmaf(yk, ih, -ph));
          const float t = sum + ph;
          const float bp = t - sum;
          corr += ((sum - (t - bp)) + (ph - bp)) + pe;
          sum = t;
        }
        y[c] = sum + corr;
      }
    }
  }
  __syncthreads();

  bool bad = false;
  float* const outY = single ? J.Y_final : J.Y;
  float* const outYt = single ? J.Yt_final : J.Yt;
  void* const outOp = single ? J.op_final : J.op;
  if (outY)
    for (int i = tid; i < rows * nu; i += kRowThreads) {
      const int r = i / nu, c = i % nu;
      const float v = Ys[r * kYsStride + c];
      bad |= !isfinite(v);
      outY[(size_t)(r0 + r) * nu + c] = v;
    }
  if (outYt)
    for (int i = tid; i < rows * nu; i += kRowThreads) {
      const int c = i / rows, r = i % rows;
      outYt[(size_t)c * J.N + r0 + r] = Ys[r * kYsStride + c];
    }
  if (outOp)
    for (int i = tid; i < rows * nu; i += kRowThreads) {
      const int c = i / rows, r = i % rows;
      store_op(outOp, (size_t)c * J.ldop + r0 + r, J.op_fmt, J.op_part, Ys[r * kYsStride + c]);
    }
  if (bad) set_status(ctrl, NMF_ERR_NONFINITE);
  if (J.gram_part && !single && (J.gram_always || extra_gram)) {
    const int E = nu * (nu + 1) / 2;
    const int E2 = gram_stride(nu);
    for (int e = tid; e < E2; e += kRowThreads) {
      if (e >= E) {
        J.gram_part[(size_t)cta * E2 + e] = make_float2(0.f, 0.f);
        continue;
      }
      int a, b;
      tri_index(e, nu, a, b);
      // four accumulators over interleaved rows (shorter dependent chains)
      DF s0{0.f, 0.f}, s1{0.f, 0.f}, s2{0.f, 0.f}, s3{0.f, 0.f};
      int r = 0;
      for (; r + 4 <= rows; r += 4) {
        df_add_product(s0, Ys[(r + 0) * kYsStride + a], Ys[(r + 0) * kYsStride + b]);
        df_add_product(s1, Ys[(r + 1) * kYsStride + a], Ys[(r + 1) * kYsStride + b]);
        df_add_product(s2, Ys[(r + 2) * kYsStride + a], Ys[(r + 2) * kYsStride + b]);
        df_add_product(s3, Ys[(r + 3) * kYsStride + a], Ys[(r + 3) * kYsStride + b]);
      }
      for (; r < rows; ++r) df_add_product(s0, Ys[r * kYsStride + a], Ys[r * kYsStride + b]);
      df_add(s0, s1.hi, s1.lo);
      df_add(s2, s3.hi, s3.lo);
      df_add(s0, s2.hi, s2.lo);
      df_norm(s0);
      J.gram_part[(size_t)cta * E2 + e] = make_float2(s0.hi, s0.lo);
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
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(total);
  cfg.blockDim = dim3(kRowThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = pdl_allowed() ? 1 : 0;
  count_launches(1);
  return cudaLaunchKernelEx(&cfg, rows_kernel, rj, ctrl);
}

}  // namespace nmf
