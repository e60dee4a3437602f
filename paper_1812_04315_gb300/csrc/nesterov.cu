// nesterov.cu -- the inner loop of NeNMF (Sec. 2) on the columns of a p x N
// unknown Y, one column per thread, fused with what the loop needs:
//
// prologue  H, W and L_c of the subproblem, reduced by the previous kernel's
//           tail (below); B of every column:
//             compressed (Alg. 1): B(:, j) = W d_j, d_j the j-th compressed
//               data vector (G side: W = F_R = F R, d_j = row j of X_R;
//               F side: W = G_L^T = (L G)^T, d_j = column j of X_L);
//             plain (eq. 2-3): B summed from the X pass partials;
// loop      f = max(0, y - grad(y) / L_c); y' = f + beta_k (f - f_prev).
//           Only the gradient at f is formed (H f - b); the gradient at the
//           extrapolated y' follows by linearity,
//           grad(y') = grad(f) + beta_k (grad(f) - grad(f_prev)).
//           Optional stop test ||P grad(f_k)||_F <= eps: per-CTA float64
//           partials, summed in a fixed order after all CTAs have published;
//           the result of the test at iteration k is read at iteration
//           k + kLag, so the cross-CTA wait overlaps compute, and the iterate
//           f_k is kept until then (cooperative launch, bounded waits);
// epilogue  the returned iterate is stored (and copied for the next X pass,
//           the snapshot, the stats); the next phase's W (f times rows of R or
//           columns of L) or Gram matrix f f^T is summed per CTA, then over
//           groups of kTailGroup CTAs by the last CTA of each group, then over
//           groups by the last group; that CTA forms H = W W^T and
//           L_c = lambda_max(H) (one warp: repeated squaring of H / trace with
//           the trace normalisation, stopping once the spectrum has collapsed
//           to rank one, then a float64 Rayleigh quotient).
#include "internal.h"

namespace nmf {
namespace {

constexpr int T = kSolveThreads;
constexpr int kLag = 2;
constexpr int kKeep = kLag + 1;
constexpr int kMaxSquarings = 16;
constexpr int kFs = T + 1;
constexpr unsigned long long kWaitNs = 2000000000ull;

struct KParams {
  SolveArgs a;
  const float* beta;  // [max_inner] extrapolation weights
  int mode;
};

__device__ __forceinline__ double block_sum_double(double v, double* red) {
  v = warp_sum(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < T / 32; ++i) s += red[i];
  return s;  // valid in thread 0
}

// g = H y - b with H (PM x PM, zero padded) in shared memory, rows read as float4.
template <int PM>
__device__ __forceinline__ void hmatvec(const float* Hs, const float* y, const float* b, float* g) {
#pragma unroll
  for (int c = 0; c < PM; ++c) {
    float s = -b[c];
    const float4* h = reinterpret_cast<const float4*>(Hs + c * PM);
#pragma unroll
    for (int d = 0; d < PM / 4; ++d) {
      const float4 v = h[d];
      s = fmaf(v.x, y[4 * d + 0], s);
      s = fmaf(v.y, y[4 * d + 1], s);
      s = fmaf(v.z, y[4 * d + 2], s);
      s = fmaf(v.w, y[4 * d + 3], s);
    }
    g[c] = s;
  }
}

template <int PM>
__device__ __forceinline__ float pg_sq(const float* f, const float* g) {
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < PM; ++c) {
    const float v = f[c] > 0.f ? g[c] : fminf(g[c], 0.f);
    s = fmaf(v, v, s);
  }
  return s;
}

// Waits (thread 0) until the stop-test arrival counter reaches `target`.
__device__ __forceinline__ bool wait_arrivals(Control* c, unsigned int target) {
  __shared__ int ok;
  if (threadIdx.x == 0) {
    cuda::atomic_ref<unsigned int, cuda::thread_scope_device> cnt(c->bar_count);
    cuda::atomic_ref<int, cuda::thread_scope_device> abrt(c->abort);
    int good = 1;
    const unsigned long long t0 = global_ns();
    while (cnt.load(cuda::memory_order_acquire) < target) {
      if (abrt.load(cuda::memory_order_relaxed)) { good = 0; break; }
      if (global_ns() - t0 > kWaitNs) {
        set_status(c, NMF_ERR_DEVICE_TIMEOUT);
        abrt.store(1, cuda::memory_order_relaxed);
        good = 0;
        break;
      }
      __nanosleep(20);
    }
    ok = good;
  }
  __syncthreads();
  return ok != 0;
}

// lambda_max of the symmetric PSD p x p matrix H (row stride p) in shared
// memory, by the whole CTA: repeated squaring of M = H / trace(H) with the
// trace renormalised each time, until trace(M^2) = 1 (rank one), then the
// float64 Rayleigh quotient of M's dominant column. M0, M1: PM x PM scratch.
// Returns 0 for H = 0 and a non-finite value for a non-finite H.
template <int PM>
__device__ double lambda_max_block(const float* H, int p, float* M0, float* M1, double* red) {
  __shared__ float tr_s;
  __shared__ double lam_s;
  const int tid = threadIdx.x;
  if (tid < 32) {
    double tr = 0.0;
    for (int c = tid; c < p; c += 32) tr += (double)H[c * p + c];
    tr = warp_sum(tr);
    if (tid == 0) red[0] = tr;
  }
  __syncthreads();
  const double tr = red[0];
  __syncthreads();
  if (!(tr > 0.0) || !isfinite(tr)) return isfinite(tr) ? 0.0 : tr;
  const float inv = (float)(1.0 / tr);
  for (int i = tid; i < PM * PM; i += T) {
    const int c = i / PM, d = i % PM;
    M0[i] = (c < p && d < p) ? H[c * p + d] * inv : 0.f;
  }
  __syncthreads();
  float* M = M0;
  float* M2 = M1;
  for (int s = 0; s < kMaxSquarings; ++s) {
    for (int i = tid; i < PM * PM; i += T) {
      const int c = i / PM, d = i % PM;
      float v = 0.f;
#pragma unroll
      for (int k = 0; k < PM; ++k) v = fmaf(M[c * PM + k], M[k * PM + d], v);
      M2[i] = v;
    }
    __syncthreads();
    if (tid < 32) {
      const float t = warp_sum(tid < PM ? M2[tid * PM + tid] : 0.f);
      if (tid == 0) tr_s = t;
    }
    __syncthreads();
    const float t2 = tr_s;
    if (t2 > 0.f) {
      const float it = 1.f / t2;
      for (int i = tid; i < PM * PM; i += T) M2[i] *= it;
    }
    __syncthreads();
    float* tmp = M;
    M = M2;
    M2 = tmp;
    // trace(M^2) of a trace-one M equals 1 exactly when M has rank one; at
    // 1 - trace(M^2) < 1e-5 the other eigenvectors' share in the chosen
    // column is < 1e-5, so the Rayleigh quotient is exact to ~1e-10.
    if (!(t2 > 0.f) || 1.f - t2 < 1e-5f) break;
  }
  if (tid < 32) {
    int jb = 0;
    for (int c = 1; c < PM; ++c)
      if (M[c * PM + c] > M[jb * PM + jb]) jb = c;
    double hv = 0.0, vc = 0.0;
    if (tid < p) {
      vc = (double)M[tid * PM + jb];
      for (int d = 0; d < p; ++d) hv = fma((double)H[tid * p + d], (double)M[d * PM + jb], hv);
    }
    const double num = warp_sum(vc * hv), den = warp_sum(vc * vc);
    if (tid == 0) lam_s = den > 0.0 ? num / den : 0.0;
  }
  __syncthreads();
  return lam_s;
}

// Fixed-order total of the stop-test partials of test j (warp 0 sums; all read flag).
__device__ __forceinline__ void test_total(const double* pg2_part, int j, int ctas, double eps2, double* tot,
                                           int* flag) {
  if (threadIdx.x < 32) {
    double t = 0.0;
    const double* sl = pg2_part + (size_t)(j % kStopSlots) * ctas;
    for (int i = threadIdx.x; i < ctas; i += 32) t += __ldcg(sl + i);
    t = warp_sum(t);
    if (threadIdx.x == 0) {
      *tot = t;
      *flag = t <= eps2;
    }
  }
  __syncthreads();
}

template <int PM>
__global__ void __launch_bounds__(T) solve_kernel(KParams kp) {
  const SolveArgs& a = kp.a;
  Control* ctrl = a.ctrl;
  if (call_failed(ctrl)) return;
  const int p = a.p, nu = a.nu, N = a.N;
  const int tid = threadIdx.x;
  const int cta = blockIdx.x;
  const int ctas = gridDim.x;
  const int col = cta * T + tid;
  const bool active = col < N;

  __shared__ __align__(16) float Hs[PM * PM];
  __shared__ float Ws[PM * NMF_MAX_SKETCH];
  __shared__ double red[T / 32];
  __shared__ int flag_s;
  __shared__ double tot_s;
  extern __shared__ __align__(16) float dyn[];

  float y[PM], b[PM], f[PM];
#pragma unroll
  for (int c = 0; c < PM; ++c) {
    y[c] = (active && c < p) ? a.Y[(size_t)c * N + col] : 0.f;
    b[c] = 0.f;
  }

  int iters = 0;
  float Lc = 0.f;
  double Lc_d = 0.0;
  if (kp.mode != MODE_EPI_ONLY) {
    const Reduced* R = a.red_in;
    for (int i = tid; i < PM * PM; i += T) {
      const int c = i / PM, d = i % PM;
      Hs[i] = (c < p && d < p) ? R->H[c * p + d] : 0.f;
    }
    if (a.bsrc != B_FROM_PARTIALS)
      for (int i = tid; i < PM * nu; i += T) {
        const int c = i / nu, k = i % nu;
        Ws[c * NMF_MAX_SKETCH + k] = c < p ? R->W[c * nu + k] : 0.f;
      }
    Lc = R->Lc;
    Lc_d = R->Lc_d;
    __syncthreads();
    if (active) {
      if (a.bsrc == B_FROM_PARTIALS) {
        // B(:, col) = sum over the X pass partials; a whole row of partials
        // per q, so the loads of all c are in flight together.
        for (int q = 0; q < a.Bparts; ++q) {
          const float* bp = a.Bpart + ((size_t)q * N + col) * a.Bld;
#pragma unroll
          for (int c = 0; c < PM; ++c)
            if (c < p) b[c] += __ldcg(bp + c);
        }
      }
    }
    if (a.bsrc != B_FROM_PARTIALS) {
      // The CTA's T data vectors go through shared memory: Ds[k][t] for k < nu.
      // Rows of X_R (N x nu) are contiguous for the whole CTA; columns of X_L
      // (nu x N) are coalesced per k. Loads are independent, so they overlap.
      float* Ds = dyn;
      const int c0 = cta * T;
      const int cols = min(T, N - c0);
      if (a.bsrc == B_FROM_ROWS) {
        const float* src = a.D + (size_t)c0 * nu;
        for (int i = tid; i < cols * nu; i += T) {
          const int t = i / nu, k = i % nu;
          Ds[k * kFs + t] = __ldg(src + i);
        }
      } else {
        for (int i = tid; i < nu * T; i += T) {
          const int k = i / T, t = i % T;
          Ds[k * kFs + t] = t < cols ? __ldg(a.D + (size_t)k * N + c0 + t) : 0.f;
        }
      }
      __syncthreads();
      if (active)
        for (int k = 0; k < nu; ++k) {
          const float dk = Ds[k * kFs + tid];
#pragma unroll
          for (int c = 0; c < PM; ++c) b[c] = fmaf(Ws[c * NMF_MAX_SKETCH + k], dk, b[c]);
        }
      __syncthreads();  // dyn is reused below
    }
  }

#pragma unroll
  for (int c = 0; c < PM; ++c) f[c] = y[c];
  double pg2_final = 0.0;

  if (kp.mode == MODE_EVAL) {
    float g[PM];
    hmatvec<PM>(Hs, f, b, g);
    const double s = block_sum_double(active ? (double)pg_sq<PM>(f, g) : 0.0, red);
    if (tid == 0) a.pg2_init[cta] = s;
  } else if (kp.mode == MODE_SOLVE && Lc > 0.f) {
    float g[PM], fp[PM], gp[PM];
    hmatvec<PM>(Hs, y, b, g);
#pragma unroll
    for (int c = 0; c < PM; ++c) {
      fp[c] = y[c];
      gp[c] = g[c];
    }
    float* keep = dyn;  // [kKeep][PM][T]: iterates whose stop test is pending
    const float inv_Lc = 1.f / Lc;
    const bool test = a.stop_test;
    const double eps2 = ctrl->eps2;
    int tests = 0, stop_j = -1;
    for (int k = 0; k < a.max_inner; ++k) {
#pragma unroll
      for (int c = 0; c < PM; ++c) f[c] = fmaxf(0.f, fmaf(-g[c], inv_Lc, y[c]));
      float gf[PM];
      hmatvec<PM>(Hs, f, b, gf);
      const float beta = __ldg(kp.beta + k);
#pragma unroll
      for (int c = 0; c < PM; ++c) {
        y[c] = fmaf(beta, f[c] - fp[c], f[c]);
        g[c] = fmaf(beta, gf[c] - gp[c], gf[c]);
        fp[c] = f[c];
        gp[c] = gf[c];
      }
      iters = k + 1;
      if (test && k + 1 >= a.min_inner) {
        const double s = block_sum_double(active ? (double)pg_sq<PM>(f, gf) : 0.0, red);
        if (tid == 0) {
          a.pg2_part[(size_t)(tests % kStopSlots) * ctas + cta] = s;
          __threadfence();
          atomicAdd(&ctrl->bar_count, 1u);
        }
        float* slot = keep + (size_t)(tests % kKeep) * PM * T;
#pragma unroll
        for (int c = 0; c < PM; ++c) slot[c * T + tid] = f[c];
        ++tests;
        if (tests > kLag) {
          const int j = tests - 1 - kLag;
          if (!wait_arrivals(ctrl, (unsigned int)(j + 1) * ctas)) return;
          test_total(a.pg2_part, j, ctas, eps2, &tot_s, &flag_s);
          if (flag_s) {
            stop_j = j;
            break;
          }
        }
      }
    }
    if (test && stop_j < 0) {
      // tests still pending when the loop ended, in order
      for (int j = tests > kLag ? tests - kLag : 0; j < tests; ++j) {
        if (!wait_arrivals(ctrl, (unsigned int)(j + 1) * ctas)) return;
        test_total(a.pg2_part, j, ctas, eps2, &tot_s, &flag_s);
        if (flag_s) {
          stop_j = j;
          break;
        }
      }
    }
    if (stop_j >= 0) {
      const float* slot = keep + (size_t)(stop_j % kKeep) * PM * T;
#pragma unroll
      for (int c = 0; c < PM; ++c) f[c] = slot[c * T + tid];
      iters = a.min_inner + stop_j;
      pg2_final = cta == 0 ? tot_s : 0.0;  // the total is global: CTA 0 carries it
    } else {
      pg2_final = block_sum_double(active ? (double)pg_sq<PM>(fp, gp) : 0.0, red);  // thread 0
    }
  }

  // ---- outputs ----
  if (kp.mode == MODE_SOLVE && active) {
    bool bad = false;
#pragma unroll
    for (int c = 0; c < PM; ++c)
      if (c < p) {
        bad |= !isfinite(f[c]);
        a.Y[(size_t)c * N + col] = f[c];
      }
    if (bad) set_status(ctrl, NMF_ERR_NONFINITE);
    if (a.record) {
#pragma unroll
      for (int c = 0; c < PM; ++c)
        if (c < p) {
          if (a.record_transposed) a.record[(size_t)col * p + c] = f[c];
          else a.record[(size_t)c * N + col] = f[c];
        }
    }
  }
  if (a.op_out && active) {
#pragma unroll
    for (int c = 0; c < PM; ++c)
      if (c < p) {
        if (a.op_bf16) static_cast<__nv_bfloat16*>(a.op_out)[(size_t)c * a.op_ld + col] = __float2bfloat16_rn(f[c]);
        else static_cast<float*>(a.op_out)[(size_t)c * a.op_ld + col] = f[c];
      }
  }
  if (kp.mode == MODE_SOLVE && tid == 0 && a.pg2_part) a.pg2_part[(size_t)kStopSlots * ctas + cta] = pg2_final;

  // ---- epilogue: the next phase's W or Gram matrix ----
  if (a.epi != EPI_NONE) {
    __syncthreads();  // dyn (keep) is reused
    const int P = a.epi == EPI_GRAM ? p * p : p * nu;
    float* Fs = dyn;             // [PM][kFs]
    float* Es = dyn + PM * kFs;  // [nu][kFs]
#pragma unroll
    for (int c = 0; c < PM; ++c) Fs[c * kFs + tid] = active ? f[c] : 0.f;
    if (a.epi == EPI_W_ROWS) {
      for (int k = 0; k < nu; ++k) Es[k * kFs + tid] = active ? a.E[(size_t)col * nu + k] : 0.f;
    } else if (a.epi == EPI_W_COLS) {
      for (int k = 0; k < nu; ++k) Es[k * kFs + tid] = active ? a.E[(size_t)k * N + col] : 0.f;
    }
    __syncthreads();
    const float* Os = a.epi == EPI_GRAM ? Fs : Es;
    const int ow = a.epi == EPI_GRAM ? p : nu;
    for (int o = tid; o < P; o += T) {
      const int c = o / ow, k = o % ow;
      float s = 0.f;
      for (int t = 0; t < T; ++t) s = fmaf(Fs[c * kFs + t], Os[k * kFs + t], s);
      a.part_out[(size_t)cta * P + o] = s;
    }
    // tail: the last CTA of each group sums the group, the last group sums all
    __threadfence();
    __syncthreads();
    const int ngroups = tail_groups(ctas);
    const int gi = cta / kTailGroup;
    const int gsz = min(kTailGroup, ctas - gi * kTailGroup);
    if (tid == 0) flag_s = atomicAdd(&a.tail_ctr[1 + gi], 1u) == (unsigned int)(gsz - 1);
    __syncthreads();
    if (flag_s) {
      __threadfence();
      for (int o = tid; o < P; o += T) {
        float s = 0.f;
        for (int i = 0; i < gsz; ++i) s += __ldcg(a.part_out + (size_t)(gi * kTailGroup + i) * P + o);
        a.group_out[(size_t)gi * P + o] = s;
      }
      __threadfence();
      __syncthreads();
      if (tid == 0) {
        a.tail_ctr[1 + gi] = 0u;
        flag_s = atomicAdd(&a.tail_ctr[0], 1u) == (unsigned int)(ngroups - 1);
      }
      __syncthreads();
      if (flag_s) {
        __threadfence();
        float* Rw = dyn;                                  // P
        float* Rh = dyn + NMF_MAX_RANK * NMF_MAX_SKETCH;  // p x p
        float* M0 = Rh + NMF_MAX_RANK * NMF_MAX_RANK;
        float* M1 = M0 + PM * PM;
        for (int o = tid; o < P; o += T) {
          float s = 0.f;
          for (int i = 0; i < ngroups; ++i) s += __ldcg(a.group_out + (size_t)i * P + o);
          Rw[o] = s;
        }
        __syncthreads();
        if (a.epi == EPI_GRAM) {
          for (int o = tid; o < p * p; o += T) Rh[o] = Rw[o];
        } else {
          for (int o = tid; o < p * p; o += T) {
            const int c = o / p, d = o % p;
            float s = 0.f;
            for (int k = 0; k < nu; ++k) s = fmaf(Rw[c * nu + k], Rw[d * nu + k], s);
            Rh[o] = s;
          }
        }
        __syncthreads();
        Reduced* out = a.red_out;
        for (int o = tid; o < p * p; o += T) out->H[o] = Rh[o];
        if (a.epi != EPI_GRAM)
          for (int o = tid; o < P; o += T) out->W[o] = Rw[o];
        const double lam = lambda_max_block<PM>(Rh, p, M0, M1, red);
        if (tid == 0) {
          out->Lc_d = lam;
          out->Lc = isfinite(lam) ? (float)lam : 0.f;
          if (!isfinite(lam)) set_status(ctrl, NMF_ERR_NONFINITE);
          a.tail_ctr[0] = 0u;
          ctrl->bar_count = 0u;  // every CTA is past its stop-test waits
        }
      }
    }
  }
  if (kp.mode == MODE_SOLVE && cta == 0 && tid == 0) {
    ctrl->iters[a.side] = iters;
    ctrl->lipschitz[a.side] = Lc;
    if (a.stats) {
      a.stats->last_inner[a.side] = iters;
      a.stats->total_inner[a.side] += iters;
      a.stats->lipschitz[a.side] = Lc_d;
    }
  }
  if (a.time_out) {
    __syncthreads();
    if (tid == 0) {
      __threadfence();
      atomicMax(a.time_out, global_ns());
    }
  }
}

template <int PM>
size_t dyn_smem(const SolveArgs& a, int mode) {
  const size_t keep = (mode == MODE_SOLVE && a.stop_test) ? (size_t)kKeep * PM * T : 0;
  size_t stage = (mode != MODE_EPI_ONLY && a.bsrc != B_FROM_PARTIALS) ? (size_t)a.nu * kFs : 0;
  if (a.epi != EPI_NONE) {
    const int erows = a.epi == EPI_GRAM ? 0 : a.nu;
    const size_t st = (size_t)(PM + erows) * kFs;
    const size_t tail = NMF_MAX_RANK * NMF_MAX_SKETCH + NMF_MAX_RANK * NMF_MAX_RANK + 2 * PM * PM;
    if (st > stage) stage = st;
    if (tail > stage) stage = tail;
  }
  return (keep > stage ? keep : stage) * sizeof(float);
}

template <int PM>
cudaError_t launch_pm(const KParams& kp, cudaStream_t s) {
  const SolveArgs& a = kp.a;
  const int ctas = solve_ctas(a.N);
  const size_t smem = dyn_smem<PM>(a, kp.mode);
  cudaError_t e = allow_dynamic_smem((const void*)solve_kernel<PM>, (int)smem);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(ctas);
  cfg.blockDim = dim3(T);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  int nattr = 0;
  if (kp.mode == MODE_SOLVE && a.stop_test) {
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    nattr = 1;
  }
  cfg.attrs = attr;
  cfg.numAttrs = nattr;
  count_launches(1);
  return cudaLaunchKernelEx(&cfg, solve_kernel<PM>, kp);
}

__global__ void beta_kernel(float* beta, int K) {
  // beta_k = (alpha_k - 1) / alpha_{k+1}, alpha_0 = 1, alpha_{k+1} = (1 + sqrt(4 alpha_k^2 + 1)) / 2.
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double al = 1.0;
  for (int k = 0; k < K; ++k) {
    const double an = 0.5 * (1.0 + sqrt(4.0 * al * al + 1.0));
    beta[k] = (float)((al - 1.0) / an);
    al = an;
  }
}

__global__ void stats_kernel(nenmf_stats_t* st, const double* pgG, int cG, const double* pgF, int cF,
                             Control* ctrl, int outer) {
  if (threadIdx.x != 0) return;
  double sG = 0.0, sF = 0.0;
  if (pgG)
    for (int i = 0; i < cG; ++i) sG += pgG[i];
  if (pgF)
    for (int i = 0; i < cF; ++i) sF += pgF[i];
  if (st) {
    st->pg_norm[0] = sqrt(sG);
    st->pg_norm[1] = sqrt(sF);
    st->status = ctrl->status;
    st->outer_done = ctrl->status == 0 ? outer : 0;
  }
}

__global__ void eps_kernel(Control* ctrl, const double* pgG, int cG, const double* pgF, int cF, double tol,
                           int tol_mode, nenmf_stats_t* st) {
  if (threadIdx.x != 0) return;
  double e2 = -1.0;
  if (tol > 0.0) {
    if (tol_mode == NENMF_TOL_ABS) {
      e2 = tol * tol;
    } else {
      double s = 0.0;
      for (int i = 0; i < cG; ++i) s += pgG[i];
      for (int i = 0; i < cF; ++i) s += pgF[i];
      e2 = tol * tol * s;
    }
  }
  ctrl->eps2 = e2;
  if (st) st->eps = e2 > 0.0 ? sqrt(e2) : 0.0;
}

int pad_rank(int p) { return p <= 4 ? 4 : p <= 8 ? 8 : p <= 12 ? 12 : p <= 16 ? 16 : p <= 24 ? 24 : 32; }

template <int PM>
int occupancy_pm(size_t smem) {
  int per = 0;
  if (allow_dynamic_smem((const void*)solve_kernel<PM>, (int)smem) != cudaSuccess)
    return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, solve_kernel<PM>, T, smem) != cudaSuccess) return 0;
  return per;
}

}  // namespace

int solve_ctas(int N) { return ceil_div(N, T); }

cudaError_t solve_launch_mode(const SolveArgs& a, const float* beta, int mode, cudaStream_t s) {
  KParams kp{a, beta, mode};
  switch (pad_rank(a.p)) {
    case 4: return launch_pm<4>(kp, s);
    case 8: return launch_pm<8>(kp, s);
    case 12: return launch_pm<12>(kp, s);
    case 16: return launch_pm<16>(kp, s);
    case 24: return launch_pm<24>(kp, s);
    default: return launch_pm<32>(kp, s);
  }
}

cudaError_t beta_launch(float* beta, int K, cudaStream_t s) {
  count_launches(1);
  beta_kernel<<<1, 32, 0, s>>>(beta, K);
  return cudaGetLastError();
}

cudaError_t stats_launch(nenmf_stats_t* stats, const double* pgG, int cG, const double* pgF, int cF, Control* ctrl,
                         int outer, cudaStream_t s) {
  count_launches(1);
  stats_kernel<<<1, 32, 0, s>>>(stats, pgG, cG, pgF, cF, ctrl, outer);
  return cudaGetLastError();
}

cudaError_t eps_launch(Control* ctrl, const double* pgG, int cG, const double* pgF, int cF, double tol, int tol_mode,
                       nenmf_stats_t* stats, cudaStream_t s) {
  count_launches(1);
  eps_kernel<<<1, 32, 0, s>>>(ctrl, pgG, cG, pgF, cF, tol, tol_mode, stats);
  return cudaGetLastError();
}

int solve_max_coresident(int p, int nu, int epi) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  SolveArgs a{};
  a.p = p;
  a.nu = nu;
  a.epi = epi;
  a.stop_test = true;
  a.bsrc = B_FROM_ROWS;
  int per = 0;
  switch (pad_rank(p)) {
    case 4: per = occupancy_pm<4>(dyn_smem<4>(a, MODE_SOLVE)); break;
    case 8: per = occupancy_pm<8>(dyn_smem<8>(a, MODE_SOLVE)); break;
    case 12: per = occupancy_pm<12>(dyn_smem<12>(a, MODE_SOLVE)); break;
    case 16: per = occupancy_pm<16>(dyn_smem<16>(a, MODE_SOLVE)); break;
    case 24: per = occupancy_pm<24>(dyn_smem<24>(a, MODE_SOLVE)); break;
    default: per = occupancy_pm<32>(dyn_smem<32>(a, MODE_SOLVE)); break;
  }
  return per * sms;
}

}  // namespace nmf
