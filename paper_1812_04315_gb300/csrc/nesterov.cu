// nesterov.cu -- the inner loop of NeNMF (Sec. 2) on the columns of a p x N
// unknown Y, one column per thread, fused with everything the loop needs:
//
// prologue  H and B of the subproblem
//             compressed (Alg. 1): W = sum of per-CTA partials (p x nu), H = W W^T,
//               B(:, j) = W d_j with d_j the j-th compressed data vector
//               (G side: W = F_R = F R, d_j = row j of X_R;
//                F side: W = G_L^T = (L G)^T, d_j = column j of X_L);
//             plain (eq. 2-3): H and B summed from partials of the previous
//               kernel and of the X pass;
//           L_c = lambda_max(H): repeated squaring of H / trace (float32,
//               4096th power) picks the top eigenvector, whose Rayleigh
//               quotient is taken in float64;
// loop      grad = H y - b; f = max(0, y - grad / L_c); y = f + beta_k (f - f_prev);
//           optional stop test ||P grad(f)||_F^2 <= eps^2 over all columns,
//           reduced in float64 in a fixed order across CTAs (cooperative launch,
//           bounded grid barrier);
// epilogue  the returned f is stored; partial products for the next phase:
//             W partials (f times rows of R, or columns of L), or Gram partials
//             f f^T (plain); optional operand copy for the next X pass,
//             snapshot and timestamp.
#include "internal.h"

namespace nmf {
namespace {

constexpr int T = kSolveThreads;
constexpr int kSquarings = 12;
constexpr int kFs = T + 1;


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

// Fixed-order sum of `count` doubles, identical in every CTA. Warp 0 computes.
__device__ __forceinline__ double ordered_sum(const double* v, int count) {
  double s = 0.0;
  const int l = threadIdx.x & 31;
  for (int i = l; i < count; i += 32) s += ((volatile const double*)v)[i];
  return warp_sum(s);
}

template <int PM>
__device__ __forceinline__ void hmatvec(const float* Hs, const float* y, const float* b, float* g) {
#pragma unroll
  for (int c = 0; c < PM; ++c) {
    float s = -b[c];
#pragma unroll
    for (int d = 0; d < PM; ++d) s = fmaf(Hs[c * PM + d], y[d], s);
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

  __shared__ float Hs[PM * PM];
  __shared__ float Ms[2][PM * PM];
  __shared__ float Ws[PM * NMF_MAX_SKETCH];
  __shared__ double red[T / 32];
  __shared__ float Lc_s;
  __shared__ double lc_d;
  __shared__ int stop_s;
  extern __shared__ float dyn[];  // epilogue staging: Fs [PM][kFs], Es [nu][kFs]

  float y[PM], b[PM], f[PM], g[PM];
#pragma unroll
  for (int c = 0; c < PM; ++c) {
    y[c] = (active && c < p) ? a.Y[(size_t)c * N + col] : 0.f;
    b[c] = 0.f;
  }

  int iters = 0;
  float Lc = 0.f;
  if (kp.mode != MODE_EPI_ONLY) {
    // ---- H (and W) ----
    if (a.bsrc == B_FROM_PARTIALS) {
      for (int i = tid; i < PM * PM; i += T) {
        const int c = i / PM, d = i % PM;
        float s = 0.f;
        if (c < p && d < p)
          for (int q = 0; q < a.Hparts; ++q) s += a.Hpart[((size_t)q * p + c) * p + d];
        Hs[i] = s;
      }
    } else {
      for (int i = tid; i < PM * nu; i += T) {
        const int c = i / nu, k = i % nu;
        float s = 0.f;
        if (c < p)
          for (int q = 0; q < a.Wparts; ++q) s += a.Wpart[((size_t)q * p + c) * nu + k];
        Ws[c * NMF_MAX_SKETCH + k] = s;
      }
      __syncthreads();
      for (int i = tid; i < PM * PM; i += T) {
        const int c = i / PM, d = i % PM;
        float s = 0.f;
        for (int k = 0; k < nu; ++k) s = fmaf(Ws[c * NMF_MAX_SKETCH + k], Ws[d * NMF_MAX_SKETCH + k], s);
        Hs[i] = s;
      }
    }
    __syncthreads();
    // ---- L_c = lambda_max(H) ----
    if (tid == 0) {
      float tr = 0.f;
      for (int c = 0; c < PM; ++c) tr += Hs[c * PM + c];
      Lc_s = tr;
    }
    __syncthreads();
    const float tr0 = Lc_s;
    if (tr0 > 0.f && isfinite(tr0)) {
      for (int i = tid; i < PM * PM; i += T) Ms[0][i] = Hs[i] / tr0;
      __syncthreads();
      int cur = 0;
      for (int s = 0; s < kSquarings; ++s) {
        const float* M = Ms[cur];
        float* M2 = Ms[cur ^ 1];
        for (int i = tid; i < PM * PM; i += T) {
          const int c = i / PM, d = i % PM;
          float v = 0.f;
#pragma unroll
          for (int k = 0; k < PM; ++k) v = fmaf(M[c * PM + k], M[k * PM + d], v);
          M2[i] = v;
        }
        __syncthreads();
        if (tid == 0) {
          float tr = 0.f;
          for (int c = 0; c < PM; ++c) tr += M2[c * PM + c];
          Lc_s = tr;
        }
        __syncthreads();
        const float tr = Lc_s;
        if (tr > 0.f)
          for (int i = tid; i < PM * PM; i += T) M2[i] /= tr;
        __syncthreads();
        cur ^= 1;
      }
      if (tid < 32) {
        // v = column of M with the largest diagonal entry; lambda = v'Hv / v'v in float64.
        const float* M = Ms[cur];
        int jbest = 0;
        for (int c = 1; c < PM; ++c)
          if (M[c * PM + c] > M[jbest * PM + jbest]) jbest = c;
        double hv = 0.0, vc = 0.0;
        if (tid < PM) {
          vc = (double)M[tid * PM + jbest];
          for (int d = 0; d < PM; ++d) hv = fma((double)Hs[tid * PM + d], (double)M[d * PM + jbest], hv);
        }
        const double num = warp_sum(vc * hv);
        const double den = warp_sum(vc * vc);
        if (tid == 0) lc_d = den > 0.0 ? num / den : 0.0;
      }
      __syncthreads();
      Lc = (float)lc_d;
    }
    // ---- B ----
    if (active) {
      if (a.bsrc == B_FROM_PARTIALS) {
#pragma unroll
        for (int c = 0; c < PM; ++c)
          if (c < p) {
            float s = 0.f;
            for (int q = 0; q < a.Bparts; ++q) s += a.Bpart[((size_t)q * N + col) * a.Bld + c];
            b[c] = s;
          }
      } else {
        for (int k = 0; k < nu; ++k) {
          const float dk = a.bsrc == B_FROM_ROWS ? a.D[(size_t)col * nu + k] : a.D[(size_t)k * N + col];
#pragma unroll
          for (int c = 0; c < PM; ++c) b[c] = fmaf(Ws[c * NMF_MAX_SKETCH + k], dk, b[c]);
        }
      }
    }
  }

  // f holds the returned iterate; before any iteration it is Y_0.
#pragma unroll
  for (int c = 0; c < PM; ++c) f[c] = y[c];
  double pg2_final = -1.0;

  if (kp.mode == MODE_EVAL) {
    hmatvec<PM>(Hs, f, b, g);
    const double s = block_sum_double(active ? (double)pg_sq<PM>(f, g) : 0.0, red);
    if (tid == 0) a.pg2_init[cta] = s;
  } else if (kp.mode == MODE_SOLVE && Lc > 0.f) {
    float fp[PM];
#pragma unroll
    for (int c = 0; c < PM; ++c) fp[c] = y[c];
    const bool test = a.stop_test;
    for (int k = 0; k < a.max_inner; ++k) {
      hmatvec<PM>(Hs, y, b, g);
#pragma unroll
      for (int c = 0; c < PM; ++c) f[c] = fmaxf(0.f, y[c] - g[c] / Lc);
      const float beta = kp.beta[k];
#pragma unroll
      for (int c = 0; c < PM; ++c) {
        y[c] = fmaf(beta, f[c] - fp[c], f[c]);
        fp[c] = f[c];
      }
      iters = k + 1;
      if (test && k + 1 >= a.min_inner) {
        hmatvec<PM>(Hs, f, b, g);
        const double s = block_sum_double(active ? (double)pg_sq<PM>(f, g) : 0.0, red);
        double* slot = a.pg2_part + (size_t)(k & 1) * ctas;
        if (tid == 0) slot[cta] = s;
        __threadfence();
        if (!grid_barrier(ctrl)) return;
        if (tid < 32) {
          const double tot = ordered_sum(slot, ctas);
          if (tid == 0) {
            stop_s = tot <= ctrl->eps2;
            lc_d = tot;
          }
        }
        __syncthreads();
        if (stop_s) {
          pg2_final = lc_d;
          break;
        }
      }
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
  if (kp.mode == MODE_SOLVE && a.pg2_part) {
    // ||P grad||^2 of the returned iterate, per CTA (for the stats).
    if (pg2_final < 0.0) {
      hmatvec<PM>(Hs, f, b, g);
      const double s = block_sum_double(active ? (double)pg_sq<PM>(f, g) : 0.0, red);
      if (tid == 0) a.pg2_part[(size_t)2 * ctas + cta] = s;
    } else if (tid == 0) {
      a.pg2_part[(size_t)2 * ctas + cta] = (cta == 0) ? pg2_final : 0.0;
    }
  }
  if (a.epi != EPI_NONE) {
    float* Fs = dyn;                 // [PM][kFs]
    float* Es = dyn + PM * kFs;      // [nu][kFs] or [PM][kFs] for the Gram
#pragma unroll
    for (int c = 0; c < PM; ++c) Fs[c * kFs + tid] = active ? f[c] : 0.f;
    if (a.epi == EPI_W_ROWS) {
      for (int k = 0; k < nu; ++k) Es[k * kFs + tid] = active ? a.E[(size_t)col * nu + k] : 0.f;
    } else if (a.epi == EPI_W_COLS) {
      for (int k = 0; k < nu; ++k) Es[k * kFs + tid] = active ? a.E[(size_t)k * N + col] : 0.f;
    }
    __syncthreads();
    if (a.epi == EPI_GRAM) {
      for (int o = tid; o < p * p; o += T) {
        const int c = o / p, d = o % p;
        float s = 0.f;
        for (int t = 0; t < T; ++t) s = fmaf(Fs[c * kFs + t], Fs[d * kFs + t], s);
        a.Hpart_out[(size_t)cta * p * p + o] = s;
      }
    } else {
      for (int o = tid; o < p * nu; o += T) {
        const int c = o / nu, k = o % nu;
        float s = 0.f;
        for (int t = 0; t < T; ++t) s = fmaf(Fs[c * kFs + t], Es[k * kFs + t], s);
        a.Wpart_out[(size_t)cta * p * nu + o] = s;
      }
    }
  }
  if (kp.mode == MODE_SOLVE && cta == 0 && tid == 0) {
    ctrl->iters[a.side] = iters;
    ctrl->lipschitz[a.side] = Lc;
    if (a.stats) {
      a.stats->last_inner[a.side] = iters;
      a.stats->total_inner[a.side] += iters;
      a.stats->lipschitz[a.side] = (double)lc_d;
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
cudaError_t launch_pm(const KParams& kp, cudaStream_t s) {
  const SolveArgs& a = kp.a;
  const int ctas = solve_ctas(a.N);
  const int erows = a.epi == EPI_GRAM ? 0 : (a.epi == EPI_NONE ? 0 : a.nu);
  const size_t smem = a.epi == EPI_NONE ? 0 : (size_t)(PM + erows) * kFs * sizeof(float);
  cudaError_t e = cudaFuncSetAttribute(solve_kernel<PM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
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

}  // namespace

int solve_ctas(int N) { return ceil_div(N, T); }

static int pad_rank(int p) {
  return p <= 4 ? 4 : p <= 8 ? 8 : p <= 12 ? 12 : p <= 16 ? 16 : p <= 24 ? 24 : 32;
}

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

template <int PM>
static int occupancy_pm(size_t smem) {
  int per = 0;
  if (cudaFuncSetAttribute(solve_kernel<PM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, solve_kernel<PM>, T, smem) != cudaSuccess) return 0;
  return per;
}

int solve_max_coresident(int p, int nu, int epi) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int PM = pad_rank(p);
  const int erows = (epi == EPI_GRAM || epi == EPI_NONE) ? 0 : nu;
  const size_t smem = epi == EPI_NONE ? 0 : (size_t)(PM + erows) * kFs * sizeof(float);
  int per = 0;
  switch (PM) {
    case 4: per = occupancy_pm<4>(smem); break;
    case 8: per = occupancy_pm<8>(smem); break;
    case 12: per = occupancy_pm<12>(smem); break;
    case 16: per = occupancy_pm<16>(smem); break;
    case 24: per = occupancy_pm<24>(smem); break;
    default: per = occupancy_pm<32>(smem); break;
  }
  return per * sms;
}

}  // namespace nmf
