// nesterov.cu -- the inner loop of NeNMF (Sec. 2) on the columns of a p x N
// unknown Y, one column per thread, fused with what the loop needs:
//
// prologue  loads that do not depend on the previous kernel first (own
//           factor, data and basis vectors), then griddepcontrol.wait
//           (the kernel is launched as a programmatic dependent of the
//           previous one, so this part overlaps its end); then every CTA
//           copies the previous kernel's per-CTA partials of W (compressed:
//           p x nu) or of the Gram matrix (plain) into shared memory with one
//           bulk copy and sums them in a fixed order, forms H = W W^T and
//           L_c = lambda_max(H) (one warp: repeated squaring of H / trace
//           with trace renormalisation until the spectrum has collapsed to
//           rank one, then a float-float Rayleigh quotient), and B:
//             compressed (Alg. 1): B(:, j) = W d_j, d_j the j-th compressed
//               data vector (G side: W = F_R = F R, d_j = row j of X_R;
//               F side: W = G_L^T = (L G)^T, d_j = column j of X_L);
//             plain (eq. 2-3): B summed from the X pass partials;
// loop      f = max(0, y - grad(y) / L_c); y' = f + beta_k (f - f_prev).
//           Only the gradient at f is formed (H f - b); the gradient at the
//           extrapolated y' follows by linearity,
//           grad(y') = grad(f) + beta_k (grad(f) - grad(f_prev)).
//           For p <= 12 the loop reads H from registers (packed upper
//           triangle). Optional stop test ||P grad(f_k)||_F <= eps
//           (stop_test.cuh), taken in blocks of kBlockU tests: each
//           iteration records its test, the block's tests are then decided
//           in order (locally when a partial already exceeds eps^2, else
//           from every CTA's tagged partial, summed in one fixed order),
//           and the first one that passed returns its kept iterate (bounded
//           waits);
// epilogue  the returned iterate is stored (and copied for the next X pass,
//           the snapshot, the stats); the next phase's W (f times rows of R or
//           columns of L) or Gram matrix f f^T is summed per CTA; for large
//           grids the last CTA of each group also sums its group.
#include <algorithm>

#include "internal.h"
#include "nnls_device.cuh"
#include "stop_test.cuh"

namespace nmf {
namespace {

constexpr int kBlockU = 6;  // stop tests per block (their iterates are kept in shared memory)

struct KParams {
  SolveArgs a;
  const float* beta;  // [max_inner] extrapolation weights
  int mode;
  unsigned long long wait_ns;  // limit of every bounded wait
  int withhold;                // failure-path testing: CTA 0 never posts its stop-test words
};

// Bulk copy global -> shared (async proxy), completion counted on an mbarrier.
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_addr(dst)),
               "l"(src), "r"(bytes), "r"(smem_addr(bar))
               : "memory");
}
__device__ __forceinline__ bool mbar_done(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred P1;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 P1, [%1], %2;\n\t"
      "selp.b32 %0, 1, 0, P1;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait for phase `parity`; false after wait_ns or on abort.
__device__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, Control* c, unsigned long long wait_ns) {
  if (mbar_done(bar, parity)) return true;
  const unsigned long long t0 = global_ns();  // the clock is read only for a wait that did not end at once
  while (!mbar_done(bar, parity)) {
    if (*((volatile int*)&c->abort) || global_ns() - t0 > wait_ns) return false;
  }
  return true;
}

__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_launch_dependents() { asm volatile("griddepcontrol.launch_dependents;"); }

// TEST, RESTART: the launch runs the stop test, the adaptive restart
// (template parameters, so launches without them carry none of their code in
// the inner loop, which then stays small enough for the instruction cache).
template <int PM, bool TEST, bool RESTART>
__global__ void __launch_bounds__(kThreadsAll, PM <= 16 ? 2 : 1) solve_kernel(KParams kp) {
  const SolveArgs& a = kp.a;
  Control* ctrl = a.ctrl;
  const int p = a.p, nu = a.nu, N = a.N;
  const int tid = threadIdx.x;
  const int NT = blockDim.x;          // all threads, for cooperative loads
  const bool colthr = tid < T;        // every thread owns a column
  const int cta = blockIdx.x;
  const int ctas = gridDim.x;
  const int col = cta * T + tid;
  const bool active = colthr && col < N;
  const int c0 = cta * T;
  const int cols = min(T, N - c0);
  const bool gram = a.bsrc == B_FROM_PARTIALS;  // plain mode: H comes reduced, no W

  __shared__ __align__(16) float Hs[PM * PM];
  __shared__ float Ws[PM * kWs];
  __shared__ __align__(8) uint64_t pbar;
  __shared__ float2 red[kThreadsAll / 32];
  __shared__ int flag_s;
  __shared__ StopShared stop_s;
  __shared__ double lam_s;
  __shared__ __align__(16) float lam_dg[2 * PM];
  extern __shared__ __align__(16) float dyn[];
  const bool epiW = a.epi == EPI_W_ROWS || a.epi == EPI_W_COLS;
  const bool stageD = kp.mode != MODE_EPI_ONLY && !gram;
  const int vecF = round_up(nu * kFs, 4);            // sub-buffers start on 16-byte boundaries
  float* Es = dyn;                                   // [nu][kFs]: basis vectors of the epilogue
  float* Ds = Es + (epiW ? vecF : 0);                // [nu][kFs]: data vectors of B
  float* scratch = Ds + (stageD ? vecF : 0);         // partial sums, pending iterates, epilogue

  // ---- independent of the previous kernel ----
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(&pbar)), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  float y[PM], b[PM], f[PM];
#pragma unroll
  for (int c = 0; c < PM; ++c) {
    y[c] = (active && c < p) ? a.Y[(size_t)c * N + col] : 0.f;
    b[c] = 0.f;
  }
  if (a.epi == EPI_W_ROWS) {
    const float* src = a.E + (size_t)c0 * nu;
    for (int i = tid; i < T * nu; i += NT) {
      const int t = i / nu, k = i % nu;
      Es[k * kFs + t] = t < cols ? __ldg(src + i) : 0.f;
    }
  } else if (a.epi == EPI_W_COLS) {
    for (int i = tid; i < nu * T; i += NT) {
      const int k = i / T, t = i % T;
      Es[k * kFs + t] = t < cols ? __ldg(a.E + (size_t)k * N + c0 + t) : 0.f;
    }
  }
  if (stageD) {
    if (a.bsrc == B_FROM_ROWS) {
      const float* src = a.D + (size_t)c0 * nu;
      for (int i = tid; i < T * nu; i += NT) {
        const int t = i / nu, k = i % nu;
        Ds[k * kFs + t] = t < cols ? __ldg(src + i) : 0.f;
      }
    } else {
      for (int i = tid; i < nu * T; i += NT) {
        const int k = i / T, t = i % T;
        Ds[k * kFs + t] = t < cols ? __ldg(a.D + (size_t)k * N + c0 + t) : 0.f;
      }
    }
  }

  // ---- everything below may read what the previous kernel wrote ----
  pdl_wait();
  if (__syncthreads_or(call_failed(ctrl))) return;  // also: the mbarrier is initialised
  pdl_launch_dependents();

  int iters = 0;
  float Lc = 0.f;
  double Lc_d = 0.0;
  if (kp.mode != MODE_EPI_ONLY) {
    // Sum of the predecessor's partials, in a fixed order (same in every CTA):
    // one bulk copy of all partials into shared memory, then float4 sums over
    // `slices` contiguous ranges of partials, then over the slices.
    const int P = gram ? p * p : p * nu;
    const int P4 = partial_stride(P);
    const int G = a.groups_in;
    float* Ps = scratch;          // [G][P4]
    float* Rw = Ps + G * P4;      // [P4]: the reduced W (or H)
    float* Red = Rw + P4;         // [slices][P4]
    if (tid == 0) bulk_load(Ps, a.part_in, (uint32_t)(G * P4) * 4u, &pbar);
    const bool got = mbar_wait_bounded(&pbar, 0u, ctrl, kp.wait_ns);
    if (__syncthreads_or(!got)) {
      if (tid == 0) {
        set_status(ctrl, NMF_ERR_DEVICE_TIMEOUT);
        *((volatile int*)&ctrl->abort) = 1;
        // the copy is in flight: wait for it (bounded) before leaving
        const unsigned long long t0 = global_ns();
        while (!mbar_done(&pbar, 0u) && global_ns() - t0 < kp.wait_ns) {
        }
      }
      __syncthreads();
      return;
    }
    {
      const int Q = P4 / 4;
      const int slices = max(1, min(G, NT / Q));
      for (int idx = tid; idx < slices * Q; idx += NT) {
        const int q = idx % Q, sl = idx / Q;
        const int g0 = sl * G / slices, g1 = (sl + 1) * G / slices;
        float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
        const float4* src = reinterpret_cast<const float4*>(Ps) + q;
#pragma unroll 4
        for (int g = g0; g < g1; ++g) {
          const float4 v = src[(size_t)g * Q];
          acc.x += v.x;
          acc.y += v.y;
          acc.z += v.z;
          acc.w += v.w;
        }
        reinterpret_cast<float4*>(Red)[sl * Q + q] = acc;
      }
      __syncthreads();
      for (int q = tid; q < Q; q += NT) {
        float4 acc = reinterpret_cast<const float4*>(Red)[q];
        for (int sl = 1; sl < slices; ++sl) {
          const float4 v = reinterpret_cast<const float4*>(Red)[sl * Q + q];
          acc.x += v.x;
          acc.y += v.y;
          acc.z += v.z;
          acc.w += v.w;
        }
        reinterpret_cast<float4*>(Rw)[q] = acc;
      }
    }
    __syncthreads();
    if (gram) {
      for (int i = tid; i < PM * PM; i += NT) {
        const int c = i / PM, d = i % PM;
        Hs[i] = (c < p && d < p) ? Rw[c * p + d] : 0.f;
      }
    } else {
      for (int i = tid; i < PM * nu; i += NT) {
        const int c = i / nu, k = i % nu;
        Ws[c * kWs + k] = c < p ? Rw[c * nu + k] : 0.f;
      }
      __syncthreads();
      for (int i = tid; i < PM * PM; i += NT) {
        const int c = i / PM, d = i % PM;
        float s = 0.f;
        for (int k = 0; k < nu; ++k) s = fmaf(Ws[c * kWs + k], Ws[d * kWs + k], s);
        Hs[i] = s;
      }
    }
    __syncthreads();
    if (active) {
      if (gram) {
        // B(:, col) = sum over the X pass partials; a whole row of partials
        // per q, so the loads of all c are in flight together.
        for (int q = 0; q < a.Bparts; ++q) {
          const float* bp = a.Bpart + ((size_t)q * N + col) * a.Bld;
#pragma unroll
          for (int c = 0; c < PM; ++c)
            if (c < p) b[c] += __ldcg(bp + c);
        }
      } else {
        for (int k = 0; k < nu; ++k) {
          const float dk = Ds[k * kFs + tid];
#pragma unroll
          for (int c = 0; c < PM; ++c) b[c] = fmaf(Ws[c * kWs + k], dk, b[c]);
        }
      }
    }
    if (active) {
      // non-finite data or a non-finite current factor: max(0, .) would turn
      // a NaN step into 0 silently, so report it (the call's later kernels stop)
      bool bad = false;
#pragma unroll
      for (int c = 0; c < PM; ++c) bad |= !isfinite(b[c]) || !isfinite(y[c]);
      if (bad) set_status(ctrl, NMF_ERR_NONFINITE);
    }
    // L_c by the whole block (the slice sums are consumed: eigenvalue scratch)
    if (kp.mode == MODE_SOLVE) lambda_max_cta<PM>(Hs, Red, lam_dg, &lam_s, p);
    __syncthreads();
    if (kp.mode == MODE_SOLVE) {
      Lc_d = lam_s;
      if (!isfinite(Lc_d)) {
        if (tid == 0) set_status(ctrl, NMF_ERR_NONFINITE);
        Lc_d = 0.0;
      }
      Lc = (float)Lc_d;
    }
  }

#pragma unroll
  for (int c = 0; c < PM; ++c) f[c] = y[c];
  double pg2_final = 0.0;

  if (kp.mode == MODE_EVAL) {
    float g[PM];
    hmatvec<PM>(Hs, f, b, g);
    const double s = block_sum_df(active ? pg_sq<PM>(f, g) : 0.f, red);
    if (tid == 0) a.pg2_init[cta] = s;
  } else if (kp.mode == MODE_SOLVE && Lc > 0.f) {
    // PM <= kPackedMax: the loop's products read H from registers
    constexpr bool packed = PM <= kPackedMax;
    float Hp[packed ? PM * (PM + 1) / 2 : 1];
    if constexpr (packed) load_packed<PM>(Hs, Hp);
    float g[PM], fp[PM], gp[PM];
    if constexpr (packed) hmatvec_packed<PM>(Hp, y, b, g);
    else hmatvec<PM>(Hs, y, b, g);
#pragma unroll
    for (int c = 0; c < PM; ++c) {
      fp[c] = y[c];
      gp[c] = g[c];
    }
    float beta_next = __ldg(kp.beta);
    int rs = 0;            // restart: iterations since this vector's last restart
    float obj_prev = 0.f;  // restart: this vector's previous objective
    float* keep = scratch;  // [kBlockU][PM][T]: iterates of the block's tests (per thread)
    const float inv_Lc = 1.f / Lc;
    constexpr bool test = TEST;
    const double eps2 = ctrl->eps2;
    const float eps2_f = eps2 < 0.0 ? 0.f : __double2float_rd(eps2);  // eps^2 rounded down to float
    int stop_j = -1, nrec = 0, base = 0;  // tests: recorded in this block, decided before it
    bool aborted = false;
    for (int k = 0; k < a.max_inner; ++k) {
#pragma unroll
      for (int c = 0; c < PM; ++c) f[c] = fmaxf(0.f, fmaf(-g[c], inv_Lc, y[c]));
      float beta = beta_next;
      if (k + 1 < a.max_inner) beta_next = __ldg(kp.beta + k + 1);  // in flight during the product
      float gf[PM];
      if constexpr (packed) hmatvec_packed<PM>(Hp, f, b, gf);
      else hmatvec<PM>(Hs, f, b, gf);
      if (RESTART) {
        // adaptive restart: this vector's objective 1/2 f^T H f - b^T f = 1/2 f^T (gf - b);
        // when it rises the vector drops its momentum (beta_0 = 0 now, beta_1 next)
        // a rise counts beyond kRestartTol of the terms' scale (float32 rounding stays below it)
        float obj = 0.f, sc = 0.f;
#pragma unroll
        for (int c = 0; c < PM; ++c) {
          obj = fmaf(f[c], gf[c] - b[c], obj);
          sc = fmaf(fabsf(f[c]), fabsf(gf[c]) + fabsf(b[c]), sc);
        }
        obj *= 0.5f;
        if (k >= 1 && obj - obj_prev > kRestartTol * sc) rs = 0;
        obj_prev = obj;
        beta = __ldg(kp.beta + rs);
        ++rs;
      }
#pragma unroll
      for (int c = 0; c < PM; ++c) {
        y[c] = fmaf(beta, f[c] - fp[c], f[c]);
        g[c] = fmaf(beta, gf[c] - gp[c], gf[c]);
        fp[c] = f[c];
        gp[c] = gf[c];
      }
      iters = k + 1;
      if (test && k + 1 >= a.min_inner) {
        stop_record<PM>(stop_s, nrec, active ? pg_sq<PM>(f, gf) : 0.f, f, keep, eps2_f);
        if (++nrec == kBlockU || k + 1 == a.max_inner) {
          const int r = stop_decide(stop_s, nrec, base, a.stop_slots, a.epoch, eps2, eps2_f, ctas,
                                    kp.withhold != 0, ctrl, kp.wait_ns);
          if (r == -2) {
            aborted = true;
            break;
          }
          if (r >= 0) {
            // the first test that passed: its iterate, as the sequential rule returns it
            const float* slot = keep + (size_t)r * PM * T;
#pragma unroll
            for (int c = 0; c < PM; ++c) f[c] = slot[c * T + tid];
            stop_j = base + r;
            break;
          }
          base += nrec;
          nrec = 0;
        }
      }
    }
    if (aborted) return;  // every thread saw the same outcome
    if (stop_j >= 0) iters = a.min_inner + stop_j;
    if (stop_j >= 0) {
      pg2_final = cta == 0 ? stop_s.total : 0.0;  // the total is global: CTA 0 carries it
    } else {
      pg2_final = block_sum_df(active ? pg_sq<PM>(fp, gp) : 0.f, red);  // thread 0
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
  if (kp.mode == MODE_SOLVE && tid == 0 && a.pg2_part) a.pg2_part[cta] = pg2_final;
  if (kp.mode == MODE_SOLVE && cta == 0 && tid == 0) {
    ctrl->iters[a.side] = iters;
    ctrl->lipschitz[a.side] = Lc;
    if (a.stats) {
      a.stats->last_inner[a.side] = iters;
      a.stats->total_inner[a.side] += iters;
      a.stats->lipschitz[a.side] = Lc_d;
    }
  }

  // ---- epilogue: this CTA's share of the next phase's W or Gram matrix ----
  if (a.epi != EPI_NONE) {
    __syncthreads();  // scratch (pending iterates) is reused
    const int P = a.epi == EPI_GRAM ? p * p : p * nu;
    const int P4 = partial_stride(P);
    float* Fs = scratch;  // [PM][kFs]
    if (colthr) {
#pragma unroll
      for (int c = 0; c < PM; ++c) Fs[c * kFs + tid] = active ? f[c] : 0.f;
    }
    __syncthreads();
    const float* Os = a.epi == EPI_GRAM ? Fs : Es;
    const int ow = a.epi == EPI_GRAM ? p : nu;
    for (int o = tid; o < P4; o += NT) {
      float s = 0.f;
      if (o < P) {
        const int c = o / ow, k = o % ow;
        const float4* fa = reinterpret_cast<const float4*>(Fs + c * kFs);
        const float4* ob = reinterpret_cast<const float4*>(Os + k * kFs);
        float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
#pragma unroll 8
        for (int t4 = 0; t4 < T / 4; ++t4) {
          const float4 x = fa[t4], z = ob[t4];
          s0 = fmaf(x.x, z.x, s0);
          s1 = fmaf(x.y, z.y, s1);
          s2 = fmaf(x.z, z.z, s2);
          s3 = fmaf(x.w, z.w, s3);
        }
        s = (s0 + s1) + (s2 + s3);
      }
      a.part_out[(size_t)cta * P4 + o] = s;
    }
    if (a.group > 1) {
      // large grids: the last CTA of each group sums the group's partials
      __threadfence();
      __syncthreads();
      const int gi = cta / a.group;
      const int gsz = min(a.group, ctas - gi * a.group);
      if (tid == 0) flag_s = atomicAdd(&a.tail_ctr[gi], 1u) == (unsigned int)(gsz - 1);
      __syncthreads();
      if (flag_s) {
        __threadfence();
        for (int o = tid; o < P4; o += NT) {
          float s = 0.f;
          for (int i = 0; i < gsz; ++i) s += __ldcg(a.part_out + (size_t)(gi * a.group + i) * P4 + o);
          a.group_out[(size_t)gi * P4 + o] = s;
        }
        if (tid == 0) a.tail_ctr[gi] = 0u;
      }
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
  const bool epiW = a.epi == EPI_W_ROWS || a.epi == EPI_W_COLS;
  const bool gram = a.bsrc == B_FROM_PARTIALS;
  const bool stageD = mode != MODE_EPI_ONLY && !gram;
  size_t scratch = 0;
  if (mode != MODE_EPI_ONLY) {
    const size_t P4 = partial_stride(gram ? a.p * a.p : a.p * a.nu);
    // partials, their sum, and the slice sums (reused as the eigenvalue scratch)
    scratch = (size_t)a.groups_in * P4 + P4 + std::max({(size_t)4 * kThreadsAll, P4, (size_t)2 * PM * lam_stride<PM>()});
  }
  if (mode == MODE_SOLVE && a.stop_test) scratch = std::max(scratch, (size_t)kBlockU * PM * T);
  if (a.epi != EPI_NONE) scratch = std::max(scratch, (size_t)PM * kFs);
  const size_t vecF = round_up_sz((size_t)a.nu * kFs, 4);
  return ((epiW ? vecF : 0) + (stageD ? vecF : 0) + scratch) * sizeof(float);
}

template <int PM>
cudaError_t launch_pm(const KParams& kp, cudaStream_t s) {
  const SolveArgs& a = kp.a;
  const int ctas = solve_ctas(a.N);
  const size_t smem = dyn_smem<PM>(a, kp.mode);
  const bool t = kp.a.stop_test, r = kp.a.restart != 0;
  const void* fn = t ? (r ? (const void*)solve_kernel<PM, true, true> : (const void*)solve_kernel<PM, true, false>)
                     : (r ? (const void*)solve_kernel<PM, false, true> : (const void*)solve_kernel<PM, false, false>);
  cudaError_t e = allow_dynamic_smem(fn, (int)smem);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(ctas);
  cfg.blockDim = dim3(kThreadsAll);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  // Programmatic dependent launch: the kernel starts while its predecessor
  // finishes and waits (griddepcontrol.wait) before touching its outputs.
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  count_launches(1);
  if (t) return r ? cudaLaunchKernelEx(&cfg, solve_kernel<PM, true, true>, kp)
               : cudaLaunchKernelEx(&cfg, solve_kernel<PM, true, false>, kp);
  return r ? cudaLaunchKernelEx(&cfg, solve_kernel<PM, false, true>, kp)
           : cudaLaunchKernelEx(&cfg, solve_kernel<PM, false, false>, kp);
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
  if (allow_dynamic_smem((const void*)solve_kernel<PM, true, true>, (int)smem) != cudaSuccess)
    return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, solve_kernel<PM, true, true>, kThreadsAll, smem) !=
      cudaSuccess)
    return 0;
  return per;
}

}  // namespace

int solve_ctas(int N) { return ceil_div(N, T); }

cudaError_t solve_launch_mode(const SolveArgs& a, const float* beta, int mode, cudaStream_t s) {
  KParams kp{a, beta, mode, wait_limit_ns(), injected_fault() == NMF_FAULT_STOP_TEST ? 1 : 0};
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

int solve_max_coresident(int p, int nu, int epi, int groups_in) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  SolveArgs a{};
  a.p = p;
  a.nu = nu;
  a.epi = epi;
  a.stop_test = true;
  a.bsrc = epi == EPI_GRAM ? B_FROM_PARTIALS : B_FROM_ROWS;
  a.groups_in = groups_in;
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
