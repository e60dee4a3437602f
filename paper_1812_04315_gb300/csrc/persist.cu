// persist.cu -- compressed NeNMF (Alg. 1) with all of its outer iterations in
// one persistent, cooperative launch.
//
// CTA c owns columns c*T .. c*T+T-1 of both unknowns: of G^T (rows of G, the
// G update of eq. 2 on X_R = X R) and of F (the F update of eq. 3 on
// X_L = L X). It loads them once, together with the matching data vectors
// (rows of X_R, columns of X_L) and basis vectors (columns of L, rows of R),
// and keeps them in shared memory for the whole solve; only the p x nu
// products that couple the columns travel through global memory:
//
//   phase (side s, outer iteration t)
//     wait     every CTA has posted the share of W this phase reads (grid
//              barrier: one counter, one polling thread per CTA, bounded);
//     reduce   all shares copied into shared memory at once (16-byte
//              asynchronous copies), then W = their sum in one fixed order
//              (the order of the per-update kernels, so both paths agree
//              bit for bit): G side W = F R (p x nu), F side W = (L G)^T;
//     prepare  H = W W^T, L_c = lambda_max(H), b_j = W d_j per column;
//     solve    the inner loop of Sec. 2 on the CTA's columns, with the
//              projected-gradient stop test across CTAs (stop_test.cuh),
//              taken in blocks of kBlockP tests;
//     share    this CTA's part of the other side's W (G side: sum_j g_j l_j^T;
//              F side: sum_j f_j r_j^T), then its arrival at the barrier.
//
// With the stop test on, a first phase forms the projected gradients at
// (G0, F0) and eps (Sec. 2's rule; the same arithmetic and order as the
// per-update path). Every wait is bounded; on a timeout the CTA records
// NMF_ERR_DEVICE_TIMEOUT, raises the abort flag and returns, and the others
// leave at their next wait. The launch is cooperative, so all CTAs are
// resident together.
#include <algorithm>

#include "internal.h"
#include "nnls_device.cuh"
#include "stop_test.cuh"

namespace nmf {
namespace {

struct PArgs {
  int n, m, p, nu;
  const float* L;
  const float* R;
  const float* XL;
  const float* XR;
  float* G;  // n x p, in/out
  float* F;  // p x m, in/out
  int max_outer, max_inner, min_inner;
  const float* beta;  // [max_inner]
  float* partG;       // [ctasG][P4]: the G side's shares of the F update's W
  float* partF;       // [ctasF][P4]: the F side's shares of the G update's W
  double* pg2G;       // [ctasG]: ||P grad||^2 of the last G update, per CTA
  double* pg2F;       // [ctasF]
  double* initG;      // [ctasG]: ||P grad_G(G0, F0)||^2, per CTA
  double* initF;      // [ctasF]
  unsigned long long* slots;  // [max_inner][C] stop-test words (zeroed per call)
  unsigned int* bar;          // barrier arrivals (zeroed per call)
  float* keep;                // [C][kBlockP][PM][T] kept iterates, or null: in shared memory
  float* record_G;            // optional [max_outer][n][p]
  float* record_F;            // optional [max_outer][p][m]
  unsigned long long* times;  // optional [max_outer + 1]
  double tol;
  int tol_mode;
  nenmf_stats_t* stats;
  Control* ctrl;
  unsigned long long wait_ns;
  int withhold;
  int ctasG, ctasF;
};

constexpr int kBlockP = kMaxStopBlock;  // stop tests per block (their iterates are kept)

__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(static_cast<uint32_t>(__cvta_generic_to_shared(dst))),
               "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Grid barrier on a counter that only grows: arrival r of every CTA lifts it
// to r * gridDim.x. After the block barrier, thread 0's release reduction
// publishes the CTA's stores with the count; the waiter's acquire load of
// the count makes them visible, and the block barrier after it passes them
// on to the CTA's threads.
__device__ __forceinline__ void grid_arrive(unsigned int* bar) {
  __syncthreads();
  if (threadIdx.x == 0) asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(bar) : "memory");
}

// Thread 0 waits for `target` arrivals; false (in every thread) on timeout,
// an abort raised elsewhere or a device error recorded by any CTA. The
// status word is loaded together with the count in every poll, so the last
// poll costs one round trip; an error recorded just before the last arrival
// may be seen one wait later (the call still ends with that status).
__device__ __forceinline__ bool grid_wait(unsigned int* bar, unsigned int target, Control* c,
                                          unsigned long long wait_ns, int* ok_s) {
  if (threadIdx.x == 0) {
    cuda::atomic_ref<unsigned int, cuda::thread_scope_device> cnt(*bar);
    int ok = 1;
    unsigned long long t0 = 0ull;  // the clock is read from the first check on
    unsigned int spins = 0;
    int status = 0;
    for (;;) {
      // the status first: the acquire load of the count orders what follows it
      status = *((volatile int*)&c->status);
      const unsigned int arrived = cnt.load(cuda::memory_order_acquire);
      if (arrived >= target) break;
      // the abort flag and the clock every 16 polls: a tighter loop notices
      // the last arrival sooner, and the wait stays bounded
      if ((++spins & 15u) != 0u) continue;
      if (*((volatile int*)&c->abort)) { ok = 0; break; }
      if (t0 == 0ull) {
        t0 = global_ns();
      } else if (global_ns() - t0 > wait_ns) {
        set_status(c, NMF_ERR_DEVICE_TIMEOUT);
        *((volatile int*)&c->abort) = 1;
        ok = 0;
        break;
      }
    }
    if (status != 0) ok = 0;
    *ok_s = ok;
  }
  __syncthreads();
  return *ok_s != 0;
}

// The first G shares (P4 floats each, contiguous) into Ps, every 16-byte
// copy in flight at once.
__device__ __forceinline__ void stage_shares(const float* part, int G, int P4, float* Ps) {
  for (int i = threadIdx.x; i < G * (P4 / 4); i += blockDim.x) cp_async16(Ps + 4 * i, part + 4 * i);
  cp_async_wait_all();
  __syncthreads();
}

// Sum of the G shares in Ps (P4 floats each) into Rw, in the order of
// solve_kernel's prologue: float4 sums over `slices` contiguous ranges of
// shares, then over the slices. Red: max(1, min(G, NT / Q)) * P4 floats.
__device__ __forceinline__ void sum_shares(const float* Ps, int G, int P4, float* Rw, float* Red) {
  const int tid = threadIdx.x, NT = blockDim.x;
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
  __syncthreads();
}

// W (p x nu, from Rw) into Ws, H = W W^T into Hs (zero padded to PM x PM).
template <int PM>
__device__ __forceinline__ void form_h(const float* Rw, int p, int nu, float* Ws, float* Hs) {
  const int tid = threadIdx.x, NT = blockDim.x;
  for (int i = tid; i < PM * nu; i += NT) {
    const int c = i / nu, k = i % nu;
    Ws[c * kWs + k] = c < p ? Rw[c * nu + k] : 0.f;
  }
  __syncthreads();
  // the upper triangle, mirrored (fmaf(a, b, s) = fmaf(b, a, s): H_dc equals H_cd bit for bit)
  constexpr int E = PM * (PM + 1) / 2;
  for (int e = tid; e < E; e += NT) {
    int c = 0, r = e;
    while (r >= PM - c) {
      r -= PM - c;
      ++c;
    }
    const int d = c + r;
    float s = 0.f;
#pragma unroll 4
    for (int k = 0; k < nu; ++k) s = fmaf(Ws[c * kWs + k], Ws[d * kWs + k], s);
    Hs[c * PM + d] = s;
    Hs[d * PM + c] = s;
  }
  __syncthreads();
}

// b = W d for this thread's column (d: column tid of Ds, nu x kFs).
template <int PM>
__device__ __forceinline__ void form_b(const float* Ws, const float* Ds, int nu, float* b) {
#pragma unroll
  for (int c = 0; c < PM; ++c) b[c] = 0.f;
#pragma unroll 4
  for (int k = 0; k < nu; ++k) {
    const float dk = Ds[k * kFs + threadIdx.x];
#pragma unroll
    for (int c = 0; c < PM; ++c) b[c] = fmaf(Ws[c * kWs + k], dk, b[c]);
  }
}

// This CTA's share of the other side's W: part[o] = sum_t Y[c][t] E[k][t],
// o = c nu + k (the epilogue of solve_kernel, same order).
// Each thread forms the outputs (c, k) and (c + 1, k): the two share the read
// of row k of Es (the reads that bound this step), and every output keeps
// the arithmetic of the one-output form (four chains over t, then
// (s0 + s1) + (s2 + s3)). From PM = 24 on, where the kernel has no
// registers to spare, one output per thread.
template <int PM>
__device__ __forceinline__ void form_share(const float* Ys, const float* Es, int p, int nu, int P4, float* part) {
  const int P = p * nu;
  if constexpr (PM >= 24) {
    for (int o = threadIdx.x; o < P4; o += blockDim.x) {
      float s = 0.f;
      if (o < P) {
        const int c = o / nu, k = o % nu;
        const float4* fa = reinterpret_cast<const float4*>(Ys + c * kFs);
        const float4* ob = reinterpret_cast<const float4*>(Es + k * kFs);
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
      part[o] = s;
    }
    return;
  }
  const int pairs = (p + 1) / 2;
  for (int task = threadIdx.x; task < pairs * nu; task += blockDim.x) {
    const int c = 2 * (task / nu), k = task % nu;
    const bool two = c + 1 < p;
    const float4* fa = reinterpret_cast<const float4*>(Ys + c * kFs);
    const float4* fb = reinterpret_cast<const float4*>(Ys + (two ? c + 1 : c) * kFs);
    const float4* ob = reinterpret_cast<const float4*>(Es + k * kFs);
    float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f, b0 = 0.f, b1 = 0.f, b2 = 0.f, b3 = 0.f;
#pragma unroll 4
    for (int t4 = 0; t4 < T / 4; ++t4) {
      const float4 z = ob[t4], x = fa[t4], y = fb[t4];
      a0 = fmaf(x.x, z.x, a0);
      a1 = fmaf(x.y, z.y, a1);
      a2 = fmaf(x.z, z.z, a2);
      a3 = fmaf(x.w, z.w, a3);
      b0 = fmaf(y.x, z.x, b0);
      b1 = fmaf(y.y, z.y, b1);
      b2 = fmaf(y.z, z.z, b2);
      b3 = fmaf(y.w, z.w, b3);
    }
    part[c * nu + k] = (a0 + a1) + (a2 + a3);
    if (two) part[(c + 1) * nu + k] = (b0 + b1) + (b2 + b3);
  }
  // the padding of the share
  for (int o = P + threadIdx.x; o < P4; o += blockDim.x) part[o] = 0.f;
}

// PM: the padded rank of H, W, the kept iterates' layout and the columns in
// shared memory. PL <= PM: the rows the inner loop's register arithmetic
// runs over (iterates, gradients, b and the packed upper triangle of H); the
// rows from p on are exact zeros (zero rows of W give zero rows of H and b,
// hence zero gradients and iterates), so leaving out those from PL on gives
// the values of the full-width loop (up to the sign of a zero).
template <int PM, int PL, bool TEST, bool RESTART>
__global__ void __launch_bounds__(kThreadsAll, 1) persist_kernel(PArgs a) {
  static_assert(PL <= PM && (PL == PM || PL <= kPackedMax), "a shorter loop rank needs H in registers");
  Control* ctrl = a.ctrl;
  const int p = a.p, nu = a.nu;
  const int tid = threadIdx.x, NT = blockDim.x;
  const int cta = blockIdx.x, C = gridDim.x;
  const int c0 = cta * T;
  const int P4 = partial_stride(p * nu);

  __shared__ __align__(16) float Hs[PM * PM];
  __shared__ float Ws[PM * kWs];
  __shared__ float2 red[kThreadsAll / 32];
  __shared__ int ok_s;
  __shared__ StopShared stop_s;
  __shared__ float pterm[TEST ? kBlockP * T : 1];  // the current block's stop-test terms, per thread
  __shared__ double lam_s, eps2_s;
  __shared__ __align__(16) float lam_dg[2 * PM];
  extern __shared__ __align__(16) float dyn[];
  const int vecF = round_up(nu * kFs, 4);
  float* const YG = dyn;                   // this CTA's columns of G^T
  float* const YF = YG + PM * kFs;         // and of F
  float* const DG = YF + PM * kFs;         // rows of X_R (data vectors of the G side)
  float* const DF = DG + vecF;             // columns of X_L
  float* const EG = DF + vecF;             // columns of L (basis vectors of the G side's share)
  float* const EF = EG + vecF;             // rows of R
  float* const scratch = EF + vecF;        // reductions, eigenvalue scratch, pending iterates
  float* keep = a.keep ? a.keep + (size_t)cta * kBlockP * PM * T : scratch;

  if (call_failed(ctrl)) return;
  // ---- resident data: factors, data and basis vectors of the CTA's columns ----
  for (int i = tid; i < PM * T; i += NT) {
    const int c = i / T, t = i % T;
    const bool g = c < p && c0 + t < a.n, f = c < p && c0 + t < a.m;
    YG[c * kFs + t] = g ? a.G[(size_t)(c0 + t) * p + c] : 0.f;
    YF[c * kFs + t] = f ? a.F[(size_t)c * a.m + c0 + t] : 0.f;
  }
  for (int i = tid; i < T * nu; i += NT) {
    const int t = i / nu, k = i % nu;  // consecutive threads: consecutive k of one row
    const bool g = c0 + t < a.n, f = c0 + t < a.m;
    DG[k * kFs + t] = g ? __ldg(a.XR + (size_t)(c0 + t) * nu + k) : 0.f;
    EF[k * kFs + t] = f ? __ldg(a.R + (size_t)(c0 + t) * nu + k) : 0.f;
  }
  for (int i = tid; i < nu * T; i += NT) {
    const int k = i / T, t = i % T;
    const bool g = c0 + t < a.n, f = c0 + t < a.m;
    EG[k * kFs + t] = g ? __ldg(a.L + (size_t)k * a.n + c0 + t) : 0.f;
    DF[k * kFs + t] = f ? __ldg(a.XL + (size_t)k * a.m + c0 + t) : 0.f;
  }
  __syncthreads();

  unsigned int rounds = 0;  // barrier arrivals so far (the same count in every CTA)
  long long total_inner_G = 0, total_inner_F = 0;  // CTA 0, thread 0: the statistics' running totals
  // ---- shares of both W's at (G0, F0) ----
  if (cta < a.ctasF) form_share<PM>(YF, EF, p, nu, P4, a.partF + (size_t)cta * P4);
  if (TEST && cta < a.ctasG) form_share<PM>(YG, EG, p, nu, P4, a.partG + (size_t)cta * P4);
  grid_arrive(a.bar);
  ++rounds;

  // ---- eps from the projected gradients at (G0, F0) ----
  if (TEST) {
    if (!grid_wait(a.bar, rounds * C, ctrl, a.wait_ns, &ok_s)) return;
    for (int s = 0; s < 2; ++s) {
      float* Rw = scratch + (size_t)C * P4;
      float* Red = Rw + P4;
      const int G = s == 0 ? a.ctasF : a.ctasG;
      stage_shares(s == 0 ? a.partF : a.partG, G, P4, scratch);
      sum_shares(scratch, G, P4, Rw, Red);
      form_h<PM>(Rw, p, nu, Ws, Hs);
      const bool active = c0 + tid < (s == 0 ? a.n : a.m);
      const float* Y = s == 0 ? YG : YF;
      float y[PM], b[PM], g[PM];
      float pg = 0.f;
      if (active) {
#pragma unroll
        for (int c = 0; c < PM; ++c) y[c] = Y[c * kFs + tid];
        form_b<PM>(Ws, s == 0 ? DG : DF, nu, b);
        hmatvec<PM>(Hs, y, b, g);
        pg = pg_sq<PM>(y, g);
      }
      const double tot = block_sum_df(pg, red);
      if (tid == 0 && cta < (s == 0 ? a.ctasG : a.ctasF)) (s == 0 ? a.initG : a.initF)[cta] = tot;
      __syncthreads();  // Ws, Hs and the scratch are reused by the next side
    }
    grid_arrive(a.bar);
    ++rounds;
    if (!grid_wait(a.bar, rounds * C, ctrl, a.wait_ns, &ok_s)) return;
    if (tid == 0) {
      // eps^2 = tol^2 (sum over the G side's CTAs, then the F side's), as eps_kernel
      double e2 = -1.0;
      if (a.tol > 0.0) {
        if (a.tol_mode == NENMF_TOL_ABS) {
          e2 = a.tol * a.tol;
        } else {
          double s = 0.0;
          for (int i = 0; i < a.ctasG; ++i) s += __ldcg(a.initG + i);
          for (int i = 0; i < a.ctasF; ++i) s += __ldcg(a.initF + i);
          e2 = a.tol * a.tol * s;
        }
      }
      eps2_s = e2;
      if (cta == 0) {
        ctrl->eps2 = e2;
        if (a.stats) a.stats->eps = e2 > 0.0 ? sqrt(e2) : 0.0;
      }
    }
    __syncthreads();
  } else if (tid == 0) {
    eps2_s = -1.0;
    if (cta == 0) ctrl->eps2 = -1.0;
  }
  const double eps2 = eps2_s;

  // ---- the outer iterations of Alg. 1 ----
  for (int t = 0; t < a.max_outer; ++t) {
    for (int s = 0; s < 2; ++s) {
      if (!grid_wait(a.bar, rounds * C, ctrl, a.wait_ns, &ok_s)) return;
      const int col = c0 + tid;
      const int ctas_s = s == 0 ? a.ctasG : a.ctasF;
      const bool mine = cta < ctas_s;  // this CTA has columns on this side
      const bool active = col < (s == 0 ? a.n : a.m);
      const int epoch = 2 * t + 1 + s;
      float* const Y = s == 0 ? YG : YF;
      float* Rw = scratch + (size_t)C * P4;
      float* Red = Rw + P4;
      const int G = s == 0 ? a.ctasF : a.ctasG;
      stage_shares(s == 0 ? a.partF : a.partG, G, P4, scratch);
      sum_shares(scratch, G, P4, Rw, Red);
      form_h<PM>(Rw, p, nu, Ws, Hs);
      float y[PL], b[PL], f[PL];
#pragma unroll
      for (int c = 0; c < PL; ++c) {
        y[c] = active ? Y[c * kFs + tid] : 0.f;
        b[c] = 0.f;
      }
      if (active) {
        form_b<PL>(Ws, s == 0 ? DG : DF, nu, b);
        bool bad = false;
#pragma unroll
        for (int c = 0; c < PL; ++c) bad |= !isfinite(b[c]) || !isfinite(y[c]);
        if (bad) set_status(ctrl, NMF_ERR_NONFINITE);
      }
      // L_c by the whole block (the reduction scratch is consumed)
      lambda_max_cta<PM>(Hs, Red, lam_dg, &lam_s, p);
      __syncthreads();
      double Lc_d = lam_s;
      if (!isfinite(Lc_d)) {
        if (tid == 0) set_status(ctrl, NMF_ERR_NONFINITE);
        Lc_d = 0.0;
      }
      const float Lc = (float)Lc_d;
      int iters = 0;
#pragma unroll
      for (int c = 0; c < PL; ++c) f[c] = y[c];
      double pg2_final = 0.0;
      if (Lc > 0.f && mine) {
        constexpr bool packed = PL <= kPackedMax;
        float Hp[packed ? PL * (PL + 1) / 2 : 1];
        if constexpr (packed) load_packed<PL, PM>(Hs, Hp);
        float g[PL], fp[PL], gp[PL];
        if constexpr (packed) hmatvec_packed<PL>(Hp, y, b, g);
        else hmatvec<PM>(Hs, y, b, g);
#pragma unroll
        for (int c = 0; c < PL; ++c) {
          fp[c] = y[c];
          gp[c] = g[c];
        }
        float beta_next = __ldg(a.beta);
        int rs = 0;
        float obj_prev = 0.f;
        const float inv_Lc = 1.f / Lc;
        const float eps2_f = eps2 < 0.0 ? 0.f : __double2float_rd(eps2);  // eps^2 rounded down to float
        int stop_j = -1, nrec = 0, base = 0;  // tests: recorded in this block, decided before it
        unsigned int wfail = 0u;              // the warp's failed votes in this block (bit per test)
        bool aborted = false;
        for (int k = 0; k < a.max_inner; ++k) {
#pragma unroll
          for (int c = 0; c < PL; ++c) f[c] = fmaxf(0.f, fmaf(-g[c], inv_Lc, y[c]));
          float beta = beta_next;
          if (k + 1 < a.max_inner) beta_next = __ldg(a.beta + k + 1);
          float gf[PL];
          if constexpr (packed) hmatvec_packed<PL>(Hp, f, b, gf);
          else hmatvec<PM>(Hs, f, b, gf);
          if (RESTART) {
            float obj = 0.f, sc = 0.f;
#pragma unroll
            for (int c = 0; c < PL; ++c) {
              obj = fmaf(f[c], gf[c] - b[c], obj);
              sc = fmaf(fabsf(f[c]), fabsf(gf[c]) + fabsf(b[c]), sc);
            }
            obj *= 0.5f;
            if (k >= 1 && obj - obj_prev > kRestartTol * sc) rs = 0;
            obj_prev = obj;
            beta = __ldg(a.beta + rs);
            ++rs;
          }
#pragma unroll
          for (int c = 0; c < PL; ++c) {
            y[c] = fmaf(beta, f[c] - fp[c], f[c]);
            g[c] = fmaf(beta, gf[c] - gp[c], gf[c]);
            fp[c] = f[c];
            gp[c] = gf[c];
          }
          iters = k + 1;
          if (TEST && k + 1 >= a.min_inner) {
            if (stop_record_term<PL>(pterm, nrec, active ? pg_sq<PL>(f, gf) : 0.f, f, keep, eps2_f))
              wfail |= 1u << nrec;
            if (++nrec == kBlockP || k + 1 == a.max_inner) {
              stop_sum_terms(stop_s, nrec, pterm, wfail);
              wfail = 0u;
              // pterm is free once summed: it gathers the other CTAs' words
              const int r = stop_decide(stop_s, nrec, base, a.slots, epoch, eps2, eps2_f, ctas_s, a.withhold != 0,
                                        ctrl, a.wait_ns, pterm, kBlockP * T);
              if (r == -2) {
                aborted = true;
                break;
              }
              if (r >= 0) {
                // the first test that passed: its iterate, as the sequential rule returns it
                const float* slot = keep + (size_t)r * PL * T;
#pragma unroll
                for (int c = 0; c < PL; ++c) f[c] = slot[c * T + tid];
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
        // ||P grad||^2 of the returned iterate: only the last update's
        // reaches the statistics
        if (stop_j >= 0) pg2_final = cta == 0 ? stop_s.total : 0.0;
        else if (t == a.max_outer - 1) pg2_final = block_sum_df(active ? pg_sq<PL>(fp, gp) : 0.f, red);
      }
      // ---- outputs of the phase ----
      if (active) {
        bool bad = false;
#pragma unroll
        for (int c = 0; c < PL; ++c) {
          bad |= c < p && !isfinite(f[c]);
          Y[c * kFs + tid] = c < p ? f[c] : 0.f;
        }
        if (bad) set_status(ctrl, NMF_ERR_NONFINITE);
        if (s == 0 && a.record_G) {
#pragma unroll
          for (int c = 0; c < PL; ++c)
            if (c < p) a.record_G[((size_t)t * a.n + col) * p + c] = f[c];
        } else if (s == 1 && a.record_F) {
#pragma unroll
          for (int c = 0; c < PL; ++c)
            if (c < p) a.record_F[((size_t)t * p + c) * a.m + col] = f[c];
        }
      }
      if (tid == 0 && mine) (s == 0 ? a.pg2G : a.pg2F)[cta] = pg2_final;
      if (cta == 0 && tid == 0) {
        ctrl->iters[s] = iters;
        ctrl->lipschitz[s] = Lc;
        if (a.stats) {
          // running totals in registers: a store, not a read-modify-write whose
          // load every thread would wait for at the barrier below
          long long tot;
          if (s == 0) {
            total_inner_G += iters;
            tot = total_inner_G;
          } else {
            total_inner_F += iters;
            tot = total_inner_F;
          }
          a.stats->last_inner[s] = iters;
          a.stats->total_inner[s] = tot;
          a.stats->lipschitz[s] = Lc_d;
        }
      }
      __syncthreads();  // Ys complete
      if (mine) form_share<PM>(Y, s == 0 ? EG : EF, p, nu, P4, (s == 0 ? a.partG : a.partF) + (size_t)cta * P4);
      if (s == 1 && a.times) {
        __syncthreads();
        if (tid == 0) {
          __threadfence();
          atomicMax(a.times + t + 1, global_ns());
        }
      }
      grid_arrive(a.bar);
      ++rounds;
    }
  }
  // ---- the final factors ----
  __syncthreads();
  for (int i = tid; i < T * PM; i += NT) {
    const int t = i / PM, c = i % PM;  // consecutive threads: consecutive entries of a row of G
    if (c < p && c0 + t < a.n) a.G[(size_t)(c0 + t) * p + c] = YG[c * kFs + t];
  }
  for (int i = tid; i < PM * T; i += NT) {
    const int c = i / T, t = i % T;
    if (c < p && c0 + t < a.m) a.F[(size_t)c * a.m + c0 + t] = YF[c * kFs + t];
  }
}

template <int PM>
size_t persist_smem(int nu, int p, int ctas, bool keep_shared) {
  const size_t vecF = round_up_sz((size_t)nu * kFs, 4);
  const size_t P4 = partial_stride(p * nu);
  // staged shares, their sum, and the slice sums (reused as the eigenvalue scratch)
  size_t scratch = (size_t)ctas * P4 + P4 + std::max({(size_t)4 * kThreadsAll, P4, (size_t)2 * PM * lam_stride<PM>()});
  if (keep_shared) scratch = std::max(scratch, (size_t)kBlockP * PM * T);
  return ((size_t)2 * PM * kFs + 4 * vecF + scratch) * sizeof(float);
}

template <int PM, int PL, bool TEST, bool RESTART>
const void* persist_fn() {
  return (const void*)persist_kernel<PM, PL, TEST, RESTART>;
}

template <int PM, int PL = PM>
const void* pick(bool test, bool restart) {
  return test ? (restart ? persist_fn<PM, PL, true, true>() : persist_fn<PM, PL, true, false>())
              : (restart ? persist_fn<PM, PL, false, true>() : persist_fn<PM, PL, false, false>());
}

const void* kernel_for(int PM, int PL, bool test, bool restart) {
  switch (PM) {
    case 4: return pick<4>(test, restart);
    case 8: return PL == 6 ? pick<8, 6>(test, restart) : pick<8>(test, restart);
    case 12: return PL == 10 ? pick<12, 10>(test, restart) : pick<12>(test, restart);
    case 16: return pick<16>(test, restart);
    case 24: return pick<24>(test, restart);
    default: return pick<32>(test, restart);
  }
}

size_t smem_for(int PM, int nu, int p, int ctas, bool keep_shared) {
  switch (PM) {
    case 4: return persist_smem<4>(nu, p, ctas, keep_shared);
    case 8: return persist_smem<8>(nu, p, ctas, keep_shared);
    case 12: return persist_smem<12>(nu, p, ctas, keep_shared);
    case 16: return persist_smem<16>(nu, p, ctas, keep_shared);
    case 24: return persist_smem<24>(nu, p, ctas, keep_shared);
    default: return persist_smem<32>(nu, p, ctas, keep_shared);
  }
}

int pad_rank_p(int p) { return p <= 4 ? 4 : p <= 8 ? 8 : p <= 12 ? 12 : p <= 16 ? 16 : p <= 24 ? 24 : 32; }
// The inner loop's rank: two rows fewer than the padding where p leaves
// them zero, for the register-resident ranks 8 and 12.
int loop_rank(int p, int PM) { return (PM == 8 || PM == 12) && p <= PM - 2 ? PM - 2 : PM; }

}  // namespace

PersistPlan persist_plan(int n, int m, int p, int nu, bool test, bool restart) {
  PersistPlan pl{};
  pl.ok = false;
  const int ctasG = ceil_div(n, T), ctasF = ceil_div(m, T);
  const int C = std::max(ctasG, ctasF);
  const int P4 = partial_stride(p * nu);
  pl.ctas = C;
  pl.PM = pad_rank_p(p);
  pl.PL = loop_rank(p, pl.PM);
  if ((long)C * P4 > kMaxReduceFloats) return pl;  // every CTA reads every share: keep that small
  if (C > kMaxStopCtas) return pl;
  int dev = 0, max_smem = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return pl;
  cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const void* fn = kernel_for(pl.PM, pl.PL, test, restart);
  cudaFuncAttributes fa{};
  if (cudaFuncGetAttributes(&fa, fn) != cudaSuccess) return pl;
  // pending iterates in shared memory when they fit, else in the workspace
  pl.keep_shared = smem_for(pl.PM, nu, p, C, true) + fa.sharedSizeBytes <= (size_t)max_smem;
  pl.smem = smem_for(pl.PM, nu, p, C, pl.keep_shared);
  if (pl.smem + fa.sharedSizeBytes > (size_t)max_smem) return pl;
  if (allow_dynamic_smem(fn, (int)pl.smem) != cudaSuccess) return pl;
  int per = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, kThreadsAll, pl.smem) != cudaSuccess) return pl;
  if ((long)per * sms < C) return pl;
  pl.ok = true;
  return pl;
}

size_t persist_keep_floats(int n, int m, int p, int nu) {
  const PersistPlan pl = persist_plan(n, m, p, nu, true, false);
  return pl.ok && !pl.keep_shared ? (size_t)pl.ctas * kBlockP * pl.PM * T : 0;
}

cudaError_t persist_launch(const PersistPlan& pl, const PersistLaunch& L, cudaStream_t s) {
  PArgs a{};
  a.n = L.n;
  a.m = L.m;
  a.p = L.p;
  a.nu = L.nu;
  a.L = L.L;
  a.R = L.R;
  a.XL = L.XL;
  a.XR = L.XR;
  a.G = L.G;
  a.F = L.F;
  a.max_outer = L.max_outer;
  a.max_inner = L.max_inner;
  a.min_inner = L.min_inner;
  a.beta = L.beta;
  a.partG = L.partG;
  a.partF = L.partF;
  a.pg2G = L.pg2G;
  a.pg2F = L.pg2F;
  a.initG = L.initG;
  a.initF = L.initF;
  a.slots = L.slots;
  a.bar = L.bar;
  a.keep = pl.keep_shared ? nullptr : L.keep;
  a.record_G = L.record_G;
  a.record_F = L.record_F;
  a.times = L.times;
  a.tol = L.tol;
  a.tol_mode = L.tol_mode;
  a.stats = L.stats;
  a.ctrl = L.ctrl;
  a.wait_ns = wait_limit_ns();
  a.withhold = injected_fault() == NMF_FAULT_STOP_TEST ? 1 : 0;
  a.ctasG = ceil_div(L.n, T);
  a.ctasF = ceil_div(L.m, T);
  const bool test = L.tol > 0.0;
  const void* fn = kernel_for(pl.PM, pl.PL, test, L.restart != 0);
  cudaError_t e = allow_dynamic_smem(fn, (int)pl.smem);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(pl.ctas);
  cfg.blockDim = dim3(kThreadsAll);
  cfg.dynamicSmemBytes = pl.smem;
  cfg.stream = s;
  // cooperative: the grid barrier needs every CTA resident at once
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  count_launches(1);
  void* args[] = {&a};
  return cudaLaunchKernelExC(&cfg, fn, args);
}

}  // namespace nmf
