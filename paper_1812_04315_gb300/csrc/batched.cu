// batched.cu -- many independent compressed NeNMF problems (Alg. 1 with the
// inner loop of Sec. 2) of different sizes in one persistent launch.
//
// Every thread-block cluster (1, 2, 4 or 8 CTAs) owns a list of problems
// chosen by the host planner and runs all outer iterations of each problem,
// one problem at a time; clusters never wait on one another. Inside a
// cluster, per factor update (G first, then F, Alg. 1):
//   W      = F R (p x nu, G side) or (L G)^T (F side): every CTA forms the
//            product over its share of the summed index in shared-memory
//            chunks; the cluster's partials are summed in rank order through
//            distributed shared memory, so every CTA holds the same W;
//   H      = W W^T and L_c = lambda_max(H) (by the whole CTA);
//   loop   every thread owns whole vectors (rows of G or columns of F) and
//          runs blocks of kBlockIters Nesterov iterations on each, state in
//          registers, recording ||P grad||^2 of every iteration; after a
//          block the cluster sums those partials and finds the first
//          iteration that passes the stop test; the vectors are then re-run
//          from the block's start to that iteration (the iterates of Sec. 2
//          do not depend on the test, so the re-run reproduces them).
// Cluster barriers (release/acquire at cluster scope) order the factor
// writes of one update before the reads of the next.
#include <algorithm>
#include <array>
#include <mutex>
#include <numeric>
#include <queue>
#include <vector>

#include "internal.h"
#include "nnls_device.cuh"

namespace nmf {
namespace {

constexpr int kBlockIters = 16;
constexpr int kBatchThreads = 256;
constexpr int kBWs = NMF_MAX_SKETCH + 1;  // row stride of W in shared memory

struct BatchDesc {
  int n, m, p, nu;
  const float* L;
  const float* R;
  const float* XL;
  const float* XR;
  float* G;
  float* F;
};

struct BatchArgs {
  const BatchDesc* desc;  // [count]
  const int* order;       // problem indices, cluster after cluster
  const int* start;       // [clusters + 1]
  const float* beta;      // [max_inner]
  float* scratch;         // per cluster: scratch_stride floats
  size_t scratch_stride;
  int max_j;              // largest n or m of the batch (scratch row length)
  int pcap, nucap;        // largest padded p and largest nu of the batch (shared-memory carve)
  int max_outer, max_inner, min_inner, tol_mode, restart;
  double tol;
  nenmf_stats_t* stats;   // [count] or null
  Control* ctrl;
};

// ---- cluster primitives ----
__device__ __forceinline__ uint32_t cl_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ uint32_t cl_size() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ void cl_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ uint32_t cl_map(const void* p, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;"
               : "=r"(r)
               : "r"((uint32_t)__cvta_generic_to_shared(p)), "r"(rank));
  return r;
}
__device__ __forceinline__ float cl_ld(uint32_t addr) {
  float v;
  asm volatile("ld.shared::cluster.f32 %0, [%1];" : "=f"(v) : "r"(addr) : "memory");
  return v;
}

// One factor update's operands. The unknown's vector j has element c at
// U[c * u_c + j * u_j]; its data vector has element k at D[k * d_k + j * d_j];
// W sums V(c, i) E(i, k) over i < Jw with V(c, i) = V[c * v_c + i * v_i] and
// E(i, k) = E[i * e_i + k * e_k].
struct Side {
  int J;
  float* U;
  int u_c, u_j;
  const float* D;
  int d_k, d_j;
  int Jw;
  const float* V;
  int v_c, v_i;
  const float* E;
  int e_i, e_k;
};

struct Shared {
  float* Vs;   // [pcap][SV] chunk of V
  float* Es;   // [nucap][SV] chunk of E
  float* Wp;   // [2][pcap * nucap] this CTA's partial of W (read by the cluster)
  float* Ws;   // [pcap][kBWs]
  float* Hs;   // [pcap * pcap]
  float* Ms;   // eigenvalue scratch
  float* dg;   // [2][pcap]: diagonal of the squared iterate (lambda_max by the whole CTA)
  float2* pgc; // [2][kBlockIters] this CTA's float-float stop-test partials (read by the cluster)
  float* red;  // [warps][kBlockIters]
  float* pgt;  // [kBlockIters][threads]: each thread's ||P grad||^2 sums per iteration of the block
  double* tot; // [kBlockIters] the cluster's totals
  int SV, wstride;
};

struct PhaseOut {
  int iters;
  double lc;
  double pg2;  // ||P grad||^2 at the returned (or evaluated) iterate
  int bad;
};

// Cluster-wide float-float sum of the first `cnt` entries of every CTA's
// pgc[buf]; the totals land in S.tot (valid after the call, every thread).
__device__ void cluster_totals(Shared& S, int buf, int cnt, uint32_t CS) {
  cl_sync();
  if ((int)threadIdx.x < cnt) {
    DF t{0.f, 0.f};
    for (uint32_t r = 0; r < CS; ++r) {
      const uint32_t a = cl_map(&S.pgc[buf * kBlockIters + threadIdx.x], r);
      df_add(t, cl_ld(a), cl_ld(a + 4));
    }
    S.tot[threadIdx.x] = (double)t.hi + (double)t.lo;
  }
  __syncthreads();
}

// The CTA's float-float sum of every thread's pgt[kk], kk < cnt, into pgc[buf].
__device__ void cta_partials(Shared& S, int buf, int cnt) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int kk = 0; kk < cnt; ++kk) {
    const float v = warp_sum(S.pgt[kk * blockDim.x + threadIdx.x]);
    if (lane == 0) S.red[w * kBlockIters + kk] = v;
  }
  __syncthreads();
  if ((int)threadIdx.x < cnt) {
    DF t{0.f, 0.f};
    for (int i = 0; i < nw; ++i) df_add(t, S.red[i * kBlockIters + threadIdx.x], 0.f);
    S.pgc[buf * kBlockIters + threadIdx.x] = make_float2(t.hi, t.lo);
  }
}

__device__ __forceinline__ void clear_pgt(Shared& S) {
#pragma unroll
  for (int kk = 0; kk < kBlockIters; ++kk) S.pgt[kk * blockDim.x + threadIdx.x] = 0.f;
}

// b = W x_j for data vector j
template <int PM>
__device__ __forceinline__ void form_b(const Side& s, const float* Ws, int nu, int j, float* b) {
#pragma unroll
  for (int c = 0; c < PM; ++c) b[c] = 0.f;
  const float* x = s.D + (size_t)j * s.d_j;
  for (int k = 0; k < nu; ++k) {
    const float xk = __ldg(x + (size_t)k * s.d_k);
#pragma unroll
    for (int c = 0; c < PM; ++c) b[c] = fmaf(Ws[c * kBWs + k], xk, b[c]);
  }
}

template <int PM>
__device__ __forceinline__ void load_u(const Side& s, int p, int j, float* u) {
  const float* src = s.U + (size_t)j * s.u_j;
#pragma unroll
  for (int c = 0; c < PM; ++c) u[c] = c < p ? src[(size_t)c * s.u_c] : 0.f;
}

template <int PM>
__device__ __forceinline__ void store_u(const Side& s, int p, int j, const float* u, int& bad) {
  float* dst = s.U + (size_t)j * s.u_j;
#pragma unroll
  for (int c = 0; c < PM; ++c)
    if (c < p) {
      bad |= !isfinite(u[c]);
      dst[(size_t)c * s.u_c] = u[c];
    }
}

struct LoopState {
  float* S_in;   // [4 PM + 2][max_j] state at the block's start (blocks after the first)
  float* S_out;  // [4 PM + 2][max_j] state at the block's end
  float* res;    // [PM][max_j] iterate at the block's end (stop test on)
  int max_j;
};

// Iterations k0 .. k1-1 of the inner loop on one vector; with pgt set,
// pgt[(k - k0) * threads + tid] accumulates ||P grad(f_k)||^2. State: y (the
// extrapolated point), g = grad at y, fp and gp = previous iterate and its
// gradient; with restart on, rs (iterations since the vector's last
// restart) and objp (its previous objective); f returns the last iterate.
template <int PL, int PM>
__device__ __forceinline__ void iterate(const float* Hs, const float* b, const float* beta, float invL, int k0, int k1,
                                        float* y, float* g, float* fp, float* gp, float* f, float* pgt, int restart,
                                        int& rs, float& objp) {
  for (int k = k0; k < k1; ++k) {
#pragma unroll
    for (int c = 0; c < PL; ++c) f[c] = fmaxf(0.f, fmaf(-g[c], invL, y[c]));
    float gf[PL];
    hmatvec_rolled<PL, PM>(Hs, f, b, gf);
    float bk;
    if (restart) {
      // the vector's objective 1/2 f^T H f - b^T f = 1/2 f^T (gf - b); a rise drops the momentum
      float obj = 0.f, sc = 0.f;
#pragma unroll
      for (int c = 0; c < PL; ++c) {
        obj = fmaf(f[c], gf[c] - b[c], obj);
        sc = fmaf(fabsf(f[c]), fabsf(gf[c]) + fabsf(b[c]), sc);
      }
      obj *= 0.5f;
      if (k >= 1 && obj - objp > kRestartTol * sc) rs = 0;
      objp = obj;
      bk = __ldg(beta + rs);
      ++rs;
    } else {
      bk = __ldg(beta + k);
    }
    if (pgt) pgt[(k - k0) * blockDim.x + threadIdx.x] += pg_sq<PL>(f, gf);
#pragma unroll
    for (int c = 0; c < PL; ++c) {
      y[c] = fmaf(bk, f[c] - fp[c], f[c]);
      g[c] = fmaf(bk, gf[c] - gp[c], gf[c]);
      fp[c] = f[c];
      gp[c] = gf[c];
    }
  }
}

// One factor update (mode 0: evaluate ||P grad||^2 at the current factor;
// mode 1: the inner solve). `ph` counts phases (double buffers). PM: the
// padded rank of W, H and the saved loop state; PL <= PM: the rows of the
// per-vector arithmetic (from p on every row is an exact zero, so leaving
// out rows PL.. gives the same values).
template <int PM, int PL>
__device__ PhaseOut phase(const Side& s, int p, int nu, int mode, double eps2, const BatchArgs& A, Shared& S,
                          const LoopState& LS, int ph) {
  const uint32_t rank = cl_rank(), CS = cl_size();
  const int tid = threadIdx.x, TB = blockDim.x;
  const int buf = ph & 1;
  PhaseOut out{0, 0.0, 0.0, 0};
  __shared__ float lam_s;

  // ---- W: this CTA's share, in chunks of TB summed vectors ----
  const int NO = PM * nu;
  float* Wp = S.Wp + buf * S.wstride;
  for (int o = tid; o < NO; o += TB) Wp[o] = 0.f;
  const int i0 = (int)((long long)s.Jw * rank / CS), i1 = (int)((long long)s.Jw * (rank + 1) / CS);
  for (int ic = i0; ic < i1; ic += TB) {
    const int i = ic + tid;
    const bool ok = i < i1;
#pragma unroll
    for (int c = 0; c < PM; ++c)
      S.Vs[c * S.SV + tid] = (ok && c < p) ? __ldg(s.V + (size_t)c * s.v_c + (size_t)i * s.v_i) : 0.f;
    for (int k = 0; k < nu; ++k)
      S.Es[k * S.SV + tid] = ok ? __ldg(s.E + (size_t)i * s.e_i + (size_t)k * s.e_k) : 0.f;
    __syncthreads();
    for (int o = tid; o < NO; o += TB) {
      const int c = o / nu, k = o % nu;
      const float4* va = reinterpret_cast<const float4*>(S.Vs + c * S.SV);
      const float4* ea = reinterpret_cast<const float4*>(S.Es + k * S.SV);
      float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
      for (int t4 = 0; t4 < TB / 4; ++t4) {
        const float4 x = va[t4], z = ea[t4];
        s0 = fmaf(x.x, z.x, s0);
        s1 = fmaf(x.y, z.y, s1);
        s2 = fmaf(x.z, z.z, s2);
        s3 = fmaf(x.w, z.w, s3);
      }
      Wp[o] += (s0 + s1) + (s2 + s3);
    }
    __syncthreads();
  }
  cl_sync();  // every CTA's partial (and the factor the partials read) is complete
  for (int o = tid; o < PM * kBWs; o += TB) S.Ws[o] = 0.f;
  __syncthreads();
  for (int o = tid; o < NO; o += TB) {
    float w = 0.f;
    for (uint32_t r = 0; r < CS; ++r) w += cl_ld(cl_map(&Wp[o], r));
    S.Ws[(o / nu) * kBWs + o % nu] = w;
  }
  __syncthreads();
  for (int i = tid; i < PM * PM; i += TB) {
    const int c = i / PM, d = i % PM;
    float h = 0.f;
    for (int k = 0; k < nu; ++k) h = fmaf(S.Ws[c * kBWs + k], S.Ws[d * kBWs + k], h);
    S.Hs[i] = h;
  }
  __syncthreads();

  const int j0 = (int)((long long)s.J * rank / CS), j1 = (int)((long long)s.J * (rank + 1) / CS);
  float invL = 0.f;
  if (mode == 1) {
    // L_c by every thread of the CTA (one upper-triangle entry each per squaring)
    __shared__ double lam_d;
    const double lam = lambda_max_cta<PM>(S.Hs, S.Ms, S.dg, &lam_d, p);
    if (tid == 0) lam_s = isfinite(lam) ? (float)lam : -1.f;
    __syncthreads();
    const float Lc = lam_s;
    out.lc = Lc;
    if (!(Lc > 0.f)) {
      // H = 0 (nothing to fit) keeps the factor; a non-finite H is reported
      out.bad = Lc < 0.f;
      cl_sync();
      return out;
    }
    invL = 1.f / Lc;
  }
  const bool test = mode == 1 && eps2 > 0.0;
  const int K = mode == 1 ? A.max_inner : 0;
  const int MJ = LS.max_j;
  float* S_in = LS.S_in;
  float* S_out = LS.S_out;
  int pbuf = buf;
  int kstop = -1;
  // kind 0: ||P grad||^2 at the current factor; 1: a block of iterations;
  // 2: the block again, up to the iterate that passed the stop test.
  for (int kb = 0, kind = mode == 0 ? 0 : 1; kind == 0 || kb < K;) {
    const int k1 = kind == 0 ? 0 : min(K, kb + kBlockIters);
    const int kend = kind == 2 ? kstop + 1 : k1;
    const bool last = k1 == K;
    if (kind != 2) clear_pgt(S);
    for (int j = j0 + tid; j < j1; j += TB) {
      float b[PL], y[PL], g[PL], fp[PL], gp[PL], f[PL];
      int rs = 0;
      float objp = 0.f;
      form_b<PL>(s, S.Ws, nu, j, b);
      if (kb == 0) {
        load_u<PL>(s, p, j, y);
        hmatvec_rolled<PL, PM>(S.Hs, y, b, g);
#pragma unroll
        for (int c = 0; c < PL; ++c) {
          fp[c] = y[c];
          gp[c] = g[c];
        }
      } else {
#pragma unroll
        for (int c = 0; c < PL; ++c) {
          y[c] = S_in[(size_t)(0 * PM + c) * MJ + j];
          g[c] = S_in[(size_t)(1 * PM + c) * MJ + j];
          fp[c] = S_in[(size_t)(2 * PM + c) * MJ + j];
          gp[c] = S_in[(size_t)(3 * PM + c) * MJ + j];
        }
        rs = (int)S_in[(size_t)(4 * PM) * MJ + j];
        objp = S_in[(size_t)(4 * PM + 1) * MJ + j];
      }
      if (kind == 0) {
        S.pgt[tid] += pg_sq<PL>(y, g);
        continue;
      }
      iterate<PL, PM>(S.Hs, b, A.beta, invL, kb, kend, y, g, fp, gp, f, kind == 1 ? S.pgt : nullptr, A.restart, rs,
                      objp);
      if (kind == 2) {
        store_u<PL>(s, p, j, f, out.bad);
        continue;
      }
      if (!last) {
#pragma unroll
        for (int c = 0; c < PL; ++c) {
          S_out[(size_t)(0 * PM + c) * MJ + j] = y[c];
          S_out[(size_t)(1 * PM + c) * MJ + j] = g[c];
          S_out[(size_t)(2 * PM + c) * MJ + j] = fp[c];
          S_out[(size_t)(3 * PM + c) * MJ + j] = gp[c];
        }
        S_out[(size_t)(4 * PM) * MJ + j] = (float)rs;
        S_out[(size_t)(4 * PM + 1) * MJ + j] = objp;
      }
      if (test) {
#pragma unroll
        for (int c = 0; c < PL; ++c) LS.res[(size_t)c * MJ + j] = f[c];
      } else if (last) {
        store_u<PL>(s, p, j, f, out.bad);
      }
    }
    if (kind == 2) break;
    const int cnt = kind == 0 ? 1 : k1 - kb;
    if (kind == 0 || test || last) {
      cta_partials(S, pbuf, cnt);
      cluster_totals(S, pbuf, cnt, CS);
      pbuf ^= 1;
    }
    if (kind == 0) {
      out.pg2 = S.tot[0];
      break;
    }
    if (test)
      for (int kk = 0; kk < cnt; ++kk)
        if (kb + kk + 1 >= A.min_inner && S.tot[kk] <= eps2) {
          kstop = kb + kk;
          break;
        }
    if (kstop >= 0 || last) {
      const int kr = kstop >= 0 ? kstop : K - 1;  // the returned iterate
      out.pg2 = S.tot[kr - kb];
      out.iters = kr + 1;
      if (kstop >= 0 && kstop < k1 - 1) {
        kind = 2;  // re-run the block from its start state (S_in is intact)
        continue;
      }
      if (test)  // the block's last iterate is the result
        for (int j = j0 + tid; j < j1; j += TB) {
          float f[PL];
#pragma unroll
          for (int c = 0; c < PL; ++c) f[c] = LS.res[(size_t)c * MJ + j];
          store_u<PL>(s, p, j, f, out.bad);
        }
      break;
    }
    float* t = S_in;
    S_in = S_out;
    S_out = t;
    kb = k1;
  }
  cl_sync();  // the factor's new values are visible to the whole cluster
  return out;
}

template <int PM, int PL = PM>
__device__ void solve_problem(const BatchDesc& d, int inst, const BatchArgs& A, Shared& S, const LoopState& LS,
                              int& ph) {
  const int p = d.p, nu = d.nu;
  // G side: rows of G (n x p), data rows of X_R, W = F R
  const Side sG{d.n, d.G, 1, p, d.XR, 1, nu, d.m, d.F, d.m, 1, d.R, nu, 1};
  // F side: columns of F (p x m), data columns of X_L, W = (L G)^T
  const Side sF{d.m, d.F, d.m, 1, d.XL, d.m, 1, d.n, d.G, 1, p, d.L, 1, d.n};
  // one call site for every update (evaluations first when eps is relative)
  const int nev = (A.tol > 0.0 && A.tol_mode == NENMF_TOL_REL) ? 2 : 0;
  double eps2 = (A.tol > 0.0 && nev == 0) ? A.tol * A.tol : -1.0;
  double ev = 0.0;
  long long totG = 0, totF = 0;  // per side (no runtime-indexed arrays: they would live in local memory)
  PhaseOut lastG{}, lastF{};
  int bad = 0;
  const int steps = nev + 2 * A.max_outer;
  for (int st = 0; st < steps; ++st) {
    const int sd = st & 1;
    const bool eval = st < nev;
    const PhaseOut o = phase<PM, PL>(sd ? sF : sG, p, nu, eval ? 0 : 1, eps2, A, S, LS, ph++);
    if (eval) {
      ev += o.pg2;
      if (st == nev - 1) eps2 = A.tol * A.tol * ev;
    } else {
      if (sd) {
        totF += o.iters;
        lastF = o;
      } else {
        totG += o.iters;
        lastG = o;
      }
      bad |= o.bad;
    }
  }
  // the problem's non-finite flag, OR-ed over the cluster
  __shared__ int bad_s;
  bad = __syncthreads_or(bad);
  if (threadIdx.x == 0) bad_s = bad;
  cl_sync();
  if (threadIdx.x == 0)
    for (uint32_t r = 0; r < cl_size(); ++r) bad |= (int)__float_as_int(cl_ld(cl_map(&bad_s, r)));
  cl_sync();
  if (cl_rank() == 0 && threadIdx.x == 0) {
    if (bad) set_status(A.ctrl, NMF_ERR_NONFINITE);
    if (A.stats) {
      nenmf_stats_t* st = A.stats + inst;
      st->status = bad ? NMF_ERR_NONFINITE : NMF_OK;
      st->outer_done = A.max_outer;
      st->eps = eps2 > 0.0 ? sqrt(eps2) : 0.0;
      st->last_inner[0] = lastG.iters;
      st->last_inner[1] = lastF.iters;
      st->total_inner[0] = totG;
      st->total_inner[1] = totF;
      st->pg_norm[0] = sqrt(fmax(lastG.pg2, 0.0));
      st->pg_norm[1] = sqrt(fmax(lastF.pg2, 0.0));
      st->lipschitz[0] = lastG.lc;
      st->lipschitz[1] = lastF.lc;
    }
  }
}

// PMAX: the largest padded rank of the batch. The kernel instantiates the
// rank classes up to PMAX only, so a batch of small ranks does not pay the
// registers of the largest class.
template <int PMAX>
__global__ void __launch_bounds__(kBatchThreads, 1) batched_kernel(BatchArgs A) {
  extern __shared__ __align__(16) float dyn[];
  const int TB = blockDim.x;
  const int pc = A.pcap, nc = A.nucap;
  Shared S;
  S.SV = TB + 4;
  S.wstride = pc * nc;
  float* q = dyn;
  S.Vs = q;
  q += pc * S.SV;
  S.Es = q;
  q += nc * S.SV;
  S.Wp = q;
  q += round_up(2 * pc * nc, 4);
  S.Ws = q;
  q += round_up(pc * kBWs, 4);
  S.Hs = q;
  q += pc * pc;
  S.Ms = q;
  q += 2 * pc * (((pc / 4) & 1) ? pc : pc + 4);
  S.dg = q;
  q += 2 * pc;
  S.pgc = reinterpret_cast<float2*>(q);
  q += 4 * kBlockIters;
  S.red = q;
  q += (kBatchThreads / 32) * kBlockIters;
  S.pgt = q;
  q += kBlockIters * TB;
  S.tot = reinterpret_cast<double*>(q);

  const int cl = blockIdx.x / (int)cl_size();
  LoopState LS;
  LS.max_j = A.max_j;
  float* base = A.scratch ? A.scratch + (size_t)cl * A.scratch_stride : nullptr;
  LS.res = base;
  LS.S_in = base ? base + (size_t)pc * A.max_j : nullptr;
  LS.S_out = base ? LS.S_in + (size_t)(4 * pc + 2) * A.max_j : nullptr;
  int ph = 0;
  for (int ii = A.start[cl]; ii < A.start[cl + 1]; ++ii) {
    const int inst = A.order[ii];
    const BatchDesc d = A.desc[inst];
    // the smallest padded rank that holds p; in the classes 8 to 16 the
    // per-vector arithmetic leaves out the two padding rows when p allows
    const int pm = d.p <= 4 ? 4 : d.p <= 8 ? 8 : d.p <= 12 ? 12 : d.p <= 16 ? 16 : d.p <= 24 ? 24 : 32;
    const bool short_loop = d.p <= pm - 2;
    if (pm == 4) solve_problem<4>(d, inst, A, S, LS, ph);
    if constexpr (PMAX >= 8)
      if (pm == 8) short_loop ? solve_problem<8, 6>(d, inst, A, S, LS, ph) : solve_problem<8>(d, inst, A, S, LS, ph);
    if constexpr (PMAX >= 12)
      if (pm == 12)
        short_loop ? solve_problem<12, 10>(d, inst, A, S, LS, ph) : solve_problem<12>(d, inst, A, S, LS, ph);
    if constexpr (PMAX >= 16)
      if (pm == 16)
        short_loop ? solve_problem<16, 14>(d, inst, A, S, LS, ph) : solve_problem<16>(d, inst, A, S, LS, ph);
    if constexpr (PMAX >= 24) if (pm == 24) solve_problem<24>(d, inst, A, S, LS, ph);
    if constexpr (PMAX >= 32) if (pm == 32) solve_problem<32>(d, inst, A, S, LS, ph);
  }
  cl_sync();  // no CTA leaves while another may read its shared memory
}

// Copies up to kDescChunk descriptors (passed by value) into the workspace.
constexpr int kDescChunk = 40;
struct DescChunk {
  BatchDesc d[kDescChunk];
  int count, first;
};
__global__ void desc_upload_kernel(BatchDesc* dst, DescChunk c) {
  const int i = threadIdx.x;
  if (i < c.count) dst[c.first + i] = c.d[i];
}
constexpr int kIntChunk = 900;
struct IntChunk {
  int v[kIntChunk];
  int count, first;
};
__global__ void int_upload_kernel(int* dst, IntChunk c) {
  for (int i = threadIdx.x; i < c.count; i += blockDim.x) dst[c.first + i] = c.v[i];
}

int pad_p(int p) { return p <= 4 ? 4 : p <= 8 ? 8 : p <= 12 ? 12 : p <= 16 ? 16 : p <= 24 ? 24 : 32; }

// The instantiation for a batch whose largest padded rank is pmax.
const void* batched_fn(int pmax) {
  switch (pad_p(pmax)) {
    case 4: return (const void*)batched_kernel<4>;
    case 8: return (const void*)batched_kernel<8>;
    case 12: return (const void*)batched_kernel<12>;
    case 16: return (const void*)batched_kernel<16>;
    case 24: return (const void*)batched_kernel<24>;
    default: return (const void*)batched_kernel<32>;
  }
}

size_t batched_smem(int pcap, int nucap, int tb) {
  const size_t sv = tb + 4;
  size_t f = pcap * sv + nucap * sv + round_up(2 * pcap * nucap, 4) + round_up(pcap * kBWs, 4) + pcap * pcap;
  f += 2 * pcap * (((pcap / 4) & 1) ? pcap : pcap + 4) + 2 * pcap + 4 * kBlockIters +
       (kBatchThreads / 32) * kBlockIters + kBlockIters * tb;
  f = round_up_sz(f, 2);
  return f * sizeof(float) + kBlockIters * sizeof(double);
}

struct BatchPlan {
  int cluster = 1, threads = kBatchThreads, clusters = 0, pmax = 4, numax = 1, max_j = 1;
  std::vector<int> order, start;
  size_t scratch_stride = 0;
  double makespan = 0.0;
};

// Co-resident clusters of a given size (cached per device, size and shared memory).
int active_clusters(int cs, int pmax, int numax, int tb) {
  static std::mutex mu;
  static std::vector<std::array<int, 4>> cache;  // {dev, cs, pmax, result}
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  {
    std::lock_guard<std::mutex> g(mu);
    for (const auto& e : cache)
      if (e[0] == dev && e[1] == cs * 1000 + tb && e[2] == pmax * 100 + numax) return e[3];
  }
  const void* fn = batched_fn(pmax);
  const size_t smem = batched_smem(pmax, numax, tb);
  int n = 0;
  if (allow_dynamic_smem(fn, (int)smem) == cudaSuccess) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(cs * 64);
    cfg.blockDim = dim3(tb);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = cs;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    if (cudaOccupancyMaxActiveClusters(&n, fn, &cfg) != cudaSuccess) {
      cudaGetLastError();
      n = 0;
    }
  }
  std::lock_guard<std::mutex> g(mu);
  cache.push_back({dev, cs * 1000 + tb, pmax * 100 + numax, n});
  return n;
}

// Estimated device cycles of one problem on a cluster of `cs` CTAs: the
// inner loops and the W and B products spread over cs * threads lanes, plus
// the per-update latency (lambda_max, cluster barriers) that does not shrink.
double problem_cycles(const nenmf_problem_t& pr, const nenmf_params_t& pa, int cs, int tb) {
  const double P = pad_p(pr.p), nm = (double)pr.n + pr.m;
  const double per_outer = (pa.max_inner * (P * P + 6.0 * P) + 2.0 * pr.nu * P) * nm;
  const double lanes = (double)cs * tb;
  const double blocks = (pa.max_inner + kBlockIters - 1) / kBlockIters;
  const double sync = 9000.0 + 2500.0 * (blocks + 1) + 300.0 * cs;
  return pa.max_outer * (2.0 * per_outer / (0.5 * lanes) + 2.0 * sync) + 20000.0;
}

// Longest-processing-time assignment of problems to `clusters` clusters.
void lpt(const std::vector<double>& cost, int clusters, BatchPlan& pl) {
  const int count = (int)cost.size();
  std::vector<int> idx(count);
  std::iota(idx.begin(), idx.end(), 0);
  std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) { return cost[a] > cost[b]; });
  using Item = std::pair<double, int>;
  std::priority_queue<Item, std::vector<Item>, std::greater<Item>> heap;
  for (int c = 0; c < clusters; ++c) heap.push({0.0, c});
  std::vector<std::vector<int>> lists(clusters);
  for (int i : idx) {
    Item it = heap.top();
    heap.pop();
    lists[it.second].push_back(i);
    it.first += cost[i];
    heap.push(it);
  }
  pl.makespan = 0.0;
  while (!heap.empty()) {
    pl.makespan = std::max(pl.makespan, heap.top().first);
    heap.pop();
  }
  pl.order.clear();
  pl.start.assign(1, 0);
  for (int c = 0; c < clusters; ++c) {
    pl.order.insert(pl.order.end(), lists[c].begin(), lists[c].end());
    pl.start.push_back((int)pl.order.size());
  }
}

nmf_status_t make_plan(int count, const nenmf_problem_t* pr, const nenmf_params_t& pa,
                       const nenmf_batch_config_t* cfg, BatchPlan& pl) {
  pl.pmax = 4;
  pl.max_j = 1;
  for (int i = 0; i < count; ++i) {
    pl.pmax = std::max(pl.pmax, pad_p(pr[i].p));
    pl.numax = std::max(pl.numax, pr[i].nu);
    pl.max_j = std::max(pl.max_j, std::max(pr[i].n, pr[i].m));
  }
  const int want = cfg ? cfg->cluster : 0;
  const int tb = cfg && cfg->threads ? cfg->threads : kBatchThreads;
  if (tb != 128 && tb != kBatchThreads) return NMF_ERR_INVALID_ARG;
  std::vector<int> sizes;
  if (want > 0) sizes.push_back(want);
  else sizes = {1, 2, 4, 8};
  bool found = false;
  BatchPlan best;
  for (int cs : sizes) {
    const int act = active_clusters(cs, pl.pmax, pl.numax, tb);
    if (act <= 0) continue;
    BatchPlan cand = pl;
    cand.cluster = cs;
    cand.threads = tb;
    cand.clusters = std::min(act, std::max(1, count));
    std::vector<double> cost(count);
    for (int i = 0; i < count; ++i) cost[i] = problem_cycles(pr[i], pa, cs, tb);
    lpt(cost, cand.clusters, cand);
    if (!found || cand.makespan < best.makespan) {
      best = cand;
      found = true;
    }
  }
  if (!found) return NMF_ERR_UNSUPPORTED;
  pl = best;
  const bool test = pa.tol > 0.0;
  const bool blocks = pa.max_inner > kBlockIters;
  pl.scratch_stride = round_up_sz((size_t)(test ? pl.pmax : 0) * pl.max_j, 64) +
                      (blocks ? round_up_sz((size_t)2 * (4 * pl.pmax + 2) * pl.max_j, 64) : 0);
  if (blocks && !test) pl.scratch_stride += round_up_sz((size_t)pl.pmax * pl.max_j, 64);
  return NMF_OK;
}

struct BatchWs {
  Control* ctrl;
  float* beta;
  BatchDesc* desc;
  int* order;
  int* start;
  float* scratch;
  size_t bytes;
};

BatchWs carve_batch(void* base, int count, const BatchPlan& pl) {
  BatchWs w{};
  Carver cv(base);
  w.ctrl = cv.take<Control>(1);
  w.beta = cv.take<float>(kMaxInnerIters);
  w.desc = cv.take<BatchDesc>(std::max(count, 1));
  w.order = cv.take<int>(std::max(count, 1));
  w.start = cv.take<int>(pl.clusters + 1);
  w.scratch = cv.take<float>(pl.scratch_stride * std::max(pl.clusters, 1));
  w.bytes = cv.size();
  return w;
}

nmf_status_t check_batch(int count, const nenmf_problem_t* pr, const nenmf_params_t* pa) {
  if (count < 0 || (count > 0 && !pr) || !pa) return NMF_ERR_INVALID_ARG;
  if (pa->max_outer < 0 || pa->max_inner < 1 || pa->max_inner > kMaxInnerIters || pa->min_inner < 1 ||
      (pa->tol_mode != NENMF_TOL_REL && pa->tol_mode != NENMF_TOL_ABS))
    return NMF_ERR_INVALID_ARG;
  if (pa->record_G || pa->record_F || pa->record_time_ns) return NMF_ERR_INVALID_ARG;
  for (int i = 0; i < count; ++i) {
    const nenmf_problem_t& q = pr[i];
    if (q.mode != NENMF_COMPRESSED) return NMF_ERR_UNSUPPORTED;
    if (q.n < 1 || q.m < 1 || q.p < 1 || q.p > NMF_MAX_RANK || q.nu < q.p || q.nu > NMF_MAX_SKETCH)
      return NMF_ERR_INVALID_ARG;
    if (!q.L || !q.R || !q.XL || !q.XR) return NMF_ERR_INVALID_ARG;
  }
  return NMF_OK;
}

}  // namespace
}  // namespace nmf

using namespace nmf;

extern "C" size_t nenmf_solve_batched_workspace_size(int count, const nenmf_problem_t* problems,
                                                     const nenmf_params_t* params,
                                                     const nenmf_batch_config_t* config) {
  if (check_batch(count, problems, params) != NMF_OK) return 0;
  BatchPlan pl;
  if (make_plan(count, problems, *params, config, pl) != NMF_OK) return 0;
  return carve_batch(nullptr, count, pl).bytes;
}

extern "C" nmf_status_t nenmf_batch_plan_info(int count, const nenmf_problem_t* problems,
                                              const nenmf_params_t* params, const nenmf_batch_config_t* config,
                                              nenmf_batch_config_t* chosen, int* clusters) {
  nmf_status_t st = check_batch(count, problems, params);
  if (st != NMF_OK) return st;
  BatchPlan pl;
  st = make_plan(count, problems, *params, config, pl);
  if (st != NMF_OK) return st;
  if (chosen) {
    chosen->cluster = pl.cluster;
    chosen->threads = pl.threads;
  }
  if (clusters) *clusters = pl.clusters;
  return NMF_OK;
}

extern "C" nmf_status_t nenmf_solve_batched(nmf_stream_t stream, int count, const nenmf_problem_t* problems,
                                            float* const* G, float* const* F, const nenmf_params_t* params,
                                            const nenmf_batch_config_t* config, nenmf_stats_t* stats,
                                            void* workspace, size_t workspace_bytes) {
  nmf_status_t st = check_batch(count, problems, params);
  if (st != NMF_OK) return st;
  if (count > 0 && (!G || !F)) return NMF_ERR_INVALID_ARG;
  for (int i = 0; i < count; ++i)
    if (!G[i] || !F[i]) return NMF_ERR_INVALID_ARG;
  if (config && config->cluster != 0 && config->cluster != 1 && config->cluster != 2 && config->cluster != 4 &&
      config->cluster != 8)
    return NMF_ERR_INVALID_ARG;
  if (count == 0) return NMF_OK;
  BatchPlan pl;
  st = make_plan(count, problems, *params, config, pl);
  if (st != NMF_OK) return st;
  const BatchWs w = carve_batch(workspace, count, pl);
  if (!workspace || workspace_bytes < w.bytes || (reinterpret_cast<uintptr_t>(workspace) & 255))
    return NMF_ERR_WORKSPACE;
  cudaStream_t s = (cudaStream_t)stream;
  NMF_CU(cudaMemsetAsync(w.ctrl, 0, sizeof(Control), s));
  NMF_CU(beta_launch(w.beta, params->max_inner, s));
  for (int first = 0; first < count; first += kDescChunk) {
    DescChunk c{};
    c.first = first;
    c.count = std::min(kDescChunk, count - first);
    for (int i = 0; i < c.count; ++i) {
      const nenmf_problem_t& q = problems[first + i];
      c.d[i] = BatchDesc{q.n, q.m, q.p, q.nu, q.L, q.R, q.XL, q.XR, G[first + i], F[first + i]};
    }
    count_launches(1);
    desc_upload_kernel<<<1, kDescChunk, 0, s>>>(w.desc, c);
    NMF_CU(cudaGetLastError());
  }
  std::vector<int> ints(pl.order);
  auto upload = [&](int* dst, const std::vector<int>& v) -> cudaError_t {
    for (int first = 0; first < (int)v.size(); first += kIntChunk) {
      IntChunk c{};
      c.first = first;
      c.count = std::min(kIntChunk, (int)v.size() - first);
      for (int i = 0; i < c.count; ++i) c.v[i] = v[first + i];
      count_launches(1);
      int_upload_kernel<<<1, 256, 0, s>>>(dst, c);
      cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  };
  NMF_CU(upload(w.order, pl.order));
  NMF_CU(upload(w.start, pl.start));

  BatchArgs a{};
  a.desc = w.desc;
  a.order = w.order;
  a.start = w.start;
  a.beta = w.beta;
  a.scratch = pl.scratch_stride ? w.scratch : nullptr;
  a.scratch_stride = pl.scratch_stride;
  a.max_j = pl.max_j;
  a.pcap = pl.pmax;
  a.nucap = pl.numax;
  a.max_outer = params->max_outer;
  a.max_inner = params->max_inner;
  a.min_inner = params->min_inner;
  a.tol_mode = params->tol_mode;
  a.restart = params->restart ? 1 : 0;
  a.tol = params->tol;
  a.stats = stats;
  a.ctrl = w.ctrl;
  const void* fn = batched_fn(pl.pmax);
  const size_t smem = batched_smem(pl.pmax, pl.numax, pl.threads);
  NMF_CU(allow_dynamic_smem(fn, (int)smem));
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(pl.clusters * pl.cluster);
  cfg.blockDim = dim3(pl.threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = pl.cluster;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  void* args[] = {&a};
  count_launches(1);
  NMF_CU(cudaLaunchKernelExC(&cfg, fn, args));
  return NMF_OK;
}

// ---- measured choice of the cluster size -----------------------------------
namespace {

constexpr int kTuneCandidates[4] = {1, 2, 4, 8};
constexpr int kTuneThreads[2] = {kBatchThreads, 128};

// Scratch copies of every problem's G and F (each 256-byte aligned), then the
// largest batched-solve workspace over the candidates.
struct TuneWs {
  std::vector<float*> G, F;
  void* solve_ws;
  size_t solve_bytes;
  size_t bytes;
};

TuneWs carve_tune(void* base, int count, const nenmf_problem_t* pr, const nenmf_params_t& trial) {
  TuneWs w{};
  Carver cv(base);
  w.G.resize(count);
  w.F.resize(count);
  for (int i = 0; i < count; ++i) {
    w.G[i] = cv.take<float>((size_t)pr[i].n * pr[i].p);
    w.F[i] = cv.take<float>((size_t)pr[i].p * pr[i].m);
  }
  size_t need = 0;
  for (int c : kTuneCandidates)
    for (int tb : kTuneThreads) {
      const nenmf_batch_config_t cfg{c, tb};
      need = std::max(need, nenmf_solve_batched_workspace_size(count, pr, &trial, &cfg));
    }
  w.solve_ws = cv.take<char>(need);
  w.solve_bytes = need;
  w.bytes = cv.size();
  return w;
}

nenmf_params_t trial_params(const nenmf_params_t& pa, int trial_outer) {
  nenmf_params_t t = pa;
  t.max_outer = trial_outer;
  t.record_G = nullptr;
  t.record_F = nullptr;
  t.record_time_ns = nullptr;
  return t;
}

}  // namespace

extern "C" size_t nenmf_batch_autotune_workspace_size(int count, const nenmf_problem_t* problems,
                                                      const nenmf_params_t* params, int trial_outer) {
  if (trial_outer < 1 || count < 1 || !params) return 0;
  const nenmf_params_t t = trial_params(*params, trial_outer);
  if (check_batch(count, problems, &t) != NMF_OK) return 0;
  return carve_tune(nullptr, count, problems, t).bytes;
}

extern "C" nmf_status_t nenmf_batch_autotune(nmf_stream_t stream, int count, const nenmf_problem_t* problems,
                                             float* const* G, float* const* F, const nenmf_params_t* params,
                                             int trial_outer, nenmf_batch_config_t* best, float* trial_ms,
                                             void* workspace, size_t workspace_bytes) {
  if (trial_outer < 1 || count < 1 || !params || !best || !G || !F) return NMF_ERR_INVALID_ARG;
  const nenmf_params_t t = trial_params(*params, trial_outer);
  nmf_status_t st = check_batch(count, problems, &t);
  if (st != NMF_OK) return st;
  for (int i = 0; i < count; ++i)
    if (!G[i] || !F[i]) return NMF_ERR_INVALID_ARG;
  const TuneWs w = carve_tune(workspace, count, problems, t);
  if (!workspace || workspace_bytes < w.bytes || (reinterpret_cast<uintptr_t>(workspace) & 255))
    return NMF_ERR_WORKSPACE;
  cudaStream_t s = (cudaStream_t)stream;
  cudaEvent_t e0, e1;
  NMF_CU(cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return NMF_ERR_CUDA;
  }
  float best_ms = -1.f;
  int best_c = 0, best_t = 0;
  st = NMF_OK;
  for (int k = 0; k < 8 && st == NMF_OK; ++k) {
    const int c = kTuneCandidates[k / 2], tb = kTuneThreads[k % 2];
    const nenmf_batch_config_t cfg{c, tb};
    if (trial_ms) trial_ms[k] = -1.f;
    if (nenmf_solve_batched_workspace_size(count, problems, &t, &cfg) == 0) continue;  // not a valid plan
    // one untimed run (first-use costs), then the timed one, each from the caller's factors
    for (int rep = 0; rep < 2 && st == NMF_OK; ++rep) {
      for (int i = 0; i < count && st == NMF_OK; ++i) {
        if (cudaMemcpyAsync(w.G[i], G[i], sizeof(float) * (size_t)problems[i].n * problems[i].p,
                            cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
            cudaMemcpyAsync(w.F[i], F[i], sizeof(float) * (size_t)problems[i].p * problems[i].m,
                            cudaMemcpyDeviceToDevice, s) != cudaSuccess)
          st = NMF_ERR_CUDA;
      }
      if (st != NMF_OK) break;
      if (rep == 1 && cudaEventRecord(e0, s) != cudaSuccess) st = NMF_ERR_CUDA;
      if (st == NMF_OK)
        st = nenmf_solve_batched(stream, count, problems, w.G.data(), w.F.data(), &t, &cfg, nullptr, w.solve_ws,
                                 w.solve_bytes);
      if (st == NMF_OK && rep == 1 && cudaEventRecord(e1, s) != cudaSuccess) st = NMF_ERR_CUDA;
    }
    if (st != NMF_OK) break;
    float ms = 0.f;
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
      st = NMF_ERR_CUDA;
      break;
    }
    int dstatus = 0;
    if (cudaMemcpy(&dstatus, w.solve_ws, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) {
      st = NMF_ERR_CUDA;
      break;
    }
    if (dstatus != 0) {
      st = (nmf_status_t)dstatus;
      break;
    }
    if (trial_ms) trial_ms[k] = ms;
    if (best_ms < 0.f || ms < best_ms) {
      best_ms = ms;
      best_c = c;
      best_t = tb;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != NMF_OK) return st;
  if (best_c == 0) return NMF_ERR_UNSUPPORTED;
  best->cluster = best_c;
  best->threads = best_t;
  return NMF_OK;
}
