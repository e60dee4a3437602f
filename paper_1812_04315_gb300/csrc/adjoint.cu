// adjoint.cu -- reverse-mode derivative of unrolled compressed NeNMF
// (Alg. 1 with the inner loop of Sec. 2 run for a fixed K iterations), with
// the bases L and R held fixed.
//
// Outer iterations are taken in reverse; each factor update is undone in
// the reverse of its forward order (F update, then G update):
//   W       = F R (G update) or (L G)^T (F update) from the forward's
//             checkpoints: strided product kernel, per-CTA partials summed in
//             a fixed order;
//   H, L_c  = W W^T, lambda_max(H) and its unit eigenvector v (one CTA);
//   vectors one thread per row of G (or column of F): the K forward
//             iterations are recomputed from the update's starting factor
//             (z_k and Y_k kept in scratch), then run backwards:
//               dF_k += (1 + beta_k) dY_{k+1},  dF_{k-1} -= beta_k dY_{k+1},
//               dz_k = 1[z_k > 0] dF_k,  dY_k = dz_k - H dz_k / L_c,
//               dB += dz_k / L_c,  dL_c += <Y_k - z_k, dz_k> / L_c;
//             the vector's own outputs: the cotangent of the starting factor
//             (dY_0 + dF_{-1}) and of its data vector (W^T dB);
//   W again dH = -(1/L_c) sum_k dz_k Y_k^T, dS = dH + dH^T + 2 dL_c v v^T,
//             dW = dS W + sum_j dB_j x_j^T (x_j the update's data vectors);
//   other   the other factor's cotangent gains dW through W's product:
//             dF += dW R^T (G update) or dG += L^T dW^T (F update).
#include <algorithm>

#include "internal.h"
#include "nnls_device.cuh"

namespace nmf {
namespace {

constexpr int kPT = 256;          // threads of the product kernels
constexpr int kProdCtas = 152;    // partials of one product (at most)
constexpr int kBT = 128;          // threads of the vector kernel
constexpr int kMaxOut = NMF_MAX_RANK * NMF_MAX_SKETCH;

// out[c][k] = sum_i V[c * v_c + i * v_i] * E[i * e_i + k * e_k], c < C1, k < C2
struct Prod {
  int C1, C2;
  long long Ni;
  const float* V;
  long long v_c, v_i;
  const float* E;
  long long e_i, e_k;
};

constexpr int kPS = kPT + 4;  // row stride of the product tiles (16-byte aligned rows)

// Shared memory: C1 + C2 rows of kPS floats (dynamic).
__global__ void __launch_bounds__(kPT) prod_partial_kernel(Prod a, float* part) {
  extern __shared__ __align__(16) float tiles[];
  float* Vs = tiles;
  float* Es = tiles + a.C1 * kPS;
  const int tid = threadIdx.x;
  const int NO = a.C1 * a.C2;
  constexpr int kAcc = kMaxOut / kPT;
  float acc[kAcc];
#pragma unroll
  for (int r = 0; r < kAcc; ++r) acc[r] = 0.f;
  for (long long i0 = (long long)blockIdx.x * kPT; i0 < a.Ni; i0 += (long long)gridDim.x * kPT) {
    const long long i = i0 + tid;
    const bool ok = i < a.Ni;
    for (int c = 0; c < a.C1; ++c) Vs[c * kPS + tid] = ok ? __ldg(a.V + c * a.v_c + i * a.v_i) : 0.f;
    for (int k = 0; k < a.C2; ++k) Es[k * kPS + tid] = ok ? __ldg(a.E + i * a.e_i + k * a.e_k) : 0.f;
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kAcc; ++r) {
      const int o = tid + r * kPT;
      if (o < NO) {
        const float4* x = reinterpret_cast<const float4*>(Vs + (o / a.C2) * kPS);
        const float4* z = reinterpret_cast<const float4*>(Es + (o % a.C2) * kPS);
        float s0 = 0.f, s1 = 0.f;
        for (int t4 = 0; t4 < kPT / 4; ++t4) {
          const float4 u = x[t4], w = z[t4];
          s0 = fmaf(u.x, w.x, s0);
          s1 = fmaf(u.y, w.y, s1);
          s0 = fmaf(u.z, w.z, s0);
          s1 = fmaf(u.w, w.w, s1);
        }
        acc[r] += s0 + s1;
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < kAcc; ++r) {
    const int o = tid + r * kPT;
    if (o < NO) part[(size_t)blockIdx.x * NO + o] = acc[r];
  }
}

// out[o] = sum of the parts in order
__global__ void prod_reduce_kernel(const float* part, int parts, int NO, float* out) {
  for (int o = threadIdx.x; o < NO; o += blockDim.x) {
    float s = 0.f;
    for (int q = 0; q < parts; ++q) s += part[(size_t)q * NO + o];
    out[o] = s;
  }
}

// Per-update state kept on the device.
struct Phase {
  float W[NMF_MAX_RANK * NMF_MAX_SKETCH];   // [p][nu]
  float H[NMF_MAX_RANK * NMF_MAX_RANK];     // [PM][PM], zero padded
  float v[NMF_MAX_RANK];
  float Lc;
  float pad[3];
  float dH[NMF_MAX_RANK * NMF_MAX_RANK];    // [p][p]: sum_k dz_k Y_k^T
  float dWB[NMF_MAX_RANK * NMF_MAX_SKETCH]; // [p][nu]: sum_j dB_j x_j^T
  float dW[NMF_MAX_RANK * NMF_MAX_SKETCH];  // [p][nu]
};

// H = W W^T (PM x PM, zero padded), L_c and v.
template <int PM>
__global__ void hsym_kernel(Phase* ph, int p, int nu) {
  __shared__ __align__(16) float Hs[PM * PM];
  __shared__ __align__(16) float Ms[2 * PM * lam_stride<PM>()];
  __shared__ float vs[PM];
  for (int i = threadIdx.x; i < PM * PM; i += blockDim.x) {
    const int c = i / PM, d = i % PM;
    float h = 0.f;
    if (c < p && d < p)
      for (int k = 0; k < nu; ++k) h = fmaf(ph->W[c * nu + k], ph->W[d * nu + k], h);
    Hs[i] = h;
  }
  for (int i = threadIdx.x; i < PM; i += blockDim.x) vs[i] = 0.f;
  __syncthreads();
  if (threadIdx.x < 32) {
    const double lam = lambda_max_warp<PM>(Hs, Ms, p, vs);
    __syncwarp();
    if (threadIdx.x == 0) ph->Lc = isfinite(lam) ? (float)lam : -1.f;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < PM * PM; i += blockDim.x) ph->H[i] = Hs[i];
  for (int i = threadIdx.x; i < NMF_MAX_RANK; i += blockDim.x) ph->v[i] = i < PM ? vs[i] : 0.f;
}

struct Vecs {
  int N, p, nu, K;
  const float* U0;  // the update's starting factor: element (c, j) at U0[c * u_c + j * u_j]
  long long u_c, u_j;
  float* dU;        // cotangent of the update's result in, of its start out (same layout)
  const float* D;   // data vectors: element (k, j) at D[k * d_k + j * d_j]
  long long d_k, d_j;
  float* dD;        // their cotangent (+=), same layout as D
  float* Ybuf;      // [PM][K][N]
  float* Zbuf;      // [PM][K][N]
  float* dZbuf;     // [PM][K][N]
  float* dB;        // [PM][N]
  float* dLpart;    // [gridDim.x] per-CTA partial of dL_c
  const float* beta;
  const Phase* ph;
  Control* ctrl;
};

template <int PM>
__global__ void __launch_bounds__(kBT) vec_bwd_kernel(Vecs a) {
  __shared__ __align__(16) float Hs[PM * PM];
  __shared__ float Ws[PM * (NMF_MAX_SKETCH + 1)];
  __shared__ float red[kBT / 32];
  const int tid = threadIdx.x;
  const int p = a.p, nu = a.nu, K = a.K, N = a.N;
  constexpr int WS = NMF_MAX_SKETCH + 1;
  for (int i = tid; i < PM * PM; i += kBT) Hs[i] = a.ph->H[i];
  for (int i = tid; i < PM * WS; i += kBT) {
    const int c = i / WS, k = i % WS;
    Ws[i] = (c < p && k < nu) ? a.ph->W[c * nu + k] : 0.f;
  }
  __syncthreads();
  const float Lc = a.ph->Lc;
  const int j = blockIdx.x * kBT + tid;
  float dl = 0.f;
  if (j < N) {
    const size_t KN = (size_t)K * N;
    float b[PM], dOut[PM];
#pragma unroll
    for (int c = 0; c < PM; ++c) {
      b[c] = 0.f;
      dOut[c] = c < p ? a.dU[c * a.u_c + j * a.u_j] : 0.f;
    }
    for (int k = 0; k < nu; ++k) {
      const float xk = __ldg(a.D + k * a.d_k + j * a.d_j);
#pragma unroll
      for (int c = 0; c < PM; ++c) b[c] = fmaf(Ws[c * WS + k], xk, b[c]);
    }
    float dB[PM];
#pragma unroll
    for (int c = 0; c < PM; ++c) dB[c] = 0.f;
    if (!(Lc > 0.f)) {
      // zero iterations in the forward: the update returned its start
      for (int k = 0; k < K; ++k)
#pragma unroll
        for (int c = 0; c < PM; ++c) a.dZbuf[c * KN + (size_t)k * N + j] = 0.f;
    } else {
      const float invL = 1.f / Lc;
      // forward, as the solver computes it (gradient at y by linearity)
      float y[PM], g[PM], fp[PM], gp[PM];
#pragma unroll
      for (int c = 0; c < PM; ++c) y[c] = c < p ? __ldg(a.U0 + c * a.u_c + j * a.u_j) : 0.f;
      hmatvec<PM>(Hs, y, b, g);
#pragma unroll
      for (int c = 0; c < PM; ++c) {
        fp[c] = y[c];
        gp[c] = g[c];
      }
      for (int k = 0; k < K; ++k) {
        float f[PM], gf[PM];
#pragma unroll
        for (int c = 0; c < PM; ++c) {
          const float z = fmaf(-g[c], invL, y[c]);
          a.Ybuf[c * KN + (size_t)k * N + j] = y[c];
          a.Zbuf[c * KN + (size_t)k * N + j] = z;
          f[c] = fmaxf(0.f, z);
        }
        hmatvec<PM>(Hs, f, b, gf);
        const float bk = __ldg(a.beta + k);
#pragma unroll
        for (int c = 0; c < PM; ++c) {
          y[c] = fmaf(bk, f[c] - fp[c], f[c]);
          g[c] = fmaf(bk, gf[c] - gp[c], gf[c]);
          fp[c] = f[c];
          gp[c] = gf[c];
        }
      }
      // backward
      float dFk[PM], dFm[PM], dYn[PM];
#pragma unroll
      for (int c = 0; c < PM; ++c) {
        dFk[c] = dOut[c];
        dFm[c] = 0.f;
        dYn[c] = 0.f;
      }
      for (int k = K - 1; k >= 0; --k) {
        const float bk = __ldg(a.beta + k);
        float dz[PM], zero[PM], hdz[PM];
#pragma unroll
        for (int c = 0; c < PM; ++c) {
          dFk[c] = fmaf(1.f + bk, dYn[c], dFk[c]);
          dFm[c] = fmaf(-bk, dYn[c], dFm[c]);
          const float z = a.Zbuf[c * KN + (size_t)k * N + j];
          const float yk = a.Ybuf[c * KN + (size_t)k * N + j];
          dz[c] = z > 0.f ? dFk[c] : 0.f;
          a.dZbuf[c * KN + (size_t)k * N + j] = dz[c];
          dl = fmaf(yk - z, dz[c], dl);
          zero[c] = 0.f;
        }
        hmatvec<PM>(Hs, dz, zero, hdz);
#pragma unroll
        for (int c = 0; c < PM; ++c) {
          dYn[c] = fmaf(-hdz[c], invL, dz[c]);
          dB[c] = fmaf(dz[c], invL, dB[c]);
          dFk[c] = dFm[c];
          dFm[c] = 0.f;
        }
      }
      dl *= invL;
#pragma unroll
      for (int c = 0; c < PM; ++c) dOut[c] = dYn[c] + dFk[c];
    }
    bool bad = false;
#pragma unroll
    for (int c = 0; c < PM; ++c) {
      if (c < p) {
        bad |= !isfinite(dOut[c]);
        a.dU[c * a.u_c + j * a.u_j] = dOut[c];
      }
      a.dB[(size_t)c * N + j] = dB[c];
    }
    if (bad) set_status(a.ctrl, NMF_ERR_NONFINITE);
    // cotangent of the data vector: W^T dB
    for (int k = 0; k < nu; ++k) {
      float s = 0.f;
#pragma unroll
      for (int c = 0; c < PM; ++c) s = fmaf(Ws[c * WS + k], dB[c], s);
      a.dD[k * a.d_k + j * a.d_j] += s;
    }
  }
  const float w = warp_sum(dl);
  if ((tid & 31) == 0) red[tid >> 5] = w;
  __syncthreads();
  if (tid == 0) {
    float s = 0.f;
    for (int i = 0; i < kBT / 32; ++i) s += red[i];
    a.dLpart[blockIdx.x] = s;
  }
}

// dW = dS W + dWB with dS = -(dH + dH^T) / L_c + 2 dL_c v v^T
__global__ void finalize_kernel(Phase* ph, int p, int nu, const float* dLpart, int parts) {
  __shared__ float dS[NMF_MAX_RANK * NMF_MAX_RANK];
  __shared__ float dL_s;
  const float Lc = ph->Lc;
  if (threadIdx.x == 0) {
    float s = 0.f;
    for (int q = 0; q < parts; ++q) s += dLpart[q];
    dL_s = s;
  }
  __syncthreads();
  const bool live = Lc > 0.f;
  for (int i = threadIdx.x; i < p * p; i += blockDim.x) {
    const int c = i / p, d = i % p;
    dS[i] = live ? -(ph->dH[c * p + d] + ph->dH[d * p + c]) / Lc + 2.f * dL_s * ph->v[c] * ph->v[d] : 0.f;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < p * nu; i += blockDim.x) {
    const int c = i / nu, k = i % nu;
    float s = ph->dWB[i];
    for (int d = 0; d < p; ++d) s = fmaf(dS[c * p + d], ph->W[d * nu + k], s);
    ph->dW[i] = s;
  }
}

// the other factor's cotangent: dV(c, i) += sum_k dW[c][k] E(i, k)
struct Prop {
  long long Ni;
  int p, nu;
  float* dV;
  long long v_c, v_i;
  const float* E;
  long long e_i, e_k;
};
__global__ void __launch_bounds__(kPT) propagate_kernel(Prop a, const Phase* ph) {
  __shared__ float dW[NMF_MAX_RANK * NMF_MAX_SKETCH];
  for (int i = threadIdx.x; i < a.p * a.nu; i += blockDim.x) dW[i] = ph->dW[i];
  __syncthreads();
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.Ni) return;
  float e[NMF_MAX_SKETCH];
  for (int k = 0; k < a.nu; ++k) e[k] = __ldg(a.E + i * a.e_i + k * a.e_k);
  for (int c = 0; c < a.p; ++c) {
    float s = 0.f;
    for (int k = 0; k < a.nu; ++k) s = fmaf(dW[c * a.nu + k], e[k], s);
    a.dV[c * a.v_c + i * a.v_i] += s;
  }
}

// dX[i][j] = sum_k L[k][i] dXL[k][j] + sum_k dXR[i][k] R[j][k], 32 x 32 tiles
__global__ void expand_dx_kernel(int n, int m, int nu, const float* L, const float* R, const float* dXL,
                                 const float* dXR, float* dX) {
  __shared__ float Lt[NMF_MAX_SKETCH][33], dXLt[NMF_MAX_SKETCH][33], dXRt[32][NMF_MAX_SKETCH + 1],
      Rt[32][NMF_MAX_SKETCH + 1];
  const int i0 = blockIdx.y * 32, j0 = blockIdx.x * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
  for (int k = ty; k < nu; k += 8) {
    Lt[k][tx] = i0 + tx < n ? L[(size_t)k * n + i0 + tx] : 0.f;
    dXLt[k][tx] = j0 + tx < m ? dXL[(size_t)k * m + j0 + tx] : 0.f;
  }
  for (int r = ty; r < 32; r += 8)
    for (int k = tx; k < nu; k += 32) {
      dXRt[r][k] = i0 + r < n ? dXR[(size_t)(i0 + r) * nu + k] : 0.f;
      Rt[r][k] = j0 + r < m ? R[(size_t)(j0 + r) * nu + k] : 0.f;
    }
  __syncthreads();
  for (int r = ty; r < 32; r += 8) {
    const int i = i0 + r, j = j0 + tx;
    if (i >= n || j >= m) continue;
    float s = 0.f;
    for (int k = 0; k < nu; ++k) s = fmaf(Lt[k][r], dXLt[k][tx], fmaf(dXRt[r][k], Rt[tx][k], s));
    dX[(size_t)i * m + j] = s;
  }
}

int pad_rank_b(int p) { return p <= 4 ? 4 : p <= 8 ? 8 : p <= 12 ? 12 : p <= 16 ? 16 : p <= 24 ? 24 : 32; }

struct BwdWs {
  Control* ctrl;
  float* beta;
  Phase* ph;
  float* part;    // [kProdCtas][kMaxOut]
  float* dLpart;  // [ceil(maxN / kBT)]
  float* Ybuf;
  float* Zbuf;
  float* dZbuf;
  float* dB;
  size_t bytes;
};

BwdWs carve_bwd(void* base, const nenmf_problem_t& pr, int K) {
  BwdWs w{};
  Carver cv(base);
  const int PM = pad_rank_b(pr.p);
  const size_t N = std::max(pr.n, pr.m);
  w.ctrl = cv.take<Control>(1);
  w.beta = cv.take<float>(kMaxInnerIters);
  w.ph = cv.take<Phase>(1);
  w.part = cv.take<float>((size_t)kProdCtas * kMaxOut);
  w.dLpart = cv.take<float>(ceil_div((int)N, kBT));
  w.Ybuf = cv.take<float>((size_t)PM * K * N);
  w.Zbuf = cv.take<float>((size_t)PM * K * N);
  w.dZbuf = cv.take<float>((size_t)PM * K * N);
  w.dB = cv.take<float>((size_t)PM * N);
  w.bytes = cv.size();
  return w;
}

cudaError_t run_prod(const Prod& a, float* part, float* out, cudaStream_t s) {
  const int ctas = (int)std::max(1LL, std::min<long long>(kProdCtas, (a.Ni + kPT - 1) / kPT));
  const int smem = (a.C1 + a.C2) * kPS * (int)sizeof(float);
  cudaError_t e = allow_dynamic_smem((const void*)prod_partial_kernel, smem);
  if (e != cudaSuccess) return e;
  count_launches(2);
  prod_partial_kernel<<<ctas, kPT, smem, s>>>(a, part);
  prod_reduce_kernel<<<1, 256, 0, s>>>(part, ctas, a.C1 * a.C2, out);
  return cudaGetLastError();
}

template <int PM>
cudaError_t run_vec(const Vecs& a, cudaStream_t s) {
  count_launches(1);
  vec_bwd_kernel<PM><<<ceil_div(a.N, kBT), kBT, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_vec(const Vecs& a, int PM, cudaStream_t s) {
  switch (PM) {
    case 4: return run_vec<4>(a, s);
    case 8: return run_vec<8>(a, s);
    case 12: return run_vec<12>(a, s);
    case 16: return run_vec<16>(a, s);
    case 24: return run_vec<24>(a, s);
    default: return run_vec<32>(a, s);
  }
}

cudaError_t launch_hsym(Phase* ph, int p, int nu, cudaStream_t s) {
  count_launches(1);
  switch (pad_rank_b(p)) {
    case 4: hsym_kernel<4><<<1, 256, 0, s>>>(ph, p, nu); break;
    case 8: hsym_kernel<8><<<1, 256, 0, s>>>(ph, p, nu); break;
    case 12: hsym_kernel<12><<<1, 256, 0, s>>>(ph, p, nu); break;
    case 16: hsym_kernel<16><<<1, 256, 0, s>>>(ph, p, nu); break;
    case 24: hsym_kernel<24><<<1, 256, 0, s>>>(ph, p, nu); break;
    default: hsym_kernel<32><<<1, 256, 0, s>>>(ph, p, nu); break;
  }
  return cudaGetLastError();
}

// One update undone. The update's unknown has N vectors; its W sums Jw
// vectors of the other factor (Vw) against the basis E; data vectors D.
struct Update {
  int N, Jw;
  const float* U0;
  long long u_c, u_j;
  float* dU;
  const float* D;
  long long d_k, d_j;
  float* dD;
  const float* Vw;  // other factor (as it was when the update ran)
  long long v_c, v_i;
  float* dVw;       // its cotangent
  const float* E;
  long long e_i, e_k;
};

nmf_status_t undo_update(const Update& u, int p, int nu, int K, const BwdWs& w, cudaStream_t s) {
  const int PM = pad_rank_b(p);
  NMF_CU(run_prod(Prod{p, nu, u.Jw, u.Vw, u.v_c, u.v_i, u.E, u.e_i, u.e_k}, w.part, w.ph->W, s));
  NMF_CU(launch_hsym(w.ph, p, nu, s));
  Vecs a{};
  a.N = u.N;
  a.p = p;
  a.nu = nu;
  a.K = K;
  a.U0 = u.U0;
  a.u_c = u.u_c;
  a.u_j = u.u_j;
  a.dU = u.dU;
  a.D = u.D;
  a.d_k = u.d_k;
  a.d_j = u.d_j;
  a.dD = u.dD;
  a.Ybuf = w.Ybuf;
  a.Zbuf = w.Zbuf;
  a.dZbuf = w.dZbuf;
  a.dB = w.dB;
  a.dLpart = w.dLpart;
  a.beta = w.beta;
  a.ph = w.ph;
  a.ctrl = w.ctrl;
  NMF_CU(launch_vec(a, PM, s));
  const long long KN = (long long)K * u.N;
  // sum_k dz_k Y_k^T over all vectors and iterations
  NMF_CU(run_prod(Prod{p, p, KN, w.dZbuf, KN, 1, w.Ybuf, 1, KN}, w.part, w.ph->dH, s));
  // sum_j dB_j x_j^T
  NMF_CU(run_prod(Prod{p, nu, u.N, w.dB, u.N, 1, u.D, u.d_j, u.d_k}, w.part, w.ph->dWB, s));
  count_launches(2);
  finalize_kernel<<<1, 256, 0, s>>>(w.ph, p, nu, w.dLpart, ceil_div(u.N, kBT));
  NMF_CU(cudaGetLastError());
  Prop pa{u.Jw, p, nu, u.dVw, u.v_c, u.v_i, u.E, u.e_i, u.e_k};
  propagate_kernel<<<ceil_div(u.Jw, kPT), kPT, 0, s>>>(pa, w.ph);
  NMF_CU(cudaGetLastError());
  return NMF_OK;
}

}  // namespace
}  // namespace nmf

using namespace nmf;

extern "C" size_t nenmf_backward_workspace_size(const nenmf_problem_t* pr, const nenmf_params_t* pa) {
  if (!pr || !pa || pr->mode != NENMF_COMPRESSED || pr->n < 1 || pr->m < 1 || pr->p < 1 ||
      pr->p > NMF_MAX_RANK || pr->nu < pr->p || pr->nu > NMF_MAX_SKETCH || pa->max_inner < 1 ||
      pa->max_inner > kMaxInnerIters)
    return 0;
  return carve_bwd(nullptr, *pr, pa->max_inner).bytes;
}

extern "C" nmf_status_t nenmf_backward(nmf_stream_t stream, const nenmf_problem_t* pr, const nenmf_params_t* pa,
                                       const float* G0, const float* F0, const float* record_G,
                                       const float* record_F, const float* dG_T, const float* dF_T, float* dXL,
                                       float* dXR, float* dG0, float* dF0, float* dX, void* workspace,
                                       size_t workspace_bytes) {
  if (!pr || !pa) return NMF_ERR_INVALID_ARG;
  if (pr->mode != NENMF_COMPRESSED) return NMF_ERR_UNSUPPORTED;
  const int n = pr->n, m = pr->m, p = pr->p, nu = pr->nu, T = pa->max_outer, K = pa->max_inner;
  if (n < 1 || m < 1 || p < 1 || p > NMF_MAX_RANK || nu < p || nu > NMF_MAX_SKETCH || T < 0 || K < 1 ||
      K > kMaxInnerIters || pa->tol > 0.0 || pa->restart)
    return NMF_ERR_INVALID_ARG;
  if (!pr->L || !pr->R || !pr->XL || !pr->XR || !G0 || !F0 || !dG_T || !dF_T || !dXL || !dXR || !dG0 || !dF0)
    return NMF_ERR_INVALID_ARG;
  if (T > 0 && (!record_G || !record_F)) return NMF_ERR_INVALID_ARG;
  const BwdWs w = carve_bwd(workspace, *pr, K);
  if (!workspace || workspace_bytes < w.bytes || (reinterpret_cast<uintptr_t>(workspace) & 255))
    return NMF_ERR_WORKSPACE;
  cudaStream_t s = (cudaStream_t)stream;
  NMF_CU(cudaMemsetAsync(w.ctrl, 0, sizeof(Control), s));
  NMF_CU(beta_launch(w.beta, K, s));
  NMF_CU(cudaMemcpyAsync(dG0, dG_T, sizeof(float) * n * p, cudaMemcpyDeviceToDevice, s));
  NMF_CU(cudaMemcpyAsync(dF0, dF_T, sizeof(float) * p * m, cudaMemcpyDeviceToDevice, s));
  NMF_CU(cudaMemsetAsync(dXL, 0, sizeof(float) * nu * m, s));
  NMF_CU(cudaMemsetAsync(dXR, 0, sizeof(float) * n * nu, s));
  for (int t = T - 1; t >= 0; --t) {
    const float* Gn = record_G + (size_t)t * n * p;                    // G after outer t
    const float* Go = t > 0 ? record_G + (size_t)(t - 1) * n * p : G0;  // G before
    const float* Fo = t > 0 ? record_F + (size_t)(t - 1) * p * m : F0;  // F before
    // F update: columns of F from Fo; W = (L G_new)^T; data X_L (nu x m)
    Update uf{m, n, Fo, (long long)m, 1, dF0, pr->XL, (long long)m, 1, dXL, Gn, 1, (long long)p, dG0, pr->L, 1,
              (long long)n};
    nmf_status_t st = undo_update(uf, p, nu, K, w, s);
    if (st != NMF_OK) return st;
    // G update: rows of G from Go; W = F_old R; data X_R (n x nu)
    Update ug{n, m, Go, 1, (long long)p, dG0, pr->XR, 1, (long long)nu, dXR, Fo, (long long)m, 1, dF0, pr->R,
              (long long)nu, 1};
    st = undo_update(ug, p, nu, K, w, s);
    if (st != NMF_OK) return st;
  }
  if (dX) {
    count_launches(1);
    expand_dx_kernel<<<dim3(ceil_div(m, 32), ceil_div(n, 32)), dim3(32, 8), 0, s>>>(n, m, nu, pr->L, pr->R, dXL,
                                                                                   dXR, dX);
    NMF_CU(cudaGetLastError());
  }
  return NMF_OK;
}
