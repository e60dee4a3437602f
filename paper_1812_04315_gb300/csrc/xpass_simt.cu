// xpass_simt.cu -- one read of X computes both products of a pass of Alg. 2:
//   Y_N = X * A   (n x nu)      and      Y_T = X^T * B   (m x nu),
// on CUDA cores in float32 (Alg. 2, the X * Q and X^T * Q steps; Alg. 1's
// X_R = X R and X_L^T = X^T L^T; plain NeNMF's X F^T and X^T G).
//
// Work split: X is cut into 64 x 64 tiles; the tile grid is cut into S_r x S_c
// rectangular regions, one per CTA. A CTA walks its region row tile by row
// tile; the N product of a row tile is complete over the region's columns and
// is written as one partial (column group cg); the T product of every column
// tile accumulates in shared memory over the region's rows and is written at
// the end as one partial (row group rg). Partials are summed later in a fixed
// order, so results are deterministic.
//
// Threads: warps 0-3 compute the N product (lane = row pair, warp = column
// block), warps 4-7 the T product (lane = X-column pair, warp = column block).
#include "internal.h"

namespace nmf {
namespace {

constexpr int kTile = 64;
constexpr int kXsStride = kTile + 1;  // padded: conflict-free row and column walks
constexpr int kSimtThreads = 256;
constexpr size_t kSimtSmemBudget = 100 * 1024;

__device__ __forceinline__ float to_f(float v) { return v; }
__device__ __forceinline__ float to_f(__nv_bfloat16 v) { return __bfloat162float(v); }

__host__ __device__ __forceinline__ int split_point(int total, int parts, int i) {
  return (int)(((long long)total * i) / parts);
}

template <typename T>
__device__ __forceinline__ void load_x_tile(float* Xs, const T* X, int ldx, int n, int m, int r0, int c0,
                                            bool vec_ok) {
  // 64 x 64 elements, 8 per thread-step.
  for (int g = threadIdx.x; g < kTile * kTile / 8; g += kSimtThreads) {
    int rr = g >> 3;
    int cc = (g & 7) * 8;
    int row = r0 + rr, col = c0 + cc;
    float v[8];
    if (row < n && vec_ok && col + 8 <= m) {
      const T* src = X + (size_t)row * ldx + col;
      if constexpr (sizeof(T) == 2) {
        uint4 raw = *reinterpret_cast<const uint4*>(src);
        const __nv_bfloat16* h = reinterpret_cast<const __nv_bfloat16*>(&raw);
#pragma unroll
        for (int j = 0; j < 8; ++j) v[j] = __bfloat162float(h[j]);
      } else {
        float4 a = *reinterpret_cast<const float4*>(src);
        float4 b = *reinterpret_cast<const float4*>(src + 4);
        v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
        v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
      }
    } else {
#pragma unroll
      for (int j = 0; j < 8; ++j)
        v[j] = (row < n && col + j < m) ? to_f(X[(size_t)row * ldx + col + j]) : 0.f;
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) Xs[rr * kXsStride + cc + j] = v[j];
  }
}

template <typename T, int NVC>
__global__ void __launch_bounds__(kSimtThreads) xpass_simt_kernel(XPassArgs a, XPassPlan pl) {
  if (call_failed(a.ctrl)) return;
  extern __shared__ float sm[];
  float* Xs = sm;                          // 64 x 65
  float* As = Xs + kTile * kXsStride;      // [k][NVC]: column k of the tile's A^T slice
  float* Bs = As + kTile * NVC;            // [r][NVC]
  float* accT = Bs + kTile * NVC;          // [region cols][NVC]
  constexpr int CPT = NVC / 4;

  const T* X = static_cast<const T*>(a.X);
  const T* opA = static_cast<const T*>(a.opA);
  const T* opB = static_cast<const T*>(a.opB);
  const int tid = threadIdx.x;
  const int rg = blockIdx.x / pl.S_c, cg = blockIdx.x % pl.S_c;
  const int rt0 = split_point(pl.tiles_r, pl.S_r, rg), rt1 = split_point(pl.tiles_r, pl.S_r, rg + 1);
  const int ct0 = split_point(pl.tiles_c, pl.S_c, cg), ct1 = split_point(pl.tiles_c, pl.S_c, cg + 1);
  const int nct = ct1 - ct0;
  const bool vec_ok = (a.ldx % 8) == 0;

  if (a.doT)
    for (int i = tid; i < nct * kTile * NVC; i += kSimtThreads) accT[i] = 0.f;

  const bool isN = tid < 128;
  const int t = tid & 127;
  const int lr = t & 31;   // row (N) or X-column (T) within the tile, plus lr + 32
  const int cb = t >> 5;   // column block of the NVC outputs

  for (int rt = rt0; rt < rt1; ++rt) {
    const int r0 = rt * kTile;
    float accN[2][CPT];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int c = 0; c < CPT; ++c) accN[i][c] = 0.f;

    for (int ct = ct0; ct < ct1; ++ct) {
      const int c0 = ct * kTile;
      __syncthreads();
      load_x_tile<T>(Xs, X, a.ldx, a.n, a.m, r0, c0, vec_ok);
      if (a.doN)
        for (int i = tid; i < NVC * kTile; i += kSimtThreads) {
          int c = i / kTile, k = i % kTile;
          As[k * NVC + c] = to_f(opA[(size_t)c * a.lda + c0 + k]);
        }
      if (a.doT && ct == ct0)
        for (int i = tid; i < NVC * kTile; i += kSimtThreads) {
          int c = i / kTile, r = i % kTile;
          Bs[r * NVC + c] = to_f(opB[(size_t)c * a.ldb + r0 + r]);
        }
      __syncthreads();
      if (isN) {
        if (a.doN) {
#pragma unroll 4
          for (int k = 0; k < kTile; ++k) {
            const float x0 = Xs[lr * kXsStride + k];
            const float x1 = Xs[(lr + 32) * kXsStride + k];
            const float* ak = As + k * NVC + cb * CPT;
#pragma unroll
            for (int c = 0; c < CPT; ++c) {
              const float av = ak[c];
              accN[0][c] = fmaf(x0, av, accN[0][c]);
              accN[1][c] = fmaf(x1, av, accN[1][c]);
            }
          }
        }
      } else if (a.doT) {
        float acc[2][CPT];
        float* at = accT + (size_t)(ct - ct0) * kTile * NVC;
#pragma unroll
        for (int c = 0; c < CPT; ++c) {
          acc[0][c] = at[lr * NVC + cb * CPT + c];
          acc[1][c] = at[(lr + 32) * NVC + cb * CPT + c];
        }
#pragma unroll 4
        for (int r = 0; r < kTile; ++r) {
          const float x0 = Xs[r * kXsStride + lr];
          const float x1 = Xs[r * kXsStride + lr + 32];
          const float* br = Bs + r * NVC + cb * CPT;
#pragma unroll
          for (int c = 0; c < CPT; ++c) {
            const float bv = br[c];
            acc[0][c] = fmaf(x0, bv, acc[0][c]);
            acc[1][c] = fmaf(x1, bv, acc[1][c]);
          }
        }
#pragma unroll
        for (int c = 0; c < CPT; ++c) {
          at[lr * NVC + cb * CPT + c] = acc[0][c];
          at[(lr + 32) * NVC + cb * CPT + c] = acc[1][c];
        }
      }
    }
    if (isN && a.doN) {
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        const int row = r0 + lr + 32 * i;
        if (row < a.n) {
          float* dst = a.partN + ((size_t)cg * a.n + row) * pl.NV + cb * CPT;
#pragma unroll
          for (int c = 0; c < CPT; ++c) dst[c] = accN[i][c];
        }
      }
    }
  }
  if (a.doT) {
    __syncthreads();
    for (int i = tid; i < nct * kTile * NVC; i += kSimtThreads) {
      const int lc = i / NVC, c = i % NVC;
      const int col = ct0 * kTile + lc;
      if (col < a.m) a.partT[((size_t)rg * a.m + col) * pl.NV + c] = accT[i];
    }
  }
}

int simt_width(int nu) { return nu <= 8 ? 8 : nu <= 16 ? 16 : nu <= 24 ? 24 : nu <= 32 ? 32 : nu <= 48 ? 48 : 64; }

size_t simt_fixed_smem(int nvc) { return (size_t)(kTile * kXsStride + 2 * kTile * nvc) * sizeof(float); }

template <typename T, int NVC>
cudaError_t launch_t(const XPassPlan& pl, const XPassArgs& a, cudaStream_t s) {
  const int maxct = ceil_div(pl.tiles_c, pl.S_c);
  size_t smem = simt_fixed_smem(NVC) + (a.doT ? (size_t)maxct * kTile * NVC * sizeof(float) : 0);
  cudaError_t e = allow_dynamic_smem((const void*)xpass_simt_kernel<T, NVC>, (int)smem);
  if (e != cudaSuccess) return e;
  count_launches(1);
  xpass_simt_kernel<T, NVC><<<pl.ctas, kSimtThreads, smem, s>>>(a, pl);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_w(const XPassPlan& pl, const XPassArgs& a, cudaStream_t s) {
  switch (simt_width(a.nu)) {
    case 8: return launch_t<T, 8>(pl, a, s);
    case 16: return launch_t<T, 16>(pl, a, s);
    case 24: return launch_t<T, 24>(pl, a, s);
    case 32: return launch_t<T, 32>(pl, a, s);
    case 48: return launch_t<T, 48>(pl, a, s);
    default: return launch_t<T, 64>(pl, a, s);
  }
}

}  // namespace

XPassPlan xpass_simt_plan(int n, int m, int nu, int num_sms) {
  XPassPlan pl{};
  pl.tile_r = pl.tile_c = kTile;
  pl.tiles_r = ceil_div(n, kTile);
  pl.tiles_c = ceil_div(m, kTile);
  pl.NV = round_up(nu, 16);
  const int nvc = simt_width(nu);
  const size_t per_ct = (size_t)kTile * nvc * sizeof(float);
  int maxct = (int)((kSimtSmemBudget - simt_fixed_smem(nvc)) / per_ct);
  if (maxct < 1) maxct = 1;
  const int target = 2 * num_sms;
  int S_c = ceil_div(pl.tiles_c, maxct);
  // square-ish regions: S_c / S_r ~ tiles_c / tiles_r
  double ideal = __builtin_sqrt((double)target * pl.tiles_c / pl.tiles_r);
  if ((int)ideal > S_c) S_c = (int)ideal;
  if (S_c > pl.tiles_c) S_c = pl.tiles_c;
  if (S_c < 1) S_c = 1;
  int S_r = target / S_c;
  if (S_r < 1) S_r = 1;
  if (S_r > pl.tiles_r) S_r = pl.tiles_r;
  pl.S_r = S_r;
  pl.S_c = S_c;
  pl.ctas = S_r * S_c;
  return pl;
}

cudaError_t xpass_simt_launch(const XPassPlan& pl, const XPassArgs& a, bool bf16, cudaStream_t s) {
  if (bf16) return launch_w<__nv_bfloat16>(pl, a, s);
  return launch_w<float>(pl, a, s);
}

}  // namespace nmf
