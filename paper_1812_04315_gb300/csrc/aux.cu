// aux.cu -- small kernels around the hot path: Gaussian sketches (Alg. 2,
// "Draw Gaussian random matrices"), the one-time bfloat16 copy of X, layout
// changes, timestamps, and the RRE of eq. (4).
#include <cuda.h>

#include <algorithm>
#include <mutex>

#include "internal.h"

namespace nmf {
namespace {

// Philox4x32-10 (Salmon et al., SC'11): round (c0..c3, k0, k1) ->
// (hi(M1 c2) ^ c1 ^ k0, lo(M1 c2), hi(M0 c0) ^ c3 ^ k1, lo(M0 c0)); the key is
// bumped by the Weyl constants before every round but the first.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
  constexpr uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u, W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k.x += W0;
      k.y += W1;
    }
    const uint32_t hi0 = __umulhi(M0, c.x), lo0 = M0 * c.x;
    const uint32_t hi1 = __umulhi(M1, c.z), lo1 = M1 * c.z;
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
  }
  return c;
}

__device__ __forceinline__ float word_to_unit(uint32_t x) {
  // ((x >> 9) + 0.5) / 2^23: 24 significant bits, exact in float32, in (0, 1).
  return ((float)(x >> 9) + 0.5f) * 1.1920928955078125e-07f;
}

__global__ void sketch_kernel(int rows, int cols, uint64_t seed, uint32_t stream_id, float* out) {
  const long long total = (long long)rows * cols;
  const long long groups = (total + 3) / 4;
  const uint2 key = make_uint2((uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32));
  for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < groups;
       g += (long long)gridDim.x * blockDim.x) {
    const uint4 w = philox4x32_10(make_uint4((uint32_t)(g & 0xffffffffu), (uint32_t)(g >> 32), stream_id, 0u), key);
    const float u0 = word_to_unit(w.x), u1 = word_to_unit(w.y), u2 = word_to_unit(w.z), u3 = word_to_unit(w.w);
    const float ra = sqrtf(-2.f * logf(u0)), rb = sqrtf(-2.f * logf(u2));
    float sa, ca, sb, cb;
    sincospif(2.f * u1, &sa, &ca);
    sincospif(2.f * u3, &sb, &cb);
    const float z[4] = {ra * ca, ra * sa, rb * cb, rb * sb};
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const long long e = 4 * g + j;
      if (e < total) out[e] = z[j];
    }
  }
}

__global__ void to_bf16_kernel(const float* X, int n, int m, __nv_bfloat16* Xb, int ldb, Control* ctrl) {
  if (call_failed(ctrl)) return;
  const long long total = (long long)n * ldb;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total / 2;
       i += (long long)gridDim.x * blockDim.x) {
    const long long e = 2 * i;
    const int r = (int)(e / ldb), c = (int)(e % ldb);  // ldb even: a pair never straddles rows
    const float a = c < m ? X[(size_t)r * m + c] : 0.f;
    const float b = c + 1 < m ? X[(size_t)r * m + c + 1] : 0.f;
    reinterpret_cast<__nv_bfloat162*>(Xb)[i] = __floats2bfloat162_rn(a, b);
  }
}

__global__ void transpose_kernel(const float* in, int R, int C, void* out, int ldo, int fmt, size_t part_stride,
                                 Control* ctrl) {
  if (ctrl && call_failed(ctrl)) return;
  __shared__ float tile[32][33];
  const int r0 = blockIdx.y * 32, c0 = blockIdx.x * 32;
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int r = r0 + i, c = c0 + threadIdx.x;
    tile[i][threadIdx.x] = (r < R && c < C) ? in[(size_t)r * C + c] : 0.f;
  }
  __syncthreads();
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int c = c0 + i, r = r0 + threadIdx.x;
    if (c < C && r < R) {
      store_op(out, (size_t)c * ldo + r, fmt, part_stride, tile[threadIdx.x][i]);
    }
  }
}

__global__ void copy_rows_kernel(const float* in, int rows, int cols, void* out, int ldo, int fmt,
                                 size_t part_stride, Control* ctrl) {
  if (ctrl && call_failed(ctrl)) return;
  const long long total = (long long)rows * cols;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(i / cols), c = (int)(i % cols);
    store_op(out, (size_t)r * ldo + c, fmt, part_stride, in[i]);
  }
}

__global__ void scale_kernel(const float* in, float* out, long long count, float alpha) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count; i += (long long)gridDim.x * blockDim.x)
    out[i] = alpha * in[i];
}

__global__ void timestamp_kernel(unsigned long long* t) {
  if (threadIdx.x == 0 && blockIdx.x == 0) *t = global_ns();
}

// RRE partials: block (bx, by) owns 256 columns and the row blocks of
// kRreRows rows by, by + gridDim.y, ... (one row block per block unless
// ceil(n / kRreRows) exceeds the grid's y limit); each thread keeps its
// column of F in registers and walks the rows; squared residuals and squared
// entries accumulate in float-float.
constexpr int kRreRows = 64;
constexpr int kRreThreads = 256;
constexpr int kRreMaxGridY = 65535;

__global__ void __launch_bounds__(kRreThreads) rre_kernel(int n, int m, int p, const float* X, const float* G,
                                                          const float* F, double* part) {
  __shared__ float Gs[kRreRows][NMF_MAX_RANK];
  __shared__ double red[2][kRreThreads / 32];
  const int j = blockIdx.x * kRreThreads + threadIdx.x;
  float f[NMF_MAX_RANK];
#pragma unroll
  for (int c = 0; c < NMF_MAX_RANK; ++c) f[c] = (j < m && c < p) ? F[(size_t)c * m + j] : 0.f;
  DF se{0.f, 0.f}, sx{0.f, 0.f};
  const int row_blocks = ceil_div(n, kRreRows);
  for (int by = blockIdx.y; by < row_blocks; by += gridDim.y) {
    const int r0 = by * kRreRows;
    const int rows = min(kRreRows, n - r0);
    __syncthreads();  // the previous row block's Gs is consumed
    for (int i = threadIdx.x; i < kRreRows * NMF_MAX_RANK; i += kRreThreads) {
      const int r = i / NMF_MAX_RANK, c = i % NMF_MAX_RANK;
      Gs[r][c] = (r < rows && c < p) ? G[(size_t)(r0 + r) * p + c] : 0.f;
    }
    __syncthreads();
    if (j < m) {
      for (int r = 0; r < rows; ++r) {
        const float x = X[(size_t)(r0 + r) * m + j];
        float gf = 0.f;
#pragma unroll
        for (int c = 0; c < NMF_MAX_RANK; ++c) gf = fmaf(Gs[r][c], f[c], gf);
        const float d = x - gf;
        df_add_product(se, d, d);
        df_add_product(sx, x, x);
      }
    }
  }
  double e = (double)se.hi + (double)se.lo, xx = (double)sx.hi + (double)sx.lo;
  e = warp_sum(e);
  xx = warp_sum(xx);
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    red[0][w] = e;
    red[1][w] = xx;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int i = 0; i < kRreThreads / 32; ++i) {
      a += red[0][i];
      b += red[1][i];
    }
    const size_t blk = (size_t)blockIdx.y * gridDim.x + blockIdx.x;
    part[2 * blk] = a;
    part[2 * blk + 1] = b;
  }
}

__global__ void rre_final_kernel(const double* part, int parts, double* out) {
  __shared__ double red[2][32];
  double a = 0.0, b = 0.0;
  for (int i = threadIdx.x; i < parts; i += 32 * 32) {
    a += part[2 * i];
    b += part[2 * i + 1];
  }
  // fixed-order tree: warp sums, then warp 0 sums the warp results
  a = warp_sum(a);
  b = warp_sum(b);
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = a;
    red[1][threadIdx.x >> 5] = b;
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    a = warp_sum(red[0][threadIdx.x]);
    b = warp_sum(red[1][threadIdx.x]);
    if (threadIdx.x == 0) {
      out[0] = a;
      out[1] = b;
    }
  }
}

int grid_for(long long work, int threads) {
  long long b = (work + threads - 1) / threads;
  if (b > 8 * 1024) b = 8 * 1024;
  return (int)(b < 1 ? 1 : b);
}

}  // namespace

cudaError_t sketch_launch(int rows, int cols, uint64_t seed, uint32_t stream_id, float* out, cudaStream_t s) {
  const long long groups = ((long long)rows * cols + 3) / 4;
  count_launches(1);
  sketch_kernel<<<grid_for(groups, 256), 256, 0, s>>>(rows, cols, seed, stream_id, out);
  return cudaGetLastError();
}

cudaError_t to_bf16_launch(const float* X, int n, int m, __nv_bfloat16* Xb, int ldb, Control* ctrl, cudaStream_t s) {
  const long long pairs = (long long)n * ldb / 2;
  count_launches(1);
  to_bf16_kernel<<<grid_for(pairs, 256), 256, 0, s>>>(X, n, m, Xb, ldb, ctrl);
  return cudaGetLastError();
}

cudaError_t transpose_launch(const float* in, int R, int C, void* out, int ldo, int fmt, Control* ctrl,
                             cudaStream_t s, size_t part_stride) {
  dim3 grid(ceil_div(C, 32), ceil_div(R, 32));
  count_launches(1);
  transpose_kernel<<<grid, dim3(32, 8), 0, s>>>(in, R, C, out, ldo, fmt, part_stride, ctrl);
  return cudaGetLastError();
}

cudaError_t copy_rows_launch(const float* in, int rows, int cols, void* out, int ldo, int fmt, Control* ctrl,
                             cudaStream_t s, size_t part_stride) {
  count_launches(1);
  copy_rows_kernel<<<grid_for((long long)rows * cols, 256), 256, 0, s>>>(in, rows, cols, out, ldo, fmt, part_stride,
                                                                          ctrl);
  return cudaGetLastError();
}

cudaError_t scale_launch(const float* in, float* out, long long count, float alpha, cudaStream_t s) {
  count_launches(1);
  scale_kernel<<<grid_for(count, 256), 256, 0, s>>>(in, out, count, alpha);
  return cudaGetLastError();
}

cudaError_t timestamp_launch(unsigned long long* t, cudaStream_t s) {
  count_launches(1);
  timestamp_kernel<<<1, 32, 0, s>>>(t);
  return cudaGetLastError();
}

int rre_parts(int n, int m) { return ceil_div(m, kRreThreads) * std::min(ceil_div(n, kRreRows), kRreMaxGridY); }

cudaError_t rre_launch(int n, int m, int p, const float* X, const float* G, const float* F, double* out, double* part,
                       int parts, cudaStream_t s) {
  dim3 grid(ceil_div(m, kRreThreads), std::min(ceil_div(n, kRreRows), kRreMaxGridY));
  count_launches(1);
  rre_kernel<<<grid, kRreThreads, 0, s>>>(n, m, p, X, G, F, part);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  count_launches(1);
  rre_final_kernel<<<1, 1024, 0, s>>>(part, parts, out);
  return cudaGetLastError();
}

}  // namespace nmf

// ---------------------------------------------------------------------------
// nmf_rre_static: nmf_rre with its partial sums in a fixed device array
// instead of a caller workspace (for callers that cannot allocate).
// ---------------------------------------------------------------------------
static __device__ __align__(256) double g_rre_static_scratch[2 * NMF_RRE_STATIC_MAX_PARTS];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_rre_static_mu;
double* g_rre_static_ptr[kMaxDevices] = {};
unsigned long long g_rre_static_ctx[kMaxDevices] = {};

// Unique id of the calling thread's current context (0 if unknown), through
// the driver entry points the runtime hands out: a cudaDeviceReset replaces
// the device's primary context, and with it the module holding the array.
unsigned long long current_context_id() {
  using GetCurrent = CUresult (*)(CUcontext*);
  using GetId = CUresult (*)(CUcontext, unsigned long long*);
  static GetCurrent get_current = nullptr;
  static GetId get_id = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_current = reinterpret_cast<GetCurrent>(f);
    f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_id = reinterpret_cast<GetId>(f);
  });
  CUcontext ctx = nullptr;
  unsigned long long id = 0;
  if (!get_current || !get_id || get_current(&ctx) != CUDA_SUCCESS || !ctx || get_id(ctx, &id) != CUDA_SUCCESS)
    return 0;
  return id;
}
}  // namespace

extern "C" nmf_status_t nmf_rre_static(nmf_stream_t stream, int n, int m, int p, const float* X, const float* G,
                                       const float* F, double* out) {
  if (n < 1 || m < 1 || p < 1 || p > NMF_MAX_RANK || !X || !G || !F || !out) return NMF_ERR_INVALID_ARG;
  const int parts = nmf::rre_parts(n, m);
  if (parts > NMF_RRE_STATIC_MAX_PARTS) return NMF_ERR_WORKSPACE;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return NMF_ERR_CUDA;
  if (dev < 0 || dev >= kMaxDevices) return NMF_ERR_UNSUPPORTED;
  double* scratch = nullptr;
  {
    // Host code cannot use the array's name as a device address: look the
    // address up with the device current, once per device and again when
    // the device's context has been replaced (after a cudaDeviceReset).
    std::lock_guard<std::mutex> lock(g_rre_static_mu);
    const unsigned long long ctx = current_context_id();
    if (!g_rre_static_ptr[dev] || (ctx != 0 && ctx != g_rre_static_ctx[dev])) {
      void* addr = nullptr;
      if (cudaGetSymbolAddress(&addr, g_rre_static_scratch) != cudaSuccess || addr == nullptr) return NMF_ERR_CUDA;
      g_rre_static_ptr[dev] = static_cast<double*>(addr);
      g_rre_static_ctx[dev] = current_context_id();  // the lookup made the primary context current
    }
    scratch = g_rre_static_ptr[dev];
  }
  if (nmf::rre_launch(n, m, p, X, G, F, out, scratch, parts, (cudaStream_t)stream) != cudaSuccess) return NMF_ERR_CUDA;
  return NMF_OK;
}
