// common.cuh -- helpers shared by the libnmf translation units.
//
// Status word: every call's workspace starts with a Control block whose
// `status` is the first device-detected error (0 = none). Kernels test it at
// entry and return at once when it is set, so a failed step turns the rest of
// the call into no-ops instead of computing on garbage.
//
// Grid barrier: used only by kernels launched cooperatively (all CTAs
// co-resident). Every wait is bounded by a %globaltimer deadline; on expiry the
// waiting CTA records NMF_ERR_DEVICE_TIMEOUT, raises `abort`, and returns, and
// every other CTA leaves at its next barrier.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>
#include <cuda/atomic>

#include "../../include/nmf.h"

namespace nmf {

constexpr int kStatusOk = NMF_OK;

// Device control block at the head of every workspace (256 bytes).
struct Control {
  int status;                // first device-detected error
  int abort;                 // raised when a CTA leaves a barrier early
  unsigned int bar_count;    // grid barrier arrivals
  unsigned int bar_gen;      // grid barrier generation
  int flags[8];              // per-call flags (e.g. CholeskyQR shift taken)
  double eps2;               // squared absolute stop threshold (< 0: test off)
  double scratch_d[4];
  int iters[4];              // inner iteration counts written by the solve kernels
  float lipschitz[4];
  char pad[256 - 4 * 4 - 8 * 4 - 8 - 4 * 8 - 4 * 4 - 4 * 4];
};
static_assert(sizeof(Control) == 256, "Control must be 256 bytes");

__device__ __forceinline__ void set_status(Control* c, int code) {
  atomicCAS(&c->status, 0, code);
}

__device__ __forceinline__ bool call_failed(const Control* c) {
  return *((volatile const int*)&c->status) != 0;
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Bounded grid-wide barrier. Returns false if the call must stop (timeout or
// an abort raised elsewhere); the caller then returns from the kernel.
constexpr unsigned long long kBarrierTimeoutNs = 2000000000ull;  // 2 s

__device__ __forceinline__ bool grid_barrier(Control* c) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    cuda::atomic_ref<unsigned int, cuda::thread_scope_device> gen(c->bar_gen);
    cuda::atomic_ref<unsigned int, cuda::thread_scope_device> cnt(c->bar_count);
    cuda::atomic_ref<int, cuda::thread_scope_device> abrt(c->abort);
    unsigned int g = gen.load(cuda::memory_order_acquire);
    unsigned int arrived = cnt.fetch_add(1u, cuda::memory_order_acq_rel) + 1u;
    int good = 1;
    if (arrived == gridDim.x * gridDim.y * gridDim.z) {
      cnt.store(0u, cuda::memory_order_relaxed);
      gen.store(g + 1u, cuda::memory_order_release);
    } else {
      unsigned long long t0 = global_ns();
      while (gen.load(cuda::memory_order_acquire) == g) {
        if (abrt.load(cuda::memory_order_relaxed)) { good = 0; break; }
        if (global_ns() - t0 > kBarrierTimeoutNs) {
          set_status(c, NMF_ERR_DEVICE_TIMEOUT);
          abrt.store(1, cuda::memory_order_relaxed);
          good = 0;
          break;
        }
        __nanosleep(32);
      }
    }
    if (abrt.load(cuda::memory_order_relaxed)) good = 0;
    ok = good;
  }
  __syncthreads();
  return ok != 0;
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Float-float ("double-float") accumulator: value = hi + lo with |lo| <=
// ulp(hi)/2 after renormalisation. Products enter exactly through fmaf
// (a*b = p + e with e = fma(a, b, -p)), sums through Knuth's TwoSum, giving
// about 48 significant bits at float32 throughput.
struct DF {
  float hi, lo;
};
__device__ __forceinline__ void df_add_product(DF& s, float a, float b) {
  float p = a * b;
  float e = fmaf(a, b, -p);
  float t = s.hi + p;
  float bb = t - s.hi;
  float err = (s.hi - (t - bb)) + (p - bb);
  s.hi = t;
  s.lo += err + e;
}
__device__ __forceinline__ void df_add(DF& s, float hi, float lo) {
  float t = s.hi + hi;
  float bb = t - s.hi;
  float err = (s.hi - (t - bb)) + (hi - bb);
  s.hi = t;
  s.lo += err + lo;
}
__device__ __forceinline__ void df_norm(DF& s) {
  float t = s.hi + s.lo;
  s.lo = s.lo - (t - s.hi);
  s.hi = t;
}

// Operand formats of an X pass. OP_BF16X3 holds a float32 value v as three
// bfloat16 parts p0 + p1 + p2 (p0 = bf16(v), p1 = bf16(v - p0), p2 =
// bf16(v - p0 - p1), each difference exact in float32), so |v - p0 - p1 - p2|
// <= 2^-27 |v|; part k of element i sits at i + k * part_stride.
enum OpFormat { OP_F32 = 0, OP_BF16 = 1, OP_BF16X3 = 3 };

__device__ __forceinline__ void split_bf16x3(float v, __nv_bfloat16& p0, __nv_bfloat16& p1, __nv_bfloat16& p2) {
  p0 = __float2bfloat16_rn(v);
  const float r1 = v - __bfloat162float(p0);
  p1 = __float2bfloat16_rn(r1);
  const float r2 = r1 - __bfloat162float(p1);
  p2 = __float2bfloat16_rn(r2);
}

__device__ __forceinline__ void store_op(void* out, size_t i, int fmt, size_t part_stride, float v) {
  if (fmt == OP_F32) {
    static_cast<float*>(out)[i] = v;
  } else if (fmt == OP_BF16) {
    static_cast<__nv_bfloat16*>(out)[i] = __float2bfloat16_rn(v);
  } else {
    __nv_bfloat16 p0, p1, p2;
    split_bf16x3(v, p0, p1, p2);
    __nv_bfloat16* o = static_cast<__nv_bfloat16*>(out);
    o[i] = p0;
    o[i + part_stride] = p1;
    o[i + 2 * part_stride] = p2;
  }
}

__host__ __device__ __forceinline__ int ceil_div(int a, int b) { return (a + b - 1) / b; }
__host__ __device__ __forceinline__ int round_up(int a, int b) { return ceil_div(a, b) * b; }
__host__ __device__ __forceinline__ size_t round_up_sz(size_t a, size_t b) { return (a + b - 1) / b * b; }

}  // namespace nmf
