// stop_test.cuh -- the projected-gradient stop test of the inner loop
// (Sec. 2: stop once ||P grad(F_k)||_F <= eps) across the CTAs of a solve
// launch, shared by the per-update and the persistent solve kernels.
//
// Every bounded wait gives up after `wait_ns` nanoseconds (or when another
// CTA raised the abort flag); the caller then records
// NMF_ERR_DEVICE_TIMEOUT and leaves. `withhold` (failure-path testing only)
// makes CTA 0 never publish its words, so the other CTAs' waits run out.
#pragma once

#include "common.cuh"
#include "internal.h"

namespace nmf {

constexpr int T = kSolveThreads;
constexpr int kLag = 4;
constexpr int kKeep = kLag + 2;  // a test's iterate is kept until its decision is read (posted one iteration late)
constexpr int kPackedMax = 12;   // largest padded rank whose H the loop keeps in registers
static_assert(kStopSlots >= 2 * kLag + 1, "stop-test slots are reused after kStopSlots tests");
constexpr int kFs = T + 4;                  // column-vector rows: 16-byte aligned, rows 4 banks apart
constexpr int kWs = NMF_MAX_SKETCH + 1;     // rows of W: consecutive rows in different banks

// Sum over the block (every warp, including the collector, which adds 0), in
// float-float arithmetic (float64 is slow on this part); the result is valid
// in thread 0.
__device__ __forceinline__ double block_sum_df(float v, float2* red) {
  DF s{v, 0.f};
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float h = __shfl_xor_sync(0xffffffffu, s.hi, o), l = __shfl_xor_sync(0xffffffffu, s.lo, o);
    DF a = (lane & o) ? DF{h, l} : s;
    const DF b = (lane & o) ? s : DF{h, l};
    df_add(a, b.hi, b.lo);
    s = a;
  }
  const int w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[w] = make_float2(s.hi, s.lo);
  __syncthreads();
  DF t{0.f, 0.f};
  if (threadIdx.x == 0)
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) df_add(t, red[i].x, red[i].y);
  return (double)t.hi + (double)t.lo;
}

// Stop test. Compute warps post their ||P grad||^2 partial of test j in
// shared memory; a dedicated collector warp (warp kWarps of the CTA) sums
// them and publishes the CTA's partial as one 64-bit word (tag << 32 | float
// bits) in global memory. If the CTA's own partial already exceeds eps^2 the
// test fails everywhere (partials are nonnegative), and the collector posts
// "go on" at once; otherwise it waits until every CTA's word for test j
// carries the tag, sums them in float-float in one fixed order (identical in
// every CTA) and posts the decision in shared memory. Compute warps read the decision of
// test j at iteration j + kLag, so they never wait on global memory. A single
// relaxed 64-bit store publishes value and tag together, so no fence or
// counter is needed; tags carry the launch epoch, so words left by earlier
// launches of the same call never match. Every test has its own row of words
// (no reuse within a launch): a CTA that decides locally may run ahead of a
// CTA that still polls.
constexpr int kWarps = T / 32;          // compute warps
constexpr int kThreadsAll = T + 32;     // plus the collector warp

__device__ __forceinline__ uint32_t stop_tag(int epoch, int j) { return ((uint32_t)epoch << 16) | (uint32_t)(j + 1); }

// Shared words: (test + 1) << 32 | payload, one 64-bit store each, so a
// reader that sees the tag sees the payload with it (no fence); zeroed at
// kernel start, so nothing a previous launch left in this shared memory
// matches a tag.
struct StopShared {
  unsigned long long part[kStopSlots][kWarps];  // payload: float bits of the warp's partial
  unsigned long long dec[kStopSlots];           // payload: 1 = stop, 0 = go on
  double dec_tot[kStopSlots];                   // the total, written before dec (collector fences)
};
__device__ __forceinline__ unsigned long long stop_word(int j, uint32_t payload) {
  return ((unsigned long long)(uint32_t)(j + 1) << 32) | payload;
}

// Collector warp: processes tests 0 .. ntests-1 in order until one passes.
// Returns false on timeout or abort.
// `ctas` CTAs (0 .. ctas-1) take part; slots holds one row of ctas words per test.
__device__ inline bool collector_loop(StopShared& S, unsigned long long* slots, int ntests, int epoch,
                                      double eps2, Control* c, unsigned long long wait_ns, bool withhold,
                                      int ctas) {
  const int lane = threadIdx.x & 31;
  const unsigned long long t0 = global_ns();
  for (int j = 0; j < ntests; ++j) {
    const int sl = j % kStopSlots;
    // 1. the CTA's partial: lane w waits for warp w's word of test j
    int ok = 1;
    float pv = 0.f;
    if (lane < kWarps) {
      unsigned long long w = *((volatile unsigned long long*)&S.part[sl][lane]);
      while ((uint32_t)(w >> 32) != (uint32_t)(j + 1)) {
        if (*((volatile int*)&c->abort) || global_ns() - t0 > wait_ns) { ok = 0; break; }
        w = *((volatile unsigned long long*)&S.part[sl][lane]);
      }
      pv = __uint_as_float((uint32_t)w);
    }
    if (!__all_sync(0xffffffffu, ok)) return false;
    float own = 0.f;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) own += __shfl_sync(0xffffffffu, pv, w);  // same order in every lane
    if (lane == 0 && !(withhold && blockIdx.x == 0)) {
      const unsigned long long word =
          ((unsigned long long)stop_tag(epoch, j) << 32) | (unsigned long long)__float_as_uint(own);
      cuda::atomic_ref<unsigned long long, cuda::thread_scope_device> r(slots[(size_t)j * ctas + blockIdx.x]);
      r.store(word, cuda::memory_order_relaxed);
    }
    // Partials are nonnegative and every sum below is monotone, so the total
    // is at least this CTA's partial: when that already exceeds eps^2 the
    // test fails in every CTA, and the decision needs no other CTA's word.
    if ((double)own > eps2) {
      if (lane == 0) {
        S.dec_tot[sl] = (double)own;
        __threadfence_block();
        *((volatile unsigned long long*)&S.dec[sl]) = stop_word(j, 0u);
      }
      continue;
    }
    // 2. every CTA's partial, summed in float-float in a fixed order
    const uint32_t tag = stop_tag(epoch, j);
    DF acc{0.f, 0.f};
    for (int i = lane; i < ctas && ok; i += 32) {
      cuda::atomic_ref<const unsigned long long, cuda::thread_scope_device> r(slots[(size_t)j * ctas + i]);
      unsigned long long w = r.load(cuda::memory_order_relaxed);
      while ((uint32_t)(w >> 32) != tag) {
        if (*((volatile int*)&c->abort) || global_ns() - t0 > wait_ns) { ok = 0; break; }
        w = r.load(cuda::memory_order_relaxed);
      }
      df_add(acc, __uint_as_float((uint32_t)w), 0.f);
    }
    if (!__all_sync(0xffffffffu, ok)) return false;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float hi = __shfl_xor_sync(0xffffffffu, acc.hi, o);
      const float lo = __shfl_xor_sync(0xffffffffu, acc.lo, o);
      DF a = (lane & o) ? DF{hi, lo} : acc;  // lower lane's value first in both lanes
      const DF b = (lane & o) ? acc : DF{hi, lo};
      df_add(a, b.hi, b.lo);
      acc = a;
    }
    const double total = (double)acc.hi + (double)acc.lo;
    const int stop = total <= eps2;
    if (lane == 0) {
      S.dec_tot[sl] = total;
      __threadfence_block();
      *((volatile unsigned long long*)&S.dec[sl]) = stop_word(j, (uint32_t)stop);
    }
    if (stop) return true;
  }
  return true;
}

// A compute warp that stopped waiting for a decision records the timeout and
// raises the abort flag (unless another CTA already did), so the call fails
// loudly instead of leaving with stale outputs.
__device__ __forceinline__ void give_up(Control* c) {
  if ((threadIdx.x & 31) == 0) {
    set_status(c, NMF_ERR_DEVICE_TIMEOUT);
    *((volatile int*)&c->abort) = 1;
  }
}

// Compute warp: the collector's decision on test j if it is posted (1 =
// stop, 0 = go on), else -2; never waits.
__device__ __forceinline__ int poll_decision(StopShared& S, int j) {
  const unsigned long long w = *((volatile unsigned long long*)&S.dec[j % kStopSlots]);
  return (uint32_t)(w >> 32) == (uint32_t)(j + 1) ? (int)(w & 1ull) : -2;
}

// Compute warp: waits for the collector's decision on test j (1 = stop, 0 =
// go on, -1 = timeout or abort).
__device__ __forceinline__ int wait_decision(StopShared& S, int j, Control* c, unsigned long long wait_ns) {
  const int sl = j % kStopSlots;
  unsigned long long w = *((volatile unsigned long long*)&S.dec[sl]);
  if ((uint32_t)(w >> 32) != (uint32_t)(j + 1)) {
    const unsigned long long t0 = global_ns();
    do {
      if (*((volatile int*)&c->abort) || global_ns() - t0 > wait_ns) return -1;
      w = *((volatile unsigned long long*)&S.dec[sl]);
    } while ((uint32_t)(w >> 32) != (uint32_t)(j + 1));
  }
  return (int)(w & 1ull);
}

}  // namespace nmf
