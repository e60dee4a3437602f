// stop_test.cuh -- the projected-gradient stop test of the inner loop
// (Sec. 2: stop once ||P grad(F_k)||_F <= eps) across the CTAs of a solve
// launch, shared by the per-update and the persistent solve kernels.
//
// Tests are taken in blocks. Inside a block every iteration only records its
// test, with no branch on the outcome, so the test's arithmetic stays off
// the loop's critical path:
//   * the thread's term of ||P grad||^2, summed over the warp;
//   * a warp vote: the total of the nonnegative terms is at least every
//     single term, so when one lane's term exceeds eps^2 the test fails
//     everywhere and the warp records +inf instead of its sum;
//   * otherwise the iterate, kept in the block's slot for that test.
// After the block, warp 0 decides its tests in order: lane i sums test i's
// warp partials in a fixed order and publishes the CTA's partial as one
// tagged 64-bit word (tag << 32 | float bits) in global memory; a CTA
// partial above eps^2 fails the test at once; for the others every CTA's
// word of that test must carry the tag, and warp 0 sums them in float-float
// in one fixed order (identical in every CTA). The words are gathered test
// by test by warp 0, or, given a free shared buffer, for all those tests at
// once by the whole CTA (one round trip to L2). The first test
// whose total is <= eps^2 stops the loop: its kept iterate is returned, as
// the sequential rule returns it; the iterations run after it inside the
// block are discarded. A single relaxed 64-bit store publishes value and tag
// together, so no fence or counter is needed; tags carry the launch (or
// phase) epoch, so words left by earlier launches never match, and every
// test has its own row of words.
//
// Every bounded wait gives up after `wait_ns` nanoseconds (or when another
// CTA raised the abort flag); the CTA then records NMF_ERR_DEVICE_TIMEOUT,
// raises the abort flag and leaves. `withhold` (failure-path testing only)
// makes CTA 0 never publish its words, so the waits of the others run out.
#pragma once

#include "common.cuh"
#include "internal.h"

namespace nmf {

constexpr int T = kSolveThreads;
constexpr int kWarps = T / 32;             // warps of a solve CTA
constexpr int kThreadsAll = T;             // threads of a solve CTA
constexpr int kPackedMax = 12;             // largest padded rank whose H the loop keeps in registers
constexpr int kFs = T + 4;                 // column-vector rows: 16-byte aligned, rows 4 banks apart
constexpr int kWs = NMF_MAX_SKETCH + 1;    // rows of W: consecutive rows in different banks
constexpr int kMaxStopBlock = 16;          // largest number of tests in one block

// Sum over the block in float-float arithmetic (float64 is slow on this
// part); the result is valid in thread 0.
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

__device__ __forceinline__ uint32_t stop_tag(int epoch, int j) { return ((uint32_t)epoch << 16) | (uint32_t)(j + 1); }

struct StopShared {
  float part[kMaxStopBlock][kWarps];  // the warps' partials of the block's tests (+inf: failed by the warp's terms)
  int result;                         // the block's outcome (see stop_decide)
  unsigned int fails;                 // the tests this CTA's partial fails on its own (bit i: test i)
  int ok;                             // the gathering of the other CTAs' words completed
  double total;                       // the total of the test that passed
};

// Records test i of the current block (every thread of the CTA, every
// iteration of the block). term: this thread's ||P grad(f)||^2 share; f:
// its iterate, kept in slot i of keep ([block][PM][T]) unless the warp
// knows the test fails; eps2_f: eps^2 rounded down to float (a float term
// exceeds eps^2 exactly when it exceeds eps2_f).
template <int PM>
__device__ __forceinline__ void stop_record(StopShared& S, int i, float term, const float* f, float* keep,
                                            float eps2_f) {
  const bool fails = __any_sync(0xffffffffu, term > eps2_f);
  const float ws = warp_sum(term);
  if (!fails) {
    float* slot = keep + (size_t)i * PM * T;
#pragma unroll
    for (int k = 0; k < PM; ++k) slot[k * T + threadIdx.x] = f[k];
  }
  if ((threadIdx.x & 31) == 0) S.part[i][threadIdx.x >> 5] = fails ? __int_as_float(0x7f800000) : ws;
}

// stop_record with the warp sum left for later: the vote and the kept
// iterate as stop_record takes them, and this thread's term (+inf when its
// warp fails the test, so that the later warp sum is +inf as stop_record
// records it) in pterm[i][T].
// Returns the warp's vote (true: the test fails in this warp).
template <int PM>
__device__ __forceinline__ bool stop_record_term(float* pterm, int i, float term, const float* f, float* keep,
                                                 float eps2_f) {
  const bool fails = __any_sync(0xffffffffu, term > eps2_f);
  if (!fails) {
    float* slot = keep + (size_t)i * PM * T;
#pragma unroll
    for (int k = 0; k < PM; ++k) slot[k * T + threadIdx.x] = f[k];
  }
  pterm[i * T + threadIdx.x] = fails ? __int_as_float(0x7f800000) : term;
  return fails;
}

// The warp sums of the block's nb tests recorded by stop_record_term, into
// S.part (the values stop_record writes): all kMaxStopBlock sums advance
// together through warp_sum's butterfly (the same steps per value, so the
// same sums), their shuffles interleaved. failed: bit i set when the warp's
// vote failed test i (warp-uniform); when every test failed, each sum is
// +inf (every lane recorded +inf) and is written as such.
__device__ __forceinline__ void stop_sum_terms(StopShared& S, int nb, const float* pterm, unsigned int failed) {
  const unsigned int all = (1u << nb) - 1u;
  if ((failed & all) == all) {
    if ((threadIdx.x & 31) == 0)
      for (int i = 0; i < nb; ++i) S.part[i][threadIdx.x >> 5] = __int_as_float(0x7f800000);
    return;
  }
  float v[kMaxStopBlock];
#pragma unroll
  for (int i = 0; i < kMaxStopBlock; ++i) v[i] = i < nb ? pterm[i * T + threadIdx.x] : 0.f;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
#pragma unroll
    for (int i = 0; i < kMaxStopBlock; ++i) v[i] += __shfl_xor_sync(0xffffffffu, v[i], o);
  if ((threadIdx.x & 31) == 0)
#pragma unroll
    for (int i = 0; i < kMaxStopBlock; ++i)
      if (i < nb) S.part[i][threadIdx.x >> 5] = v[i];
}

// Every CTA's word of the tests not in `fails` (nb tests, ctas words each)
// into stage[i * ctas + q] as floats, all loads of a thread in flight
// together: one round trip to L2 instead of one per test. False when a wait
// gave up (in every thread).
__device__ inline bool stop_stage_words(const unsigned long long* slots, int nb, int base, int epoch, int ctas,
                                        unsigned int fails, float* stage, Control* c, unsigned long long wait_ns,
                                        int* ok_s) {
  constexpr int kInFlight = 8;
  const int NT = blockDim.x, total = nb * ctas;
  unsigned long long t0 = 0ull;  // the clock is read only once a word is found missing
  bool ok = true;
  for (int i0 = threadIdx.x; i0 < total && ok; i0 += kInFlight * NT) {
    unsigned long long w[kInFlight];
#pragma unroll
    for (int u = 0; u < kInFlight; ++u) {
      const int idx = i0 + u * NT;
      w[u] = 0ull;
      if (idx < total && !((fails >> (idx / ctas)) & 1u)) {
        cuda::atomic_ref<const unsigned long long, cuda::thread_scope_device> r(slots[(size_t)base * ctas + idx]);
        w[u] = r.load(cuda::memory_order_relaxed);
      }
    }
#pragma unroll
    for (int u = 0; u < kInFlight; ++u) {
      const int idx = i0 + u * NT;
      if (idx >= total) continue;
      const int i = idx / ctas;
      if ((fails >> i) & 1u) continue;
      const uint32_t tag = stop_tag(epoch, base + i);
      cuda::atomic_ref<const unsigned long long, cuda::thread_scope_device> r(slots[(size_t)base * ctas + idx]);
      while ((uint32_t)(w[u] >> 32) != tag) {
        if (t0 == 0ull) t0 = global_ns();
        if (*((volatile int*)&c->abort) || global_ns() - t0 > wait_ns) {
          ok = false;
          break;
        }
        w[u] = r.load(cuda::memory_order_relaxed);
      }
      if (!ok) break;
      stage[idx] = __uint_as_float((uint32_t)w[u]);
    }
  }
  if (threadIdx.x == 0) *ok_s = 1;
  __syncthreads();
  if (!ok) *ok_s = 0;
  __syncthreads();
  return *ok_s != 0;
}

// Decides the nb tests base .. base+nb-1 just recorded (every thread calls
// it; block barriers only). `ctas` CTAs (0 .. ctas-1) take part; slots holds
// one row of ctas words per test. Returns the block index of the first test
// that passed (its iterate is in keep slot i; S.total holds its total), -1
// when none did, -2 when a wait gave up (status and abort flag are set).
// With `stage` (stage_cap floats of shared memory, free during the call) and
// nb * ctas <= stage_cap, the other CTAs' words of every undecided test are
// gathered at once by the whole block before warp 0 sums them; otherwise
// warp 0 gathers them test by test. Both take the same sums in the same
// order, so the outcome and the totals are the same.
__device__ inline int stop_decide(StopShared& S, int nb, int base, unsigned long long* slots, int epoch, double eps2,
                                  float eps2_f, int ctas, bool withhold, Control* c, unsigned long long wait_ns,
                                  float* stage = nullptr, int stage_cap = 0) {
  __syncthreads();  // the block's partials are in S.part
  const bool staged = stage != nullptr && nb * ctas <= stage_cap;
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    float own = 0.f;
    if (lane < nb) {
      // this CTA's partial of test base + lane: its warps' partials in order
#pragma unroll
      for (int w = 0; w < kWarps; ++w) own += S.part[lane][w];
      if (!(withhold && blockIdx.x == 0)) {
        const unsigned long long word =
            ((unsigned long long)stop_tag(epoch, base + lane) << 32) | (unsigned long long)__float_as_uint(own);
        cuda::atomic_ref<unsigned long long, cuda::thread_scope_device> r(
            slots[(size_t)(base + lane) * ctas + blockIdx.x]);
        r.store(word, cuda::memory_order_relaxed);
      }
    }
    // A CTA partial above eps^2 fails the test in every CTA (partials are
    // nonnegative and the sums below monotone): no other CTA's word needed.
    const unsigned int fails = __ballot_sync(0xffffffffu, lane < nb && own > eps2_f);
    if (lane == 0) S.fails = fails;
  }
  if (staged) {
    __syncthreads();
    const unsigned int fails = S.fails;
    if ((~fails & ((1u << nb) - 1u)) == 0u) return -1;  // every test failed on this CTA's own partial
    if (!stop_stage_words(slots, nb, base, epoch, ctas, fails, stage, c, wait_ns, &S.ok)) {
      if (threadIdx.x == 0) {
        S.result = -2;
        set_status(c, NMF_ERR_DEVICE_TIMEOUT);
        *((volatile int*)&c->abort) = 1;
      }
      __syncthreads();
      return -2;
    }
    if (threadIdx.x < 32) {
      const int lane = threadIdx.x;
      int result = -1;
      double total = 0.0;
      for (int i = 0; i < nb; ++i) {
        if ((fails >> i) & 1u) continue;
        // every CTA's partial of test base + i, summed in float-float in a fixed order
        DF acc{0.f, 0.f};
        for (int q = lane; q < ctas; q += 32) df_add(acc, stage[i * ctas + q], 0.f);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          const float hi = __shfl_xor_sync(0xffffffffu, acc.hi, o);
          const float lo = __shfl_xor_sync(0xffffffffu, acc.lo, o);
          DF a = (lane & o) ? DF{hi, lo} : acc;  // lower lane's value first in both lanes
          const DF b = (lane & o) ? acc : DF{hi, lo};
          df_add(a, b.hi, b.lo);
          acc = a;
        }
        const double tot = (double)acc.hi + (double)acc.lo;
        if (tot <= eps2) {
          result = i;
          total = tot;
          break;
        }
      }
      if (lane == 0) {
        S.result = result;
        S.total = total;
      }
    }
    __syncthreads();
    return S.result;
  }
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    __syncwarp();  // lane 0's S.fails
    const unsigned int fails = S.fails;
    int result = -1;
    double total = 0.0;
    for (int i = 0; i < nb; ++i) {
      if ((fails >> i) & 1u) continue;
      // every CTA's partial of test base + i, summed in float-float in a fixed order
      const uint32_t tag = stop_tag(epoch, base + i);
      const unsigned long long* row = slots + (size_t)(base + i) * ctas;
      unsigned long long t0 = 0ull;  // the clock is read only once a word is found missing
      int ok = 1;
      DF acc{0.f, 0.f};
      for (int q = lane; q < ctas && ok; q += 32) {
        cuda::atomic_ref<const unsigned long long, cuda::thread_scope_device> r(row[q]);
        unsigned long long w = r.load(cuda::memory_order_relaxed);
        while ((uint32_t)(w >> 32) != tag) {
          if (t0 == 0ull) t0 = global_ns();
          if (*((volatile int*)&c->abort) || global_ns() - t0 > wait_ns) {
            ok = 0;
            break;
          }
          w = r.load(cuda::memory_order_relaxed);
        }
        df_add(acc, __uint_as_float((uint32_t)w), 0.f);
      }
      if (!__all_sync(0xffffffffu, ok)) {
        result = -2;
        break;
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const float hi = __shfl_xor_sync(0xffffffffu, acc.hi, o);
        const float lo = __shfl_xor_sync(0xffffffffu, acc.lo, o);
        DF a = (lane & o) ? DF{hi, lo} : acc;  // lower lane's value first in both lanes
        const DF b = (lane & o) ? acc : DF{hi, lo};
        df_add(a, b.hi, b.lo);
        acc = a;
      }
      const double tot = (double)acc.hi + (double)acc.lo;
      if (tot <= eps2) {
        result = i;
        total = tot;
        break;
      }
    }
    if (lane == 0) {
      S.result = result;
      S.total = total;
      if (result == -2) {
        set_status(c, NMF_ERR_DEVICE_TIMEOUT);
        *((volatile int*)&c->abort) = 1;
      }
    }
  }
  __syncthreads();
  return S.result;
}

}  // namespace nmf
