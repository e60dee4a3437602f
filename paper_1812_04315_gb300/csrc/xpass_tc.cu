// xpass_tc.cu -- one pass over a bfloat16 X on the tcgen05 tensor cores:
//   Y_N = X * A (n x nu) and Y_T = X^T * B (m x nu) from a single read of X,
// the two products of every pass of Alg. 2 (and Alg. 1's X R, X^T L^T, plain
// NeNMF's X F^T, X^T G).
//
// Tiles. X is cut into 128 x 128 tiles; a CTA owns a rectangle of tiles
// (row tiles rt0..rt1, column tiles ct0..ct1) and walks it row by row. The
// bfloat16 copy of X is stored tile by tile, each tile already in the byte
// order the MMAs read from shared memory (two 128 x 64 boxes, 128-byte
// swizzle), so a tile is one contiguous 32 KB bulk copy. One X tile lands in
// shared memory once and feeds two MMAs:
//   N product: D_N[128 rows x NV] += X_tile (K-major, K = tile columns) * A^T tile
//   T product: D_T[ct][128 cols x NV] += X_tile^T (MN-major view of the same
//              bytes, K = tile rows) * B^T tile
// D_N (double buffered) completes at the end of a row of tiles and is drained
// by the epilogue warps as one partial of the CTA's column group; every D_T[ct]
// accumulates over the CTA's row tiles in TMEM and is drained at the end as
// one partial of its row group. Partials are summed in a fixed order later.
// The epilogue stages each warp's 32 rows in shared memory so that its global
// stores cover whole 128-byte lines.
//
// Warps: 0 = TMA producer, 1 = MMA issuer (and TMEM owner), 2..5 = epilogue
// (TMEM lane quarter = warp % 4). Every mbarrier wait is bounded; on expiry
// the CTA records NMF_ERR_DEVICE_TIMEOUT, stops issuing work, waits (bounded)
// for its own copies in flight, frees its TMEM and exits.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <mutex>

#include "internal.h"

namespace nmf {
namespace {

constexpr int kTM = 128;             // tile rows (M of the N product)
constexpr int kTK = 128;             // tile columns (M of the T product)
constexpr int kBoxK = 64;            // bf16 elements per 128-byte swizzle row
constexpr int kMaxStages = 4;
constexpr int kThreads = 192;
constexpr size_t kSmemBudget = 220 * 1024;
constexpr int kXStageBytes = kTM * kTK * 2;  // 32 KB
constexpr uint32_t kMaxTmemCols = 512;
constexpr int kStg = 36;                     // floats per staged row (16-byte rows, 4 banks apart)
constexpr int kStageArea = 4 * 32 * kStg * 4;  // epilogue staging: 4 warps x 32 rows

struct TcParams {
  const uint8_t* Xt;  // bfloat16 tiles, tile (rt, ct) at byte (rt * tiles_c + ct) * kXStageBytes
  int n, m, stages;
  int tiles_r, tiles_c, S_r, S_c;
  int doN, doT;
  float* partN;
  float* partT;
  Control* ctrl;
  uint32_t tmem_cols;
  unsigned long long wait_ns;  // limit of every bounded wait
  int withhold;                // failure-path testing: CTA 0 arms its first stage and issues no copy
};

__host__ __device__ __forceinline__ int split_point(int total, int parts, int i) {
  return (int)(((long long)total * i) / parts);
}

// ---- PTX wrappers ---------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}
__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n\t.reg .pred P1;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 P1, [%1], %2;\n\t"
      "selp.b32 %0, 1, 0, P1;\n\t}"
      : "=r"(done)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return done != 0;
}
// Bounded wait: false when the deadline passed or the CTA is aborting.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag,
                                          unsigned long long wait_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = global_ns();  // the clock is read only for a wait that did not end at once
  while (!mbar_try_wait(bar, parity)) {
    if (*abort_flag) return false;
    if (global_ns() - t0 > wait_ns) {
      *abort_flag = 1;
      return false;
    }
  }
  return true;
}
// Bounded wait that ignores the abort flag (draining work already in flight).
__device__ __forceinline__ void mbar_drain(uint64_t* bar, uint32_t parity, unsigned long long wait_ns) {
  const unsigned long long t0 = global_ns();
  while (!mbar_try_wait(bar, parity) && global_ns() - t0 < wait_ns) {
  }
}
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::"r"(
          smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(x), "r"(y)
      : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                       uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float* v) {
  uint32_t r[8];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Shared-memory matrix descriptor (tcgen05): start, leading and stride byte
// offsets (>> 4), descriptor version 1, 128-byte swizzle (layout type 2).
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFF);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}
// Instruction descriptor, kind::f16: fp32 accumulate, bf16 A and B,
// A major-ness (0 = K-major, 1 = MN-major), B K-major, N >> 3, M >> 4.
__host__ __device__ constexpr uint32_t instr_desc(int M, int N, int a_mn_major) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)a_mn_major << 15) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

// Stores a warp's block of 32 rows x NV floats (row r in lane r's v[]) to dst
// (row stride NV), rows from `valid` on skipped: through shared memory, in
// rounds of W columns, so that each store instruction covers whole lines.
template <int NV>
__device__ __forceinline__ void store_block(const float* v, float* stg, float* dst, int valid, int lane) {
  constexpr int W = NV % 32 == 0 ? 32 : 16;
  constexpr int W4 = W / 4;
#pragma unroll
  for (int c0 = 0; c0 < NV; c0 += W) {
#pragma unroll
    for (int c = 0; c < W; c += 4)
      *reinterpret_cast<float4*>(stg + lane * kStg + c) =
          make_float4(v[c0 + c], v[c0 + c + 1], v[c0 + c + 2], v[c0 + c + 3]);
    __syncwarp();
#pragma unroll
    for (int g = lane; g < 32 * W4; g += 32) {
      const int r = g / W4, c4 = g % W4;
      if (r < valid)
        *reinterpret_cast<float4*>(dst + (size_t)r * NV + c0 + 4 * c4) =
            *reinterpret_cast<const float4*>(stg + r * kStg + 4 * c4);
    }
    __syncwarp();
  }
}

// Epilogue warps 2..5 (TMEM lane quarter = warp % 4): D_N of every row of
// tiles as it completes (double buffered: tfull / tempty), then every D_T
// once the MMA issuer's last commit (tdone) has landed. stage_area: 4 x 32
// staged rows of kStg floats.
//
// ACC accumulators per output, ACC NV TMEM columns: ACC = 1: D_N buffer b at
// b NV, D_T[ci] at (2 + ci) NV. ACC = 3 (L, S_a, S_b of the three-part pass,
// summed here as L + (S_a + S_b)): D_N buffer b at 3 b NV, D_T[ci] at
// (6 + 3 ci) NV.
template <int NV, int ACC>
__device__ __forceinline__ void load_acc(uint32_t taddr, float* v) {
#pragma unroll
  for (int c = 0; c < NV; c += 8) tmem_ld8(taddr + (uint32_t)c, v + c);
  if constexpr (ACC == 3) {
    float a[NV], b[NV];
#pragma unroll
    for (int c = 0; c < NV; c += 8) {
      tmem_ld8(taddr + (uint32_t)(NV + c), a + c);
      tmem_ld8(taddr + (uint32_t)(2 * NV + c), b + c);
    }
    tmem_ld_wait();
#pragma unroll
    for (int c = 0; c < NV; ++c) v[c] += a[c] + b[c];
  } else {
    tmem_ld_wait();
  }
}

template <int NV, int ACC>
__device__ __forceinline__ void epilogue(const TcParams& P, uint32_t tmem, float* stage_area, uint64_t* tfull,
                                         uint64_t* tempty, uint64_t* tdone, volatile int* abort_flag, int rt0, int ct0,
                                         int nrt, int nct, int rg, int cg) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int q = warp & 3;
  const uint32_t lane_off = (uint32_t)(q * 32) << 16;
  float* stg = stage_area + (warp - 2) * 32 * kStg;
  float v[NV];
  if (P.doN) {
    for (int ri = 0; ri < nrt; ++ri) {
      const int buf = ri & 1;
      if (!mbar_wait(&tfull[buf], (uint32_t)(ri >> 1) & 1u, abort_flag, P.wait_ns)) break;
      tc_fence_after();
      load_acc<NV, ACC>(tmem + lane_off + (uint32_t)(buf * ACC * NV), v);
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&tempty[buf]);
      const int row0 = (rt0 + ri) * kTM + q * 32;
      store_block<NV>(v, stg, P.partN + ((size_t)cg * P.n + row0) * NV, P.n - row0, lane);
    }
  }
  if (P.doT && mbar_wait(tdone, 0u, abort_flag, P.wait_ns)) {
    tc_fence_after();
    for (int ci = 0; ci < nct; ++ci) {
      load_acc<NV, ACC>(tmem + lane_off + (uint32_t)((2 + ci) * ACC * NV), v);
      const int col0 = (ct0 + ci) * kTK + q * 32;
      store_block<NV>(v, stg, P.partT + ((size_t)rg * P.m + col0) * NV, P.m - col0, lane);
    }
  } else if (!P.doT) {
    mbar_wait(tdone, 0u, abort_flag, P.wait_ns);
  }
}

// The MMA issuer's last commit (tdone) completes only when every MMA has
// finished reading shared memory and writing TMEM; after an abort nobody
// else waited for it, so the issuer drains it before the TMEM is freed.
__device__ __forceinline__ void teardown(const TcParams& P, uint32_t tmem, uint64_t* tdone, volatile int* abort_flag) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (warp == 1 && lane == 0 && *abort_flag) mbar_drain(tdone, 0u, P.wait_ns);
  tc_fence_before();
  __syncthreads();
  if (*abort_flag && threadIdx.x == 0) set_status(P.ctrl, NMF_ERR_DEVICE_TIMEOUT);
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(P.tmem_cols));
  }
}

template <int NV>
__global__ void __launch_bounds__(kThreads, 1)
    xpass_tc_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB, TcParams P) {
  // launched as a programmatic dependent: the operands come from the previous kernel
  asm volatile("griddepcontrol.wait;" ::: "memory");
  if (call_failed(P.ctrl)) return;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  constexpr int opBox = NV * kBoxK * 2;          // one NV x 64 operand box
  constexpr int stageBytes = kXStageBytes + 4 * opBox;
  const int kStages = P.stages;
  __shared__ uint64_t full[kMaxStages], empty[kMaxStages], tfull[2], tempty[2], tdone;
  __shared__ uint32_t tmem_base_s;
  __shared__ int abort_s;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int rg = blockIdx.x / P.S_c, cg = blockIdx.x % P.S_c;
  const int rt0 = split_point(P.tiles_r, P.S_r, rg), rt1 = split_point(P.tiles_r, P.S_r, rg + 1);
  const int ct0 = split_point(P.tiles_c, P.S_c, cg), ct1 = split_point(P.tiles_c, P.S_c, cg + 1);
  const int nrt = rt1 - rt0, nct = ct1 - ct0;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], 4);
    }
    mbar_init(&tdone, 1);
    abort_s = 0;
    mbar_fence_init();
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base_s)),
                 "r"(P.tmem_cols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base_s;
  volatile int* abort_flag = &abort_s;

  if (warp == 0) {
    // ---------------- TMA producer ----------------
    if (lane == 0) {
      const uint32_t bytes = kXStageBytes + (P.doN ? 2 * opBox : 0) + (P.doT ? 2 * opBox : 0);
      int it = 0;
      for (int rt = rt0; rt < rt1 && !*abort_flag; ++rt) {
        for (int ct = ct0; ct < ct1; ++ct, ++it) {
          const int s = it % kStages;
          const uint32_t ph = (uint32_t)(it / kStages) & 1u;
          if (!mbar_wait(&empty[s], ph ^ 1u, abort_flag, P.wait_ns)) break;
          uint8_t* st = smem + (size_t)s * stageBytes;
          mbar_arrive_expect_tx(&full[s], bytes);
          if (P.withhold && blockIdx.x == 0 && it == 0) continue;  // failure-path testing: the stage never fills
          bulk_load(st, P.Xt + ((size_t)rt * P.tiles_c + ct) * kXStageBytes, (uint32_t)kXStageBytes, &full[s]);
          if (P.doN) {
            tma_load_2d(st + kXStageBytes, &mapA, &full[s], ct * kTK, 0);
            tma_load_2d(st + kXStageBytes + opBox, &mapA, &full[s], ct * kTK + kBoxK, 0);
          }
          if (P.doT) {
            tma_load_2d(st + kXStageBytes + 2 * opBox, &mapB, &full[s], rt * kTM, 0);
            tma_load_2d(st + kXStageBytes + 3 * opBox, &mapB, &full[s], rt * kTM + kBoxK, 0);
          }
        }
      }
      if (*abort_flag) {
        // let the copies already issued land before the CTA exits
        const int issued = it;
        for (int j = issued - kStages < 0 ? 0 : issued - kStages; j < issued; ++j)
          mbar_drain(&full[j % kStages], (uint32_t)(j / kStages) & 1u, P.wait_ns);
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      const uint32_t idN = instr_desc(kTM, NV, 0);
      const uint32_t idT = instr_desc(kTK, NV, 1);
      int it = 0;
      bool ok = true;
      for (int ri = 0; ri < nrt && ok; ++ri) {
        const int buf = ri & 1;
        const uint32_t dN = tmem + (uint32_t)(buf * NV);
        if (P.doN) {
          if (!mbar_wait(&tempty[buf], ((uint32_t)(ri >> 1) & 1u) ^ 1u, abort_flag, P.wait_ns)) { ok = false; break; }
          tc_fence_after();
        }
        for (int ci = 0; ci < nct; ++ci, ++it) {
          const int s = it % kStages;
          const uint32_t ph = (uint32_t)(it / kStages) & 1u;
          if (!mbar_wait(&full[s], ph, abort_flag, P.wait_ns)) { ok = false; break; }
          tc_fence_after();
          const uint32_t st = smem_u32(smem + (size_t)s * stageBytes);
          const uint32_t xa = st, opa = st + kXStageBytes, opb = st + kXStageBytes + 2 * opBox;
          // N and T steps alternate: an MMA into the accumulator the previous
          // MMA wrote waits for it, so consecutive MMAs go to different ones
          const uint32_t dT = tmem + (uint32_t)((2 + ci) * NV);
#pragma unroll
          for (int kk = 0; kk < kTK / 16; ++kk) {
            const uint32_t boff = (uint32_t)((kk >> 2) * opBox + (kk & 3) * 32);
            if (P.doN) {
              const uint32_t off = (uint32_t)((kk >> 2) * (kXStageBytes / 2) + (kk & 3) * 32);
              tc_mma(dN, smem_desc(xa + off, 16, 1024), smem_desc(opa + boff, 16, 1024), idN,
                     (ci > 0 || kk > 0) ? 1u : 0u);
            }
            if (P.doT)
              tc_mma(dT, smem_desc(xa + (uint32_t)(kk * 2048), kXStageBytes / 2, 1024), smem_desc(opb + boff, 16, 1024),
                     idT, (ri > 0 || kk > 0) ? 1u : 0u);
          }
          tc_commit(&empty[s]);
        }
        if (ok && P.doN) tc_commit(&tfull[buf]);
      }
      tc_commit(&tdone);
    }
  } else {
    epilogue<NV, 1>(P, tmem, reinterpret_cast<float*>(smem + (size_t)kStages * stageBytes), tfull, tempty, &tdone,
                    abort_flag, rt0, ct0, nrt, nct, rg, cg);
  }
  teardown(P, tmem, &tdone, abort_flag);
}


// ---- float32 X as three bfloat16 parts -------------------------------------
// X = X0 + X1 + X2 and every operand A = A0 + A1 + A2 (OP_BF16X3): each part
// rounds the float32 residual of the previous ones, so |X - X0 - X1 - X2| <=
// 2^-27 |X|. The six products X_j A_i with i + j <= 2 leave out terms below
// 2^-26 |x a|. The leading term X_0 A_0 has a TMEM accumulator L of its own
// and the five others (at most 2^-8 of it) go to two more, S_a and S_b:
// tensor-core accumulation rounds the running sum at every MMA, so adding
// the small terms into the large sum would round it six times as often as a
// one-part pass does. With the operand parts stacked (A_0; A_1; A_2), the
// small terms take two MMAs of width 2 NV and one of width NV per step:
//   X_0 [A_1 | A_2] -> [S_a | S_b],  X_1 [A_0 | A_1] -> [S_a | S_b],  X_2 A_0 -> S_a.
// The epilogue forms L + (S_a + S_b). A pass is then as accurate as the
// one-part pass is on its own inputs, from 6 bytes of X per element instead
// of 4 (the parts are formed once per call).
//
// A tile's three parts arrive as three 32 KB stages of the X ring. The
// operand slices change less often and have rings of their own: the A slice
// (3 NV rows x 128 columns, the tile's columns) per tile, the B slice per row
// of tiles, each double buffered. Part j of a tile feeds the MMAs with
// operand parts 0 .. 2 - j.
//
// (The one-part bfloat16 pass stays on xpass_tc_kernel, operands with every
// stage: on this ring, with five X stages and a separate operand producer, it
// measured 187 against 182 us per dual product at n = m = 10^4, nu = 20.)
constexpr int kMaxStagesRing = 6;
__host__ __device__ constexpr int op_box_bytes(int NV, int parts) { return parts * NV * kBoxK * 2; }  // rows x 128 B
__host__ __device__ constexpr int op_tile_bytes(int NV, int parts) { return 2 * op_box_bytes(NV, parts); }

// Warps of the ring kernel: 0 = X producer, 1 = MMA issuer (and TMEM owner),
// 2..5 = epilogue, 6 = operand producer.
constexpr int kRingWarps = 7;

template <int NV, int PARTS>
__global__ void __launch_bounds__(kRingWarps * 32, 1)
    xpass_ring_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB, TcParams P) {
  // launched as a programmatic dependent: the operands come from the previous kernel
  asm volatile("griddepcontrol.wait;" ::: "memory");
  if (call_failed(P.ctrl)) return;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  constexpr int box = op_box_bytes(NV, PARTS);
  constexpr int opTile = op_tile_bytes(NV, PARTS);
  constexpr int ACC = PARTS == 3 ? 3 : 1;  // accumulators per output (see load_acc)
  const int kStages = P.stages;
  uint8_t* xring = smem;
  uint8_t* aring = xring + (size_t)kStages * kXStageBytes;
  uint8_t* bring = aring + 2 * opTile;
  float* stage_area = reinterpret_cast<float*>(bring + 2 * opTile);
  __shared__ uint64_t xfull[kMaxStagesRing], xempty[kMaxStagesRing], afull[2], aempty[2], bfull[2], bempty[2];
  __shared__ uint64_t tfull[2], tempty[2], tdone;
  __shared__ uint32_t tmem_base_s;
  __shared__ int abort_s;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int rg = blockIdx.x / P.S_c, cg = blockIdx.x % P.S_c;
  const int rt0 = split_point(P.tiles_r, P.S_r, rg), rt1 = split_point(P.tiles_r, P.S_r, rg + 1);
  const int ct0 = split_point(P.tiles_c, P.S_c, cg), ct1 = split_point(P.tiles_c, P.S_c, cg + 1);
  const int nrt = rt1 - rt0, nct = ct1 - ct0;

  if (threadIdx.x == 0) {
    for (int st = 0; st < kStages; ++st) {
      mbar_init(&xfull[st], 1);
      mbar_init(&xempty[st], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&afull[b], 1);
      mbar_init(&aempty[b], 1);
      mbar_init(&bfull[b], 1);
      mbar_init(&bempty[b], 1);
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], 4);
    }
    mbar_init(&tdone, 1);
    abort_s = 0;
    mbar_fence_init();
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base_s)),
                 "r"(P.tmem_cols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base_s;
  volatile int* abort_flag = &abort_s;

  if (warp == 0) {
    // ---------------- X producer: the tiles' parts through the X ring ----------------
    if (lane == 0) {
      int it = 0;
      bool ok = true;
      for (int rt = rt0; rt < rt1 && ok && !*abort_flag; ++rt)
        for (int ct = ct0; ct < ct1 && ok; ++ct)
          for (int j = 0; j < PARTS; ++j, ++it) {
            const int st = it % kStages;
            if (!mbar_wait(&xempty[st], ((uint32_t)(it / kStages) & 1u) ^ 1u, abort_flag, P.wait_ns)) {
              ok = false;
              break;
            }
            mbar_arrive_expect_tx(&xfull[st], (uint32_t)kXStageBytes);
            if (P.withhold && blockIdx.x == 0 && it == 0) continue;  // failure-path testing: the stage never fills
            bulk_load(xring + (size_t)st * kXStageBytes,
                      P.Xt + (((size_t)rt * P.tiles_c + ct) * PARTS + j) * kXStageBytes, (uint32_t)kXStageBytes,
                      &xfull[st]);
          }
      if (*abort_flag)  // let the copies already issued land before the CTA exits
        for (int k = it - kStages < 0 ? 0 : it - kStages; k < it; ++k)
          mbar_drain(&xfull[k % kStages], (uint32_t)(k / kStages) & 1u, P.wait_ns);
    }
  } else if (warp == kRingWarps - 1) {
    // ---------------- operand producer: B per row of tiles, A per tile ----------------
    // (its own thread, so the X ring runs ahead of the operand rings)
    if (lane == 0) {
      int at = 0, bt = 0;
      bool ok = true;
      for (int rt = rt0; rt < rt1 && ok && !*abort_flag; ++rt) {
        if (P.doT) {
          const int b = bt & 1;
          if (!mbar_wait(&bempty[b], ((uint32_t)(bt >> 1) & 1u) ^ 1u, abort_flag, P.wait_ns)) break;
          mbar_arrive_expect_tx(&bfull[b], (uint32_t)opTile);
          tma_load_2d(bring + (size_t)b * opTile, &mapB, &bfull[b], rt * kTM, 0);
          tma_load_2d(bring + (size_t)b * opTile + box, &mapB, &bfull[b], rt * kTM + kBoxK, 0);
          ++bt;
        }
        for (int ct = ct0; ct < ct1 && P.doN; ++ct) {
          const int a = at & 1;
          if (!mbar_wait(&aempty[a], ((uint32_t)(at >> 1) & 1u) ^ 1u, abort_flag, P.wait_ns)) {
            ok = false;
            break;
          }
          mbar_arrive_expect_tx(&afull[a], (uint32_t)opTile);
          tma_load_2d(aring + (size_t)a * opTile, &mapA, &afull[a], ct * kTK, 0);
          tma_load_2d(aring + (size_t)a * opTile + box, &mapA, &afull[a], ct * kTK + kBoxK, 0);
          ++at;
        }
      }
      if (*abort_flag) {
        for (int k = at - 2 < 0 ? 0 : at - 2; k < at; ++k) mbar_drain(&afull[k & 1], (uint32_t)(k >> 1) & 1u, P.wait_ns);
        for (int k = bt - 2 < 0 ? 0 : bt - 2; k < bt; ++k) mbar_drain(&bfull[k & 1], (uint32_t)(k >> 1) & 1u, P.wait_ns);
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      const uint32_t idN1 = instr_desc(kTM, NV, 0), idN2 = instr_desc(kTM, 2 * NV, 0);
      const uint32_t idT1 = instr_desc(kTK, NV, 1), idT2 = instr_desc(kTK, 2 * NV, 1);
      int it = 0, at = 0, bt = 0;
      bool ok = true;
      for (int ri = 0; ri < nrt && ok; ++ri) {
        const int buf = ri & 1;
        const uint32_t dN = tmem + (uint32_t)(buf * ACC * NV);  // PARTS = 3: L, then S_a, S_b
        int b = 0;
        if (P.doN) {
          if (!mbar_wait(&tempty[buf], ((uint32_t)(ri >> 1) & 1u) ^ 1u, abort_flag, P.wait_ns)) { ok = false; break; }
          tc_fence_after();
        }
        if (P.doT) {
          b = bt & 1;
          if (!mbar_wait(&bfull[b], (uint32_t)(bt >> 1) & 1u, abort_flag, P.wait_ns)) { ok = false; break; }
          tc_fence_after();
        }
        const uint32_t opb = smem_u32(bring + (size_t)b * opTile);
        for (int ci = 0; ci < nct && ok; ++ci) {
          int a = 0;
          if (P.doN) {
            a = at & 1;
            if (!mbar_wait(&afull[a], (uint32_t)(at >> 1) & 1u, abort_flag, P.wait_ns)) { ok = false; break; }
            tc_fence_after();
          }
          const uint32_t opa = smem_u32(aring + (size_t)a * opTile);
          for (int j = 0; j < PARTS; ++j, ++it) {
            const int st = it % kStages;
            if (!mbar_wait(&xfull[st], (uint32_t)(it / kStages) & 1u, abort_flag, P.wait_ns)) { ok = false; break; }
            tc_fence_after();
            const uint32_t xa = smem_u32(xring + (size_t)st * kXStageBytes);
            // Per K step: part 0 issues L and [S_a | S_b] MMAs, parts 1 and 2
            // one [S_a | S_b] or S_a MMA; N and T alternate so that
            // consecutive MMAs go to different accumulators.
            const uint32_t dT = tmem + (uint32_t)((2 + ci) * ACC * NV);
            const bool firstN = ci == 0 && j == 0, firstT = ri == 0 && j == 0;
            // operand rows of the small-term MMA: A_1 (j = 0) or A_0 (j = 1, 2)
            const uint32_t srow = (uint32_t)(j == 0 ? NV * 128 : 0);
            const uint32_t idNs = j == 2 ? idN1 : idN2, idTs = j == 2 ? idT1 : idT2;
#pragma unroll
            for (int kk = 0; kk < kTK / 16; ++kk) {
              const uint32_t xoffN = (uint32_t)((kk >> 2) * (kXStageBytes / 2) + (kk & 3) * 32);
              const uint32_t xoffT = (uint32_t)(kk * 2048);
              const uint32_t boff = (uint32_t)((kk >> 2) * box + (kk & 3) * 32);
              const uint32_t acc = kk > 0 ? 1u : 0u;
              if (j == 0) {
                if (P.doN)
                  tc_mma(dN, smem_desc(xa + xoffN, 16, 1024), smem_desc(opa + boff, 16, 1024), idN1,
                         firstN ? acc : 1u);
                if (P.doT)
                  tc_mma(dT, smem_desc(xa + xoffT, kXStageBytes / 2, 1024), smem_desc(opb + boff, 16, 1024), idT1,
                         firstT ? acc : 1u);
              }
              if constexpr (PARTS == 3) {
                if (P.doN)
                  tc_mma(dN + NV, smem_desc(xa + xoffN, 16, 1024), smem_desc(opa + boff + srow, 16, 1024), idNs,
                         firstN ? acc : 1u);
                if (P.doT)
                  tc_mma(dT + NV, smem_desc(xa + xoffT, kXStageBytes / 2, 1024),
                         smem_desc(opb + boff + srow, 16, 1024), idTs, firstT ? acc : 1u);
              }
            }
            tc_commit(&xempty[st]);
          }
          if (ok && P.doN) {
            tc_commit(&aempty[a]);
            ++at;
          }
        }
        if (ok && P.doT) {
          tc_commit(&bempty[b]);
          ++bt;
        }
        if (ok && P.doN) tc_commit(&tfull[buf]);
      }
      tc_commit(&tdone);
    }
  } else {
    epilogue<NV, ACC>(P, tmem, stage_area, tfull, tempty, &tdone, abort_flag, rt0, ct0, nrt, nct, rg, cg);
  }
  teardown(P, tmem, &tdone, abort_flag);
}

// ---- host side -------------------------------------------------------------
PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

// 2D bf16 map over a row-major [rows][ld] array, box box_cols x box_rows, 128-byte swizzle.
bool make_map(CUtensorMap* map, const void* base, int ld, int rows, int box_cols, int box_rows) {
  auto fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {(cuuint64_t)ld, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
  cuuint32_t box[2] = {(cuuint32_t)box_cols, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

uint32_t tmem_cols_for(int NV, int maxct, int acc) {
  const uint32_t need = (uint32_t)((2 + maxct) * acc * NV);
  uint32_t c = 32;
  while (c < need) c <<= 1;
  return c;
}

int max_col_tiles(int NV, int acc) { return (int)(kMaxTmemCols / (acc * NV)) - 2; }

size_t tc_stage_bytes(int NV) { return (size_t)(kXStageBytes + 4 * NV * kBoxK * 2); }
int tc_stages(int NV) {
  int st = (int)((kSmemBudget - 1024 - kStageArea) / tc_stage_bytes(NV));
  return st > kMaxStages ? kMaxStages : st;
}
size_t tc_smem_bytes(int NV) { return (size_t)tc_stages(NV) * tc_stage_bytes(NV) + kStageArea + 1024; }

// X (n x m float32, row-major) to bfloat16 tiles of kTM x kTK: tile (rt, ct)
// at element (rt * tiles_c + ct) * kTM * kTK, laid out as the two 128 x 64
// boxes the kernel's shared memory holds, box h at byte h * kTM * 128, row r
// at byte r * 128 of its box, the 16-byte chunk j of a row at chunk
// j ^ (r mod 8) (the 128-byte swizzle). Entries outside X are zero. One
// thread per 8 consecutive elements of a row: the reads of a warp are
// contiguous, and every 8 threads fill one 128-byte row of a box.
//
// parts = 3: every element is stored as its three bfloat16 parts
// (split_bf16x3), part j of tile (rt, ct) at byte ((rt * tiles_c + ct) * 3 +
// j) * 32 KB, in the same layout.
template <int PARTS>
__global__ void to_tiles_kernel(const float* __restrict__ X, int n, int m, int tiles_r, int tiles_c,
                                uint4* __restrict__ Xt, Control* ctrl) {
  if (call_failed(ctrl)) return;
  const long long chunks_row = (long long)tiles_c * (kTK / 8);
  const long long total = (long long)tiles_r * kTM * chunks_row;
  const bool vec = (m & 3) == 0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(i / chunks_row), cj = (int)(i % chunks_row);
    const int c0 = cj * 8;
    float v[8];
    if (vec && r < n && c0 + 8 <= m) {
      const float4* src = reinterpret_cast<const float4*>(X + (size_t)r * m + c0);
      const float4 a = __ldcs(src), b = __ldcs(src + 1);
      v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
      v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
    } else {
#pragma unroll
      for (int k = 0; k < 8; ++k) v[k] = (r < n && c0 + k < m) ? X[(size_t)r * m + c0 + k] : 0.f;
    }
    uint4 out[PARTS];
    if constexpr (PARTS == 1) {
      uint32_t* o = reinterpret_cast<uint32_t*>(&out[0]);
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const __nv_bfloat162 h = __floats2bfloat162_rn(v[2 * k], v[2 * k + 1]);
        o[k] = *reinterpret_cast<const uint32_t*>(&h);
      }
    } else {
      __nv_bfloat16* o0 = reinterpret_cast<__nv_bfloat16*>(&out[0]);
      __nv_bfloat16* o1 = reinterpret_cast<__nv_bfloat16*>(&out[1]);
      __nv_bfloat16* o2 = reinterpret_cast<__nv_bfloat16*>(&out[2]);
#pragma unroll
      for (int k = 0; k < 8; ++k) split_bf16x3(v[k], o0[k], o1[k], o2[k]);
    }
    const int rt = r / kTM, rr = r % kTM, ct = cj / (kTK / 8), h = (cj / 8) & 1, j = cj & 7;
    const size_t byte = ((size_t)rt * tiles_c + ct) * PARTS * kXStageBytes + (size_t)h * (kTM * 128) +
                        (size_t)rr * 128 + (size_t)((j ^ (rr & 7)) * 16);
#pragma unroll
    for (int q = 0; q < PARTS; ++q) Xt[(byte + (size_t)q * kXStageBytes) / 16] = out[q];
  }
}

// Launch with programmatic dependent launch allowed: the kernel's CTAs may
// start while the previous kernel on the stream finishes, and wait
// (griddepcontrol.wait) before reading anything it wrote.
cudaError_t launch_pdl(const void* fn, int ctas, int threads, size_t smem, cudaStream_t s, const CUtensorMap& mA,
                       const CUtensorMap& mB, const TcParams& P) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(ctas);
  cfg.blockDim = dim3(threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = pdl_allowed() ? 1 : 0;
  void* args[] = {const_cast<CUtensorMap*>(&mA), const_cast<CUtensorMap*>(&mB), const_cast<TcParams*>(&P)};
  return cudaLaunchKernelExC(&cfg, fn, args);
}

template <int NV>
cudaError_t launch_nv(const CUtensorMap& mA, const CUtensorMap& mB, const TcParams& P, int ctas, cudaStream_t s) {
  const size_t smem = tc_smem_bytes(NV);
  cudaError_t e = allow_dynamic_smem((const void*)xpass_tc_kernel<NV>, (int)smem);
  if (e != cudaSuccess) return e;
  count_launches(1);
  return launch_pdl((const void*)xpass_tc_kernel<NV>, ctas, kThreads, smem, s, mA, mB, P);
}

// Ring kernel: X ring stages that fit beside the two operand rings (double
// buffered) and the epilogue staging.
int ring_stages(int NV, int parts) {
  const long room = (long)kSmemBudget - 1024 - kStageArea - 4l * op_tile_bytes(NV, parts);
  const long st = room / kXStageBytes;
  return (int)(st > kMaxStagesRing ? kMaxStagesRing : st);
}
size_t ring_smem_bytes(int NV, int parts) {
  return (size_t)ring_stages(NV, parts) * kXStageBytes + 4 * (size_t)op_tile_bytes(NV, parts) + kStageArea + 1024;
}

template <int NV, int PARTS>
cudaError_t launch_ring(const CUtensorMap& mA, const CUtensorMap& mB, const TcParams& P, int ctas, cudaStream_t s) {
  const size_t smem = ring_smem_bytes(NV, PARTS);
  cudaError_t e = allow_dynamic_smem((const void*)xpass_ring_kernel<NV, PARTS>, (int)smem);
  if (e != cudaSuccess) return e;
  count_launches(1);
  return launch_pdl((const void*)xpass_ring_kernel<NV, PARTS>, ctas, kRingWarps * 32, smem, s, mA, mB, P);
}

}  // namespace

bool xpass_tc_available() {
  static int avail = -1;
  if (avail < 0) {
    int dev = 0, major = 0, minor = 0;
    avail = 0;
    if (cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev) == cudaSuccess)
      avail = (major == 10 && minor == 3 && encode_fn() != nullptr) ? 1 : 0;
  }
  return avail == 1;
}

// Region grid: the S_r x S_c split of the tile grid with at most `num_sms`
// CTAs that minimises the largest region (tiles per CTA), subject to the
// TMEM budget on column tiles per region.
XPassPlan xpass_tc_plan(int n, int m, int nu, int num_sms, int parts) {
  XPassPlan pl{};
  pl.parts = parts;
  pl.tile_r = kTM;
  pl.tile_c = kTK;
  pl.tiles_r = ceil_div(n, kTM);
  pl.tiles_c = ceil_div(m, kTK);
  pl.NV = round_up(nu, 16);
  const int maxct = max_col_tiles(pl.NV, parts == 3 ? 3 : 1);
  long best = -1;
  int bestr = 1, bestc = pl.tiles_c;
  for (int S_c = 1; S_c <= pl.tiles_c; ++S_c) {
    if (ceil_div(pl.tiles_c, S_c) > maxct) continue;
    for (int S_r = 1; S_r <= pl.tiles_r && S_r * S_c <= num_sms; ++S_r) {
      const long worst = (long)ceil_div(pl.tiles_r, S_r) * ceil_div(pl.tiles_c, S_c);
      if (best < 0 || worst < best || (worst == best && S_r * S_c < bestr * bestc)) {
        best = worst;
        bestr = S_r;
        bestc = S_c;
      }
    }
  }
  pl.S_r = bestr;
  pl.S_c = bestc;
  pl.ctas = bestr * bestc;
  pl.tiled = 1;
  return pl;
}

cudaError_t xpass_tc_convert(const XPassPlan& pl, const float* X, int n, int m, void* Xt, Control* ctrl,
                             cudaStream_t s) {
  // a grid-stride loop over 16-byte chunks, eight 256-thread CTAs per SM
  const long long chunks = (long long)pl.tiles_r * kTM * pl.tiles_c * (kTK / 8);
  const long long ctas = std::min<long long>((chunks + 255) / 256, 8ll * device_sm_count());
  count_launches(1);
  if (pl.parts == 3)
    to_tiles_kernel<3><<<(int)ctas, 256, 0, s>>>(X, n, m, pl.tiles_r, pl.tiles_c, static_cast<uint4*>(Xt), ctrl);
  else
    to_tiles_kernel<1><<<(int)ctas, 256, 0, s>>>(X, n, m, pl.tiles_r, pl.tiles_c, static_cast<uint4*>(Xt), ctrl);
  return cudaGetLastError();
}

cudaError_t xpass_tc_launch(const XPassPlan& pl, const XPassArgs& a, cudaStream_t s) {
  CUtensorMap mA, mB;
  if (!pl.tiled || (reinterpret_cast<uintptr_t>(a.X) & 15u)) return cudaErrorInvalidValue;
  if (pl.parts != 1 && (pl.parts != 3 || pl.NV > kSplitMaxNV)) return cudaErrorInvalidValue;
  // operands: parts x NV rows (part k at rows k NV .. k NV + NV - 1), one box holds them all
  const int oprows = pl.parts * pl.NV;
  if (!make_map(&mA, a.opA, a.lda, oprows, kBoxK, oprows)) return cudaErrorInvalidValue;
  if (!make_map(&mB, a.opB, a.ldb, oprows, kBoxK, oprows)) return cudaErrorInvalidValue;
  TcParams P{};
  P.Xt = static_cast<const uint8_t*>(a.X);
  P.n = a.n;
  P.m = a.m;
  P.stages = pl.parts == 3 ? ring_stages(pl.NV, pl.parts) : tc_stages(pl.NV);
  P.tiles_r = pl.tiles_r;
  P.tiles_c = pl.tiles_c;
  P.S_r = pl.S_r;
  P.S_c = pl.S_c;
  P.doN = a.doN;
  P.doT = a.doT;
  P.partN = a.partN;
  P.partT = a.partT;
  P.ctrl = a.ctrl;
  P.tmem_cols = tmem_cols_for(pl.NV, ceil_div(pl.tiles_c, pl.S_c), pl.parts == 3 ? 3 : 1);
  P.wait_ns = wait_limit_ns();
  P.withhold = injected_fault() == NMF_FAULT_XPASS_COPY ? 1 : 0;
  if (pl.parts == 3) {
    switch (pl.NV) {
      case 16: return launch_ring<16, 3>(mA, mB, P, pl.ctas, s);
      case 32: return launch_ring<32, 3>(mA, mB, P, pl.ctas, s);
      default: return cudaErrorInvalidValue;
    }
  }

  switch (pl.NV) {
    case 16: return launch_nv<16>(mA, mB, P, pl.ctas, s);
    case 32: return launch_nv<32>(mA, mB, P, pl.ctas, s);
    case 48: return launch_nv<48>(mA, mB, P, pl.ctas, s);
    case 64: return launch_nv<64>(mA, mB, P, pl.ctas, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace nmf
