// nnls_device.cuh -- device pieces of the Nesterov inner loop (Sec. 2)
// shared by the single-problem and the batched solvers: the product H y - b
// with the symmetric H in shared memory, the projected-gradient norm of the
// stop test, and L_c = lambda_max(H).
#pragma once

#include "common.cuh"

namespace nmf {

constexpr int kMaxSquarings = 16;
// Adaptive restart: a vector's objective counts as risen when the rise
// exceeds this fraction of sum_c |f_c| (|grad_c| + |b_c|), the scale of the
// terms it is computed from, so float32 rounding near convergence does not
// restart the momentum.
constexpr float kRestartTol = 1e-5f;

// g = H y - b with the symmetric H (PM x PM, zero padded) in shared memory:
// row d of H is column d, so g accumulates y_d times row d (read as float4)
// over d; the PM sums advance together and hide each other's latency.
template <int PM>
__device__ __forceinline__ void hmatvec(const float* Hs, const float* y, const float* b, float* g) {
#pragma unroll
  for (int c = 0; c < PM; ++c) g[c] = -b[c];
#pragma unroll
  for (int d = 0; d < PM; ++d) {
    const float4* h = reinterpret_cast<const float4*>(Hs + d * PM);
    const float yd = y[d];
#pragma unroll
    for (int c4 = 0; c4 < PM / 4; ++c4) {
      const float4 v = h[c4];
      g[4 * c4 + 0] = fmaf(v.x, yd, g[4 * c4 + 0]);
      g[4 * c4 + 1] = fmaf(v.y, yd, g[4 * c4 + 1]);
      g[4 * c4 + 2] = fmaf(v.z, yd, g[4 * c4 + 2]);
      g[4 * c4 + 3] = fmaf(v.w, yd, g[4 * c4 + 3]);
    }
  }
}

// Index of H_ij in the packed upper triangle (row-major, i <= j).
template <int PM>
__host__ __device__ constexpr int packed_index(int i, int j) {
  return i <= j ? i * PM - i * (i - 1) / 2 + (j - i) : j * PM - j * (j - 1) / 2 + (i - j);
}
// Small PM: the upper triangle of H held in registers (every index below is
// a compile-time constant), loaded once per solve; LD is the row stride of
// Hs (its padded rank, >= PM).
template <int PM, int LD = PM>
__device__ __forceinline__ void load_packed(const float* Hs, float* Hp) {
#pragma unroll
  for (int i = 0; i < PM; ++i)
#pragma unroll
    for (int j = i; j < PM; ++j) Hp[packed_index<PM>(i, j)] = Hs[i * LD + j];
}
// g = H y - b from the packed registers: the operations of hmatvec in the
// same order (H is exactly symmetric: H_cd and H_dc are the same products
// summed in the same order), so the results are identical.
template <int PM>
__device__ __forceinline__ void hmatvec_packed(const float* Hp, const float* y, const float* b, float* g) {
#pragma unroll
  for (int c = 0; c < PM; ++c) g[c] = -b[c];
#pragma unroll
  for (int d = 0; d < PM; ++d)
#pragma unroll
    for (int c = 0; c < PM; ++c) g[c] = fmaf(Hp[packed_index<PM>(d, c)], y[d], g[c]);
}

// The same product with the loop over d kept rolled: one row of H live at a
// time, for kernels with enough warps per SM to hide the shared-memory
// latency and too many other live values to hold more of H. LD: the row
// stride of Hs (a multiple of 4, >= PM); with PM < LD only the first PM rows
// and columns take part (the others must be zero in y, which makes their
// terms exact zeros).
template <int PM, int LD = PM>
__device__ __forceinline__ void hmatvec_rolled(const float* Hs, const float* y, const float* b, float* g) {
  static_assert(LD % 4 == 0 && LD >= PM, "rows of H are read as float4");
#pragma unroll
  for (int c = 0; c < PM; ++c) g[c] = -b[c];
#pragma unroll 1
  for (int d = 0; d < PM; ++d) {
    const float4* h = reinterpret_cast<const float4*>(Hs + d * LD);
    float yd = 0.f;
#pragma unroll
    for (int e = 0; e < PM; ++e) yd = (e == d) ? y[e] : yd;
#pragma unroll
    for (int c4 = 0; c4 < (PM + 3) / 4; ++c4) {
      const float4 v = h[c4];
      if (4 * c4 + 0 < PM) g[4 * c4 + 0] = fmaf(v.x, yd, g[4 * c4 + 0]);
      if (4 * c4 + 1 < PM) g[4 * c4 + 1] = fmaf(v.y, yd, g[4 * c4 + 1]);
      if (4 * c4 + 2 < PM) g[4 * c4 + 2] = fmaf(v.z, yd, g[4 * c4 + 2]);
      if (4 * c4 + 3 < PM) g[4 * c4 + 3] = fmaf(v.w, yd, g[4 * c4 + 3]);
    }
  }
}

template <int PM>
__device__ __forceinline__ float pg_sq(const float* f, const float* g) {
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < PM; ++c) {
    const float v = f[c] > 0.f ? g[c] : fminf(g[c], 0.f);
    s = fmaf(v, v, s);
  }
  return s;
}

// Row stride of the squaring buffers: PM or PM + 4, whichever is an odd
// number of float4s, so rows read as float4 by eight lanes hit eight
// different bank groups.
template <int PM>
__host__ __device__ constexpr int lam_stride() { return ((PM / 4) & 1) ? PM : PM + 4; }

// lambda_max of the symmetric PSD matrix H (PM x PM in shared memory, zero
// outside p x p), by one warp. Repeated squaring with trace normalisation:
// A_0 = H, A_{s+1} = (A_s / tr A_s)^2; the lanes share the PM (PM + 1) / 2
// entries of the upper triangle (A stays symmetric), each a dot product of
// two rows. tr(A_{s+1}) = tr(M^2) for the trace-one M = A_s / tr(A_s), which
// reaches 1 exactly when M has rank one; at 1 - tr(M^2) < 1e-5 the other
// eigenvectors' share in the dominant column is < 1e-5, so its Rayleigh
// quotient (float-float arithmetic) is exact to ~1e-10. Ms is 2 PM
// lam_stride<PM>() floats of 16-byte aligned scratch. The result is valid in
// every lane; 0 for H = 0, non-finite for a non-finite H. With v set, lanes
// c < p also store the unit eigenvector's entry v[c] (the dominant column,
// normalised).
template <int PM>
__device__ double lambda_max_warp(const float* Hs, float* Ms, int p, float* v = nullptr) {
  constexpr int LS = lam_stride<PM>();
  constexpr int E = PM * (PM + 1) / 2;
  constexpr int NPL = (E + 31) / 32;
  const int lane = threadIdx.x & 31;
  const float tr = warp_sum(lane < p ? Hs[lane * PM + lane] : 0.f);
  if (!(tr > 0.f) || !isfinite(tr)) return isfinite(tr) ? 0.0 : (double)tr;
  float* A = Ms;
  float* B = Ms + PM * LS;
  for (int i = lane; i < PM * PM; i += 32) A[(i / PM) * LS + i % PM] = Hs[i];
  // this lane's upper-triangle entries (i << 8 | j), -1 past the end
  int pr[NPL];
  {
    int i = 0, e = lane;
#pragma unroll
    for (int q = 0; q < NPL; ++q) {
      while (i < PM && e >= PM - i) {
        e -= PM - i;
        ++i;
      }
      pr[q] = i < PM ? (i << 8) | (i + e) : -1;
      e += 32;
    }
  }
  __syncwarp();
  float t = tr;
  for (int s = 0; s < kMaxSquarings; ++s) {
    const float sc = __fdividef(1.f, t);  // any positive scale normalises; t2 below is measured
    const float sc2 = sc * sc;
    float dsum = 0.f;
#pragma unroll
    for (int q = 0; q < NPL; ++q) {
      if (pr[q] < 0) continue;
      const int i = pr[q] >> 8, j = pr[q] & 255;
      const float4* ri = reinterpret_cast<const float4*>(A + i * LS);
      const float4* rj = reinterpret_cast<const float4*>(A + j * LS);
      float s0 = 0.f, s1 = 0.f;
#pragma unroll
      for (int d4 = 0; d4 < PM / 4; ++d4) {
        const float4 x = ri[d4], z = rj[d4];
        s0 = fmaf(x.x, z.x, s0);
        s1 = fmaf(x.y, z.y, s1);
        s0 = fmaf(x.z, z.z, s0);
        s1 = fmaf(x.w, z.w, s1);
      }
      const float v = (s0 + s1) * sc2;
      B[i * LS + j] = v;
      B[j * LS + i] = v;
      if (i == j) dsum += v;
    }
    const float t2 = warp_sum(dsum);  // trace of the new A (= tr(M^2), tr(M) = 1 to rounding)
    __syncwarp();                      // every lane has read A and written B
    float* tmp = A;
    A = B;
    B = tmp;
    t = t2;
    if (!(t2 > 0.f) || 1.f - t2 < 1e-5f) break;
  }
  // dominant column jb = argmax diag(A); v_c = A[c][jb] = A[jb][c]
  float best = lane < p ? A[lane * LS + lane] : -1.f;
  int jb = lane;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float ob = __shfl_xor_sync(0xffffffffu, best, o);
    const int oj = __shfl_xor_sync(0xffffffffu, jb, o);
    if (ob > best || (ob == best && oj < jb)) {
      best = ob;
      jb = oj;
    }
  }
  const float* vrow = A + jb * LS;  // v (broadcast reads)
  const float vc = lane < p ? vrow[lane] : 0.f;
  // (H v)_c, then v^T H v and v^T v, all in float-float
  DF hv{0.f, 0.f};
  if (lane < p) {
#pragma unroll
    for (int d = 0; d < PM; ++d) df_add_product(hv, Hs[lane * PM + d], vrow[d]);
  }
  DF num{0.f, 0.f}, den{0.f, 0.f};
  df_add_product(num, vc, hv.hi);
  num.lo = fmaf(vc, hv.lo, num.lo);
  df_add_product(den, vc, vc);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float nh = __shfl_xor_sync(0xffffffffu, num.hi, o), nl = __shfl_xor_sync(0xffffffffu, num.lo, o);
    const float dh = __shfl_xor_sync(0xffffffffu, den.hi, o), dl = __shfl_xor_sync(0xffffffffu, den.lo, o);
    // the lower lane's value first, so both lanes compute the same sum
    DF a = (lane & o) ? DF{nh, nl} : num, b = (lane & o) ? num : DF{nh, nl};
    df_add(a, b.hi, b.lo);
    num = a;
    a = (lane & o) ? DF{dh, dl} : den;
    b = (lane & o) ? den : DF{dh, dl};
    df_add(a, b.hi, b.lo);
    den = a;
  }
  df_norm(num);
  df_norm(den);
  if (!(den.hi > 0.f)) return 0.0;
  if (v != nullptr && lane < p) v[lane] = vc * rsqrtf(den.hi + den.lo);
  // num / den in float-float: q0, then one correction from the exact residual
  const float q0 = num.hi / den.hi;
  const float ph = q0 * den.hi;
  const float pe = fmaf(q0, den.hi, -ph);
  const float r = ((num.hi - ph) - pe) + (num.lo - q0 * den.lo);
  return (double)q0 + (double)(r / den.hi);
}

// lambda_max of H like lambda_max_warp, by every thread of the block: the
// upper-triangle entries of each squaring are shared over all threads, with
// a barrier per squaring; the trace of the new iterate is summed by every
// thread from a double-buffered diagonal in one fixed order, so all threads
// take the same branch and the result is deterministic. Ms: 2 PM
// lam_stride<PM>() floats, dg: 2 PM floats, lam_out: one double (shared).
// Returns the value in every thread.
template <int PM>
__device__ double lambda_max_cta(const float* Hs, float* Ms, float* dg, double* lam_out, int p) {
  constexpr int LS = lam_stride<PM>();
  constexpr int E = PM * (PM + 1) / 2;
  const int tid = threadIdx.x, NT = blockDim.x;
  // the trace: every diagonal load issued first, then the sum in index order
  float dgl[PM];
#pragma unroll
  for (int c = 0; c < PM; ++c) dgl[c] = c < p ? Hs[c * PM + c] : 0.f;
  float tr = 0.f;
#pragma unroll
  for (int c = 0; c < PM; ++c)
    if (c < p) tr += dgl[c];
  if (!(tr > 0.f) || !isfinite(tr)) {
    // every thread sees the same trace: a uniform exit
    const double r = isfinite(tr) ? 0.0 : (double)tr;
    if (tid == 0) *lam_out = r;
    __syncthreads();
    return r;
  }
  float* A = Ms;
  float* B = Ms + PM * LS;
  for (int i = tid; i < PM * PM; i += NT) A[(i / PM) * LS + i % PM] = Hs[i];
  __syncthreads();
  // this thread's upper-triangle entries (i << 8 | j), found once
  constexpr int kPairs = (E + 127) / 128;  // blocks of at least 128 threads
  int pr[kPairs];
#pragma unroll
  for (int q = 0; q < kPairs; ++q) {
    const int e0 = tid + q * NT;
    int i = 0, e = e0;
    while (i < PM && e >= PM - i) {
      e -= PM - i;
      ++i;
    }
    pr[q] = e0 < E ? (i << 8) | (i + e) : -1;
  }
  float t = tr;
  int par = 0;
  for (int s = 0; s < kMaxSquarings; ++s) {
    const float sc = __fdividef(1.f, t);
    const float sc2 = sc * sc;
#pragma unroll
    for (int q = 0; q < kPairs; ++q) {
      if (pr[q] < 0) continue;
      const int i = pr[q] >> 8, j = pr[q] & 255;
      const float4* ri = reinterpret_cast<const float4*>(A + i * LS);
      const float4* rj = reinterpret_cast<const float4*>(A + j * LS);
      float s0 = 0.f, s1 = 0.f;
#pragma unroll
      for (int d4 = 0; d4 < PM / 4; ++d4) {
        const float4 x = ri[d4], z = rj[d4];
        s0 = fmaf(x.x, z.x, s0);
        s1 = fmaf(x.y, z.y, s1);
        s0 = fmaf(x.z, z.z, s0);
        s1 = fmaf(x.w, z.w, s1);
      }
      const float v = (s0 + s1) * sc2;
      B[i * LS + j] = v;
      B[j * LS + i] = v;
      if (i == j) dg[par * PM + i] = v;
    }
    __syncthreads();
    // the new trace, same order in every thread: float4 lanes, then a short tree
    float4 tq = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int c4 = 0; c4 < PM / 4; ++c4) {
      const float4 v = reinterpret_cast<const float4*>(dg + par * PM)[c4];
      tq.x += v.x;
      tq.y += v.y;
      tq.z += v.z;
      tq.w += v.w;
    }
    const float t2 = (tq.x + tq.y) + (tq.z + tq.w);
    float* tmp = A;
    A = B;
    B = tmp;
    t = t2;
    par ^= 1;
    if (!(t2 > 0.f) || 1.f - t2 < 1e-5f) break;
  }
  if (tid < 32) {
    // dominant column and its float-float Rayleigh quotient (one warp)
    const int lane = tid;
    float best = lane < p ? A[lane * LS + lane] : -1.f;
    int jb = lane;
    // lanes from PM on hold nothing (-1 here, zeros below): the butterflies
    // start at the smallest power of two covering PM lanes (the same results)
    constexpr int o0 = PM > 16 ? 16 : PM > 8 ? 8 : PM > 4 ? 4 : 2;
#pragma unroll
    for (int o = o0; o > 0; o >>= 1) {
      const float ob = __shfl_xor_sync(0xffffffffu, best, o);
      const int oj = __shfl_xor_sync(0xffffffffu, jb, o);
      if (ob > best || (ob == best && oj < jb)) {
        best = ob;
        jb = oj;
      }
    }
    const float* vrow = A + jb * LS;
    const float vc = lane < p ? vrow[lane] : 0.f;
    // (H v)_lane in four independent float-float sums, combined in a fixed order
    DF hv{0.f, 0.f};
    if (lane < p) {
      DF h1{0.f, 0.f}, h2{0.f, 0.f}, h3{0.f, 0.f};
#pragma unroll
      for (int d = 0; d < PM; d += 4) {
        df_add_product(hv, Hs[lane * PM + d], vrow[d]);
        df_add_product(h1, Hs[lane * PM + d + 1], vrow[d + 1]);
        df_add_product(h2, Hs[lane * PM + d + 2], vrow[d + 2]);
        df_add_product(h3, Hs[lane * PM + d + 3], vrow[d + 3]);
      }
      df_add(hv, h1.hi, h1.lo);
      df_add(h2, h3.hi, h3.lo);
      df_add(hv, h2.hi, h2.lo);
    }
    DF num{0.f, 0.f}, den{0.f, 0.f};
    df_add_product(num, vc, hv.hi);
    num.lo = fmaf(vc, hv.lo, num.lo);
    df_add_product(den, vc, vc);
#pragma unroll
    for (int o = o0; o > 0; o >>= 1) {
      const float nh = __shfl_xor_sync(0xffffffffu, num.hi, o), nl = __shfl_xor_sync(0xffffffffu, num.lo, o);
      const float dh = __shfl_xor_sync(0xffffffffu, den.hi, o), dl = __shfl_xor_sync(0xffffffffu, den.lo, o);
      DF a = (lane & o) ? DF{nh, nl} : num, b = (lane & o) ? num : DF{nh, nl};
      df_add(a, b.hi, b.lo);
      num = a;
      a = (lane & o) ? DF{dh, dl} : den;
      b = (lane & o) ? den : DF{dh, dl};
      df_add(a, b.hi, b.lo);
      den = a;
    }
    df_norm(num);
    df_norm(den);
    if (lane == 0) {
      double lam = 0.0;
      if (den.hi > 0.f) {
        const float q0 = num.hi / den.hi;
        const float ph = q0 * den.hi;
        const float pe = fmaf(q0, den.hi, -ph);
        const float r = ((num.hi - ph) - pe) + (num.lo - q0 * den.lo);
        lam = (double)q0 + (double)(r / den.hi);
      }
      *lam_out = lam;
    }
  }
  __syncthreads();
  return *lam_out;
}

}  // namespace nmf
