// peaks.cu -- measured FP64 and FP32 FMA throughput of this GPU, and the
// nu x nu factorisation of the orthonormalisation (LDL^T, then U^-1) timed
// in float64 against float-float: one CTA of 256 threads, one entry per
// thread, a barrier per step, as the orthonormalisation kernel does it.
// Prints one JSON object. Built and run by `python bench.py --peaks`; it is
// a measurement, not part of the library.
#include <cstdio>
#include <cstdlib>
#include <cmath>
#include <vector>
#include <cuda_runtime.h>

__global__ void dfma_kernel(double* out, int iters, double a, double b) {
  double x0 = threadIdx.x, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3, x4 = x0 + 4, x5 = x0 + 5, x6 = x0 + 6, x7 = x0 + 7;
  for (int i = 0; i < iters; ++i) {
    x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
    x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
}
__global__ void ffma_kernel(float* out, int iters, float a, float b) {
  float x0 = threadIdx.x, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3, x4 = x0 + 4, x5 = x0 + 5, x6 = x0 + 6, x7 = x0 + 7;
  for (int i = 0; i < iters; ++i) {
    x0 = fmaf(x0, a, b); x1 = fmaf(x1, a, b); x2 = fmaf(x2, a, b); x3 = fmaf(x3, a, b);
    x4 = fmaf(x4, a, b); x5 = fmaf(x5, a, b); x6 = fmaf(x6, a, b); x7 = fmaf(x7, a, b);
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
}

constexpr int kAs = 65;
struct FF { float hi, lo; };
__device__ __forceinline__ FF ff_quick(float a, float b) { const float s = a + b; return FF{s, b - (s - a)}; }
__device__ __forceinline__ FF ff_add(FF x, FF y) {
  const float s = x.hi + y.hi; const float bb = s - x.hi;
  float e = (x.hi - (s - bb)) + (y.hi - bb); e += x.lo + y.lo; return ff_quick(s, e);
}
__device__ __forceinline__ FF ff_neg(FF x) { return FF{-x.hi, -x.lo}; }
__device__ __forceinline__ FF ff_mul(FF x, FF y) {
  const float p = x.hi * y.hi; float e = fmaf(x.hi, y.hi, -p); e = fmaf(x.hi, y.lo, e); e = fmaf(x.lo, y.hi, e);
  return ff_quick(p, e);
}
__device__ __forceinline__ FF ff_div(FF x, FF y) {
  const float q1 = x.hi / y.hi; const FF r = ff_add(x, ff_neg(ff_mul(y, FF{q1, 0.f})));
  const float q2 = r.hi / y.hi; return ff_quick(q1, q2);
}
__device__ __forceinline__ void tri_index(int e, int nu, int& a, int& b) {
  a = 0; while (e >= nu - a) { e -= nu - a; ++a; } b = a + e;
}

// out[0] = cycles of LDL^T + U^-1 (float64), out[1] = the same in float-float, each summed over reps
__global__ void factor_kernel(const double* S, int nu, int reps, long long* out, double* res) {
  extern __shared__ double dyn[];
  double* Ad = dyn;
  double* Id = Ad + 64 * kAs;
  float* Ahi = reinterpret_cast<float*>(Id + 64 * kAs);
  float* Alo = Ahi + 64 * kAs;
  float* Ihi = Alo + 64 * kAs;
  float* Ilo = Ihi + 64 * kAs;
  __shared__ double Dinv_d[64];
  __shared__ float Dinv_hi[64], Dinv_lo[64];
  const int tid = threadIdx.x, NT = blockDim.x, E = nu * (nu + 1) / 2;
  long long c64 = 0, cff = 0;
  for (int rep = 0; rep < reps; ++rep) {
    for (int e = tid; e < nu * nu; e += NT) {
      const int a = e / nu, b = e % nu;
      Ad[a * kAs + b] = S[e];
      Ahi[a * kAs + b] = (float)S[e];
      Alo[a * kAs + b] = (float)(S[e] - (double)(float)S[e]);
    }
    __syncthreads();
    long long t0 = clock64();
    // float64: LDL^T right-looking, one barrier per step
    for (int j = 0; j < nu; ++j) {
      const double inv = 1.0 / Ad[j * kAs + j];
      if (tid == 0) Dinv_d[j] = inv;
      for (int e = tid; e < E; e += NT) {
        int i, k; tri_index(e, nu, i, k);
        if (i <= j) continue;
        Ad[i * kAs + k] -= (Ad[j * kAs + i] * inv) * Ad[j * kAs + k];
      }
      __syncthreads();
    }
    for (int e = tid; e < E; e += NT) { int i, k; tri_index(e, nu, i, k); if (i < k) Ad[i * kAs + k] *= Dinv_d[i]; }
    for (int e = tid; e < nu * kAs; e += NT) Id[e] = (e / kAs == e % kAs) ? 1.0 : 0.0;
    __syncthreads();
    for (int k = nu - 1; k >= 1; --k) {
      const int w = nu - k;
      for (int t = tid; t < k * w; t += NT) { const int i = t / w, c = k + t % w; Id[i * kAs + c] -= Ad[i * kAs + k] * Id[k * kAs + c]; }
      __syncthreads();
    }
    long long t1 = clock64();
    // float-float: the same steps
    for (int j = 0; j < nu; ++j) {
      const FF d{Ahi[j * kAs + j], Alo[j * kAs + j]};
      const FF inv = ff_div(FF{1.f, 0.f}, d);
      if (tid == 0) { Dinv_hi[j] = inv.hi; Dinv_lo[j] = inv.lo; }
      for (int e = tid; e < E; e += NT) {
        int i, k; tri_index(e, nu, i, k);
        if (i <= j) continue;
        const FF l = ff_mul(FF{Ahi[j * kAs + i], Alo[j * kAs + i]}, inv);
        const FF v = ff_add(FF{Ahi[i * kAs + k], Alo[i * kAs + k]}, ff_neg(ff_mul(l, FF{Ahi[j * kAs + k], Alo[j * kAs + k]})));
        Ahi[i * kAs + k] = v.hi; Alo[i * kAs + k] = v.lo;
      }
      __syncthreads();
    }
    for (int e = tid; e < E; e += NT) {
      int i, k; tri_index(e, nu, i, k);
      if (i < k) { const FF u = ff_mul(FF{Ahi[i * kAs + k], Alo[i * kAs + k]}, FF{Dinv_hi[i], Dinv_lo[i]}); Ahi[i * kAs + k] = u.hi; Alo[i * kAs + k] = u.lo; }
    }
    for (int e = tid; e < nu * kAs; e += NT) { Ihi[e] = (e / kAs == e % kAs) ? 1.f : 0.f; Ilo[e] = 0.f; }
    __syncthreads();
    for (int k = nu - 1; k >= 1; --k) {
      const int w = nu - k;
      for (int t = tid; t < k * w; t += NT) {
        const int i = t / w, c = k + t % w;
        const FF v = ff_add(FF{Ihi[i * kAs + c], Ilo[i * kAs + c]}, ff_neg(ff_mul(FF{Ahi[i * kAs + k], Alo[i * kAs + k]}, FF{Ihi[k * kAs + c], Ilo[k * kAs + c]})));
        Ihi[i * kAs + c] = v.hi; Ilo[i * kAs + c] = v.lo;
      }
      __syncthreads();
    }
    long long t2 = clock64();
    c64 += t1 - t0; cff += t2 - t1;
  }
  if (tid == 0) {
    out[0] = c64; out[1] = cff;
    double md = 0;  // agreement of the two inverses (float-float value vs float64)
    for (int i = 0; i < nu; ++i) for (int c = i; c < nu; ++c) md = fmax(md, fabs(((double)Ihi[i * kAs + c] + (double)Ilo[i * kAs + c]) - Id[i * kAs + c]) / fmax(1e-300, fabs(Id[i * kAs + c])));
    res[0] = md;
  }
}

int main() {
  int dev = 0, sms = 0, clk = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&clk, cudaDevAttrClockRate, dev);
  const int blocks = sms * 8, threads = 256, iters = 1 << 14;
  double* od; float* of;
  cudaMalloc(&od, sizeof(double) * blocks * threads);
  cudaMalloc(&of, sizeof(float) * blocks * threads);
  cudaEvent_t e0, e1; cudaEventCreate(&e0); cudaEventCreate(&e1);
  float ms = 0;
  for (int w = 0; w < 2; ++w) dfma_kernel<<<blocks, threads>>>(od, iters / 16, 1.0000001, 1e-9);
  cudaEventRecord(e0); dfma_kernel<<<blocks, threads>>>(od, iters / 16, 1.0000001, 1e-9); cudaEventRecord(e1);
  cudaEventSynchronize(e1); cudaEventElapsedTime(&ms, e0, e1);
  const double f64 = 2.0 * 8 * (iters / 16) * (double)blocks * threads / (ms * 1e-3) / 1e12;
  for (int w = 0; w < 2; ++w) ffma_kernel<<<blocks, threads>>>(of, iters, 1.0000001f, 1e-9f);
  cudaEventRecord(e0); ffma_kernel<<<blocks, threads>>>(of, iters, 1.0000001f, 1e-9f); cudaEventRecord(e1);
  cudaEventSynchronize(e1); cudaEventElapsedTime(&ms, e0, e1);
  const double f32 = 2.0 * 8 * iters * (double)blocks * threads / (ms * 1e-3) / 1e12;
  printf("{\"fp64_fma_tflops\": %.4f, \"fp32_fma_tflops\": %.3f, \"sms\": %d, \"clock_khz\": %d", f64, f32, sms, clk);
  for (int nu : {20, 26, 42, 64}) {
    std::vector<double> A((nu + 8) * nu), S(nu * nu);
    srand(nu);
    for (auto& x : A) x = (double)rand() / RAND_MAX - 0.5;
    for (int i = 0; i < nu; ++i) for (int j = 0; j < nu; ++j) { double s = 0; for (int k = 0; k < nu + 8; ++k) s += A[k * nu + i] * A[k * nu + j]; S[i * nu + j] = s + (i == j ? 1e-3 : 0); }
    double* Sd; long long* cyc; double* res;
    cudaMalloc(&Sd, sizeof(double) * nu * nu); cudaMalloc(&cyc, 16); cudaMalloc(&res, 8);
    cudaMemcpy(Sd, S.data(), sizeof(double) * nu * nu, cudaMemcpyHostToDevice);
    const size_t smem = (size_t)64 * kAs * (2 * sizeof(double) + 4 * sizeof(float));
    cudaFuncSetAttribute(factor_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    factor_kernel<<<1, 256, smem>>>(Sd, nu, 2, cyc, res);
    factor_kernel<<<1, 256, smem>>>(Sd, nu, 20, cyc, res);
    long long c[2]; double r;
    cudaMemcpy(c, cyc, 16, cudaMemcpyDeviceToHost); cudaMemcpy(&r, res, 8, cudaMemcpyDeviceToHost);
    printf(", \"nu%d\": {\"f64_cycles\": %lld, \"ff_cycles\": %lld, \"max_rel_diff\": %.2e}", nu, c[0] / 20, c[1] / 20, r);
    cudaFree(Sd); cudaFree(cyc); cudaFree(res);
  }
  printf("}\n");
  return cudaGetLastError() == cudaSuccess ? 0 : 1;
}
