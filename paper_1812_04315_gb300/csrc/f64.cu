// f64.cu -- float64 twins of nmf_compress (Alg. 2 and the compression step
// of Alg. 1) and nenmf_solve (Alg. 1 / plain NeNMF with the inner loop of
// Sec. 2): the same steps in the same order, computed in float64 on the GPU.
// They exist for parity at tight tolerances on small problems, not for speed
// (float64 runs at 1/64 of the float32 rate here): every product is a
// deterministic one-output-per-thread loop, the small factorisations run in
// one thread, and each inner solve is one CTA.
#include <math.h>

#include "internal.h"

// Returns the failing runtime status from a helper that returns cudaError_t.
#define F64_CU(call)                            \
  do {                                          \
    cudaError_t e_ = (call);                    \
    if (e_ != cudaSuccess) return e_;           \
  } while (0)

namespace nmf {
namespace {

constexpr int kMaxP64 = 32;
constexpr int kNnlsThreads = 256;
constexpr double kRestartTol64 = 1e-5;  // the float32 path's restart threshold (a relative rise)

int grid64(long long work, int threads) {
  long long b = (work + threads - 1) / threads;
  const long long cap = 8ll * device_sm_count();
  if (b > cap) b = cap;
  return (int)(b < 1 ? 1 : b);
}

// C (M x N, row stride ldc) = A (M x K) B (K x N) with A(i, k) = A[i ars + k acs]
// and B(k, j) = B[k brs + j bcs]; one output per thread, k ascending.
__global__ void gemm_f64_kernel(int M, int N, int K, const double* __restrict__ A, long long ars, long long acs,
                                const double* __restrict__ B, long long brs, long long bcs, double* __restrict__ C,
                                long long ldc, int accumulate, double alpha, Control* ctrl) {
  if (call_failed(ctrl)) return;
  const long long total = (long long)M * N;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const long long i = idx / N, j = idx % N;
    double s = 0.0;
    for (int k = 0; k < K; ++k) s = fma(A[i * ars + k * acs], B[k * brs + j * bcs], s);
    C[i * ldc + j] = accumulate ? C[i * ldc + j] + alpha * s : alpha * s;
  }
}

cudaError_t gemm64(int M, int N, int K, const double* A, long long ars, long long acs, const double* B, long long brs,
                   long long bcs, double* C, long long ldc, Control* ctrl, cudaStream_t s) {
  count_launches(1);
  gemm_f64_kernel<<<grid64((long long)M * N, 256), 256, 0, s>>>(M, N, K, A, ars, acs, B, brs, bcs, C, ldc, 0, 1.0,
                                                                  ctrl);
  return cudaGetLastError();
}

// C += alpha A B (same layouts as gemm64).
cudaError_t gemm64_acc(int M, int N, int K, const double* A, long long ars, long long acs, const double* B,
                       long long brs, long long bcs, double* C, long long ldc, double alpha, Control* ctrl,
                       cudaStream_t s) {
  count_launches(1);
  gemm_f64_kernel<<<grid64((long long)M * N, 256), 256, 0, s>>>(M, N, K, A, ars, acs, B, brs, bcs, C, ldc, 1, alpha,
                                                                  ctrl);
  return cudaGetLastError();
}

__global__ void widen_kernel(const float* in, long long count, double* out) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count;
       i += (long long)gridDim.x * blockDim.x)
    out[i] = (double)in[i];
}

// out (C x R) = in^T for in (R x C).
__global__ void transpose_f64_kernel(const double* in, int R, int C, double* out, Control* ctrl) {
  if (ctrl && call_failed(ctrl)) return;
  const long long total = (long long)R * C;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const long long r = idx / C, c = idx % C;
    out[c * R + r] = in[idx];
  }
}

cudaError_t transpose64(const double* in, int R, int C, double* out, Control* ctrl, cudaStream_t s) {
  count_launches(1);
  transpose_f64_kernel<<<grid64((long long)R * C, 256), 256, 0, s>>>(in, R, C, out, ctrl);
  return cudaGetLastError();
}

// S = R^T R (R upper triangular, positive diagonal) by the Cholesky
// recurrence, then R^{-1} by back substitution; one thread. S is k x k; A
// (scratch) and Rinv are k x k. With `shift_ok`, a pivot that is not safely
// positive (below 1e-24 of the largest diagonal entry) restarts the
// factorisation of S + 1e-14 tr(S) I (shifted CholeskyQR, Fukaya et al.
// 2020): the passes that follow restore orthogonality. Without it, such a
// pivot is NMF_ERR_NOT_SPD.
__global__ void chol_inv_f64_kernel(const double* S, int k, double* A, double* Rinv, int shift_ok, Control* ctrl) {
  if (call_failed(ctrl) || threadIdx.x != 0 || blockIdx.x != 0) return;
  double tr = 0.0, md = 0.0;
  for (int i = 0; i < k; ++i) {
    tr += S[i * k + i];
    md = fmax(md, S[i * k + i]);
  }
  if (!isfinite(tr)) {
    set_status(ctrl, NMF_ERR_NONFINITE);
    return;
  }
  if (!(md > 0.0)) {
    set_status(ctrl, NMF_ERR_NOT_SPD);
    return;
  }
  const double floor = 1e-24 * md;
  bool ok = false;
  for (int attempt = 0; attempt < 2 && !ok; ++attempt) {
    if (attempt == 1 && !shift_ok) break;
    const double shift = attempt == 1 ? 1e-14 * tr : 0.0;
    ok = true;
    for (int j = 0; j < k && ok; ++j) {
      for (int i = 0; i < j; ++i) {
        double v = S[i * k + j];
        for (int l = 0; l < i; ++l) v -= A[l * k + i] * A[l * k + j];
        A[i * k + j] = v / A[i * k + i];
      }
      double d = S[j * k + j] + shift;
      for (int l = 0; l < j; ++l) d -= A[l * k + j] * A[l * k + j];
      if (!(d > floor)) {
        ok = false;
      } else {
        A[j * k + j] = sqrt(d);
      }
    }
  }
  if (!ok) {
    set_status(ctrl, NMF_ERR_NOT_SPD);
    return;
  }
  // R^{-1}, column c: x_c = 1 / R_cc, x_i = -(sum_{l = i+1..c} R_il x_l) / R_ii
  for (int c = 0; c < k; ++c) {
    for (int i = c + 1; i < k; ++i) Rinv[i * k + c] = 0.0;
    Rinv[c * k + c] = 1.0 / A[c * k + c];
    for (int i = c - 1; i >= 0; --i) {
      double s = 0.0;
      for (int l = i + 1; l <= c; ++l) s += A[i * k + l] * Rinv[l * k + c];
      Rinv[i * k + c] = -s / A[i * k + i];
    }
  }
}

struct Orth64 {
  double* S;     // k x k
  double* A;     // k x k
  double* Rinv;  // k x k
  double* T;     // N x k
};

// Q (N x k) with orthonormal columns and span(Q) = span(Y): CholeskyQR in
// three passes (the first one shifted when needed). Y and Q may alias.
cudaError_t orth64(const double* Y, int N, int k, double* Q, const Orth64& w, Control* ctrl, cudaStream_t s) {
  const double* src = Y;
  for (int pass = 0; pass < 3; ++pass) {
    // S = src^T src
    F64_CU(gemm64(k, k, N, src, 1, k, src, k, 1, w.S, k, ctrl, s));
    count_launches(1);
    chol_inv_f64_kernel<<<1, 1, 0, s>>>(w.S, k, w.A, w.Rinv, pass == 0 ? 1 : 0, ctrl);
    F64_CU(cudaGetLastError());
    // out = src R^{-1}
    double* out = pass == 2 ? Q : w.T;
    if (out == src) out = pass == 2 ? w.T : Q;
    F64_CU(gemm64(N, k, k, src, k, 1, w.Rinv, k, 1, out, k, ctrl, s));
    src = out;
  }
  if (src != Q) F64_CU(cudaMemcpyAsync(Q, src, sizeof(double) * (size_t)N * k, cudaMemcpyDeviceToDevice, s));
  return cudaSuccess;
}

// beta_k = (alpha_k - 1) / alpha_{k+1}, alpha_0 = 1,
// alpha_{k+1} = (1 + sqrt(4 alpha_k^2 + 1)) / 2 (Sec. 2), in float64.
__global__ void beta_f64_kernel(double* beta, int K) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double a = 1.0;
  for (int k = 0; k < K; ++k) {
    const double an = (1.0 + sqrt(4.0 * a * a + 1.0)) / 2.0;
    beta[k] = (a - 1.0) / an;
    a = an;
  }
}

// lambda_max of the symmetric p x p H by cyclic Jacobi rotations (one
// thread; A is p x p scratch), written to *lam; with V (p x p scratch) and
// v (p), also the unit eigenvector of lambda_max (the rotations accumulated).
__global__ void lambda_f64_kernel(const double* H, int p, double* A, double* lam, double* V, double* v,
                                  Control* ctrl) {
  if (call_failed(ctrl) || threadIdx.x != 0 || blockIdx.x != 0) return;
  if (V)
    for (int i = 0; i < p * p; ++i) V[i] = (i / p == i % p) ? 1.0 : 0.0;
  double nrm = 0.0;
  for (int i = 0; i < p * p; ++i) {
    A[i] = H[i];
    nrm += H[i] * H[i];
  }
  if (!isfinite(nrm)) {
    set_status(ctrl, NMF_ERR_NONFINITE);
    *lam = 0.0;
    return;
  }
  for (int sweep = 0; sweep < 64; ++sweep) {
    double off = 0.0;
    for (int i = 0; i < p; ++i)
      for (int j = i + 1; j < p; ++j) off += A[i * p + j] * A[i * p + j];
    if (off <= 1e-36 * nrm) break;
    for (int i = 0; i < p; ++i)
      for (int j = i + 1; j < p; ++j) {
        const double aij = A[i * p + j];
        if (aij == 0.0) continue;
        // rotation zeroing A_ij (Golub and Van Loan, Alg. 8.5.1)
        const double tau = (A[j * p + j] - A[i * p + i]) / (2.0 * aij);
        const double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
        const double c = 1.0 / sqrt(1.0 + t * t), sn = t * c;
        for (int l = 0; l < p; ++l) {  // columns i, j
          const double x = A[l * p + i], y = A[l * p + j];
          A[l * p + i] = c * x - sn * y;
          A[l * p + j] = sn * x + c * y;
        }
        for (int l = 0; l < p; ++l) {  // rows i, j
          const double x = A[i * p + l], y = A[j * p + l];
          A[i * p + l] = c * x - sn * y;
          A[j * p + l] = sn * x + c * y;
        }
        if (V)
          for (int l = 0; l < p; ++l) {  // V J: eigenvectors in the columns of V
            const double x = V[l * p + i], y = V[l * p + j];
            V[l * p + i] = c * x - sn * y;
            V[l * p + j] = sn * x + c * y;
          }
      }
  }
  int im = 0;
  for (int i = 1; i < p; ++i)
    if (A[i * p + i] > A[im * p + im]) im = i;
  *lam = A[im * p + im];
  if (V)
    for (int l = 0; l < p; ++l) v[l] = V[l * p + im];
}

// Fixed-order sum over the block of one double per thread (valid in thread 0).
__device__ double block_sum64(double v, double* red) {
  red[threadIdx.x] = v;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  const double r = red[0];
  __syncthreads();
  return r;
}

__device__ __forceinline__ double pg_term(double f, double g) {
  const double v = f > 0.0 ? g : fmin(g, 0.0);
  return v * v;
}

// sum ||P grad||^2 over the columns of a p x N unknown F with grad = H F - B,
// added to *out (one CTA).
__global__ void pg2_f64_kernel(const double* H, const double* B, const double* F, int p, int N, double* out,
                               Control* ctrl) {
  __shared__ double red[kNnlsThreads];
  __shared__ double Hs[kMaxP64 * kMaxP64];
  if (call_failed(ctrl)) return;
  for (int i = threadIdx.x; i < p * p; i += blockDim.x) Hs[i] = H[i];
  __syncthreads();
  double acc = 0.0;
  for (int j = threadIdx.x; j < N; j += blockDim.x) {
    for (int c = 0; c < p; ++c) {
      double g = -B[(size_t)c * N + j];
      for (int d = 0; d < p; ++d) g = fma(Hs[c * p + d], F[(size_t)d * N + j], g);
      acc += pg_term(F[(size_t)c * N + j], g);
    }
  }
  const double s = block_sum64(acc, red);
  if (threadIdx.x == 0) *out += s;
}

__global__ void eps_f64_kernel(double* pg2_init, double tol, int tol_mode, double* eps2, nenmf_stats_t* st) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double e2 = -1.0;
  if (tol > 0.0) e2 = tol_mode == NENMF_TOL_ABS ? tol * tol : tol * tol * (*pg2_init);
  *eps2 = e2;
  if (st) st->eps = e2 > 0.0 ? sqrt(e2) : 0.0;
}

// The inner loop of Sec. 2 on the columns of a p x N unknown (F in, F out),
// one CTA: Y_0 = F, F_{-1} = F; per k: F_k = max(0, Y_k - (H Y_k - B) / L_c),
// Y_{k+1} = F_k + beta_{r} (F_k - F_{k-1}) (r: iterations since the column's
// last restart, or k without restart); stop once k + 1 >= min_inner and
// ||P grad(F_k)||_F^2 <= eps^2. Y, Fp (p x N), obj (N), r (N) are scratch.
__global__ void nnls_f64_kernel(const double* H, const double* B, double* F, int p, int N, const double* lam_p,
                                const double* beta, int max_inner, int min_inner, const double* eps2_p, int restart,
                                double* Y, double* Fp, double* obj, int* rc, nenmf_stats_t* st, int side,
                                Control* ctrl) {
  __shared__ double red[kNnlsThreads];
  __shared__ double Hs[kMaxP64 * kMaxP64];
  __shared__ int stop_s;
  if (call_failed(ctrl)) return;
  for (int i = threadIdx.x; i < p * p; i += blockDim.x) Hs[i] = H[i];
  const double Lc = *lam_p;
  const double eps2 = *eps2_p;
  for (int j = threadIdx.x; j < N; j += blockDim.x) {
    for (int c = 0; c < p; ++c) {
      Y[(size_t)c * N + j] = F[(size_t)c * N + j];
      Fp[(size_t)c * N + j] = F[(size_t)c * N + j];
    }
    rc[j] = 0;
    obj[j] = 0.0;
  }
  __syncthreads();
  int iters = 0;
  double pg2 = 0.0;
  if (Lc > 0.0) {
    for (int k = 0; k < max_inner; ++k) {
      double acc = 0.0;
      for (int j = threadIdx.x; j < N; j += blockDim.x) {
        double y[kMaxP64], f[kMaxP64], hf[kMaxP64];
        for (int c = 0; c < p; ++c) y[c] = Y[(size_t)c * N + j];
        for (int c = 0; c < p; ++c) {
          double g = -B[(size_t)c * N + j];
          for (int d = 0; d < p; ++d) g = fma(Hs[c * p + d], y[d], g);
          f[c] = fmax(0.0, y[c] - g / Lc);
        }
        for (int c = 0; c < p; ++c) {
          double h = 0.0;
          for (int d = 0; d < p; ++d) h = fma(Hs[c * p + d], f[d], h);
          hf[c] = h;
        }
        int r = restart ? rc[j] : k;
        if (restart) {
          // 1/2 f^T H f - b^T f and its term scale sum |f| (|H f - b| + |b|)
          double o = 0.0, sc = 0.0;
          for (int c = 0; c < p; ++c) {
            const double b = B[(size_t)c * N + j];
            o += 0.5 * f[c] * hf[c] - b * f[c];
            sc += fabs(f[c]) * (fabs(hf[c] - b) + fabs(b));
          }
          if (k >= 1 && o - obj[j] > kRestartTol64 * sc) r = 0;
          obj[j] = o;
          rc[j] = r + 1;
        }
        const double bt = beta[r];
        for (int c = 0; c < p; ++c) {
          const double fp = Fp[(size_t)c * N + j];
          Y[(size_t)c * N + j] = f[c] + bt * (f[c] - fp);
          Fp[(size_t)c * N + j] = f[c];
          F[(size_t)c * N + j] = f[c];
          acc += pg_term(f[c], hf[c] - B[(size_t)c * N + j]);
        }
      }
      pg2 = block_sum64(acc, red);
      iters = k + 1;
      if (threadIdx.x == 0) stop_s = (eps2 >= 0.0 && k + 1 >= min_inner && pg2 <= eps2) ? 1 : 0;
      __syncthreads();
      if (stop_s) break;
      __syncthreads();
    }
  } else {
    // H = 0: the subproblem is constant; Y_0 is returned after zero iterations
    double acc = 0.0;
    for (int j = threadIdx.x; j < N; j += blockDim.x)
      for (int c = 0; c < p; ++c) acc += pg_term(F[(size_t)c * N + j], -B[(size_t)c * N + j]);
    pg2 = block_sum64(acc, red);
  }
  if (threadIdx.x == 0 && st) {
    st->last_inner[side] = iters;
    st->total_inner[side] += iters;
    st->pg_norm[side] = sqrt(pg2);
    st->lipschitz[side] = Lc;
  }
}

// ---- reverse mode (the derivative of K unrolled inner iterations) ----------
// Tapes are [p][K][N] (row c of every iteration contiguous), so that
// dH = -(1/L_c) sum_k dz_k Y_k^T is one product over the (k, j) pairs.

// K iterations of the inner loop (no stop test, no restart) on the columns
// of Y0 (p x N), recording Y_k (the point the step starts from) and z_k
// (before the projection); Fout = F_{K-1}. With L_c <= 0, Fout = Y0.
__global__ void nnls_tape_f64_kernel(const double* H, const double* B, const double* Y0, double* Fout, int p, int N,
                                     int K, const double* lam_p, const double* beta, double* tapeY, double* tapeZ,
                                     Control* ctrl) {
  __shared__ double Hs[kMaxP64 * kMaxP64];
  if (call_failed(ctrl)) return;
  for (int i = threadIdx.x; i < p * p; i += blockDim.x) Hs[i] = H[i];
  __syncthreads();
  const double Lc = *lam_p;
  const size_t KN = (size_t)K * N;
  for (int j = threadIdx.x; j < N; j += blockDim.x) {
    double y[kMaxP64], f[kMaxP64], fp[kMaxP64];
    for (int c = 0; c < p; ++c) y[c] = fp[c] = f[c] = Y0[(size_t)c * N + j];
    if (Lc > 0.0) {
      for (int k = 0; k < K; ++k) {
        for (int c = 0; c < p; ++c) {
          double g = -B[(size_t)c * N + j];
          for (int d = 0; d < p; ++d) g = fma(Hs[c * p + d], y[d], g);
          const double z = y[c] - g / Lc;
          tapeY[c * KN + (size_t)k * N + j] = y[c];
          tapeZ[c * KN + (size_t)k * N + j] = z;
          f[c] = fmax(0.0, z);
        }
        for (int c = 0; c < p; ++c) {
          y[c] = f[c] + beta[k] * (f[c] - fp[c]);
          fp[c] = f[c];
        }
      }
    }
    for (int c = 0; c < p; ++c) Fout[(size_t)c * N + j] = f[c];
  }
}

// The adjoint of those K iterations for cotangent dOut (p x N), k = K-1..0:
//   dF_k = dOut [k = K-1] + carry + (1 + beta_k) dY_{k+1},  carry' = -beta_k dY_{k+1};
//   dz_k = 1[z_k > 0] dF_k;  dY_k = dz_k - H dz_k / L_c;
//   dB += dz_k / L_c;  dL_c += <Y_k - z_k, dz_k> / L_c;
// then dY0 = dY_0 + carry (F_{-1} = Y_0). Writes dY0 and dB (p x N), dz_k to
// tapeDZ, and dL_c (summed over the block in a fixed order) to *dL.
// With L_c <= 0 the map is the identity: dY0 = dOut, dB = 0, dL = 0.
__global__ void nnls_adj_f64_kernel(const double* H, const double* dOut, int p, int N, int K, const double* lam_p,
                                    const double* beta, const double* tapeY, const double* tapeZ, double* tapeDZ,
                                    double* dY0, double* dB, double* dL, Control* ctrl) {
  __shared__ double red[kNnlsThreads];
  __shared__ double Hs[kMaxP64 * kMaxP64];
  if (call_failed(ctrl)) return;
  for (int i = threadIdx.x; i < p * p; i += blockDim.x) Hs[i] = H[i];
  __syncthreads();
  const double Lc = *lam_p;
  const size_t KN = (size_t)K * N;
  double acc = 0.0;
  for (int j = threadIdx.x; j < N; j += blockDim.x) {
    if (!(Lc > 0.0)) {
      for (int c = 0; c < p; ++c) {
        dY0[(size_t)c * N + j] = dOut[(size_t)c * N + j];
        dB[(size_t)c * N + j] = 0.0;
      }
      continue;
    }
    double dyn[kMaxP64], carry[kMaxP64], dz[kMaxP64], db[kMaxP64];
    for (int c = 0; c < p; ++c) dyn[c] = carry[c] = db[c] = 0.0;
    for (int k = K - 1; k >= 0; --k) {
      for (int c = 0; c < p; ++c) {
        const double dF = (k == K - 1 ? dOut[(size_t)c * N + j] : 0.0) + carry[c] + (1.0 + beta[k]) * dyn[c];
        carry[c] = -beta[k] * dyn[c];
        const size_t t = c * KN + (size_t)k * N + j;
        const double z = tapeZ[t];
        dz[c] = z > 0.0 ? dF : 0.0;
        tapeDZ[t] = dz[c];
        db[c] += dz[c] / Lc;
        acc += (tapeY[t] - z) * dz[c] / Lc;
      }
      for (int c = 0; c < p; ++c) {
        double h = 0.0;
        for (int d = 0; d < p; ++d) h = fma(Hs[c * p + d], dz[d], h);
        dyn[c] = dz[c] - h / Lc;
      }
    }
    for (int c = 0; c < p; ++c) {
      dY0[(size_t)c * N + j] = dyn[c] + carry[c];
      dB[(size_t)c * N + j] = db[c];
    }
  }
  const double s = block_sum64(acc, red);
  if (threadIdx.x == 0) *dL = s;
}

// dH (p x p) := (dH + dL v v^T), then S := dH + dH^T (one thread per entry).
__global__ void dh_finish_f64_kernel(double* dH, const double* dL, const double* v, int p, double* S,
                                     Control* ctrl) {
  if (call_failed(ctrl)) return;
  __shared__ double T[kMaxP64 * kMaxP64];
  for (int i = threadIdx.x; i < p * p; i += blockDim.x) T[i] = dH[i] + (*dL) * v[i / p] * v[i % p];
  __syncthreads();
  for (int i = threadIdx.x; i < p * p; i += blockDim.x) S[i] = T[i] + T[(i % p) * p + i / p];
}

// dH *= -1 / L_c (0 when L_c <= 0: the solve made no step).
__global__ void scale_by_lam_kernel(double* dH, int p, const double* lam_p, Control* ctrl) {
  if (call_failed(ctrl)) return;
  const double Lc = *lam_p;
  for (int i = threadIdx.x; i < p * p; i += blockDim.x) dH[i] = Lc > 0.0 ? -dH[i] / Lc : 0.0;
}

__global__ void finish_f64_kernel(nenmf_stats_t* st, int outer, Control* ctrl) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  st->outer_done = outer;
  st->status = ctrl->status;
}

}  // namespace
}  // namespace nmf

using namespace nmf;

namespace {

struct Compress64Ws {
  Control* ctrl;
  float* sk;      // float draw of a sketch (seeded path)
  double* omL;    // m x nu
  double* omR;    // nu x n
  double* QL;     // n x nu
  double* QR;     // m x nu (Q_R^T)
  double* T1;     // max(n, m) x nu
  Orth64 o;
  size_t bytes;
};

Compress64Ws carve_compress64(void* base, int n, int m, int nu) {
  Compress64Ws w{};
  Carver cv(base);
  const size_t big = (size_t)(n > m ? n : m) * nu;
  w.ctrl = cv.take<Control>(1);
  w.sk = cv.take<float>(big);
  w.omL = cv.take<double>((size_t)m * nu);
  w.omR = cv.take<double>((size_t)nu * n);
  w.QL = cv.take<double>((size_t)n * nu);
  w.QR = cv.take<double>((size_t)m * nu);
  w.T1 = cv.take<double>(big);
  w.o.S = cv.take<double>((size_t)nu * nu);
  w.o.A = cv.take<double>((size_t)nu * nu);
  w.o.Rinv = cv.take<double>((size_t)nu * nu);
  w.o.T = cv.take<double>(big);
  w.bytes = cv.size();
  return w;
}

// The caller's workspace: present, 256-byte aligned, large enough.
bool ws64_ok(const void* ws, size_t bytes, size_t need) {
  return ws && (reinterpret_cast<uintptr_t>(ws) & 255u) == 0 && bytes >= need;
}

bool compress64_args_ok(int n, int m, int nu, int q) {
  return n >= 1 && m >= 1 && nu >= 1 && nu <= NMF_MAX_SKETCH && nu <= n && nu <= m && q >= 0 && q <= 64;
}

struct Solve64Ws {
  Control* ctrl;
  double* Gt;     // p x n
  double* Bm;     // p x max(n, m)
  double* Y;      // p x max(n, m)
  double* Fp;     // p x max(n, m)
  double* obj;    // max(n, m)
  int* rc;        // max(n, m)
  double* W;      // max(p, nu) x max(p, nu): F R (p x nu) or L G (nu x p)
  double* H;      // p x p
  double* J;      // p x p Jacobi scratch
  double* lam;
  double* beta;   // max_inner (kMaxInnerIters)
  double* pg2;    // initial joint ||P grad||^2
  double* eps2;
  size_t bytes;
};

Solve64Ws carve_solve64(void* base, const nenmf_problem_f64_t& pr) {
  Solve64Ws w{};
  Carver cv(base);
  const int N = pr.n > pr.m ? pr.n : pr.m;
  const int k = pr.mode == NENMF_COMPRESSED ? (pr.p > pr.nu ? pr.p : pr.nu) : pr.p;
  w.ctrl = cv.take<Control>(1);
  w.Gt = cv.take<double>((size_t)pr.p * pr.n);
  w.Bm = cv.take<double>((size_t)pr.p * N);
  w.Y = cv.take<double>((size_t)pr.p * N);
  w.Fp = cv.take<double>((size_t)pr.p * N);
  w.obj = cv.take<double>(N);
  w.rc = cv.take<int>(N);
  w.W = cv.take<double>((size_t)k * k);
  w.H = cv.take<double>((size_t)pr.p * pr.p);
  w.J = cv.take<double>((size_t)pr.p * pr.p);
  w.lam = cv.take<double>(1);
  w.beta = cv.take<double>(kMaxInnerIters);
  w.pg2 = cv.take<double>(1);
  w.eps2 = cv.take<double>(1);
  w.bytes = cv.size();
  return w;
}

bool problem64_ok(const nenmf_problem_f64_t* pr) {
  if (!pr) return false;
  if (pr->n < 1 || pr->m < 1 || pr->p < 1 || pr->p > kMaxP64 || pr->p > pr->n || pr->p > pr->m) return false;
  if (pr->mode == NENMF_PLAIN) return pr->X != nullptr;
  if (pr->mode != NENMF_COMPRESSED) return false;
  return pr->nu >= pr->p && pr->nu <= NMF_MAX_SKETCH && pr->nu <= pr->n && pr->nu <= pr->m && pr->L && pr->R &&
         pr->XL && pr->XR;
}

// H (p x p) and B (p x N) of the G update (the unknown is G^T, N = n).
cudaError_t g_side(const nenmf_problem_f64_t& pr, const double* F, const Solve64Ws& w, cudaStream_t s) {
  const int n = pr.n, m = pr.m, p = pr.p, nu = pr.nu;
  Control* c = w.ctrl;
  if (pr.mode == NENMF_PLAIN) {
    F64_CU(gemm64(p, p, m, F, m, 1, F, 1, m, w.H, p, c, s));         // F F^T
    F64_CU(gemm64(p, n, m, F, m, 1, pr.X, 1, m, w.Bm, n, c, s));     // F X^T
  } else {
    F64_CU(gemm64(p, nu, m, F, m, 1, pr.R, nu, 1, w.W, nu, c, s));   // F_R = F R
    F64_CU(gemm64(p, p, nu, w.W, nu, 1, w.W, 1, nu, w.H, p, c, s));  // F_R F_R^T
    F64_CU(gemm64(p, n, nu, w.W, nu, 1, pr.XR, 1, nu, w.Bm, n, c, s));  // F_R X_R^T
  }
  return cudaSuccess;
}

// H (p x p) and B (p x m) of the F update, from G^T (p x n).
cudaError_t f_side(const nenmf_problem_f64_t& pr, const double* Gt, const Solve64Ws& w, cudaStream_t s) {
  const int n = pr.n, m = pr.m, p = pr.p, nu = pr.nu;
  Control* c = w.ctrl;
  if (pr.mode == NENMF_PLAIN) {
    F64_CU(gemm64(p, p, n, Gt, n, 1, Gt, 1, n, w.H, p, c, s));       // G^T G
    F64_CU(gemm64(p, m, n, Gt, n, 1, pr.X, m, 1, w.Bm, m, c, s));    // G^T X
  } else {
    F64_CU(gemm64(nu, p, n, pr.L, n, 1, Gt, 1, n, w.W, p, c, s));    // G_L = L G (nu x p)
    F64_CU(gemm64(p, p, nu, w.W, 1, p, w.W, p, 1, w.H, p, c, s));    // G_L^T G_L
    F64_CU(gemm64(p, m, nu, w.W, 1, p, pr.XL, m, 1, w.Bm, m, c, s));  // G_L^T X_L
  }
  return cudaSuccess;
}

cudaError_t inner64(const nenmf_problem_f64_t& pr, double* U, int N, const nenmf_params_t& pa, const Solve64Ws& w,
                    nenmf_stats_t* st, int side, cudaStream_t s) {
  count_launches(2);
  lambda_f64_kernel<<<1, 1, 0, s>>>(w.H, pr.p, w.J, w.lam, nullptr, nullptr, w.ctrl);
  nnls_f64_kernel<<<1, kNnlsThreads, 0, s>>>(w.H, w.Bm, U, pr.p, N, w.lam, w.beta, pa.max_inner, pa.min_inner,
                                              w.eps2, pa.restart, w.Y, w.Fp, w.obj, w.rc, st, side, w.ctrl);
  return cudaGetLastError();
}

// ---- reverse mode, host side ----------------------------------------------
struct Back64Ws {
  Control* ctrl;
  double* snapGt;  // [T][p][n]: G^t transposed before outer iteration t
  double* snapF;   // [T][p][m]
  double* Gt;      // p x n (running forward; then G^{t+1} of the sweep)
  double* F;       // p x m
  double* tYg;     // [p][K][n] tapes of the G update
  double* tZg;
  double* tDg;
  double* tYf;     // [p][K][m] tapes of the F update
  double* tZf;
  double* tDf;
  double* FR;      // p x nu
  double* GL;      // nu x p
  double* HG;      // p x p
  double* HF;
  double* dH;      // p x p
  double* S;       // p x p
  double* J;       // p x p Jacobi scratch
  double* V;       // p x p eigenvectors
  double* vG;      // p
  double* vF;
  double* lamG;
  double* lamF;
  double* dL;
  double* Bg;      // p x n
  double* Bf;      // p x m
  double* dBg;     // p x n
  double* dBf;     // p x m
  double* dGt;     // p x n (cotangent of G^T)
  double* dGo;     // p x n (cotangent of the previous G^T)
  double* dG;      // n x p
  double* dFo;     // p x m (cotangent of the previous F)
  double* dF;      // p x m
  double* dGL;     // nu x p
  double* dFR;     // p x nu
  double* beta;    // K
  size_t bytes;
};

Back64Ws carve_back64(void* base, const nenmf_problem_f64_t& pr, int T, int K) {
  Back64Ws w{};
  Carver cv(base);
  const size_t n = pr.n, m = pr.m, p = pr.p, nu = pr.nu;
  w.ctrl = cv.take<Control>(1);
  w.snapGt = cv.take<double>((size_t)T * p * n);
  w.snapF = cv.take<double>((size_t)T * p * m);
  w.Gt = cv.take<double>(p * n);
  w.F = cv.take<double>(p * m);
  w.tYg = cv.take<double>(p * K * n);
  w.tZg = cv.take<double>(p * K * n);
  w.tDg = cv.take<double>(p * K * n);
  w.tYf = cv.take<double>(p * K * m);
  w.tZf = cv.take<double>(p * K * m);
  w.tDf = cv.take<double>(p * K * m);
  w.FR = cv.take<double>(p * nu);
  w.GL = cv.take<double>(nu * p);
  w.HG = cv.take<double>(p * p);
  w.HF = cv.take<double>(p * p);
  w.dH = cv.take<double>(p * p);
  w.S = cv.take<double>(p * p);
  w.J = cv.take<double>(p * p);
  w.V = cv.take<double>(p * p);
  w.vG = cv.take<double>(p);
  w.vF = cv.take<double>(p);
  w.lamG = cv.take<double>(1);
  w.lamF = cv.take<double>(1);
  w.dL = cv.take<double>(1);
  w.Bg = cv.take<double>(p * n);
  w.Bf = cv.take<double>(p * m);
  w.dBg = cv.take<double>(p * n);
  w.dBf = cv.take<double>(p * m);
  w.dGt = cv.take<double>(p * n);
  w.dGo = cv.take<double>(p * n);
  w.dG = cv.take<double>(n * p);
  w.dFo = cv.take<double>(p * m);
  w.dF = cv.take<double>(p * m);
  w.dGL = cv.take<double>(nu * p);
  w.dFR = cv.take<double>(p * nu);
  w.beta = cv.take<double>(K > 0 ? K : 1);
  w.bytes = cv.size();
  return w;
}

bool back64_args_ok(const nenmf_problem_f64_t* pr, const nenmf_params_t* pa) {
  return problem64_ok(pr) && pr->mode == NENMF_COMPRESSED && pa && pa->max_outer >= 0 && pa->max_outer <= 4096 &&
         pa->max_inner >= 1 && pa->max_inner <= 1024 && pa->tol <= 0.0 && !pa->restart;
}

// The G update's H, B (the unknown is G^T) from F, with lambda_max and its eigenvector.
cudaError_t back_g_inputs(const nenmf_problem_f64_t& pr, const double* F, const Back64Ws& w, cudaStream_t s) {
  const int n = pr.n, m = pr.m, p = pr.p, nu = pr.nu;
  F64_CU(gemm64(p, nu, m, F, m, 1, pr.R, nu, 1, w.FR, nu, w.ctrl, s));      // F_R = F R
  F64_CU(gemm64(p, p, nu, w.FR, nu, 1, w.FR, 1, nu, w.HG, p, w.ctrl, s));   // F_R F_R^T
  F64_CU(gemm64(p, n, nu, w.FR, nu, 1, pr.XR, 1, nu, w.Bg, n, w.ctrl, s));  // F_R X_R^T
  count_launches(1);
  lambda_f64_kernel<<<1, 1, 0, s>>>(w.HG, p, w.J, w.lamG, w.V, w.vG, w.ctrl);
  return cudaGetLastError();
}

// The F update's H, B from G^T.
cudaError_t back_f_inputs(const nenmf_problem_f64_t& pr, const double* Gt, const Back64Ws& w, cudaStream_t s) {
  const int n = pr.n, m = pr.m, p = pr.p, nu = pr.nu;
  F64_CU(gemm64(nu, p, n, pr.L, n, 1, Gt, 1, n, w.GL, p, w.ctrl, s));      // G_L = L G
  F64_CU(gemm64(p, p, nu, w.GL, 1, p, w.GL, p, 1, w.HF, p, w.ctrl, s));    // G_L^T G_L
  F64_CU(gemm64(p, m, nu, w.GL, 1, p, pr.XL, m, 1, w.Bf, m, w.ctrl, s));   // G_L^T X_L
  count_launches(1);
  lambda_f64_kernel<<<1, 1, 0, s>>>(w.HF, p, w.J, w.lamF, w.V, w.vF, w.ctrl);
  return cudaGetLastError();
}

// S = dH + dH^T of one inner solve: dH = -(1/L_c) sum_k dz_k Y_k^T + dL v v^T.
cudaError_t back_sym_dh(int p, int N, int K, const double* tD, const double* tY, const double* lam, const double* v,
                        const Back64Ws& w, cudaStream_t s) {
  // dH = sum over (k, j) of dz (p x KN) times Y^T, scaled by -1/L_c on the device
  F64_CU(gemm64(p, p, K * N, tD, (long long)K * N, 1, tY, 1, (long long)K * N, w.dH, p, w.ctrl, s));
  count_launches(1);
  scale_by_lam_kernel<<<1, kMaxP64 * kMaxP64, 0, s>>>(w.dH, p, lam, w.ctrl);
  count_launches(1);
  dh_finish_f64_kernel<<<1, kMaxP64 * kMaxP64, 0, s>>>(w.dH, w.dL, v, p, w.S, w.ctrl);
  return cudaGetLastError();
}

}  // namespace

extern "C" {

size_t nmf_compress_f64_workspace_size(int n, int m, int nu) {
  if (!compress64_args_ok(n, m, nu, 0)) return 0;
  return carve_compress64(nullptr, n, m, nu).bytes;
}

nmf_status_t nmf_compress_f64(nmf_stream_t stream, int n, int m, int nu, int q, const double* X,
                              const double* omega_L, const double* omega_R, uint64_t seed, double* L, double* R,
                              double* XL, double* XR, void* workspace, size_t workspace_bytes) {
  if (!compress64_args_ok(n, m, nu, q) || !X || !L || !R || !XL || !XR) return NMF_ERR_INVALID_ARG;
  if ((omega_L == nullptr) != (omega_R == nullptr)) return NMF_ERR_INVALID_ARG;
  const Compress64Ws w = carve_compress64(workspace, n, m, nu);
  if (!ws64_ok(workspace, workspace_bytes, w.bytes)) return NMF_ERR_WORKSPACE;
  cudaStream_t s = (cudaStream_t)stream;
  Control* c = w.ctrl;
  NMF_CU(cudaMemsetAsync(c, 0, sizeof(Control), s));
  const double* OL = omega_L;
  const double* OR = omega_R;
  if (!OL) {
    // the float32 path's Philox draw (streams 0 and 1), widened
    NMF_CU(sketch_launch(m, nu, seed, 0u, w.sk, s));
    count_launches(1);
    widen_kernel<<<grid64((long long)m * nu, 256), 256, 0, s>>>(w.sk, (long long)m * nu, w.omL);
    NMF_CU(sketch_launch(nu, n, seed, 1u, w.sk, s));
    count_launches(1);
    widen_kernel<<<grid64((long long)nu * n, 256), 256, 0, s>>>(w.sk, (long long)nu * n, w.omR);
    NMF_CU(cudaGetLastError());
    OL = w.omL;
    OR = w.omR;
  }
  // Alg. 2: Q_L = orth(X Omega_L); Q_R^T = orth((Omega_R X)^T) = orth(X^T Omega_R^T)
  NMF_CU(gemm64(n, nu, m, X, m, 1, OL, nu, 1, w.T1, nu, c, s));
  NMF_CU(orth64(w.T1, n, nu, w.QL, w.o, c, s));
  NMF_CU(gemm64(m, nu, n, X, 1, m, OR, 1, n, w.T1, nu, c, s));
  NMF_CU(orth64(w.T1, m, nu, w.QR, w.o, c, s));
  for (int k = 0; k < q; ++k) {
    // Q~_L = orth(X^T Q_L), Q_L = orth(X Q~_L); Q~_R^T = orth(X Q_R^T), Q_R^T = orth(X^T Q~_R^T)
    NMF_CU(gemm64(m, nu, n, X, 1, m, w.QL, nu, 1, w.T1, nu, c, s));
    NMF_CU(orth64(w.T1, m, nu, w.T1, w.o, c, s));
    NMF_CU(gemm64(n, nu, m, X, m, 1, w.T1, nu, 1, w.QL, nu, c, s));
    NMF_CU(orth64(w.QL, n, nu, w.QL, w.o, c, s));
    NMF_CU(gemm64(n, nu, m, X, m, 1, w.QR, nu, 1, w.T1, nu, c, s));
    NMF_CU(orth64(w.T1, n, nu, w.T1, w.o, c, s));
    NMF_CU(gemm64(m, nu, n, X, 1, m, w.T1, nu, 1, w.QR, nu, c, s));
    NMF_CU(orth64(w.QR, m, nu, w.QR, w.o, c, s));
  }
  // L = Q_L^T (nu x n), R = Q_R^T (m x nu); X_L = L X, X_R = X R
  NMF_CU(transpose64(w.QL, n, nu, L, c, s));
  NMF_CU(cudaMemcpyAsync(R, w.QR, sizeof(double) * (size_t)m * nu, cudaMemcpyDeviceToDevice, s));
  NMF_CU(gemm64(nu, m, n, w.QL, 1, nu, X, m, 1, XL, m, c, s));
  NMF_CU(gemm64(n, nu, m, X, m, 1, w.QR, nu, 1, XR, nu, c, s));
  return NMF_OK;
}

size_t nenmf_solve_f64_workspace_size(const nenmf_problem_f64_t* problem) {
  if (!problem64_ok(problem)) return 0;
  return carve_solve64(nullptr, *problem).bytes;
}

nmf_status_t nenmf_solve_f64(nmf_stream_t stream, const nenmf_problem_f64_t* problem, double* G, double* F,
                             const nenmf_params_t* params, nenmf_stats_t* stats, void* workspace,
                             size_t workspace_bytes) {
  if (!problem64_ok(problem) || !params || !G || !F) return NMF_ERR_INVALID_ARG;
  const nenmf_problem_f64_t pr = *problem;
  const nenmf_params_t pa = *params;
  if (pa.max_outer < 0 || pa.max_outer > 32000 || pa.max_inner < 1 || pa.max_inner > kMaxInnerIters ||
      pa.min_inner < 1)
    return NMF_ERR_INVALID_ARG;
  if (pa.tol_mode != NENMF_TOL_REL && pa.tol_mode != NENMF_TOL_ABS) return NMF_ERR_INVALID_ARG;
  if (pa.record_G || pa.record_F || pa.record_time_ns) return NMF_ERR_UNSUPPORTED;
  const Solve64Ws w = carve_solve64(workspace, pr);
  if (!ws64_ok(workspace, workspace_bytes, w.bytes)) return NMF_ERR_WORKSPACE;
  cudaStream_t s = (cudaStream_t)stream;
  Control* c = w.ctrl;
  const int n = pr.n, m = pr.m, p = pr.p;
  NMF_CU(cudaMemsetAsync(c, 0, sizeof(Control), s));
  NMF_CU(cudaMemsetAsync(w.pg2, 0, sizeof(double), s));
  if (stats) NMF_CU(cudaMemsetAsync(stats, 0, sizeof(nenmf_stats_t), s));
  count_launches(1);
  beta_f64_kernel<<<1, 1, 0, s>>>(w.beta, pa.max_inner);
  NMF_CU(cudaGetLastError());
  NMF_CU(transpose64(G, n, p, w.Gt, c, s));
  if (pa.tol > 0.0 && pa.tol_mode == NENMF_TOL_REL) {
    // eps = tol ||[P grad_G ; P grad_F]||_F at (G0, F0), of the objective being solved
    NMF_CU(g_side(pr, F, w, s));
    count_launches(1);
    pg2_f64_kernel<<<1, kNnlsThreads, 0, s>>>(w.H, w.Bm, w.Gt, p, n, w.pg2, c);
    NMF_CU(f_side(pr, w.Gt, w, s));
    count_launches(1);
    pg2_f64_kernel<<<1, kNnlsThreads, 0, s>>>(w.H, w.Bm, F, p, m, w.pg2, c);
    NMF_CU(cudaGetLastError());
  }
  count_launches(1);
  eps_f64_kernel<<<1, 1, 0, s>>>(w.pg2, pa.tol, pa.tol_mode, w.eps2, stats);
  NMF_CU(cudaGetLastError());
  for (int t = 0; t < pa.max_outer; ++t) {
    NMF_CU(g_side(pr, F, w, s));
    NMF_CU(inner64(pr, w.Gt, n, pa, w, stats, 0, s));
    NMF_CU(f_side(pr, w.Gt, w, s));
    NMF_CU(inner64(pr, F, m, pa, w, stats, 1, s));
  }
  NMF_CU(transpose64(w.Gt, p, n, G, c, s));
  if (stats) {
    count_launches(1);
    finish_f64_kernel<<<1, 1, 0, s>>>(stats, pa.max_outer, c);
    NMF_CU(cudaGetLastError());
  }
  return NMF_OK;
}

}  // extern "C"

extern "C" {

size_t nenmf_backward_f64_workspace_size(const nenmf_problem_f64_t* problem, const nenmf_params_t* params) {
  if (!back64_args_ok(problem, params)) return 0;
  return carve_back64(nullptr, *problem, params->max_outer, params->max_inner).bytes;
}

nmf_status_t nenmf_backward_f64(nmf_stream_t stream, const nenmf_problem_f64_t* problem,
                                const nenmf_params_t* params, const double* G0, const double* F0,
                                const double* dG_T, const double* dF_T, double* dXL, double* dXR, double* dG0,
                                double* dF0, double* dX, void* workspace, size_t workspace_bytes) {
  if (problem && problem->mode != NENMF_COMPRESSED) return NMF_ERR_UNSUPPORTED;
  if (!back64_args_ok(problem, params) || !G0 || !F0 || !dG_T || !dF_T || !dXL || !dXR || !dG0 || !dF0)
    return NMF_ERR_INVALID_ARG;
  const nenmf_problem_f64_t pr = *problem;
  const int T = params->max_outer, K = params->max_inner;
  const Back64Ws w = carve_back64(workspace, pr, T, K);
  if (!ws64_ok(workspace, workspace_bytes, w.bytes)) return NMF_ERR_WORKSPACE;
  cudaStream_t s = (cudaStream_t)stream;
  Control* c = w.ctrl;
  const int n = pr.n, m = pr.m, p = pr.p, nu = pr.nu;
  NMF_CU(cudaMemsetAsync(c, 0, sizeof(Control), s));
  count_launches(1);
  beta_f64_kernel<<<1, 1, 0, s>>>(w.beta, K);
  NMF_CU(cudaGetLastError());
  // forward, keeping (G^t, F^t) before every outer iteration
  NMF_CU(transpose64(G0, n, p, w.Gt, c, s));
  NMF_CU(cudaMemcpyAsync(w.F, F0, sizeof(double) * (size_t)p * m, cudaMemcpyDeviceToDevice, s));
  for (int t = 0; t < T; ++t) {
    NMF_CU(cudaMemcpyAsync(w.snapGt + (size_t)t * p * n, w.Gt, sizeof(double) * (size_t)p * n,
                           cudaMemcpyDeviceToDevice, s));
    NMF_CU(cudaMemcpyAsync(w.snapF + (size_t)t * p * m, w.F, sizeof(double) * (size_t)p * m,
                           cudaMemcpyDeviceToDevice, s));
    NMF_CU(back_g_inputs(pr, w.F, w, s));
    count_launches(1);
    nnls_tape_f64_kernel<<<1, kNnlsThreads, 0, s>>>(w.HG, w.Bg, w.Gt, w.Gt, p, n, K, w.lamG, w.beta, w.tYg, w.tZg,
                                                     c);
    NMF_CU(back_f_inputs(pr, w.Gt, w, s));
    count_launches(1);
    nnls_tape_f64_kernel<<<1, kNnlsThreads, 0, s>>>(w.HF, w.Bf, w.F, w.F, p, m, K, w.lamF, w.beta, w.tYf, w.tZf, c);
    NMF_CU(cudaGetLastError());
  }
  // reverse sweep
  NMF_CU(cudaMemcpyAsync(w.dG, dG_T, sizeof(double) * (size_t)n * p, cudaMemcpyDeviceToDevice, s));
  NMF_CU(cudaMemcpyAsync(w.dF, dF_T, sizeof(double) * (size_t)p * m, cudaMemcpyDeviceToDevice, s));
  NMF_CU(cudaMemsetAsync(dXL, 0, sizeof(double) * (size_t)nu * m, s));
  NMF_CU(cudaMemsetAsync(dXR, 0, sizeof(double) * (size_t)n * nu, s));
  for (int t = T - 1; t >= 0; --t) {
    const double* Gt0 = w.snapGt + (size_t)t * p * n;
    const double* Fs = w.snapF + (size_t)t * p * m;
    // recompute the two updates of outer iteration t with their tapes
    NMF_CU(back_g_inputs(pr, Fs, w, s));
    count_launches(1);
    nnls_tape_f64_kernel<<<1, kNnlsThreads, 0, s>>>(w.HG, w.Bg, Gt0, w.Gt, p, n, K, w.lamG, w.beta, w.tYg, w.tZg, c);
    NMF_CU(back_f_inputs(pr, w.Gt, w, s));
    count_launches(1);
    nnls_tape_f64_kernel<<<1, kNnlsThreads, 0, s>>>(w.HF, w.Bf, Fs, w.F, p, m, K, w.lamF, w.beta, w.tYf, w.tZf, c);
    NMF_CU(cudaGetLastError());
    // F update: (dF_old, dH_F, dB_F); dG_L = G_L (dH_F + dH_F^T) + X_L dB_F^T; dX_L += G_L dB_F; dG += L^T dG_L
    count_launches(1);
    nnls_adj_f64_kernel<<<1, kNnlsThreads, 0, s>>>(w.HF, w.dF, p, m, K, w.lamF, w.beta, w.tYf, w.tZf, w.tDf, w.dFo,
                                                    w.dBf, w.dL, c);
    NMF_CU(cudaGetLastError());
    NMF_CU(back_sym_dh(p, m, K, w.tDf, w.tYf, w.lamF, w.vF, w, s));
    NMF_CU(gemm64(nu, p, p, w.GL, p, 1, w.S, p, 1, w.dGL, p, c, s));
    NMF_CU(gemm64_acc(nu, p, m, pr.XL, m, 1, w.dBf, 1, m, w.dGL, p, 1.0, c, s));
    NMF_CU(gemm64_acc(nu, m, p, w.GL, p, 1, w.dBf, m, 1, dXL, m, 1.0, c, s));
    NMF_CU(gemm64_acc(n, p, nu, pr.L, 1, n, w.dGL, p, 1, w.dG, p, 1.0, c, s));
    // G update on G^T: (dG^T_old, dH_G, dB_G); dF_R = (dH_G + dH_G^T) F_R + dB_G X_R;
    // dX_R += dB_G^T F_R; dF = dF_old + dF_R R^T; dG = (dG^T_old)^T
    NMF_CU(transpose64(w.dG, n, p, w.dGt, c, s));
    count_launches(1);
    nnls_adj_f64_kernel<<<1, kNnlsThreads, 0, s>>>(w.HG, w.dGt, p, n, K, w.lamG, w.beta, w.tYg, w.tZg, w.tDg, w.dGo,
                                                    w.dBg, w.dL, c);
    NMF_CU(cudaGetLastError());
    NMF_CU(back_sym_dh(p, n, K, w.tDg, w.tYg, w.lamG, w.vG, w, s));
    NMF_CU(gemm64(p, nu, p, w.S, p, 1, w.FR, nu, 1, w.dFR, nu, c, s));
    NMF_CU(gemm64_acc(p, nu, n, w.dBg, n, 1, pr.XR, nu, 1, w.dFR, nu, 1.0, c, s));
    NMF_CU(gemm64_acc(n, nu, p, w.dBg, 1, n, w.FR, nu, 1, dXR, nu, 1.0, c, s));
    NMF_CU(cudaMemcpyAsync(w.dF, w.dFo, sizeof(double) * (size_t)p * m, cudaMemcpyDeviceToDevice, s));
    NMF_CU(gemm64_acc(p, m, nu, w.dFR, nu, 1, pr.R, 1, nu, w.dF, m, 1.0, c, s));
    NMF_CU(transpose64(w.dGo, p, n, w.dG, c, s));
  }
  NMF_CU(cudaMemcpyAsync(dG0, w.dG, sizeof(double) * (size_t)n * p, cudaMemcpyDeviceToDevice, s));
  NMF_CU(cudaMemcpyAsync(dF0, w.dF, sizeof(double) * (size_t)p * m, cudaMemcpyDeviceToDevice, s));
  if (dX) {
    // dX = L^T dX_L + dX_R R^T
    NMF_CU(gemm64(n, m, nu, pr.L, 1, n, dXL, m, 1, dX, m, c, s));
    NMF_CU(gemm64_acc(n, m, nu, dXR, nu, 1, pr.R, 1, nu, dX, m, 1.0, c, s));
  }
  return NMF_OK;
}

}  // extern "C"
