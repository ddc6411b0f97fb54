// Small dense factorizations, one CTA with the matrix resident in shared
// memory:
//   * inverse of the upper-triangular S11 for T = S11^{-1} S12 (Eq. (2.8));
//   * Cholesky factor of a (shifted) Gram matrix and the inverse of that
//     factor, the building block of the row orthonormalisation between
//     power steps (Section 5.3) and of the pseudo-inverse R^+ in
//     U = V* R^+ (Eq. (3.5)).
// Both inverses run the same right-looking, in-place scheme: step t fixes
// row t of the inverse's diagonal and column, then folds row t of the
// triangle into every later column; all (i, j) of a step run in parallel.
#include "kernels.cuh"

namespace curid {

namespace {

constexpr int kSmallThreads = 1024;

// In-place inverse of the upper triangle of a (k x k, row stride ld) for
// rows/columns < kk; everything at or after kk is set to zero.
// On entry the strictly upper part and diagonal hold U; on exit they hold
// U^{-1} (upper triangular).  Uses `row` (k reals) as scratch.
template <typename real>
__device__ void inv_upper_inplace(real* a, int k, int ld, int kk, real* row) {
  const int tid = threadIdx.x;
  for (int t = 0; t < kk; ++t) {
    // finalize column t: X[t][t] = 1/U[t][t]; X[i][t] = -acc[i][t] * X[t][t]
    __syncthreads();
    const real d = real(1) / a[t * ld + t];
    for (int i = tid; i < t; i += kSmallThreads) a[i * ld + t] = -a[i * ld + t] * d;
    for (int j = t + 1 + tid; j < kk; j += kSmallThreads) row[j] = a[t * ld + j];
    __syncthreads();
    if (tid == 0) a[t * ld + t] = d;
    __syncthreads();
    // acc[i][j] += X[i][t] * U[t][j] for i <= t < j  (acc[t][j] starts at 0)
    const int rows = t + 1, cols = kk - t - 1;
    for (int e = tid; e < rows * cols; e += kSmallThreads) {
      const int i = e / cols, j = t + 1 + e % cols;
      const real x = a[i * ld + t];
      const real prev = i == t ? real(0) : a[i * ld + j];
      a[i * ld + j] = prev + x * row[j];
    }
  }
  __syncthreads();
  for (int e = tid; e < k * k; e += kSmallThreads) {
    const int i = e / k, j = e % k;
    if (i >= kk || j >= kk || j < i) a[i * ld + j] = real(0);
  }
  __syncthreads();
}

template <typename real>
__global__ void __launch_bounds__(kSmallThreads, 1)
upper_tri_inverse_kernel(const real* __restrict__ S11, int k, const int* __restrict__ k_eff,
                         real* __restrict__ X) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  real* a = reinterpret_cast<real*>(smem_raw);
  real* row = a + (int64_t)k * k;
  const int kk = k_eff ? min(k, *k_eff) : k;
  for (int e = threadIdx.x; e < k * k; e += kSmallThreads) a[e] = S11[e];
  inv_upper_inplace(a, k, k, kk, row);
  for (int e = threadIdx.x; e < k * k; e += kSmallThreads) X[e] = a[e];
}

// Cholesky of G + shift I, lower factor L in the lower triangle of a, then
// Linv = L^{-1} written (lower triangular) to out.  Retries with a 100x
// larger shift (up to 3 times) on a non-positive pivot; FLAG_BREAKDOWN if
// every attempt fails.
template <typename real>
__global__ void __launch_bounds__(kSmallThreads, 1)
chol_inverse_kernel(const real* __restrict__ G, int l, real rel_shift, real* __restrict__ out,
                    StatusBlock* status) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  real* a = reinterpret_cast<real*>(smem_raw);
  real* row = a + (int64_t)l * l;
  __shared__ int s_fail;
  __shared__ real s_d;
  const int tid = threadIdx.x;
  real tr = real(0);
  for (int i = 0; i < l; ++i) tr += G[(int64_t)i * l + i];
  real shift = rel_shift * tr;
  bool done = false;
  for (int attempt = 0; attempt < 4 && !done; ++attempt) {
    __syncthreads();
    // a := G + shift I (the factorization reads and writes the lower triangle)
    for (int e = tid; e < l * l; e += kSmallThreads) {
      const int i = e / l, j = e % l;
      a[e] = G[e] + (i == j ? shift : real(0));
    }
    if (tid == 0) s_fail = 0;
    __syncthreads();
    // right-looking Cholesky on the lower triangle (rows i >= column j)
    for (int j = 0; j < l; ++j) {
      if (tid == 0) {
        const real d = a[j * l + j];
        if (!(d > real(0)) || !isfinite(d)) s_fail = 1;
        s_d = d > real(0) ? sqrt(d) : real(1);
        a[j * l + j] = s_d;
      }
      __syncthreads();
      if (s_fail) break;
      const real inv = real(1) / s_d;
      for (int i = j + 1 + tid; i < l; i += kSmallThreads) a[i * l + j] *= inv;
      __syncthreads();
      const int w = l - j - 1;
      for (int e = tid; e < w * w; e += kSmallThreads) {
        const int i = j + 1 + e / w, t = j + 1 + e % w;
        if (t <= i) a[i * l + t] -= a[i * l + j] * a[t * l + j];
      }
      __syncthreads();
    }
    __syncthreads();
    if (!s_fail) done = true;
    shift = shift > real(0) ? shift * real(100)
                            : tr * (sizeof(real) == 8 ? real(1e-13) : real(1e-5));
  }
  if (!done) {
    if (tid == 0) set_flag(&status->flags, FLAG_BREAKDOWN);
    for (int e = tid; e < l * l; e += kSmallThreads) out[e] = (e / l == e % l) ? real(1) : real(0);
    return;
  }
  // transpose the factor into the upper triangle: U = L^T, invert, transpose back
  __syncthreads();
  for (int e = tid; e < l * l; e += kSmallThreads) {
    const int i = e / l, j = e % l;
    if (j > i) a[e] = a[j * l + i];
  }
  __syncthreads();
  inv_upper_inplace(a, l, l, l, row);
  // (L^{-1}) = (U^{-1})^T
  for (int e = tid; e < l * l; e += kSmallThreads) {
    const int i = e / l, j = e % l;
    out[e] = a[j * l + i];
  }
}

// C[i][j] = sum_t A[i][t] * B[j][t] accumulated and stored in float64
// (A: M x K, B: N x K, row-major).  The last factor of U = V* R^+ (Eq. (3.5))
// multiplies a well-conditioned matrix by the inverse of the skeleton's
// triangle; its cancellation needs float64 accumulation even for FP32 data.
template <typename real>
__global__ void gemm_nt_f64acc_kernel(int M, int N, int K, const real* __restrict__ A,
                                      int64_t lda, const real* __restrict__ B, int64_t ldb,
                                      double* __restrict__ C, int64_t ldc) {
  __shared__ double As[16][17];
  __shared__ double Bs[16][17];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int i = blockIdx.y * 16 + ty, j = blockIdx.x * 16 + tx;
  double acc = 0.0;
  for (int t0 = 0; t0 < K; t0 += 16) {
    const int ia = blockIdx.y * 16 + ty, ta = t0 + tx;
    As[ty][tx] = (ia < M && ta < K) ? (double)A[(int64_t)ia * lda + ta] : 0.0;
    const int jb = blockIdx.x * 16 + ty;
    Bs[ty][tx] = (jb < N && ta < K) ? (double)B[(int64_t)jb * ldb + ta] : 0.0;
    __syncthreads();
#pragma unroll
    for (int t = 0; t < 16; ++t) acc = fma(As[ty][t], Bs[tx][t], acc);
    __syncthreads();
  }
  if (i < M && j < N) C[(int64_t)i * ldc + j] = acc;
}

template <typename real>
size_t small_smem(int k) {
  return (size_t)k * k * sizeof(real) + (size_t)k * sizeof(real);
}

}  // namespace

template <typename real>
bool upper_tri_inverse_fits(const Ctx& ctx, int k) {
  return small_smem<real>(k) <= ctx.smem_optin;
}
template <typename real>
bool chol_inverse_fits(const Ctx& ctx, int l) {
  return small_smem<real>(l) <= ctx.smem_optin;
}

template <typename real>
curid_status upper_tri_inverse(const Ctx& ctx, const real* S11, int k, const int* k_eff,
                               real* X) {
  if (k <= 0) return CURID_OK;
  const size_t smem = small_smem<real>(k);
  if (smem > ctx.smem_optin) return CURID_UNSUPPORTED;
  auto fn = upper_tri_inverse_kernel<real>;
  CURID_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  fn<<<1, kSmallThreads, smem, ctx.stream>>>(S11, k, k_eff, X);
  CURID_LAUNCHED(ctx);
  return CURID_OK;
}

template <typename real>
curid_status chol_inverse(const Ctx& ctx, const real* G, int l, double rel_shift, real* Linv) {
  if (l <= 0) return CURID_OK;
  const size_t smem = small_smem<real>(l);
  if (smem > ctx.smem_optin) return CURID_UNSUPPORTED;
  auto fn = chol_inverse_kernel<real>;
  CURID_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  fn<<<1, kSmallThreads, smem, ctx.stream>>>(G, l, (real)rel_shift, Linv, ctx.status);
  CURID_LAUNCHED(ctx);
  return CURID_OK;
}

template <typename real>
curid_status gemm_nt_f64acc(const Ctx& ctx, int64_t M, int64_t N, int64_t K, const real* A,
                            int64_t lda, const real* B, int64_t ldb, double* C, int64_t ldc) {
  if (M <= 0 || N <= 0) return CURID_OK;
  dim3 grid((unsigned)((N + 15) / 16), (unsigned)((M + 15) / 16));
  gemm_nt_f64acc_kernel<real><<<grid, dim3(16, 16), 0, ctx.stream>>>((int)M, (int)N, (int)K, A,
                                                                     lda, B, ldb, C, ldc);
  CURID_LAUNCHED(ctx);
  return CURID_OK;
}

template curid_status gemm_nt_f64acc<float>(const Ctx&, int64_t, int64_t, int64_t, const float*,
                                            int64_t, const float*, int64_t, double*, int64_t);
template curid_status gemm_nt_f64acc<double>(const Ctx&, int64_t, int64_t, int64_t,
                                             const double*, int64_t, const double*, int64_t,
                                             double*, int64_t);
template bool upper_tri_inverse_fits<float>(const Ctx&, int);
template bool upper_tri_inverse_fits<double>(const Ctx&, int);
template bool chol_inverse_fits<float>(const Ctx&, int);
template bool chol_inverse_fits<double>(const Ctx&, int);
template curid_status upper_tri_inverse<float>(const Ctx&, const float*, int, const int*, float*);
template curid_status upper_tri_inverse<double>(const Ctx&, const double*, int, const int*,
                                                double*);
template curid_status chol_inverse<float>(const Ctx&, const float*, int, double, float*);
template curid_status chol_inverse<double>(const Ctx&, const double*, int, double, double*);

}  // namespace curid
