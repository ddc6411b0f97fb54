// Small dense factorizations of order <= 256:
//   * Cholesky factor of a (shifted) Gram matrix, the building block of the
//     row orthonormalisation between power steps (Section 5.3) and of the
//     pseudo-inverse R^+ in U = V* R^+ (Eq. (3.5)); one CTA, the matrix in
//     shared memory;
//   * explicit inverses of triangles through the blocked triangular solve
//     (tri.cu) with an identity right-hand side;
//   * the float64-accumulated product that ends the U chain.
#include "kernels.cuh"

namespace curid {

namespace {

constexpr int kSmallThreads = 512;  // 128 registers per thread for the block loops
constexpr int kSmallWarps = kSmallThreads / 32;
// Cholesky factor of G + shift I, blocked right-looking on 32 x 32 blocks,
// the matrix padded to a multiple of 32 with an identity tail so no block
// needs bounds checks.  Per block column: warp 0 factors the diagonal block
// (lanes = rows) and inverts it (lanes = columns); every warp then finishes
// panel rows A21 <- A21 L11^{-T} with shuffles; the trailing update
// A22 -= A21 A21^T is spread one 32 x 32 block per warp.  The lower factor
// overwrites G (upper part zeroed).  A non-positive or non-finite pivot
// retries with a 100x larger shift (4 attempts), then FLAG_BREAKDOWN.
template <typename real>
__global__ void __launch_bounds__(kSmallThreads, 1)
chol_kernel(real* __restrict__ G, int l, real rel_shift, StatusBlock* status) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int LP = (l + 31) & ~31;
  const int ld = LP + 1;
  const int nb = LP / 32;
  real* a = reinterpret_cast<real*>(smem_raw);
  real* W = a + (size_t)LP * ld;  // 32 x 33 inverse of the current diagonal block
  __shared__ int s_fail;
  __shared__ real s_tr;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (warp == 0) {
    real tr = real(0);
    for (int i = lane; i < l; i += 32) tr += G[(int64_t)i * l + i];
    tr = warp_sum(tr);
    if (lane == 0) s_tr = tr;
  }
  __syncthreads();
  const real tr = s_tr;
  real shift = rel_shift * tr;
  bool done = false;
  for (int attempt = 0; attempt < 4 && !done; ++attempt) {
    for (int e = tid; e < LP * LP; e += kSmallThreads) {
      const int i = e / LP, j = e % LP;
      real v;
      if (i < l && j < l) v = G[(int64_t)i * l + j] + (i == j ? shift : real(0));
      else v = i == j ? real(1) : real(0);
      a[i * ld + j] = v;
    }
    if (tid == 0) s_fail = 0;
    __syncthreads();
    for (int kb = 0; kb < LP; kb += 32) {
      if (warp == 0) {
        // (1) factor the diagonal block; lane i owns row kb + i
        real* Dk = a + kb * ld + kb;
        int fail = 0;
        for (int j = 0; j < 32; ++j) {
          real d = Dk[j * ld + j];
          if (!(d > real(0)) || !isfinite(d)) fail = 1;
          d = fail ? real(1) : sqrt(d);
          __syncwarp();
          if (lane == j) Dk[j * ld + j] = d;
          real lij = real(0);
          if (lane > j) {
            lij = Dk[lane * ld + j] / d;
            Dk[lane * ld + j] = lij;
          }
          __syncwarp();
          if (lane > j)
            for (int t = j + 1; t <= lane; ++t) Dk[lane * ld + t] -= lij * Dk[t * ld + j];
          __syncwarp();
        }
        // (1b) W = L11^{-1}; lane c computes column c
        real x[32];
#pragma unroll
        for (int i = 0; i < 32; ++i) {
          real sum = i == lane ? real(1) : real(0);
#pragma unroll
          for (int t = 0; t < i; ++t) sum -= Dk[i * ld + t] * x[t];
          x[i] = i >= lane ? sum / Dk[i * ld + i] : real(0);
        }
#pragma unroll
        for (int i = 0; i < 32; ++i) W[i * 33 + lane] = x[i];
        if (lane == 0) s_fail = fail;
      }
      __syncthreads();
      if (s_fail) break;
      // (2) panel rows below: A21(i, c) <- sum_{s <= c} A21(i, s) W(c, s)
      for (int i = kb + 32 + warp; i < LP; i += kSmallWarps) {
        const real ais = a[i * ld + kb + lane];
        real out = real(0);
#pragma unroll
        for (int s2 = 0; s2 < 32; ++s2) {
          const real v = __shfl_sync(0xffffffffu, ais, s2);
          out += v * W[lane * 33 + s2];
        }
        a[i * ld + kb + lane] = out;
      }
      __syncthreads();
      // (3) trailing update, one 32 x 32 block (bi >= bj > kb) per warp
      const int b0 = kb / 32 + 1;
      const int m = nb - b0;
      const int nblocks = m * (m + 1) / 2;
      for (int q = warp; q < nblocks; q += kSmallWarps) {
        int bi = 0;
        while ((bi + 1) * (bi + 2) / 2 <= q) ++bi;
        const int bj = q - bi * (bi + 1) / 2;
        const int i0 = (b0 + bi) * 32, j0 = (b0 + bj) * 32;
        real col[32];
#pragma unroll
        for (int s2 = 0; s2 < 32; ++s2) col[s2] = a[(j0 + lane) * ld + kb + s2];
        for (int r = 0; r < 32; ++r) {
          const real* ar = a + (i0 + r) * ld + kb;
          real sum = real(0);
#pragma unroll
          for (int s2 = 0; s2 < 32; ++s2) sum += ar[s2] * col[s2];
          a[(i0 + r) * ld + j0 + lane] -= sum;
        }
      }
      __syncthreads();
    }
    __syncthreads();
    if (!s_fail) done = true;
    shift = shift > real(0) ? shift * real(100)
                            : tr * (sizeof(real) == 8 ? real(1e-13) : real(1e-5));
    __syncthreads();
  }
  if (!done) {
    if (tid == 0) set_flag(&status->flags, FLAG_BREAKDOWN);
    for (int e = tid; e < l * l; e += kSmallThreads) G[e] = (e / l == e % l) ? real(1) : real(0);
    return;
  }
  for (int e = tid; e < l * l; e += kSmallThreads) {
    const int i = e / l, j = e % l;
    G[e] = j <= i ? a[i * ld + j] : real(0);
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
size_t chol_smem(int l) {
  const int LP = (l + 31) & ~31;
  return ((size_t)LP * (LP + 1) + 32 * 33) * sizeof(real);
}

}  // namespace

template <typename real>
bool upper_tri_inverse_fits(const Ctx& ctx, int k) {
  return tri_solve_fits<real>(ctx, k);
}
template <typename real>
bool chol_inverse_fits(const Ctx& ctx, int l) {
  return l <= 256 && chol_smem<real>(l) <= ctx.smem_optin && tri_solve_fits<real>(ctx, l);
}

template <typename real>
curid_status upper_tri_inverse(const Ctx& ctx, const real* S11, int k, const int* k_eff,
                               real* X) {
  return tri_solve<real>(ctx, k, S11, k, true, false, nullptr, 0, X, k, k, k_eff);
}

template <typename real>
curid_status cholesky(const Ctx& ctx, real* G, int l, double rel_shift) {
  if (l <= 0) return CURID_OK;
  if (!chol_inverse_fits<real>(ctx, l)) return CURID_UNSUPPORTED;
  const size_t smem = chol_smem<real>(l);
  auto fn = chol_kernel<real>;
  CURID_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  fn<<<1, kSmallThreads, smem, ctx.stream>>>(G, l, (real)rel_shift, ctx.status);
  CURID_LAUNCHED(ctx);
  return CURID_OK;
}

template <typename real>
curid_status chol_inverse(const Ctx& ctx, real* G, int l, double rel_shift, real* Linv) {
  CURID_TRY(cholesky<real>(ctx, G, l, rel_shift));
  return tri_solve<real>(ctx, l, G, l, false, false, nullptr, 0, Linv, l, l, nullptr);
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
template curid_status cholesky<float>(const Ctx&, float*, int, double);
template curid_status cholesky<double>(const Ctx&, double*, int, double);
template curid_status chol_inverse<float>(const Ctx&, float*, int, double, float*);
template curid_status chol_inverse<double>(const Ctx&, double*, int, double, double*);

}  // namespace curid
