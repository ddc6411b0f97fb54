// General dense products on the CUDA cores (FP32 and FP64 FMA), used for
// the FP64 path, the Gram matrices and triangular applies of the row
// orthonormalisation, T = S11^{-1} S12 and the U product chain.
//
// C[M x N] = alpha * op(A) op(B) + beta * C, row-major, with
//   op(A)(m, k) = ta ? A[k*lda + m] : A[m*lda + k]
//   op(B)(k, n) = tb ? B[n*ldb + k] : B[k*ldb + n]
// When the output has fewer tiles than the GPU has SMs the K range is split
// and the partial tiles are summed in a fixed order by a second kernel, so
// results are bitwise reproducible run to run.
#include "kernels.cuh"

namespace curid {

template <typename real>
struct GemmTile;
template <>
struct GemmTile<float> {
  static constexpr int BM = 128, BN = 128, BK = 16, TM = 8, TN = 8;
};
template <>
struct GemmTile<double> {
  static constexpr int BM = 64, BN = 64, BK = 16, TM = 4, TN = 4;
};

template <typename real, bool TA, bool TB>
__global__ void __launch_bounds__((GemmTile<real>::BM / GemmTile<real>::TM) *
                                  (GemmTile<real>::BN / GemmTile<real>::TN))
gemm_simt_kernel(int M, int N, int K, int kchunk, const real* __restrict__ A,
                 int64_t lda, const real* __restrict__ B, int64_t ldb,
                 real* __restrict__ C, int64_t ldc, real alpha, real beta,
                 real* __restrict__ partial) {
  using Tl = GemmTile<real>;
  constexpr int BM = Tl::BM, BN = Tl::BN, BK = Tl::BK, TM = Tl::TM, TN = Tl::TN;
  constexpr int RX = BN / TN, RY = BM / TM, NT = RX * RY;
  constexpr int LA = BM * BK / NT, LB = BN * BK / NT;  // tile elements each thread loads
  // two stages: the next K tile is fetched into registers while the current
  // one is multiplied, then stored into the other buffer (one barrier per tile)
  __shared__ real As[2][BK][BM + 4];
  __shared__ real Bs[2][BK][BN + 4];
  const int tid = threadIdx.x;
  const int tx = tid % RX, ty = tid / RX;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const int kbeg = blockIdx.z * kchunk;
  const int kend = min(K, kbeg + kchunk);
  real acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = real(0);

  // element e = tid + i NT of a tile; consecutive threads walk the operand's
  // contiguous dimension
  real ra[LA], rb[LB];
  auto fetch = [&](int k0) {
#pragma unroll
    for (int i = 0; i < LA; ++i) {
      const int e = tid + i * NT;
      const int mm = TA ? e % BM : e / BK, kk = TA ? e / BM : e % BK;
      const int gm = m0 + mm, gk = k0 + kk;
      ra[i] = (gm < M && gk < kend) ? (TA ? A[(int64_t)gk * lda + gm] : A[(int64_t)gm * lda + gk])
                                    : real(0);
    }
#pragma unroll
    for (int i = 0; i < LB; ++i) {
      const int e = tid + i * NT;
      const int nn = TB ? e / BK : e % BN, kk = TB ? e % BK : e / BN;
      const int gn = n0 + nn, gk = k0 + kk;
      rb[i] = (gn < N && gk < kend) ? (TB ? B[(int64_t)gn * ldb + gk] : B[(int64_t)gk * ldb + gn])
                                    : real(0);
    }
  };
  auto stash = [&](int buf) {
#pragma unroll
    for (int i = 0; i < LA; ++i) {
      const int e = tid + i * NT;
      const int mm = TA ? e % BM : e / BK, kk = TA ? e / BM : e % BK;
      As[buf][kk][mm] = ra[i];
    }
#pragma unroll
    for (int i = 0; i < LB; ++i) {
      const int e = tid + i * NT;
      const int nn = TB ? e / BK : e % BN, kk = TB ? e % BK : e / BN;
      Bs[buf][kk][nn] = rb[i];
    }
  };

  int buf = 0;
  if (kbeg < kend) {
    fetch(kbeg);
    stash(0);
  }
  __syncthreads();
  for (int k0 = kbeg; k0 < kend; k0 += BK) {
    const bool more = k0 + BK < kend;
    if (more) fetch(k0 + BK);
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      real a[TM], b[TN];
#pragma unroll
      for (int i = 0; i < TM; ++i) a[i] = As[buf][kk][ty + i * RY];
#pragma unroll
      for (int j = 0; j < TN; ++j) b[j] = Bs[buf][kk][tx + j * RX];
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    if (more) stash(buf ^ 1);
    __syncthreads();
    buf ^= 1;
  }
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    const int gm = m0 + ty + i * RY;
    if (gm >= M) continue;
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const int gn = n0 + tx + j * RX;
      if (gn >= N) continue;
      if (partial) {
        partial[((int64_t)blockIdx.z * M + gm) * N + gn] = acc[i][j];
      } else {
        real* c = C + (int64_t)gm * ldc + gn;
        *c = beta == real(0) ? alpha * acc[i][j] : alpha * acc[i][j] + beta * *c;
      }
    }
  }
}

template <typename real>
__global__ void splitk_reduce_kernel(int M, int N, int splits,
                                     const real* __restrict__ partial,
                                     real* __restrict__ C, int64_t ldc,
                                     real alpha, real beta) {
  const int64_t total = (int64_t)M * N;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    real s = real(0);
    for (int z = 0; z < splits; ++z) s += partial[(int64_t)z * total + e];
    const int64_t gm = e / N, gn = e % N;
    real* c = C + gm * ldc + gn;
    *c = beta == real(0) ? alpha * s : alpha * s + beta * *c;
  }
}

template <typename real>
int gemm_splits(int64_t M, int64_t N, int64_t K, int num_sms) {
  using Tl = GemmTile<real>;
  const int64_t tiles = ((M + Tl::BM - 1) / Tl::BM) * ((N + Tl::BN - 1) / Tl::BN);
  // K chunks of at least 256 (float32) / 64 (float64: a 64th of the float32
  // rate per SM on GB300, so even short products need more than one SM)
  const int64_t kmin = sizeof(real) == 8 ? 64 : 256;
  if (tiles >= num_sms || K < 2 * kmin) return 1;
  int64_t s = (2 * num_sms + tiles - 1) / tiles;
  s = std::min<int64_t>(s, K / kmin);
  return (int)std::max<int64_t>(1, s);
}

template <typename real>
size_t gemm_partial_elems(int64_t M, int64_t N, int64_t K, int num_sms) {
  const int s = gemm_splits<real>(M, N, K, num_sms);
  return s > 1 ? (size_t)s * M * N : 0;
}

template <typename real>
curid_status gemm(const Ctx& ctx, bool ta, bool tb, int64_t M, int64_t N,
                  int64_t K, real alpha, const real* A, int64_t lda,
                  const real* B, int64_t ldb, real beta, real* C, int64_t ldc,
                  real* partial, size_t partial_cap) {
  using Tl = GemmTile<real>;
  if (M <= 0 || N <= 0) return CURID_OK;
  if (K <= 0) {
    // C = beta * C
    if (beta == real(0)) {
      for (int64_t r = 0; r < M; ++r)
        CURID_CUDA(cudaMemsetAsync(C + r * ldc, 0, N * sizeof(real), ctx.stream));
      return CURID_OK;
    }
    return CURID_UNSUPPORTED;
  }
  // K is split to fill the SMs this caller's decomposition can expect to
  // have: all of them one at a time, a share of them with several in flight
  int splits = gemm_splits<real>(M, N, K, std::max(1, ctx.num_sms / std::max(1, ctx.concurrency)));
  if (splits > 1 && (partial == nullptr || (size_t)splits * M * N > partial_cap)) {
    splits = partial ? (int)std::max<size_t>(1, partial_cap / (size_t)(M * N)) : 1;
  }
  const int kchunk = (int)(((K + splits - 1) / splits + Tl::BK - 1) / Tl::BK * Tl::BK);
  splits = (int)((K + kchunk - 1) / kchunk);
  dim3 grid((unsigned)((N + Tl::BN - 1) / Tl::BN), (unsigned)((M + Tl::BM - 1) / Tl::BM),
            (unsigned)splits);
  constexpr int NT = (Tl::BM / Tl::TM) * (Tl::BN / Tl::TN);
  real* part = splits > 1 ? partial : nullptr;
#define CURID_GEMM_LAUNCH(TA_, TB_)                                                  \
  gemm_simt_kernel<real, TA_, TB_><<<grid, NT, 0, ctx.stream>>>(                     \
      (int)M, (int)N, (int)K, kchunk, A, lda, B, ldb, C, ldc, alpha, beta, part)
  if (!ta && !tb) CURID_GEMM_LAUNCH(false, false);
  else if (!ta && tb) CURID_GEMM_LAUNCH(false, true);
  else if (ta && !tb) CURID_GEMM_LAUNCH(true, false);
  else CURID_GEMM_LAUNCH(true, true);
#undef CURID_GEMM_LAUNCH
  CURID_LAUNCHED(ctx);
  if (splits > 1) {
    const int64_t total = M * N;
    const int blocks = (int)std::min<int64_t>((total + 255) / 256, 8 * ctx.num_sms);
    splitk_reduce_kernel<real><<<blocks, 256, 0, ctx.stream>>>((int)M, (int)N, splits,
                                                                partial, C, ldc, alpha, beta);
    CURID_LAUNCHED(ctx);
  }
  return CURID_OK;
}

template int gemm_splits<float>(int64_t, int64_t, int64_t, int);
template int gemm_splits<double>(int64_t, int64_t, int64_t, int);
template size_t gemm_partial_elems<float>(int64_t, int64_t, int64_t, int);
template size_t gemm_partial_elems<double>(int64_t, int64_t, int64_t, int);
template curid_status gemm<float>(const Ctx&, bool, bool, int64_t, int64_t, int64_t, float,
                                  const float*, int64_t, const float*, int64_t, float, float*,
                                  int64_t, float*, size_t);
template curid_status gemm<double>(const Ctx&, bool, bool, int64_t, int64_t, int64_t, double,
                                   const double*, int64_t, const double*, int64_t, double,
                                   double*, int64_t, double*, size_t);

}  // namespace curid
