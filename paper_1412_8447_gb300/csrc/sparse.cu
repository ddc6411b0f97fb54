// Sparse A (the paper's motivating case for CUR, Section 1: C and R keep
// A's sparsity): the products of the randomized sketch (Algorithm 4,
// Eq. (5.1); the power steps of Section 5.3) and the gathers C = A(:, J),
// R = A(I, :) read A from its compressed rows (CSR) and compressed columns
// (CSC); everything after them works on the dense l x n sample and the
// dense k-row skeletons as for a dense A.
//
// Products: out (R x L) = sum over the stored entries e of list r of
// val[e] * in[idx[e], :], one warp per output row r, lanes over the L
// columns (up to 256 per pass), four entries' rows of `in` loaded before
// they are used.  With in = X^T (the sample operand transposed) the lists of
// the CSC give (X A)^T and those of the CSR give (X A^T)^T.  The work is a
// gather of l-wide rows per stored entry, bound by memory latency and
// bandwidth, not a dense contraction: it runs on the CUDA cores.
#include "kernels.cuh"

namespace curid {

namespace {

constexpr int kSpThreads = 256;
constexpr int kSpCols = 256;  // columns of `in` / `out` per pass (8 per lane)

template <typename real>
__global__ void __launch_bounds__(kSpThreads)
spmm_rows_kernel(int64_t R, const int64_t* __restrict__ ptr, const int32_t* __restrict__ idx,
                 const real* __restrict__ val, int64_t nrows_in, const real* __restrict__ in,
                 int64_t ldi, int L, real* __restrict__ out, int64_t ldo) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (kSpThreads / 32);
  for (int64_t r = blockIdx.x * (int64_t)(kSpThreads / 32) + (threadIdx.x >> 5); r < R;
       r += warps) {
    real acc[kSpCols / 32];
#pragma unroll
    for (int u = 0; u < kSpCols / 32; ++u) acc[u] = real(0);
    const int64_t e0 = ptr[r], e1 = ptr[r + 1];
    for (int64_t e = e0; e < e1; e += 4) {
      int64_t c[4];
      real v[4];
#pragma unroll
      for (int s = 0; s < 4; ++s) {
        const bool in_range = e + s < e1;
        const int64_t ci = in_range ? (int64_t)idx[e + s] : 0;
        c[s] = (ci >= 0 && ci < nrows_in) ? ci : 0;  // an index out of range reads row 0
        v[s] = in_range ? val[e + s] : real(0);
      }
      real x[4][kSpCols / 32];
#pragma unroll
      for (int s = 0; s < 4; ++s)
#pragma unroll
        for (int u = 0; u < kSpCols / 32; ++u) {
          const int col = lane + 32 * u;
          x[s][u] = col < L ? in[c[s] * ldi + col] : real(0);
        }
#pragma unroll
      for (int s = 0; s < 4; ++s)
#pragma unroll
        for (int u = 0; u < kSpCols / 32; ++u) acc[u] = fma(v[s], x[s][u], acc[u]);
    }
#pragma unroll
    for (int u = 0; u < kSpCols / 32; ++u) {
      const int col = lane + 32 * u;
      if (col < L) out[r * ldo + col] = acc[u];
    }
  }
}

// The same product for long lists: one CTA per list, its 16 warps taking
// interleaved groups of four entries, the warps' partial sums added in
// shared memory in warp order (deterministic).
constexpr int kSpBlockThreads = 512;

template <typename real>
__global__ void __launch_bounds__(kSpBlockThreads)
spmm_lists_block_kernel(int64_t R, const int64_t* __restrict__ ptr,
                        const int32_t* __restrict__ idx, const real* __restrict__ val,
                        int64_t nrows_in, const real* __restrict__ in, int64_t ldi, int L,
                        real* __restrict__ out, int64_t ldo) {
  constexpr int kW = kSpBlockThreads / 32;
  __shared__ real part[kW][kSpCols];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int64_t r = blockIdx.x; r < R; r += gridDim.x) {
    real acc[kSpCols / 32];
#pragma unroll
    for (int u = 0; u < kSpCols / 32; ++u) acc[u] = real(0);
    const int64_t e0 = ptr[r], e1 = ptr[r + 1];
    for (int64_t e = e0 + 4 * warp; e < e1; e += 4 * kW) {
      int64_t c[4];
      real v[4];
#pragma unroll
      for (int s = 0; s < 4; ++s) {
        const bool in_range = e + s < e1;
        const int64_t ci = in_range ? (int64_t)idx[e + s] : 0;
        c[s] = (ci >= 0 && ci < nrows_in) ? ci : 0;
        v[s] = in_range ? val[e + s] : real(0);
      }
      real x[4][kSpCols / 32];
#pragma unroll
      for (int s = 0; s < 4; ++s)
#pragma unroll
        for (int u = 0; u < kSpCols / 32; ++u) {
          const int col = lane + 32 * u;
          x[s][u] = col < L ? in[c[s] * ldi + col] : real(0);
        }
#pragma unroll
      for (int s = 0; s < 4; ++s)
#pragma unroll
        for (int u = 0; u < kSpCols / 32; ++u) acc[u] = fma(v[s], x[s][u], acc[u]);
    }
#pragma unroll
    for (int u = 0; u < kSpCols / 32; ++u) part[warp][lane + 32 * u] = acc[u];
    __syncthreads();
    for (int col = threadIdx.x; col < L; col += kSpBlockThreads) {
      real sum = real(0);
      for (int w = 0; w < kW; ++w) sum += part[w][col];
      out[r * ldo + col] = sum;
    }
    __syncthreads();
  }
}

// Row t of dst (k x cols, leading dimension ldd, zeroed first) receives the
// stored entries of list sel[t] (clamped to [0, lists)); with dst2 non-null
// the same values go to column t of dst2 (cols x k, leading dimension ld2).
template <typename real>
__global__ void scatter_lists_kernel(const int32_t* __restrict__ sel, int k, int64_t lists,
                                     const int64_t* __restrict__ ptr,
                                     const int32_t* __restrict__ idx,
                                     const real* __restrict__ val, int64_t cols,
                                     real* __restrict__ dst, int64_t ldd, real* __restrict__ dst2,
                                     int64_t ld2) {
  for (int t = blockIdx.x; t < k; t += gridDim.x) {
    int64_t s = sel[t];
    if (s < 0 || s >= lists) s = 0;
    for (int64_t e = ptr[s] + threadIdx.x; e < ptr[s + 1]; e += blockDim.x) {
      const int64_t c = idx[e];
      if (c < 0 || c >= cols) continue;
      dst[(int64_t)t * ldd + c] = val[e];
      if (dst2) dst2[c * ld2 + t] = val[e];
    }
  }
}

}  // namespace

template <typename real>
curid_status spmm_rows(const Ctx& ctx, int64_t R, const int64_t* ptr, const int32_t* idx,
                       const real* val, int64_t nnz, int64_t nrows_in, const real* in,
                       int64_t ldi, int64_t L, real* out, int64_t ldo) {
  if (R <= 0 || L <= 0) return CURID_OK;
  // lists of more than 64 entries on average: a CTA per list; else a warp
  const bool long_lists = nnz > 64 * R;
  const unsigned blocks =
      long_lists ? (unsigned)std::min<int64_t>(R, 32LL * ctx.num_sms)
                 : (unsigned)std::max<int64_t>(
                       1, std::min<int64_t>((R + kSpThreads / 32 - 1) / (kSpThreads / 32),
                                            64LL * ctx.num_sms));
  for (int64_t c0 = 0; c0 < L; c0 += kSpCols) {
    const int w = (int)std::min<int64_t>(kSpCols, L - c0);
    if (long_lists)
      spmm_lists_block_kernel<real><<<blocks, kSpBlockThreads, 0, ctx.stream>>>(
          R, ptr, idx, val, nrows_in, in + c0, ldi, w, out + c0, ldo);
    else
      spmm_rows_kernel<real><<<blocks, kSpThreads, 0, ctx.stream>>>(R, ptr, idx, val, nrows_in,
                                                                    in + c0, ldi, w, out + c0,
                                                                    ldo);
    CURID_LAUNCHED(ctx);
  }
  return CURID_OK;
}

template <typename real>
curid_status scatter_lists(const Ctx& ctx, const int32_t* sel, int k, int64_t lists,
                           const int64_t* ptr, const int32_t* idx, const real* val, int64_t cols,
                           real* dst, int64_t ldd, real* dst2, int64_t ld2) {
  if (k <= 0) return CURID_OK;
  CURID_CUDA(cudaMemset2DAsync(dst, (size_t)ldd * sizeof(real), 0, (size_t)cols * sizeof(real),
                               (size_t)k, ctx.stream));
  if (dst2)
    CURID_CUDA(cudaMemset2DAsync(dst2, (size_t)ld2 * sizeof(real), 0, (size_t)k * sizeof(real),
                                 (size_t)cols, ctx.stream));
  scatter_lists_kernel<real><<<(unsigned)std::min(k, 65535), 256, 0, ctx.stream>>>(
      sel, k, lists, ptr, idx, val, cols, dst, ldd, dst2, ld2);
  CURID_LAUNCHED(ctx);
  return CURID_OK;
}

#define CURID_SP_INST(real)                                                                    \
  template curid_status spmm_rows<real>(const Ctx&, int64_t, const int64_t*, const int32_t*,   \
                                        const real*, int64_t, int64_t, const real*, int64_t,   \
                                        int64_t, real*, int64_t);                              \
  template curid_status scatter_lists<real>(const Ctx&, const int32_t*, int, int64_t,          \
                                            const int64_t*, const int32_t*, const real*,       \
                                            int64_t, real*, int64_t, real*, int64_t);
CURID_SP_INST(float)
CURID_SP_INST(double)
#undef CURID_SP_INST

}  // namespace curid
