// Column and row gathers (C = A(:, J[:k]), R = A(I[:k], :), Eq. (3.1)), the
// split of S1 into S11 and S12 (Eq. (2.7)), and plain 2-D copies.
// Memory-bound; all writes are coalesced, reads are coalesced wherever the
// index set allows (rows of R are contiguous; a column of C is a stride-lda
// walk, so each warp reads 32 rows of one skeleton column).
#include <type_traits>

#include "kernels.cuh"

namespace curid {

namespace {

// element conversion between storage types (bfloat16 <-> float exact or
// round-to-nearest; float <-> double by the language rules)
template <typename D, typename S>
__device__ __forceinline__ D cvt(S x) {
  return static_cast<D>(x);
}
template <>
__device__ __forceinline__ float cvt<float, __nv_bfloat16>(__nv_bfloat16 x) {
  return __bfloat162float(x);
}
template <>
__device__ __forceinline__ __nv_bfloat16 cvt<__nv_bfloat16, float>(float x) {
  return __float2bfloat16_rn(x);
}
template <>
__device__ __forceinline__ __nv_bfloat16 cvt<__nv_bfloat16, __nv_bfloat16>(__nv_bfloat16 x) {
  return x;
}

// out^T layout (transpose == true): out[i*ldo + r] = A[r*lda + J[i]].  A
// column is a stride-lda walk, so every element costs one 32-byte sector;
// each thread keeps four of them in flight.
template <typename S, typename D>
__global__ void gather_cols_t_kernel(const S* __restrict__ A, int64_t m, int64_t n, int64_t lda,
                                     const int32_t* __restrict__ J, int k,
                                     D* __restrict__ out, int64_t ldo) {
  const int i = blockIdx.y;
  int64_t col = J[i];
  if (col < 0 || col >= n) col = 0;  // indices come from the device; never read out of range
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t r0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r0 < m; r0 += 4 * stride) {
    S v[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int64_t r = r0 + u * stride;
      v[u] = r < m ? A[r * lda + col] : S(0.f);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int64_t r = r0 + u * stride;
      if (r < m) out[(int64_t)i * ldo + r] = cvt<D>(v[u]);
    }
  }
}

// out[r*ldo + i] = A[r*lda + J[i]] through a 32 x 32 shared tile
template <typename S, typename D>
__global__ void gather_cols_kernel(const S* __restrict__ A, int64_t m, int64_t n, int64_t lda,
                                   const int32_t* __restrict__ J, int k,
                                   D* __restrict__ out, int64_t ldo) {
  __shared__ D tile[32][33];
  const int i0 = blockIdx.y * 32;
  const int64_t r0 = blockIdx.x * 32LL;
  const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
  for (int yy = ty; yy < 32; yy += 8) {
    const int i = i0 + yy;
    const int64_t r = r0 + tx;
    int64_t col = i < k ? (int64_t)J[i] : 0;
    if (col < 0 || col >= n) col = 0;
    tile[yy][tx] = (i < k && r < m) ? cvt<D>(A[r * lda + col]) : cvt<D>(0.f);
  }
  __syncthreads();
  for (int yy = ty; yy < 32; yy += 8) {
    const int64_t r = r0 + yy;
    const int i = i0 + tx;
    if (r < m && i < k) out[r * ldo + i] = tile[tx][yy];
  }
}

template <typename S, typename D>
__global__ void gather_rows_kernel(const S* __restrict__ A, int64_t m, int64_t n, int64_t lda,
                                   const int32_t* __restrict__ I, D* __restrict__ out,
                                   int64_t ldo) {
  const int i = blockIdx.y;
  int64_t row = I[i];
  if (row < 0 || row >= m) row = 0;
  const S* src = A + row * lda;
  D* dst = out + (int64_t)i * ldo;
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < n;
       c += (int64_t)gridDim.x * blockDim.x)
    dst[c] = cvt<D>(src[c]);
}

// Rows of one element type copied as 16-byte vectors V (rows, leading
// dimensions and n in whole vectors; checked by the launcher).
template <typename V>
__global__ void gather_rows_vec_kernel(const V* __restrict__ A, int64_t m, int64_t nv,
                                       int64_t ldav, const int32_t* __restrict__ I,
                                       V* __restrict__ out, int64_t ldov) {
  const int i = blockIdx.y;
  int64_t row = I[i];
  if (row < 0 || row >= m) row = 0;
  const V* src = A + row * ldav;
  V* dst = out + (int64_t)i * ldov;
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < nv;
       c += (int64_t)gridDim.x * blockDim.x)
    dst[c] = src[c];
}

template <typename real>
__global__ void split_s_kernel(const real* __restrict__ S, int64_t lds,
                               const int32_t* __restrict__ J, int k, int64_t n,
                               real* __restrict__ S11, real* __restrict__ S12) {
  const int i = blockIdx.y;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n;
       t += (int64_t)gridDim.x * blockDim.x) {
    int64_t col = J[t];
    if (col < 0 || col >= n) col = 0;
    const real v = S[(int64_t)i * lds + col];
    if (t < k) S11[(int64_t)i * k + t] = v;
    else S12[(int64_t)i * (n - k) + (t - k)] = v;
  }
}

template <typename S, typename D>
__global__ void copy2d_kernel(const S* __restrict__ src, int64_t lds, D* __restrict__ dst,
                              int64_t ldd, int64_t rows, int64_t cols) {
  const int64_t total = rows * cols;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / cols, c = e % cols;
    dst[r * ldd + c] = cvt<D>(src[r * lds + c]);
  }
}

template <typename real>
__global__ void add_transpose_kernel(const real* __restrict__ src, int64_t lds,
                                     real* __restrict__ dst, int64_t ldd, int64_t rows,
                                     int64_t cols) {
  const int64_t total = rows * cols;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / cols, c = e % cols;
    dst[r * ldd + c] += src[c * lds + r];
  }
}

// x -> (hi, lo): hi = x with the 13 low mantissa bits cleared (exactly a
// TF32 value, which the tensor cores use unchanged), lo = x - hi (exact in
// float32; the tensor cores read it to about 2^-10 of itself, 2^-21 of x).
// hi may be x itself.
__global__ void split_tf32_kernel(const float* x, int64_t ldx, float* hi, int64_t ldh,
                                  float* __restrict__ lo, int64_t ldl, int64_t rows,
                                  int64_t cols) {
  const int64_t total = rows * cols;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / cols, c = e % cols;
    const float v = x[r * ldx + c];
    const float h = __uint_as_float(__float_as_uint(v) & 0xffffe000u);
    hi[r * ldh + c] = h;
    lo[r * ldl + c] = v - h;
  }
}

template <typename real>
__global__ void add2d_kernel(const real* __restrict__ src, int64_t lds, real* __restrict__ dst,
                             int64_t ldd, int64_t rows, int64_t cols) {
  const int64_t total = rows * cols;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / cols, c = e % cols;
    dst[r * ldd + c] += src[r * lds + c];
  }
}

// dst (k x 2k, leading dimension ldd) = [S11^T | lam I] from S11 (k x k)
template <typename real>
__global__ void aug_transpose_kernel(const real* __restrict__ S11, int64_t lds, int k, real lam,
                                     real* __restrict__ dst, int64_t ldd) {
  const int64_t total = 2LL * k * k;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / (2 * k), j = e % (2 * k);
    dst[i * ldd + j] = j < k ? S11[j * lds + i] : (j - k == i ? lam : real(0));
  }
}

// dst[c*ldd + r] = src[r*lds + c] through a 32 x 32 shared tile
template <typename real>
__global__ void transpose2d_kernel(const real* __restrict__ src, int64_t lds,
                                   real* __restrict__ dst, int64_t ldd, int64_t rows,
                                   int64_t cols) {
  __shared__ real tile[32][33];
  const int64_t r0 = blockIdx.y * 32LL, c0 = blockIdx.x * 32LL;
  const int tx = threadIdx.x, ty = threadIdx.y;
  for (int yy = ty; yy < 32; yy += 8) {
    const int64_t r = r0 + yy, c = c0 + tx;
    tile[yy][tx] = (r < rows && c < cols) ? src[r * lds + c] : real(0);
  }
  __syncthreads();
  for (int yy = ty; yy < 32; yy += 8) {
    const int64_t c = c0 + yy, r = r0 + tx;
    if (r < rows && c < cols) dst[c * ldd + r] = tile[tx][yy];
  }
}

inline unsigned blocks_for(int64_t work, int num_sms) {
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>((work + 255) / 256, 16LL * num_sms));
}

}  // namespace

template <typename S, typename D>
curid_status gather_cols_as(const Ctx& ctx, const S* A, int64_t m, int64_t n, int64_t lda,
                            const int32_t* J, int k, D* out, int64_t ldo, bool transpose) {
  if (k <= 0 || m <= 0) return CURID_OK;
  if (transpose) {
    dim3 grid((unsigned)std::max<int64_t>(1, std::min<int64_t>((m + 1023) / 1024, 64)),
              (unsigned)k);
    gather_cols_t_kernel<S, D><<<grid, 256, 0, ctx.stream>>>(A, m, n, lda, J, k, out, ldo);
  } else {
    dim3 grid((unsigned)((m + 31) / 32), (unsigned)((k + 31) / 32));
    gather_cols_kernel<S, D><<<grid, dim3(32, 8), 0, ctx.stream>>>(A, m, n, lda, J, k, out, ldo);
  }
  CURID_LAUNCHED(ctx);
  return CURID_OK;
}

template <typename S, typename D>
curid_status gather_rows_as(const Ctx& ctx, const S* A, int64_t m, int64_t n, int64_t lda,
                            const int32_t* I, int k, D* out, int64_t ldo) {
  if (k <= 0 || n <= 0) return CURID_OK;
  constexpr int64_t w = 16 / sizeof(S);  // elements per 16-byte vector
  if constexpr (std::is_same<S, D>::value && 16 % sizeof(S) == 0) {
    if (n % w == 0 && lda % w == 0 && ldo % w == 0 &&
        (reinterpret_cast<uintptr_t>(A) & 15) == 0 && (reinterpret_cast<uintptr_t>(out) & 15) == 0) {
      const int64_t nv = n / w;
      dim3 grid((unsigned)std::min<int64_t>((nv + 255) / 256, 64), (unsigned)k);
      gather_rows_vec_kernel<uint4><<<grid, 256, 0, ctx.stream>>>(
          reinterpret_cast<const uint4*>(A), m, nv, lda / w, I, reinterpret_cast<uint4*>(out),
          ldo / w);
      CURID_LAUNCHED(ctx);
      return CURID_OK;
    }
  }
  dim3 grid((unsigned)std::min<int64_t>((n + 255) / 256, 64), (unsigned)k);
  gather_rows_kernel<S, D><<<grid, 256, 0, ctx.stream>>>(A, m, n, lda, I, out, ldo);
  CURID_LAUNCHED(ctx);
  return CURID_OK;
}

template <typename S, typename D>
curid_status convert2d(const Ctx& ctx, const S* src, int64_t lds, D* dst, int64_t ldd,
                       int64_t rows, int64_t cols) {
  if (rows <= 0 || cols <= 0) return CURID_OK;
  copy2d_kernel<S, D><<<blocks_for(rows * cols, ctx.num_sms), 256, 0, ctx.stream>>>(
      src, lds, dst, ldd, rows, cols);
  CURID_LAUNCHED(ctx);
  return CURID_OK;
}

template <typename real>
curid_status gather_cols(const Ctx& ctx, const real* A, int64_t m, int64_t n, int64_t lda,
                         const int32_t* J, int k, real* out, int64_t ldo, bool transpose) {
  return gather_cols_as<real, real>(ctx, A, m, n, lda, J, k, out, ldo, transpose);
}

template <typename real>
curid_status gather_rows(const Ctx& ctx, const real* A, int64_t m, int64_t n, int64_t lda,
                         const int32_t* I, int k, real* out, int64_t ldo) {
  return gather_rows_as<real, real>(ctx, A, m, n, lda, I, k, out, ldo);
}

template <typename real>
curid_status split_s(const Ctx& ctx, const real* S, int64_t lds, const int32_t* J, int k,
                     int64_t n, real* S11, real* S12) {
  if (k <= 0) return CURID_OK;
  dim3 grid((unsigned)std::min<int64_t>((n + 255) / 256, 64), (unsigned)k);
  split_s_kernel<real><<<grid, 256, 0, ctx.stream>>>(S, lds, J, k, n, S11, S12);
  CURID_LAUNCHED(ctx);
  return CURID_OK;
}

template <typename real>
curid_status copy2d(const Ctx& ctx, const real* src, int64_t lds, real* dst, int64_t ldd,
                    int64_t rows, int64_t cols) {
  return convert2d<real, real>(ctx, src, lds, dst, ldd, rows, cols);
}

template <typename real>
curid_status add_transpose(const Ctx& ctx, const real* src, int64_t lds, real* dst, int64_t ldd,
                           int64_t rows, int64_t cols) {
  if (rows <= 0 || cols <= 0) return CURID_OK;
  add_transpose_kernel<real><<<blocks_for(rows * cols, ctx.num_sms), 256, 0, ctx.stream>>>(
      src, lds, dst, ldd, rows, cols);
  CURID_LAUNCHED(ctx);
  return CURID_OK;
}

curid_status split_tf32(const Ctx& ctx, const float* x, int64_t ldx, float* hi, int64_t ldh,
                        float* lo, int64_t ldl, int64_t rows, int64_t cols) {
  if (rows <= 0 || cols <= 0) return CURID_OK;
  split_tf32_kernel<<<blocks_for(rows * cols, ctx.num_sms), 256, 0, ctx.stream>>>(
      x, ldx, hi, ldh, lo, ldl, rows, cols);
  CURID_LAUNCHED(ctx);
  return CURID_OK;
}

template <typename real>
curid_status aug_transpose(const Ctx& ctx, const real* S11, int64_t lds, int k, real lam,
                           real* dst, int64_t ldd) {
  if (k <= 0) return CURID_OK;
  aug_transpose_kernel<real><<<blocks_for(2LL * k * k, ctx.num_sms), 256, 0, ctx.stream>>>(
      S11, lds, k, lam, dst, ldd);
  CURID_LAUNCHED(ctx);
  return CURID_OK;
}

template <typename real>
curid_status add2d(const Ctx& ctx, const real* src, int64_t lds, real* dst, int64_t ldd,
                   int64_t rows, int64_t cols) {
  if (rows <= 0 || cols <= 0) return CURID_OK;
  add2d_kernel<real><<<blocks_for(rows * cols, ctx.num_sms), 256, 0, ctx.stream>>>(
      src, lds, dst, ldd, rows, cols);
  CURID_LAUNCHED(ctx);
  return CURID_OK;
}

template <typename real>
curid_status transpose2d(const Ctx& ctx, const real* src, int64_t lds, real* dst, int64_t ldd,
                         int64_t rows, int64_t cols) {
  if (rows <= 0 || cols <= 0) return CURID_OK;
  dim3 grid((unsigned)((cols + 31) / 32), (unsigned)((rows + 31) / 32));
  transpose2d_kernel<real><<<grid, dim3(32, 8), 0, ctx.stream>>>(src, lds, dst, ldd, rows, cols);
  CURID_LAUNCHED(ctx);
  return CURID_OK;
}

#define CURID_INST(real)                                                                       \
  template curid_status gather_cols<real>(const Ctx&, const real*, int64_t, int64_t, int64_t,  \
                                          const int32_t*, int, real*, int64_t, bool);          \
  template curid_status gather_rows<real>(const Ctx&, const real*, int64_t, int64_t, int64_t,  \
                                          const int32_t*, int, real*, int64_t);                \
  template curid_status split_s<real>(const Ctx&, const real*, int64_t, const int32_t*, int,   \
                                      int64_t, real*, real*);                                  \
  template curid_status copy2d<real>(const Ctx&, const real*, int64_t, real*, int64_t, int64_t, \
                                     int64_t);                                                 \
  template curid_status add_transpose<real>(const Ctx&, const real*, int64_t, real*, int64_t,   \
                                            int64_t, int64_t);                                 \
  template curid_status transpose2d<real>(const Ctx&, const real*, int64_t, real*, int64_t,     \
                                          int64_t, int64_t);                                   \
  template curid_status add2d<real>(const Ctx&, const real*, int64_t, real*, int64_t, int64_t,  \
                                    int64_t);                                                  \
  template curid_status aug_transpose<real>(const Ctx&, const real*, int64_t, int, real, real*, \
                                            int64_t);
CURID_INST(float)
CURID_INST(double)
#undef CURID_INST

using bf16_t = __nv_bfloat16;
template curid_status gather_cols_as<bf16_t, float>(const Ctx&, const bf16_t*, int64_t, int64_t,
                                                    int64_t, const int32_t*, int, float*, int64_t,
                                                    bool);
template curid_status gather_cols_as<bf16_t, bf16_t>(const Ctx&, const bf16_t*, int64_t,
                                                     int64_t, int64_t, const int32_t*, int,
                                                     bf16_t*, int64_t, bool);
template curid_status gather_rows_as<bf16_t, float>(const Ctx&, const bf16_t*, int64_t, int64_t,
                                                    int64_t, const int32_t*, int, float*,
                                                    int64_t);
template curid_status convert2d<float, bf16_t>(const Ctx&, const float*, int64_t, bf16_t*,
                                               int64_t, int64_t, int64_t);
template curid_status convert2d<float, double>(const Ctx&, const float*, int64_t, double*,
                                               int64_t, int64_t, int64_t);
template curid_status convert2d<double, float>(const Ctx&, const double*, int64_t, float*,
                                               int64_t, int64_t, int64_t);
template curid_status convert2d<float, float>(const Ctx&, const float*, int64_t, float*,
                                              int64_t, int64_t, int64_t);
template curid_status convert2d<double, double>(const Ctx&, const double*, int64_t, double*,
                                                int64_t, int64_t, int64_t);

}  // namespace curid
