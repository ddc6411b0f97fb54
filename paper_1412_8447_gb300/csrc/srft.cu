// Structured sampling matrix of the accelerated randomized scheme (Section
// 5.2, Eq. (5.2)): Omega = sqrt(m / l) R F D, l x m.  Real form of the
// paper's construction: D = diag(d) with random signs d_t = +-1 (the real
// unit circle), F the orthonormal DCT-II, F(f, t) = c_f cos(pi f (2t+1) / (2m))
// with c_0 = sqrt(1/m) and c_f = sqrt(2/m), and R the l sampled rows f_i.
// So Omega(i, t) = s_i d_t cos(pi f_i (2t+1) / (2m)), s_i = sqrt(1/l) for
// f_i = 0 and sqrt(2/l) otherwise.
//
// The matrix is formed explicitly and applied by the same tensor-core
// product as a Gaussian Omega: with l of a few hundred the product Omega A
// reads A once from HBM either way, which is all a fast transform would save
// on this GPU.
//
// Angles: r = f (2t+1) mod 4m indexes cos(pi r / (2m)); split r = 256 a + b,
// cos = cos(a) cos(b) - sin(a) sin(b) from two float64 tables of sincospi
// values in shared memory (4m / 256 and 256 entries), so every element costs
// two table reads and three float64 operations and is accurate to a few
// float64 ulp.  Each CTA covers 16 rows and 2048 columns; a thread walks its
// 8 columns (stride 256) with the angle index advanced by 512 f mod 4m.
#include "kernels.cuh"

namespace curid {

namespace {

constexpr int kSrftThreads = 256;
constexpr int kSrftCols = 8 * kSrftThreads;  // columns per CTA
constexpr int kSrftRows = 16;                 // rows per CTA
constexpr int kSrftB = 256;                   // low part of the angle index

template <typename real>
__global__ void __launch_bounds__(kSrftThreads)
srft_kernel(int m, int l, const int32_t* __restrict__ rows, const int8_t* __restrict__ signs,
            real* __restrict__ out, int64_t ld) {
  extern __shared__ double2 srft_tab[];  // [na] (cos, sin) of pi 256 a / (2m), then [256]
  const int na = (4 * m + kSrftB - 1) / kSrftB;
  double2* ta = srft_tab;
  double2* tb = srft_tab + na;
  const int tid = threadIdx.x;
  for (int a = tid; a < na; a += kSrftThreads) {
    double s, c;
    sincospi((double)(kSrftB * a) / (2.0 * m), &s, &c);
    ta[a] = make_double2(c, s);
  }
  for (int b = tid; b < kSrftB; b += kSrftThreads) {
    double s, c;
    sincospi((double)b / (2.0 * m), &s, &c);
    tb[b] = make_double2(c, s);
  }
  __syncthreads();
  const int t0 = blockIdx.x * kSrftCols + tid;
  const int64_t four_m = 4LL * m;
  double d[8];
#pragma unroll
  for (int u = 0; u < 8; ++u) {
    const int t = t0 + u * kSrftThreads;
    d[u] = (t < m && signs[t] < 0) ? -1.0 : 1.0;
  }
  const int i_end = min(l, (int)(blockIdx.y + 1) * kSrftRows);
  for (int i = blockIdx.y * kSrftRows; i < i_end; ++i) {
    const int64_t f = (((int64_t)rows[i] % four_m) + four_m) % four_m;
    const double scale = sqrt((f == 0 ? 1.0 : 2.0) / (double)l);
    int r = (int)((f * (2LL * t0 + 1)) % four_m);
    const int step = (int)((2 * kSrftThreads * f) % four_m);
    real* o = out + (int64_t)i * ld;
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int t = t0 + u * kSrftThreads;
      if (t < m) {
        const double2 A = ta[r / kSrftB], B = tb[r % kSrftB];
        const double c = fma(A.x, B.x, -A.y * B.y);
        o[t] = (real)(c * scale * d[u]);
      }
      r += step;
      if (r >= four_m) r -= (int)four_m;
    }
  }
}

}  // namespace

template <typename real>
size_t srft_smem_bytes(int64_t m) {
  return (size_t)((4 * m + kSrftB - 1) / kSrftB + kSrftB) * sizeof(double2);
}

template <typename real>
curid_status srft_fill(const Ctx& ctx, int64_t m, int64_t l, const int32_t* rows,
                       const int8_t* signs, real* out, int64_t ld) {
  if (m <= 0 || l <= 0) return CURID_OK;
  if (m > (1LL << 28) || (l + kSrftRows - 1) / kSrftRows > 65535) return CURID_UNSUPPORTED;
  const size_t smem = srft_smem_bytes<real>(m);
  if (smem > ctx.smem_optin) return CURID_UNSUPPORTED;
  auto fn = srft_kernel<real>;
  CURID_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  dim3 grid((unsigned)((m + kSrftCols - 1) / kSrftCols),
            (unsigned)((l + kSrftRows - 1) / kSrftRows));
  fn<<<grid, kSrftThreads, smem, ctx.stream>>>((int)m, (int)l, rows, signs, out, ld);
  CURID_LAUNCHED(ctx);
  return CURID_OK;
}

template curid_status srft_fill<float>(const Ctx&, int64_t, int64_t, const int32_t*,
                                       const int8_t*, float*, int64_t);
template curid_status srft_fill<double>(const Ctx&, int64_t, int64_t, const int32_t*,
                                        const int8_t*, double*, int64_t);

}  // namespace curid
