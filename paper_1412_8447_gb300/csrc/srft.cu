// Structured sampling matrix of the accelerated randomized scheme (Section
// 5.2, Eq. (5.2)): Omega = sqrt(m / l) R F D, l x m.  Real form of the
// paper's construction: D = diag(d) with random signs d_t = +-1 (the real
// unit circle), F the orthonormal DCT-II, F(f, t) = c_f cos(pi f (2t+1) / (2m))
// with c_0 = sqrt(1/m) and c_f = sqrt(2/m), and R the l sampled rows f_i.
// So Omega(i, t) = s_i d_t cos(pi f_i (2t+1) / (2m)), s_i = sqrt(1/l) for
// f_i = 0 and sqrt(2/l) otherwise.
//
// Two ways to apply it.  srft_fill forms Omega explicitly, for the same
// tensor-core product as a Gaussian Omega.  srft_apply computes Y = Omega A
// without forming it: each CTA reads a few whole columns of A once (one
// coalesced pass over A in all), transforms them in shared memory with the
// fast DCT of srft_fft.cuh (O(m log m) per column, Makhoul's reordering, two
// real columns per complex transform) and writes the l sampled rows.
//
// Angles: r = f (2t+1) mod 4m indexes cos(pi r / (2m)); split r = 256 a + b,
// cos = cos(a) cos(b) - sin(a) sin(b) from two float64 tables of sincospi
// values in shared memory (4m / 256 and 256 entries), so every element costs
// two table reads and three float64 operations and is accurate to a few
// float64 ulp.  Each CTA covers 16 rows and 2048 columns; a thread walks its
// 8 columns (stride 256) with the angle index advanced by 512 f mod 4m.
#include <cstdlib>
#include <cstring>

#include "kernels.cuh"
#include "srft_fft.cuh"

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

// ---- fast application ----
constexpr int kApplyThreads = 512;
constexpr int kApplyUnroll = 4;  // rows of A in flight per thread

// 2 NS consecutive entries of one row of A (cnt of them inside the matrix)
template <typename real, int NS>
__device__ __forceinline__ void load_cols(const real* __restrict__ p, int cnt, bool vec,
                                          real (&v)[2 * NS]) {
  if (vec && cnt == 2 * NS) {
    if constexpr (sizeof(real) == 4 && NS == 1) {
      const float2 q = __ldg(reinterpret_cast<const float2*>(p));
      v[0] = q.x;
      v[1] = q.y;
    } else if constexpr (sizeof(real) == 4) {
#pragma unroll
      for (int c = 0; c < NS / 2; ++c) {
        const float4 q = __ldg(reinterpret_cast<const float4*>(p) + c);
        v[4 * c] = q.x;
        v[4 * c + 1] = q.y;
        v[4 * c + 2] = q.z;
        v[4 * c + 3] = q.w;
      }
    } else {
#pragma unroll
      for (int c = 0; c < NS; ++c) {
        const double2 q = __ldg(reinterpret_cast<const double2*>(p) + c);
        v[2 * c] = q.x;
        v[2 * c + 1] = q.y;
      }
    }
  } else {
#pragma unroll
    for (int c = 0; c < 2 * NS; ++c) v[c] = c < cnt ? __ldg(p + c) : (real)0;
  }
}

// Y(:, c0 : c0 + 2 NS) = sqrt(m / l) R F D A(:, c0 : c0 + 2 NS): columns
// c0 + 2s and c0 + 2s + 1 are the real and imaginary parts of sequence s.
template <typename real, int NS>
__global__ void __launch_bounds__(kApplyThreads)
srft_apply_kernel(const real* __restrict__ A, int m, int n, int64_t lda,
                  const int8_t* __restrict__ signs, const int32_t* __restrict__ rows, int l,
                  real* __restrict__ Y, int64_t ldy, FftPlan plan, int vec, real scale0,
                  real scale1) {
  extern __shared__ __align__(16) unsigned char srft_apply_smem[];
  cplx<real>* z = reinterpret_cast<cplx<real>*>(srft_apply_smem);
  const int c0 = blockIdx.x * 2 * NS;
  const int cnt = min(2 * NS, n - c0);
  const real* Ab = A + c0;
  const int bd = blockDim.x;
  // ---- D A, reordered even rows first, odd rows reversed ----
  for (int t0 = threadIdx.x; t0 < m; t0 += kApplyUnroll * bd) {
    real v[kApplyUnroll][2 * NS];
#pragma unroll
    for (int u = 0; u < kApplyUnroll; ++u) {
      const int t = t0 + u * bd;
      if (t < m) load_cols<real, NS>(Ab + (int64_t)t * lda, cnt, vec != 0, v[u]);
    }
#pragma unroll
    for (int u = 0; u < kApplyUnroll; ++u) {
      const int t = t0 + u * bd;
      if (t < m) {
        const real d = signs[t] < 0 ? (real)-1 : (real)1;
        const int p = fft_reorder(t, m);
#pragma unroll
        for (int s = 0; s < NS; ++s) z[s * m + p] = {v[u][2 * s] * d, v[u][2 * s + 1] * d};
      }
    }
  }
  __syncthreads();
  // ---- in-place mixed-radix DFT of every sequence ----
  int L = m;
  for (int j = 0; j < plan.nst; ++j) {
    const int r = plan.radix[j];
    switch (r) {
      case 4: fft_stage<real, 4, NS>(z, m, L, threadIdx.x, bd); break;
      case 2: fft_stage<real, 2, NS>(z, m, L, threadIdx.x, bd); break;
      case 3: fft_stage<real, 3, NS>(z, m, L, threadIdx.x, bd); break;
      case 5: fft_stage<real, 5, NS>(z, m, L, threadIdx.x, bd); break;
      default: fft_stage<real, 7, NS>(z, m, L, threadIdx.x, bd); break;
    }
    L /= r;
    __syncthreads();
  }
  // ---- the l sampled rows, scaled ----
  const int64_t four_m = 4LL * m;
  for (int i = threadIdx.x; i < l; i += bd) {
    const int64_t f = rows[i];
    const real sc = (((f % four_m) + four_m) % four_m) == 0 ? scale0 : scale1;
    real* yi = Y + (int64_t)i * ldy + c0;
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      real x1, x2;
      const real sg = fft_dct_pair<real>(z + s * m, plan, m, f, &x1, &x2);
      if (2 * s < cnt) yi[2 * s] = sg * sc * x1;
      if (2 * s + 1 < cnt) yi[2 * s + 1] = sg * sc * x2;
    }
  }
}

template <typename real, int NS>
curid_status launch_apply(const Ctx& ctx, const real* A, int64_t m, int64_t n, int64_t lda,
                          int64_t l, const int32_t* rows, const int8_t* signs, real* Y,
                          int64_t ldy, const FftPlan& plan) {
  const size_t smem = (size_t)NS * m * sizeof(cplx<real>);
  const size_t vbytes = 2 * NS * sizeof(real) >= 16 ? 16 : 2 * NS * sizeof(real);
  const int vec = (reinterpret_cast<uintptr_t>(A) % vbytes == 0 &&
                   (lda * sizeof(real)) % vbytes == 0) ? 1 : 0;
  auto fn = srft_apply_kernel<real, NS>;
  CURID_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const int64_t grid = (n + 2 * NS - 1) / (2 * NS);
  fn<<<(unsigned)grid, kApplyThreads, smem, ctx.stream>>>(
      A, (int)m, (int)n, lda, signs, rows, (int)l, Y, ldy, plan, vec,
      (real)std::sqrt(1.0 / (double)l), (real)std::sqrt(2.0 / (double)l));
  CURID_LAUNCHED(ctx);
  return CURID_OK;
}

}  // namespace

template <typename real>
curid_status srft_apply(const Ctx& ctx, const real* A, int64_t m, int64_t n, int64_t lda,
                        int64_t l, const int32_t* rows, const int8_t* signs, real* Y,
                        int64_t ldy) {
  if (m <= 0 || n <= 0 || l <= 0) return CURID_OK;
  if (m > INT32_MAX / 4 || n > INT32_MAX || l > INT32_MAX) return CURID_UNSUPPORTED;
  const FftPlan plan = fft_plan(m);
  if (plan.nst < 0) return CURID_UNSUPPORTED;
  const size_t seq = (size_t)m * sizeof(cplx<real>);
  // two sequences (four columns) per CTA where they fit, else one; the
  // environment variable CURID_SRFT_COLS (2 or 4) picks one of them
  int ns = 2 * seq <= ctx.smem_optin ? 2 : (seq <= ctx.smem_optin ? 1 : 0);
  if (const char* env = std::getenv("CURID_SRFT_COLS")) {
    if (std::strcmp(env, "2") == 0 && seq <= ctx.smem_optin) ns = 1;
    if (std::strcmp(env, "4") == 0 && 2 * seq <= ctx.smem_optin) ns = 2;
  }
  if (ns == 2) return launch_apply<real, 2>(ctx, A, m, n, lda, l, rows, signs, Y, ldy, plan);
  if (ns == 1) return launch_apply<real, 1>(ctx, A, m, n, lda, l, rows, signs, Y, ldy, plan);
  return CURID_UNSUPPORTED;
}

template curid_status srft_apply<float>(const Ctx&, const float*, int64_t, int64_t, int64_t,
                                        int64_t, const int32_t*, const int8_t*, float*, int64_t);
template curid_status srft_apply<double>(const Ctx&, const double*, int64_t, int64_t, int64_t,
                                         int64_t, const int32_t*, const int8_t*, double*,
                                         int64_t);

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
