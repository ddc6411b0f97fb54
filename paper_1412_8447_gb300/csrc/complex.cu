// Complex A (the paper states the method over C, Section 1): each entry
// a = x + iy becomes the real 2 x 2 block [[x, -y], [y, x]] (the matrix of
// multiplication by a), so A (m x n) becomes a real 2m x 2n matrix E(A) with
// E(AB) = E(A) E(B) and E(A^*) = E(A)^T.  The columns 2j and 2j + 1 of E(A)
// are orthogonal with equal norms, and a left orthogonal factor keeps them
// so; greedy column pivoting therefore takes them as a pair in consecutive
// steps (after the first, the second keeps the largest norm), 2k real steps
// are the k complex steps, the real T of E is E(T), and the real pipeline's
// U is E(U) with its rows and columns swapped within the pairs taken odd
// member first.  A sketch uses E(Omega) with a complex Gaussian Omega, so
// every sample is E of the complex sample up to a left orthogonal factor.
//
// Kernels here: the embedding, and the extraction of J, I (pair check),
// T and U from the real results.
#include "kernels.cuh"

namespace curid {

namespace {

// E (2m x 2n, lde) from A (m x n complex, interleaved, lda complex entries)
template <typename real>
__global__ void embed_complex_kernel(const real* __restrict__ A, int64_t m, int64_t n,
                                     int64_t lda, real* __restrict__ E, int64_t lde) {
  const int64_t total = m * n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / n, j = e % n;
    const real x = A[2 * (i * lda + j)], y = A[2 * (i * lda + j) + 1];
    real* r0 = E + (2 * i) * lde + 2 * j;
    real* r1 = r0 + lde;
    r0[0] = x;
    r0[1] = -y;
    r1[0] = y;
    r1[1] = x;
  }
}

// Complex pivots from the real ones: the first k pairs (either member
// first), then the unselected pairs in ascending order; a pair that is not
// {2j, 2j + 1} flags a breakdown (two complex pivots of equal norm to within
// rounding interleaved).
__global__ void extract_pivots_kernel(const int32_t* __restrict__ Jp, int k, int64_t n,
                                      int32_t* __restrict__ J, StatusBlock* status,
                                      bool halve_ranks) {
  if (halve_ranks && blockIdx.x == 0 && threadIdx.x == 0) {
    // the status block's ranks count real steps: two per complex pivot.  The
    // embedding's rank is even in exact arithmetic; an odd count means the
    // rank cut-off or the tolerance stop fell between the two members of a
    // pair (one fell below the threshold within rounding of the other): the
    // complex rank is rounded down and flagged.
    if ((status->k_eff | status->k_row) & 1) set_flag(&status->flags, FLAG_RANK_DEFICIENT);
    if (status->k_done & 1) set_flag(&status->flags, FLAG_BREAKDOWN);
    status->k_done >>= 1;
    status->k_eff >>= 1;
    status->k_row >>= 1;
  }
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int a = Jp[2 * t], b = Jp[2 * t + 1];
    const bool ok = t < k ? ((a ^ 1) == b) : ((a & 1) == 0 && b == a + 1);
    if (!ok) set_flag(&status->flags, FLAG_BREAKDOWN);
    J[t] = a >> 1;
  }
}

// Row of the real result that carries the real (even) / imaginary (odd)
// member of pair t, given which member the pivot order took first.
__device__ __forceinline__ int even_of(const int32_t* P, int t) {
  return (P[2 * t] & 1) ? 2 * t + 1 : 2 * t;
}
__device__ __forceinline__ int odd_of(const int32_t* P, int t) {
  return (P[2 * t] & 1) ? 2 * t : 2 * t + 1;
}

// T (k x cols complex, interleaved, ldt complex) from the real Tp
// (2k x 2 cols, ldtp): T(t, c) = Tp(even_t, 2c) + i Tp(odd_t, 2c).
template <typename real, typename out_t>
__global__ void extract_t_kernel(const real* __restrict__ Tp, int64_t ldtp,
                                 const int32_t* __restrict__ Jp, int k, int64_t cols,
                                 out_t* __restrict__ T, int64_t ldt) {
  const int64_t total = (int64_t)k * cols;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int t = (int)(e / cols);
    const int64_t c = e % cols;
    T[2 * (t * ldt + c)] = (out_t)Tp[even_of(Jp, t) * ldtp + 2 * c];
    T[2 * (t * ldt + c) + 1] = (out_t)Tp[odd_of(Jp, t) * ldtp + 2 * c];
  }
}

// U (k x k complex float64, interleaved) from the real Up (2k x 2k):
// U(t, s) = Up(even_J(t), even_I(s)) + i Up(odd_J(t), even_I(s)).
__global__ void extract_u_kernel(const double* __restrict__ Up, const int32_t* __restrict__ Jp,
                                 const int32_t* __restrict__ Ip, int k, double* __restrict__ U) {
  const int64_t total = (int64_t)k * k;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int t = (int)(e / k), s = (int)(e % k);
    const int c = even_of(Ip, s);
    U[2 * e] = Up[(int64_t)even_of(Jp, t) * 2 * k + c];
    U[2 * e + 1] = Up[(int64_t)odd_of(Jp, t) * 2 * k + c];
  }
}

unsigned grid_for(int64_t total, int num_sms) {
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>((total + 255) / 256, 16LL * num_sms));
}

}  // namespace

template <typename real>
curid_status embed_complex(const Ctx& ctx, const real* A, int64_t m, int64_t n, int64_t lda,
                           real* E, int64_t lde) {
  if (m <= 0 || n <= 0) return CURID_OK;
  embed_complex_kernel<real><<<grid_for(m * n, ctx.num_sms), 256, 0, ctx.stream>>>(A, m, n, lda,
                                                                                  E, lde);
  CURID_LAUNCHED(ctx);
  return CURID_OK;
}

curid_status extract_pivots(const Ctx& ctx, const int32_t* Jp, int k, int64_t n, int32_t* J,
                            bool halve_ranks) {
  if (n <= 0) return CURID_OK;
  extract_pivots_kernel<<<grid_for(n, ctx.num_sms), 256, 0, ctx.stream>>>(Jp, k, n, J,
                                                                         ctx.status, halve_ranks);
  CURID_LAUNCHED(ctx);
  return CURID_OK;
}

template <typename real>
curid_status extract_t(const Ctx& ctx, const real* Tp, int64_t ldtp, const int32_t* Jp, int k,
                       int64_t cols, real* T, int64_t ldt) {
  if (k <= 0 || cols <= 0) return CURID_OK;
  extract_t_kernel<real, real><<<grid_for((int64_t)k * cols, ctx.num_sms), 256, 0, ctx.stream>>>(
      Tp, ldtp, Jp, k, cols, T, ldt);
  CURID_LAUNCHED(ctx);
  return CURID_OK;
}

curid_status extract_u(const Ctx& ctx, const double* Up, const int32_t* Jp, const int32_t* Ip,
                       int k, double* U) {
  if (k <= 0) return CURID_OK;
  extract_u_kernel<<<grid_for((int64_t)k * k, ctx.num_sms), 256, 0, ctx.stream>>>(Up, Jp, Ip, k,
                                                                                 U);
  CURID_LAUNCHED(ctx);
  return CURID_OK;
}

template curid_status embed_complex<float>(const Ctx&, const float*, int64_t, int64_t, int64_t,
                                           float*, int64_t);
template curid_status embed_complex<double>(const Ctx&, const double*, int64_t, int64_t, int64_t,
                                            double*, int64_t);
template curid_status extract_t<float>(const Ctx&, const float*, int64_t, const int32_t*, int,
                                       int64_t, float*, int64_t);
template curid_status extract_t<double>(const Ctx&, const double*, int64_t, const int32_t*, int,
                                        int64_t, double*, int64_t);

}  // namespace curid
