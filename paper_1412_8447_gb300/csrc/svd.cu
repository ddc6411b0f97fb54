// Singular value decomposition of the k x k triangle S11 for the truncated-
// SVD interpolation matrix (Section 4.1: T from a stabilised pseudo-inverse
// of S11, dropping singular values below a threshold).
//
// One-sided Jacobi (Hestenes): the columns a_i of W = S11 are rotated in
// pairs until they are mutually orthogonal, W V = U diag(sigma) with
// sigma_i = ||a_i||; V accumulates the rotations.  A pair (p, q) with Gram
// entries alpha = ||a_p||^2, beta = ||a_q||^2, gamma = a_p . a_q is rotated
// when |gamma| > sqrt(k) eps sqrt(alpha beta): zeta = (beta - alpha) /
// (2 gamma), t = sign(zeta) / (|zeta| + sqrt(1 + zeta^2)), c = 1 /
// sqrt(1 + t^2), s = c t, a_p <- c a_p - s a_q, a_q <- s a_p + c a_q (the
// rotation that zeroes gamma).  A sweep visits every pair once in k' - 1
// rounds of k'/2 disjoint pairs (round-robin "circle" order, k' = k rounded
// up to even, the extra player idle): pair 0 of round r is (r, k' - 1), pair
// i > 0 is ((r + i) mod (k' - 1), (r - i) mod (k' - 1)).  One cooperative
// launch; a warp per pair, lanes over the k entries; a grid barrier after
// every round; sweeps stop when one rotates nothing (or after 40).
//
// Layout: W^T and V^T row-major (row i = column i), so a pair's columns are
// contiguous rows.
#include <cooperative_groups.h>

#include <cmath>
#include <limits>

#include "kernels.cuh"

namespace cg = cooperative_groups;

namespace curid {

namespace {

constexpr int kSvdThreads = 256;
constexpr int kSvdWarps = kSvdThreads / 32;
constexpr int kSvdMaxK = 256;  // k / 32 entries per lane in registers
constexpr int kSvdMaxSweeps = 40;

template <typename real>
__global__ void __launch_bounds__(kSvdThreads)
jacobi_svd_kernel(int k, real* __restrict__ Wt, real* __restrict__ Vt, int* __restrict__ rotations,
                  real tol) {
  cg::grid_group grid = cg::this_grid();
  constexpr int E = kSvdMaxK / 32;
  const int lane = threadIdx.x & 31;
  const int gw = blockIdx.x * kSvdWarps + (threadIdx.x >> 5);
  const int nw = gridDim.x * kSvdWarps;
  const int kp = k + (k & 1);
  for (int sweep = 0; sweep < kSvdMaxSweeps; ++sweep) {
    for (int r = 0; r < kp - 1; ++r) {
      for (int i = gw; i < kp / 2; i += nw) {
        int p, q;
        if (i == 0) {
          p = r;
          q = kp - 1;
        } else {
          p = (r + i) % (kp - 1);
          q = (r - i + kp - 1) % (kp - 1);
        }
        if (p >= k || q >= k) continue;
        real a[E], b[E];
        real al = real(0), be = real(0), ga = real(0);
#pragma unroll
        for (int u = 0; u < E; ++u) {
          const int c = lane + 32 * u;
          a[u] = c < k ? Wt[(int64_t)p * k + c] : real(0);
          b[u] = c < k ? Wt[(int64_t)q * k + c] : real(0);
          al = fma(a[u], a[u], al);
          be = fma(b[u], b[u], be);
          ga = fma(a[u], b[u], ga);
        }
        al = warp_sum(al);
        be = warp_sum(be);
        ga = warp_sum(ga);
        if (ga != real(0) && fabs(ga) > tol * sqrt(al * be)) {
          const real zeta = (be - al) / (real(2) * ga);
          const real t = copysign(real(1), zeta) / (fabs(zeta) + sqrt(real(1) + zeta * zeta));
          const real cs = real(1) / sqrt(real(1) + t * t), sn = cs * t;
#pragma unroll
          for (int u = 0; u < E; ++u) {
            const int c = lane + 32 * u;
            if (c < k) {
              Wt[(int64_t)p * k + c] = cs * a[u] - sn * b[u];
              Wt[(int64_t)q * k + c] = sn * a[u] + cs * b[u];
              const real vp = Vt[(int64_t)p * k + c], vq = Vt[(int64_t)q * k + c];
              Vt[(int64_t)p * k + c] = cs * vp - sn * vq;
              Vt[(int64_t)q * k + c] = sn * vp + cs * vq;
            }
          }
          if (lane == 0) atomicAdd(&rotations[sweep], 1);
        }
      }
      grid.sync();
    }
    if (*(volatile int*)&rotations[sweep] == 0) break;
  }
}

// f[i] = 1 / sigma_i^2 for sigma_i = ||row i of W^T|| > rtol * max sigma,
// else 0 (one CTA).
template <typename real>
__global__ void tsvd_filter_kernel(int k, const real* __restrict__ Wt, real rtol,
                                   real* __restrict__ f) {
  __shared__ real s_max[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  real mx = real(0);
  for (int i = warp; i < k; i += nwarp) {
    real s = real(0);
    for (int c = lane; c < k; c += 32) s = fma(Wt[(int64_t)i * k + c], Wt[(int64_t)i * k + c], s);
    s = warp_sum(s);
    if (lane == 0) f[i] = s;  // sigma_i^2 for now
    mx = s > mx ? s : mx;
  }
  if (lane == 0) s_max[warp] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    real m = real(0);
    for (int w = 0; w < nwarp; ++w) m = s_max[w] > m ? s_max[w] : m;
    s_max[0] = m;
  }
  __syncthreads();
  const real cut = rtol * rtol * s_max[0];
  for (int i = threadIdx.x; i < k; i += blockDim.x) {
    const real s2 = f[i];
    f[i] = (s2 > cut && s2 > real(0)) ? real(1) / s2 : real(0);
  }
}

template <typename real>
__global__ void identity_kernel(real* __restrict__ X, int k) {
  const int64_t total = (int64_t)k * k;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x)
    X[e] = (e / k == e % k) ? real(1) : real(0);
}

template <typename real>
__global__ void scale_rows_kernel(real* __restrict__ B, int64_t ldb, int64_t rows, int64_t cols,
                                  const real* __restrict__ f) {
  const int64_t total = rows * cols;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / cols, c = e % cols;
    B[r * ldb + c] *= f[r];
  }
}

}  // namespace

template <typename real>
bool jacobi_svd_fits(int k) {
  return k >= 1 && k <= kSvdMaxK;
}

template <typename real>
curid_status jacobi_svd(const Ctx& ctx, int k, real* Wt, real* Vt, int* rotations) {
  if (!jacobi_svd_fits<real>(k)) return CURID_UNSUPPORTED;
  CURID_CUDA(cudaMemsetAsync(rotations, 0, kSvdMaxSweeps * sizeof(int), ctx.stream));
  const int pairs = (k + 1) / 2;
  const int G = std::max(1, std::min(ctx.num_sms, (pairs + kSvdWarps - 1) / kSvdWarps));
  real tol = std::sqrt((real)k) * std::numeric_limits<real>::epsilon();
  void* args[] = {&k, &Wt, &Vt, &rotations, &tol};
  CURID_CUDA(cudaLaunchCooperativeKernel((void*)jacobi_svd_kernel<real>, dim3(G),
                                         dim3(kSvdThreads), args, 0, ctx.stream));
  if (ctx.launches) ++*ctx.launches;
  return CURID_OK;
}

template <typename real>
curid_status identity_fill(const Ctx& ctx, real* X, int k) {
  if (k <= 0) return CURID_OK;
  const unsigned blocks = (unsigned)std::max<int64_t>(
      1, std::min<int64_t>(((int64_t)k * k + 255) / 256, 16LL * ctx.num_sms));
  identity_kernel<real><<<blocks, 256, 0, ctx.stream>>>(X, k);
  CURID_LAUNCHED(ctx);
  return CURID_OK;
}

template <typename real>
curid_status tsvd_filter(const Ctx& ctx, int k, const real* Wt, double rtol, real* f) {
  tsvd_filter_kernel<real><<<1, 1024, 0, ctx.stream>>>(k, Wt, (real)rtol, f);
  CURID_LAUNCHED(ctx);
  return CURID_OK;
}

template <typename real>
curid_status scale_rows(const Ctx& ctx, real* B, int64_t ldb, int64_t rows, int64_t cols,
                        const real* f) {
  if (rows <= 0 || cols <= 0) return CURID_OK;
  const unsigned blocks = (unsigned)std::max<int64_t>(
      1, std::min<int64_t>((rows * cols + 255) / 256, 16LL * ctx.num_sms));
  scale_rows_kernel<real><<<blocks, 256, 0, ctx.stream>>>(B, ldb, rows, cols, f);
  CURID_LAUNCHED(ctx);
  return CURID_OK;
}

#define CURID_SVD_INST(real)                                                                 \
  template bool jacobi_svd_fits<real>(int);                                                  \
  template curid_status jacobi_svd<real>(const Ctx&, int, real*, real*, int*);               \
  template curid_status tsvd_filter<real>(const Ctx&, int, const real*, double, real*);      \
  template curid_status identity_fill<real>(const Ctx&, real*, int);                         \
  template curid_status scale_rows<real>(const Ctx&, real*, int64_t, int64_t, int64_t,       \
                                         const real*);
CURID_SVD_INST(float)
CURID_SVD_INST(double)
#undef CURID_SVD_INST

}  // namespace curid
