// Small dense factorizations of order <= 256:
//   * Cholesky factor of a (shifted) Gram matrix, the building block of the
//     row orthonormalisation between power steps (Section 5.3) and of the
//     pseudo-inverse R^+ in U = V* R^+ (Eq. (3.5)); one CTA, the matrix in
//     shared memory;
//   * explicit inverses of triangles through the blocked triangular solve
//     (tri.cu) with an identity right-hand side;
//   * the float64-accumulated product that ends the U chain.
#include <type_traits>
#include <utility>

#include "kernels.cuh"

namespace curid {

namespace {

constexpr int kSmallThreads = 512;  // 128 registers per thread for the block loops
constexpr int kSmallWarps = kSmallThreads / 32;
constexpr unsigned kFull = 0xffffffffu;

// Row stride of a 32 x 32 block: padded so every row starts on 16 bytes
// (vector loads) and the 32 rows a warp reads column-wise fall in distinct
// 16-byte bank groups.
template <typename real>
struct CholBlk {
  static constexpr int LD = 32 + 16 / (int)sizeof(real);
  using V = typename std::conditional<sizeof(real) == 4, float4, double2>::type;
  static constexpr int VN = 16 / (int)sizeof(real);  // elements per vector
};

__host__ __device__ inline int lower_block(int bi, int bj) { return bi * (bi + 1) / 2 + bj; }

template <typename real>
__device__ __forceinline__ real* chol_block(real* a, int bi, int bj) {
  return a + (size_t)lower_block(bi, bj) * 32 * CholBlk<real>::LD;
}

// Trailing update of block (b + 1 + bi, b + 1 + bj) by one warp:
// C -= P_i P_j^T with P_i, P_j the finished panel blocks of block column b.
// Lane t keeps row t of P_j in registers; the rows of P_i are read as
// broadcast vectors, four output rows at a time.
template <typename real>
__device__ __forceinline__ void chol_trail_block(real* a, int b, int bi, int bj, int lane) {
  using B = CholBlk<real>;
  using V = typename B::V;
  constexpr int LD = B::LD;
  const real* Pi = chol_block(a, b + 1 + bi, b);
  const real* Pj = chol_block(a, b + 1 + bj, b);
  real* C = chol_block(a, b + 1 + bi, b + 1 + bj);
  real col[32];
#pragma unroll
  for (int s = 0; s < 32; s += B::VN) {
    const V v = *reinterpret_cast<const V*>(Pj + lane * LD + s);
    if constexpr (B::VN == 4) {
      col[s] = v.x; col[s + 1] = v.y; col[s + 2] = v.z; col[s + 3] = v.w;
    } else {
      col[s] = v.x; col[s + 1] = v.y;
    }
  }
  for (int r = 0; r < 32; r += 4) {
    real sum[4] = {real(0), real(0), real(0), real(0)};
#pragma unroll
    for (int s = 0; s < 32; s += B::VN) {
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const V v = *reinterpret_cast<const V*>(Pi + (r + u) * LD + s);
        if constexpr (B::VN == 4) {
          sum[u] = fma(v.x, col[s], sum[u]);
          sum[u] = fma(v.y, col[s + 1], sum[u]);
          sum[u] = fma(v.z, col[s + 2], sum[u]);
          sum[u] = fma(v.w, col[s + 3], sum[u]);
        } else {
          sum[u] = fma(v.x, col[s], sum[u]);
          sum[u] = fma(v.y, col[s + 1], sum[u]);
        }
      }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) C[(r + u) * LD + lane] -= sum[u];
  }
}

// Trailing block number q = bi (bi + 1) / 2 + bj.
template <typename real>
__device__ __forceinline__ void chol_trail_q(real* a, int b, int q, int lane) {
  int bi = 0;
  while ((bi + 1) * (bi + 2) / 2 <= q) ++bi;
  chol_trail_block(a, b, bi, q - bi * (bi + 1) / 2, lane);
}

// Diagonal block and W = L_bb^{-1} by one warp with the block in registers:
// lane t holds column t of the Schur complement (c) and column t of the
// running inverse (x).  At step j the pivot column comes from lane j by
// shuffles, and lane t's own entry (j, t) is, by symmetry, L(t, j) times the
// pivot.  Every 4 steps both arrays shift down by 4 rows, so all register
// indices are compile-time constants while the step loop stays rolled; the
// routine is not inlined, so one compact copy serves both call sites (long
// straight-line code run by one warp is bound by instruction fetch).  Writes L (lower
// part) into D and W; returns nonzero on a non-positive or non-finite pivot.
__device__ __noinline__ int chol_diag_warp(float* D, float* W, int t) {
  constexpr int LD = CholBlk<float>::LD;
  float c[32], x[32];
#pragma unroll
  for (int i = 0; i < 32; ++i) {
    c[i] = D[i * LD + t];
    x[i] = i == t ? 1.f : 0.f;
  }
  int fail = 0;
#pragma unroll 1
  for (int j0 = 0; j0 < 32; j0 += 4) {
    // c[k], x[k] hold row j0 + k
#pragma unroll
    for (int jj = 0; jj < 4; ++jj) {
      const int j = j0 + jj;
      const float d = __shfl_sync(kFull, c[jj], j);
      if (!(d > 0.f) || !isfinite(d)) fail = 1;
      const float inv = fail ? 1.f : rsqrtf(d);
      const float ltj = c[jj] * inv;  // lane t > j: L(t, j)
      if (t > j) D[t * LD + j] = ltj;
      if (t == j) D[j * LD + j] = d * inv;
      x[jj] *= inv;  // W(j, t)
      W[j * 33 + t] = x[jj];
      const float q = inv * ltj, p = inv * x[jj];
#pragma unroll
      for (int i = jj + 1; i < 32; ++i) {
        const float cij = __shfl_sync(kFull, c[i], j);  // unscaled (j0 + i, j)
        if (t > j) c[i] = fmaf(-cij, q, c[i]);
        x[i] = fmaf(-cij, p, x[i]);
      }
    }
#pragma unroll
    for (int i = 0; i < 28; ++i) {
      c[i] = c[i + 4];
      x[i] = x[i + 4];
    }
#pragma unroll
    for (int i = 28; i < 32; ++i) c[i] = x[i] = 0.f;
  }
  return fail;
}

// Diagonal block and W = L_bb^{-1} in one sweep over the 32 x 64 augmented
// block [A_bb | I] by the whole CTA (512 threads): thread (r, c) =
// (tid / 16, tid % 16) holds A(r, c), A(r, c + 16), W(r, c), W(r, c + 16) in
// registers.  Step j: the owners publish column j of A, row j of W and the
// pivot's 1 / sqrt; one barrier; every thread then applies the rank-1
// updates of its elements.  Buffers alternate with j's parity, so one barrier
// per step orders each publication after the previous reads.  Used for
// float64, whose per-sub-partition rate makes one warp far too slow.
// Returns nonzero on a non-positive or non-finite pivot (same in all threads).
template <typename real>
__device__ __forceinline__ int chol_diag_cta(real* D, real* W, real* pcol, real* prow, real* piv,
                                             int tid) {
  constexpr int LD = CholBlk<real>::LD;
  const int r = tid >> 4, c = tid & 15;
  real a0 = D[r * LD + c], a1 = D[r * LD + c + 16];
  real w0 = r == c ? real(1) : real(0), w1 = r == c + 16 ? real(1) : real(0);
  int fail = 0;
  for (int j = 0; j < 32; ++j) {
    real* colA = pcol + (j & 1) * 32;
    real* rowW = prow + (j & 1) * 32;
    const real aj = j < 16 ? a0 : a1;
    if (c == (j & 15)) colA[r] = aj;
    if (r == j) {
      rowW[c] = w0;
      rowW[c + 16] = w1;
      if (c == (j & 15)) {
        const bool bad = !(aj > real(0)) || !isfinite(aj);
        const real inv = bad ? real(1) : rsqrt(aj);
        piv[(j & 1) * 2] = inv;
        piv[(j & 1) * 2 + 1] = bad ? real(-1) : aj * inv;
      }
    }
    __syncthreads();
    const real inv = piv[(j & 1) * 2], sj = piv[(j & 1) * 2 + 1];
    if (sj < real(0)) fail = 1;
    if (r > j) {
      // A(r, c) -= L(r, j) L(c, j) and W(r, c) -= L(r, j) W(j, c) / s_j
      // both take colA[r] / s_j^2 times an unscaled published value
      const real m = colA[r] * (inv * inv);
      if (c > j && c <= r) a0 = fma(-m, colA[c], a0);
      if (c + 16 > j && c + 16 <= r) a1 = fma(-m, colA[c + 16], a1);
      if (c == j) a0 = colA[r] * inv;
      if (c + 16 == j) a1 = colA[r] * inv;
      if (c <= j) w0 = fma(-m, rowW[c], w0);
      if (c + 16 <= j) w1 = fma(-m, rowW[c + 16], w1);
    } else if (r == j) {
      if (c == j) a0 = fabs(sj);
      if (c + 16 == j) a1 = fabs(sj);
      w0 *= inv;
      w1 *= inv;
    }
  }
  D[r * LD + c] = a0;
  D[r * LD + c + 16] = a1;
  W[r * 33 + c] = w0;
  W[r * 33 + c + 16] = w1;
  return fail;
}

// Cholesky factor of G + shift I, blocked right-looking on 32 x 32 blocks of
// the lower triangle (packed in shared memory, diagonal blocks held whole),
// the order padded to a multiple of 32 with an identity tail.  Per block
// column b:
//  (1) the diagonal block is factored and W = L_bb^{-1} formed in one
//      elimination sweep: by warp 0 with the block in registers (float32),
//      or by the whole CTA with one barrier per column (float64);
//  (2) every warp finishes panel rows A_ib <- A_ib L_bb^{-T} (W column in
//      registers, row entries as broadcast vector loads);
//  (3) the trailing update A_ij -= A_ib A_jb^T runs one 32 x 32 block per
//      warp, the A_jb row of each lane in registers and the A_ib rows read
//      as broadcast vectors.
// The lower factor overwrites G (upper part zeroed).  A non-positive or
// non-finite pivot retries with a 100x larger shift (4 attempts), then sets
// FLAG_BREAKDOWN.
template <typename real>
__global__ void __launch_bounds__(kSmallThreads, 1)
chol_kernel(real* __restrict__ G, int l, int64_t ldg, real rel_shift, StatusBlock* status) {
  using B = CholBlk<real>;
  using V = typename B::V;
  constexpr int LD = B::LD;
  constexpr bool kLookahead = sizeof(real) == 4;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int LP = (l + 31) & ~31;
  const int nb = LP / 32;
  real* a = reinterpret_cast<real*>(smem_raw);
  real* W = a + (size_t)lower_block(nb, 0) * 32 * LD;  // 32 x 33, W = L_bb^{-1}
  __shared__ real pcol[64], prow[64], piv[4];  // published pivot column / W row / 1/sqrt
  __shared__ int s_fail;
  __shared__ real s_tr;
  int s_fail_local = 0;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (warp == 0) {
    real tr = real(0);
    for (int i = lane; i < l; i += 32) tr += G[(int64_t)i * ldg + i];
    tr = warp_sum(tr);
    if (lane == 0) s_tr = tr;
  }
  __syncthreads();
  const real tr = s_tr;
  real shift = rel_shift * tr;
  bool done = false;
  for (int attempt = 0; attempt < 4 && !done; ++attempt) {
    // lower blocks of G + shift I (diagonal blocks whole), identity tail;
    // a warp loads four rows before it stores any, so each thread keeps up
    // to 32 loads in flight
    for (int i0 = warp; i0 < LP; i0 += 4 * kSmallWarps) {
      real v[4][8];
#pragma unroll
      for (int h = 0; h < 4; ++h) {
        const int i = i0 + h * kSmallWarps, bi = i >> 5;
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int j = 32 * u + lane;
          v[h][u] = (u <= bi && i < l && j < l) ? G[(int64_t)i * ldg + j] : real(0);
        }
      }
#pragma unroll
      for (int h = 0; h < 4; ++h) {
        const int i = i0 + h * kSmallWarps, bi = i >> 5, r = i & 31;
        if (i >= LP) continue;
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int j = 32 * u + lane;
          if (u <= bi) {
            real x = v[h][u];
            if (i == j) x += (i < l) ? shift : real(1);
            chol_block(a, bi, u)[r * LD + lane] = x;
          }
        }
      }
    }
    if (tid == 0) s_fail = 0;
    __syncthreads();
    // float32 looks ahead: warp 0 factors diagonal block b + 1 while the
    // other warps finish the trailing update of step b (step b = -1 only
    // factors block 0)
    for (int b = kLookahead ? -1 : 0; b < nb; ++b) {
      if (b >= 0) {
        if constexpr (!kLookahead) {
          s_fail_local = chol_diag_cta(chol_block(a, b, b), W, pcol, prow, piv, tid);
          if (tid == 0) s_fail = s_fail_local;
          __syncthreads();
        }
        if (s_fail) break;
        // (2) panel rows: A_ib(r, c) <- sum_{s <= c} A_ib(r, s) W(c, s)
        if (b + 1 < nb) {
          real w[32];
#pragma unroll
          for (int s = 0; s < 32; ++s) w[s] = W[lane * 33 + s];
          for (int i = (b + 1) * 32 + warp; i < LP; i += kSmallWarps) {
            real* row = chol_block(a, i >> 5, b) + (i & 31) * LD;
            real out = real(0);
#pragma unroll
            for (int s = 0; s < 32; s += B::VN) {
              const V v = *reinterpret_cast<const V*>(row + s);
              if constexpr (B::VN == 4) {
                out = fma(v.x, w[s], out);
                out = fma(v.y, w[s + 1], out);
                out = fma(v.z, w[s + 2], out);
                out = fma(v.w, w[s + 3], out);
              } else {
                out = fma(v.x, w[s], out);
                out = fma(v.y, w[s + 1], out);
              }
            }
            __syncwarp();
            row[lane] = out;
          }
        }
        __syncthreads();
      }
      // (3) trailing update of blocks (bi, bj), b < bj <= bi, numbered
      // q = bi (bi + 1) / 2 + bj from the next diagonal block q = 0
      const int m = nb - b - 1;
      const int nblocks = b >= 0 ? m * (m + 1) / 2 : 0;
      if constexpr (kLookahead) {
        // Warp 0 (diagonal factorization, the critical path) shares its
        // scheduler with warps 4, 8, 12 (warp % 4); those stay idle here so
        // it issues at full rate, and the 12 warps on the other three
        // schedulers take the trailing blocks.
        if (warp == 0) {
          if (m > 0) {
            if (b >= 0) chol_trail_block(a, b, 0, 0, lane);
            __syncwarp();
            const int fail = chol_diag_warp(chol_block(a, b + 1, b + 1), W, lane);
            if (lane == 0) s_fail = fail;
          }
        } else if (warp & 3) {
          constexpr int kWorkers = kSmallWarps - kSmallWarps / 4;
          const int idx = warp - (warp >> 2) - 1;  // 0 .. kWorkers - 1
          for (int q = 1 + idx; q < nblocks; q += kWorkers) chol_trail_q(a, b, q, lane);
        }
      } else {
        for (int q = warp; q < nblocks; q += kSmallWarps) chol_trail_q(a, b, q, lane);
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
    for (int e = tid; e < l * l; e += kSmallThreads)
      G[(int64_t)(e / l) * ldg + e % l] = (e / l == e % l) ? real(1) : real(0);
    return;
  }
  for (int i = warp; i < l; i += kSmallWarps) {
    const int bi = i >> 5, r = i & 31;
    for (int j = lane; j < l; j += 32)
      G[(int64_t)i * ldg + j] = j <= i ? chol_block(a, bi, j >> 5)[r * LD + (j & 31)] : real(0);
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
  const int nb = (l + 31) / 32;
  return ((size_t)lower_block(nb, 0) * 32 * CholBlk<real>::LD + 32 * 33) * sizeof(real);
}

}  // namespace

template <typename real>
bool upper_tri_inverse_fits(const Ctx& ctx, int k) {
  return tri_solve_fits<real>(ctx, k);
}
template <typename real>
bool chol_one_cta(const Ctx& ctx, int l) {
  return l <= 256 && chol_smem<real>(l) <= ctx.smem_optin;
}

template <typename real>
bool chol_inverse_fits(const Ctx& ctx, int l) {
  return l > 0 && l <= kMaxDenseOrder && chol_one_cta<real>(ctx, kCholBlock<real>()) &&
         tri_solve_fits<real>(ctx, l);
}

template <typename real>
curid_status upper_tri_inverse(const Ctx& ctx, const real* S11, int k, const int* k_eff,
                               real* X) {
  return tri_solve<real>(ctx, k, S11, k, true, false, nullptr, 0, X, k, k, k_eff);
}

template <typename real>
curid_status chol_launch(const Ctx& ctx, real* G, int l, int64_t ldg, double rel_shift) {
  const size_t smem = chol_smem<real>(l);
  auto fn = chol_kernel<real>;
  CURID_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  fn<<<1, kSmallThreads, smem, ctx.stream>>>(G, l, ldg, (real)rel_shift, ctx.status);
  CURID_LAUNCHED(ctx);
  return CURID_OK;
}

// G (l x l, leading dimension l) += shift * trace(G) * I, one CTA.
template <typename real>
__global__ void add_trace_shift_kernel(real* G, int l, real rel_shift) {
  __shared__ real s_red[32];
  real tr = real(0);
  for (int i = threadIdx.x; i < l; i += blockDim.x) tr += G[(int64_t)i * l + i];
  tr = warp_sum(tr);
  if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = tr;
  __syncthreads();
  if (threadIdx.x < 32) {
    tr = threadIdx.x < (int)(blockDim.x >> 5) ? s_red[threadIdx.x] : real(0);
    tr = warp_sum(tr);
    if (threadIdx.x == 0) s_red[0] = tr;
  }
  __syncthreads();
  const real sh = rel_shift * s_red[0];
  for (int i = threadIdx.x; i < l; i += blockDim.x) G[(int64_t)i * l + i] += sh;
}

// zero the strict upper triangle of G (l x l, leading dimension l)
template <typename real>
__global__ void zero_upper_kernel(real* G, int l) {
  const int64_t total = (int64_t)l * l;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x)
    if (e % l > e / l) G[e] = real(0);
}

// Cholesky of order l beyond one CTA: right-looking over diagonal blocks of
// kCholBlock, each factored by chol_kernel; the panel L21^T = L11^{-1} G12
// is solved in place in G's upper part (G is symmetric, so G12 = G21^T),
// the trailing block is updated with G22 -= (L21^T)^T L21^T, and L21 is
// written below the diagonal by a transpose.  The shift uses the trace of
// the whole matrix, as in the one-CTA kernel.
template <typename real>
curid_status chol_blocked(const Ctx& ctx, real* G, int l, double rel_shift) {
  if (rel_shift > 0) {
    add_trace_shift_kernel<real><<<1, 512, 0, ctx.stream>>>(G, l, (real)rel_shift);
    CURID_LAUNCHED(ctx);
  }
  const int bs = kCholBlock<real>();
  for (int kb = 0; kb < l; kb += bs) {
    const int b = std::min(bs, l - kb), rest = l - kb - b;
    real* D = G + (int64_t)kb * l + kb;
    CURID_TRY(chol_launch<real>(ctx, D, b, l, 0.0));
    if (rest == 0) break;
    real* G12 = D + b;
    real* G21 = D + (int64_t)b * l;
    real* G22 = G21 + b;
    CURID_TRY(tri_solve<real>(ctx, b, D, l, false, false, G12, l, G12, l, rest, nullptr));
    CURID_TRY(gemm<real>(ctx, true, false, rest, rest, b, real(-1), G12, l, G12, l, real(1), G22,
                         l, nullptr, 0));
    CURID_TRY(transpose2d<real>(ctx, G12, l, G21, l, b, rest));
  }
  const int64_t total = (int64_t)l * l;
  const unsigned g = (unsigned)std::max<int64_t>(1, std::min<int64_t>((total + 255) / 256,
                                                                      8LL * ctx.num_sms));
  zero_upper_kernel<real><<<g, 256, 0, ctx.stream>>>(G, l);
  CURID_LAUNCHED(ctx);
  return CURID_OK;
}

template <typename real>
curid_status cholesky(const Ctx& ctx, real* G, int l, double rel_shift) {
  if (l <= 0) return CURID_OK;
  if (chol_one_cta<real>(ctx, l)) return chol_launch<real>(ctx, G, l, l, rel_shift);
  if (!chol_inverse_fits<real>(ctx, l)) return CURID_UNSUPPORTED;
  return chol_blocked<real>(ctx, G, l, rel_shift);
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

template <typename real>
curid_status chol_qr_rows(const Ctx& ctx, real** X, real** tmp, int64_t r, int64_t c, int64_t ld,
                          real* G, real* partial, size_t partial_cap, int passes, bool tc_gram,
                          real* li) {
  const double shift = sizeof(real) == 4 ? 1e-5 : 1e-13;
  for (int pass = 0; pass < passes; ++pass) {
    bool tc = false;
    if constexpr (sizeof(real) == 4) {
      if (tc_gram) {
        CURID_TRY(gram_tf32(ctx, *X, r, c, ld, G, partial, partial_cap));
        tc = true;
      }
    }
    if (!tc)
      CURID_TRY(gemm<real>(ctx, false, true, r, r, c, real(1), *X, ld, *X, ld, real(0), G, r,
                           partial, partial_cap));
    CURID_TRY(cholesky<real>(ctx, G, (int)r, pass == 0 ? shift : 0.0));
    bool applied = false;
    if constexpr (sizeof(real) == 4) {
      if (tc && li) {
        // X <- L^{-1} X as tensor-core products: L^{-1} explicitly (a
        // triangular solve with the identity); the product splits both
        // operands into TF32 parts and remainders in shared memory, so it
        // carries float32 accuracy.  The products take at most 256 rows of
        // L^{-1} at a time (the MMA's N); rows r0..r0+mr-1 of a lower
        // triangular L^{-1} need only the first r0 + mr rows of X.
        const int64_t ldp = (r + 3) & ~int64_t(3);  // 16-byte rows for the tensor-core loads
        CURID_TRY(tri_solve<float>(ctx, (int)r, G, r, false, false, nullptr, 0, li, ldp, r,
                                   nullptr));
        const int64_t chunks = (r + 255) / 256;
        const int64_t rows = ((r + chunks - 1) / chunks + 15) / 16 * 16;
        for (int64_t r0 = 0; r0 < r; r0 += rows) {
          const int64_t mr = std::min(rows, r - r0), kk = r0 + mr;
          CURID_TRY(gemm_tf32(ctx, false, false, mr, c, kk, li + r0 * ldp, ldp, *X, ld,
                              *tmp + r0 * ld, ld, partial, partial_cap, true));
        }
        applied = true;
      }
    }
    if (!applied)
      CURID_TRY(tri_solve<real>(ctx, (int)r, G, r, false, false, *X, ld, *tmp, ld, c, nullptr));
    std::swap(*X, *tmp);
  }
  return CURID_OK;
}

curid_status gram_tf32(const Ctx& ctx, const float* X, int64_t r, int64_t c, int64_t ld, float* G,
                       float* partial, size_t partial_cap) {
  return gemm_tf32(ctx, false, true, r, r, c, X, ld, X, ld, G, r, partial, partial_cap, true);
}

template curid_status chol_qr_rows<float>(const Ctx&, float**, float**, int64_t, int64_t, int64_t,
                                          float*, float*, size_t, int, bool, float*);
template curid_status chol_qr_rows<double>(const Ctx&, double**, double**, int64_t, int64_t,
                                           int64_t, double*, double*, size_t, int, bool,
                                           double*);
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
