// Blocked triangular solve op(T) X = B for many right-hand sides.
//
// Used for every triangular step of the path: the T solve S11 T = S12
// (Eq. (2.8)), the applies X <- L^{-1} X of the Cholesky-QR row
// orthonormalisation (Section 5.3), the preconditioning S_W11^{-T} R and
// the explicit inverses of the U = V* R^+ chain (Eq. (3.5)).
//
// One CTA solves for NC columns of X with the whole triangle resident in
// shared memory, stored as 32 x 32 blocks of its lower triangle (upper or
// transposed inputs are loaded through an index map: an upper triangle with
// rows and columns reversed is lower).  The CTA first inverts its diagonal
// blocks (one warp per block, one lane per column), then sweeps the block
// rows: X_b = D_b^{-1} (B_b - sum_{t<b} L_bt X_t), each thread holding two
// rows of NC / 32 columns.  Rows and columns at or after the numerical rank kk
// are treated as an identity block with a zero right-hand side, so the
// solution is zero there (the singular S11 case of Section 2.3).
#include "kernels.cuh"

namespace curid {

namespace {

constexpr int kTB = 32;           // block order
constexpr int kTriThreads = 512;

// NC right-hand-side columns per CTA; block rows padded to LD so that every
// row starts on 16 bytes (vector loads of VN entries); in the sweep a thread
// owns one column and RPT rows of a block row.
template <typename real>
struct TriCols;
template <>
struct TriCols<float> {
  static constexpr int NC = 64, LD = 36, VN = 4;
  using V = float4;
};
template <>
struct TriCols<double> {
  static constexpr int NC = 32, LD = 34, VN = 2;
  using V = double2;
};

__host__ __device__ inline int packed_block(int bi, int bj) { return bi * (bi + 1) / 2 + bj; }

template <typename real>
struct TriParams {
  int k, nb;
  const real* T;
  int64_t ldt;
  bool trans, reverse;  // op: element (i, j) of the lower triangle used
  const real* B;        // nullptr: identity right-hand side
  int64_t ldb;
  real* X;
  int64_t ldx;
  int64_t N;
  const int* kk;        // numerical rank (device) or nullptr
  int kk_off;           // this triangle starts at row/column kk_off of the full one
};

// lower-triangle element (i, j), i >= j, in the solve's index space, read
// from the caller's triangle
template <typename real>
__device__ __forceinline__ real tri_elem(const TriParams<real>& P, int i, int j, int kk) {
  const int oi = P.reverse ? P.k - 1 - i : i;
  const int oj = P.reverse ? P.k - 1 - j : j;
  if (oi >= kk || oj >= kk || i >= P.k) return i == j ? real(1) : real(0);
  return P.trans ? P.T[(int64_t)oj * P.ldt + oi] : P.T[(int64_t)oi * P.ldt + oj];
}

template <typename real>
__global__ void __launch_bounds__(kTriThreads, 1) tri_solve_kernel(TriParams<real> P) {
  using TC = TriCols<real>;
  using V = typename TC::V;
  constexpr int NC = TC::NC, LD = TC::LD, VN = TC::VN;
  constexpr int CPT = NC / 32;                 // columns per lane when loading
  constexpr int RPT = kTB * NC / kTriThreads;  // rows per thread in the sweep
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int nb = P.nb;
  const int KP = nb * kTB;
  real* Ls = reinterpret_cast<real*>(smem_raw);                 // packed blocks, 32 x 33
  real* Xs = Ls + (size_t)packed_block(nb, 0) * kTB * LD;  // KP x NC
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int kk = P.kk ? max(0, min(P.k, *P.kk - P.kk_off)) : P.k;
  const int64_t c0 = (int64_t)blockIdx.x * NC;

  // triangle -> packed lower blocks (identity past k and past the rank): a
  // warp per block, lane = column, rows in batches of 8 loads in flight
  const int nblk = packed_block(nb, 0);
  for (int blk = warp; blk < nblk; blk += kTriThreads / 32) {
    int bi = 0;
    while (packed_block(bi + 1, 0) <= blk) ++bi;
    const int bj = blk - packed_block(bi, 0);
    real* dst = Ls + (size_t)blk * kTB * LD;
    const int j = bj * kTB + lane;
    for (int r0 = 0; r0 < kTB; r0 += 8) {
      real v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int i = bi * kTB + r0 + u;
        v[u] = j <= i ? tri_elem(P, i, j, kk) : real(0);
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) dst[(r0 + u) * LD + lane] = v[u];
    }
  }
  // right-hand side columns c0..c0+NC (identity when B is null), rows in
  // batches of 4 per warp
  for (int i0 = warp * 4; i0 < KP; i0 += 4 * (kTriThreads / 32)) {
    real v[4][CPT];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int i = i0 + u;
      const int oi = P.reverse ? P.k - 1 - i : i;
#pragma unroll
      for (int q = 0; q < CPT; ++q) {
        const int64_t col = c0 + lane + 32 * q;
        real x = real(0);
        if (i < P.k && oi < kk && col < P.N)
          x = P.B ? P.B[(int64_t)oi * P.ldb + col] : (oi == col ? real(1) : real(0));
        v[u][q] = x;
      }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int q = 0; q < CPT; ++q)
        if (i0 + u < KP) Xs[(i0 + u) * NC + lane + 32 * q] = v[u][q];
  }
  __syncthreads();
  // invert each diagonal block: warp b, lane j solves D x = e_j
  if (warp < nb) {
    real* D = Ls + (size_t)packed_block(warp, warp) * kTB * LD;
    real x[kTB];
#pragma unroll
    for (int i = 0; i < kTB; ++i) {
      real s = i == lane ? real(1) : real(0);
#pragma unroll
      for (int t = 0; t < i; ++t) s -= D[i * LD + t] * x[t];
      x[i] = i >= lane ? s / D[i * LD + i] : real(0);
    }
    __syncwarp();
#pragma unroll
    for (int i = 0; i < kTB; ++i) D[i * LD + lane] = x[i];
  }
  __syncthreads();
  // block-row sweep: thread (g, col) owns rows g*RPT .. g*RPT+RPT-1 of each
  // block row and column col; the triangle's rows are read as broadcast
  // vectors of VN entries, the X column once per entry
  const int col = tid % NC, r0 = (tid / NC) * RPT;
  for (int b = 0; b < nb; ++b) {
    real acc[RPT];
#pragma unroll
    for (int u = 0; u < RPT; ++u) acc[u] = Xs[(b * kTB + r0 + u) * NC + col];
    for (int t = 0; t < b; ++t) {
      const real* Lbt = Ls + (size_t)packed_block(b, t) * kTB * LD;
      const real* Xt = Xs + (t * kTB) * NC;
#pragma unroll 2
      for (int s = 0; s < kTB; s += VN) {
        real xv[VN];
#pragma unroll
        for (int v = 0; v < VN; ++v) xv[v] = Xt[(s + v) * NC + col];
#pragma unroll
        for (int u = 0; u < RPT; ++u) {
          const V l = *reinterpret_cast<const V*>(Lbt + (r0 + u) * LD + s);
          if constexpr (VN == 4) {
            acc[u] -= l.x * xv[0];
            acc[u] -= l.y * xv[1];
            acc[u] -= l.z * xv[2];
            acc[u] -= l.w * xv[3];
          } else {
            acc[u] -= l.x * xv[0];
            acc[u] -= l.y * xv[1];
          }
        }
      }
    }
    // X_b = D_b^{-1} acc: stage acc, then multiply (D_b^{-1} is stored
    // lower triangular with zeros above the diagonal)
#pragma unroll
    for (int u = 0; u < RPT; ++u) Xs[(b * kTB + r0 + u) * NC + col] = acc[u];
    __syncthreads();
    const real* D = Ls + (size_t)packed_block(b, b) * kTB * LD;
    real out[RPT];
#pragma unroll
    for (int u = 0; u < RPT; ++u) out[u] = real(0);
    const int smax = r0 + RPT;  // entries past the thread's last row are zero
    for (int s = 0; s < smax; s += VN) {
      real xv[VN];
#pragma unroll
      for (int v = 0; v < VN; ++v) xv[v] = Xs[(b * kTB + s + v) * NC + col];
#pragma unroll
      for (int u = 0; u < RPT; ++u) {
        const V d = *reinterpret_cast<const V*>(D + (r0 + u) * LD + s);
        if constexpr (VN == 4) {
          out[u] += d.x * xv[0];
          out[u] += d.y * xv[1];
          out[u] += d.z * xv[2];
          out[u] += d.w * xv[3];
        } else {
          out[u] += d.x * xv[0];
          out[u] += d.y * xv[1];
        }
      }
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < RPT; ++u) Xs[(b * kTB + r0 + u) * NC + col] = out[u];
    __syncthreads();
  }
  // store (rows at and after the rank are zero already)
  for (int e = tid; e < P.k * NC; e += kTriThreads) {
    const int i = e / NC, c = e % NC;
    const int64_t col = c0 + c;
    if (col >= P.N) continue;
    const int oi = P.reverse ? P.k - 1 - i : i;
    P.X[(int64_t)oi * P.ldx + col] = Xs[i * NC + c];
  }
}

template <typename real>
size_t tri_smem(int k) {
  const int nb = (k + kTB - 1) / kTB;
  return ((size_t)packed_block(nb, 0) * kTB * TriCols<real>::LD +
          (size_t)nb * kTB * TriCols<real>::NC) *
         sizeof(real);
}

}  // namespace

template <typename real>
bool tri_one_cta(const Ctx& ctx, int k) {
  return k > 0 && (k + kTB - 1) / kTB <= kTriThreads / 32 && tri_smem<real>(k) <= ctx.smem_optin;
}

template <typename real>
bool tri_solve_fits(const Ctx& ctx, int k) {
  return k > 0 && k <= kMaxDenseOrder && tri_one_cta<real>(ctx, kCholBlock<real>());
}

template <typename real>
curid_status tri_launch(const Ctx& ctx, int k, const real* T, int64_t ldt, bool upper, bool trans,
                        const real* B, int64_t ldb, real* X, int64_t ldx, int64_t N,
                        const int* kk, int kk_off) {
  TriParams<real> P;
  P.k = k;
  P.nb = (k + kTB - 1) / kTB;
  P.T = T;
  P.ldt = ldt;
  // op(T) is lower when (lower and not transposed) or (upper and transposed);
  // otherwise reverse the order of rows and columns to make it lower.
  P.trans = trans;
  P.reverse = upper != trans;
  P.B = B;
  P.ldb = ldb;
  P.X = X;
  P.ldx = ldx;
  P.N = N;
  P.kk = kk;
  P.kk_off = kk_off;
  const size_t smem = tri_smem<real>(k);
  auto fn = tri_solve_kernel<real>;
  CURID_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const int64_t grid = (N + TriCols<real>::NC - 1) / TriCols<real>::NC;
  fn<<<(unsigned)grid, kTriThreads, smem, ctx.stream>>>(P);
  CURID_LAUNCHED(ctx);
  return CURID_OK;
}

// X (k x N, leading dimension ldx) = I
template <typename real>
__global__ void set_identity_kernel(real* X, int64_t ldx, int k, int64_t N) {
  const int64_t total = (int64_t)k * N;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / N, j = e % N;
    X[i * ldx + j] = i == j ? real(1) : real(0);
  }
}

// Orders beyond one CTA: block substitution over diagonal blocks of
// kCholBlock, each solved in place by tri_solve_kernel (every CTA of that
// kernel reads all of its columns before writing them, so X may be B), the
// blocks not yet solved updated by GEMM.  Lower: forward, top block first;
// upper: backward.  A device rank kk is passed to every block with its
// offset, so rows at and after kk stay zero.
template <typename real>
curid_status tri_blocked(const Ctx& ctx, int k, const real* T, int64_t ldt, bool upper,
                         const real* B, int64_t ldb, real* X, int64_t ldx, int64_t N,
                         const int* kk) {
  if (B == nullptr) {
    const int64_t total = (int64_t)k * N;
    const unsigned g = (unsigned)std::max<int64_t>(1, std::min<int64_t>((total + 255) / 256,
                                                                        16LL * ctx.num_sms));
    set_identity_kernel<real><<<g, 256, 0, ctx.stream>>>(X, ldx, k, N);
    CURID_LAUNCHED(ctx);
  } else if (B != X || ldb != ldx) {
    CURID_TRY(copy2d<real>(ctx, B, ldb, X, ldx, k, N));
  }
  const int bs = kCholBlock<real>();
  const int nb = (k + bs - 1) / bs;
  for (int t = 0; t < nb; ++t) {
    const int i = upper ? nb - 1 - t : t;
    const int off = i * bs, b = std::min(bs, k - off);
    real* Xi = X + (int64_t)off * ldx;
    CURID_TRY(tri_launch<real>(ctx, b, T + (int64_t)off * ldt + off, ldt, upper, false, Xi, ldx, Xi,
                               ldx, N, kk, off));
    if (!upper && off + b < k) {
      CURID_TRY(gemm<real>(ctx, false, false, k - off - b, N, b, real(-1),
                           T + (int64_t)(off + b) * ldt + off, ldt, Xi, ldx, real(1),
                           X + (int64_t)(off + b) * ldx, ldx, nullptr, 0));
    } else if (upper && off > 0) {
      CURID_TRY(gemm<real>(ctx, false, false, off, N, b, real(-1), T + off, ldt, Xi, ldx, real(1),
                           X, ldx, nullptr, 0));
    }
  }
  return CURID_OK;
}

template <typename real>
curid_status tri_solve(const Ctx& ctx, int k, const real* T, int64_t ldt, bool upper, bool trans,
                       const real* B, int64_t ldb, real* X, int64_t ldx, int64_t N,
                       const int* kk) {
  if (k <= 0 || N <= 0) return CURID_OK;
  if (tri_one_cta<real>(ctx, k))
    return tri_launch<real>(ctx, k, T, ldt, upper, trans, B, ldb, X, ldx, N, kk, 0);
  if (!tri_solve_fits<real>(ctx, k) || trans) return CURID_UNSUPPORTED;
  return tri_blocked<real>(ctx, k, T, ldt, upper, B, ldb, X, ldx, N, kk);
}

template bool tri_solve_fits<float>(const Ctx&, int);
template bool tri_solve_fits<double>(const Ctx&, int);
template curid_status tri_solve<float>(const Ctx&, int, const float*, int64_t, bool, bool,
                                       const float*, int64_t, float*, int64_t, int64_t,
                                       const int*);
template curid_status tri_solve<double>(const Ctx&, int, const double*, int64_t, bool, bool,
                                        const double*, int64_t, double*, int64_t, int64_t,
                                        const int*);

}  // namespace curid
