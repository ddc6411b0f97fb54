// Reverse-mode derivative of the CUR-ID with the skeletons frozen.
//
// With J and I fixed, C = A(:, J[:k]), B = A(:, J[k:]), R = A(I[:k], :);
// the deterministic column ID's T = S11^{-1} S12 equals C^+ B (A P = Q S
// gives C = Q1 S11 and Q1^T B = S12, Section 2.3 and Eq. (2.8)), and
// U = V* R^+ with V* = [I T] P^T (Eq. (3.5)).  Given cotangents (Cbar, Ubar,
// Rbar) of the outputs (C, U, R), Abar follows the chain rule through those
// two maps:
//   U = V* R^+ :  Vsbar = Ubar R^{+T};  M = V Ubar (V = V*^T);
//                 Rbar += -R^{+T} M R^{+T} + (R R^T)^{-1} M^T (I - R^+ R)
//   T = C^+ B  :  Tbar = Vsbar(:, J[k:]);  K = (C^T C)^{-1} Tbar;
//                 Cbar += (B - C T) K^T - C K T^T;  Bbar = C K
//   Abar = Cbar -> columns J[:k], Bbar -> columns J[k:], Rbar -> rows I[:k].
//
// Working precision throughout, without forming R R^T or C^T C from raw
// data: Cholesky QR of the rows of R and of C^T gives R = L_R Q_R and
// C^T = L_C Q_C^T (Q orthonormal rows), so R^+ = Q_R^T L_R^{-1},
// (R R^T)^{-1} = L_R^{-T} L_R^{-1}, (C^T C)^{-1} = L_C^{-T} L_C^{-1}, and
// with P = Q_R M = (V* Q_R^T)^T Ubar the R-term becomes
//   Rbar + ((R R^T)^{-1} Ubar^T) V* - (L_R^{-T} P L_R^{-T} + (R R^T)^{-1} P^T) Q_R,
// while B K^T = A Kf^T with Kf the k x n matrix holding K in columns J[k:]
// and zeros in columns J[:k], and Abar starts as C Kf (Bbar in columns J[k:],
// zero elsewhere) before Cbar and Rbar are scattered in.
#include <utility>

#include "kernels.cuh"

using namespace curid;

namespace {

inline unsigned grid_for(int64_t work, int num_sms) {
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>((work + 255) / 256, 16LL * num_sms));
}

// dst (k x n, leading dimension n): column J[t] holds e_t (identity head) or
// zero for t < k, column J[k + c] holds src(:, c).  J is a permutation of
// 0..n-1, so every entry of dst is written once.
template <typename real>
__global__ void assemble_cols_kernel(int k, int n, const int32_t* __restrict__ J, int identity_head,
                                     const real* __restrict__ src, int64_t lds,
                                     real* __restrict__ dst) {
  const int64_t total = (int64_t)k * n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / n), p = (int)(e % n);
    const int col = min(max(J[p], 0), n - 1);  // indices come from the device
    real v;
    if (p < k) v = (identity_head && p == i) ? real(1) : real(0);
    else v = src[(int64_t)i * lds + (p - k)];
    dst[(int64_t)i * n + col] = v;
  }
}

// Abar[r][J[t]] += src[r][t] (r < m, t < k)
template <typename real>
__global__ void scatter_add_cols_kernel(int64_t m, int k, int n, const int32_t* __restrict__ J,
                                        const real* __restrict__ src, real* __restrict__ dst,
                                        int64_t ldd) {
  const int64_t total = m * k;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / k;
    const int t = (int)(e % k);
    const int col = min(max(J[t], 0), n - 1);
    dst[r * ldd + col] += src[e];
  }
}

// Abar[I[t]][c] += src[t][c] (t < k, c < n)
template <typename real>
__global__ void scatter_add_rows_kernel(int k, int64_t n, int64_t m, const int32_t* __restrict__ I,
                                        const real* __restrict__ src, real* __restrict__ dst,
                                        int64_t ldd) {
  const int t = blockIdx.y;
  const int64_t row = min(max((int64_t)I[t], int64_t(0)), m - 1);
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < n;
       c += (int64_t)gridDim.x * blockDim.x)
    dst[row * ldd + c] += src[(int64_t)t * n + c];
}

// dst (rows x cols, packed) = src cast to real, or zero when src is null
template <typename real, typename src_t>
__global__ void cast_copy_kernel(int64_t rows, int64_t cols, const src_t* __restrict__ src,
                                 int64_t lds, real* __restrict__ dst) {
  const int64_t total = rows * cols;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / cols, c = e % cols;
    dst[e] = src ? (real)src[r * lds + c] : real(0);
  }
}

template <typename real, typename src_t>
curid_status cast_copy(const Ctx& ctx, int64_t rows, int64_t cols, const src_t* src, int64_t lds,
                       real* dst) {
  if (rows <= 0 || cols <= 0) return CURID_OK;
  cast_copy_kernel<real, src_t>
      <<<grid_for(rows * cols, ctx.num_sms), 256, 0, ctx.stream>>>(rows, cols, src, lds, dst);
  CURID_LAUNCHED(ctx);
  return CURID_OK;
}

template <typename real>
struct AdjPlan {
  StatusBlock* status = nullptr;
  real *R1 = nullptr, *R2 = nullptr;    // k x n: R, Cholesky-QR ping-pong
  real *C1 = nullptr, *C2 = nullptr;    // k x m: C^T, ping-pong
  real *G = nullptr;                    // k x k Gram scratch
  real *Lr = nullptr, *Lc = nullptr;    // k x k: L_R, L_C
  real *Lri = nullptr, *Lci = nullptr;  // k x k: inverses
  real *Ub = nullptr;                   // k x k: Ubar in working precision
  real *Vs = nullptr;                   // k x n: V*
  real *Nm = nullptr, *Pm = nullptr, *X1 = nullptr, *W1 = nullptr, *W2 = nullptr;  // k x k
  real *G1 = nullptr, *Wc = nullptr, *S = nullptr, *S11 = nullptr;             // k x k
  real *Vsb = nullptr;                  // k x n: Vsbar
  real *Tb = nullptr, *K = nullptr;     // k x (n - k)
  real *Kf = nullptr;                   // k x n
  real *Rt = nullptr;                   // k x n: total Rbar
  real *Ct = nullptr;                   // m x k: total Cbar
  real *partial = nullptr;
  size_t partial_cap = 0;
  size_t bytes = 0;
};

template <typename real>
void adj_plan(const Ctx& ctx, int64_t m, int64_t n, int k, void* base, AdjPlan<real>* P) {
  Carver cv(base);
  const int64_t nk = std::max<int64_t>(1, n - k);
  const size_t kk = (size_t)k * k;
  P->status = cv.take<StatusBlock>(1);
  P->R1 = cv.take<real>((size_t)k * n);
  P->R2 = cv.take<real>((size_t)k * n);
  P->C1 = cv.take<real>((size_t)k * m);
  P->C2 = cv.take<real>((size_t)k * m);
  P->G = cv.take<real>(kk);
  P->Lr = cv.take<real>(kk);
  P->Lc = cv.take<real>(kk);
  P->Lri = cv.take<real>(kk);
  P->Lci = cv.take<real>(kk);
  P->Ub = cv.take<real>(kk);
  P->Vs = cv.take<real>((size_t)k * n);
  P->Nm = cv.take<real>(kk);
  P->Pm = cv.take<real>(kk);
  P->X1 = cv.take<real>(kk);
  P->W1 = cv.take<real>(kk);
  P->W2 = cv.take<real>(kk);
  P->G1 = cv.take<real>(kk);
  P->Wc = cv.take<real>(kk);
  P->S = cv.take<real>(kk);
  P->S11 = cv.take<real>(kk);
  P->Vsb = cv.take<real>((size_t)k * n);
  P->Tb = cv.take<real>((size_t)k * nk);
  P->K = cv.take<real>((size_t)k * nk);
  P->Kf = cv.take<real>((size_t)k * n);
  P->Rt = cv.take<real>((size_t)k * n);
  P->Ct = cv.take<real>((size_t)m * k);
  size_t part = 0;
  const int s = ctx.num_sms;
  const int64_t shapes[][3] = {{k, k, n},     {k, k, m},     {k, n, k}, {k, nk, k}, {k, k, nk},
                               {m, k, n},     {m, k, k},     {m, n, k}, {k, k, k}};
  for (const auto& sh : shapes)
    part = std::max(part, gemm_partial_elems<real>(sh[0], sh[1], sh[2], s));
  P->partial_cap = part;
  P->partial = part ? cv.take<real>(part) : nullptr;
  P->bytes = cv.used;
}

template <typename real>
curid_status adjoint_run(const Ctx& ctx0, const real* A, int64_t m, int64_t n, int64_t lda, int k,
                         const int32_t* J, const int32_t* I, const real* T, int64_t ldt,
                         const real* Cbar, const double* Ubar, const real* Rbar, real* Abar,
                         int64_t ldab, void* ws, size_t ws_bytes) {
  Ctx ctx = ctx0;
  AdjPlan<real> P;
  adj_plan<real>(ctx, m, n, k, nullptr, &P);
  if (!ws || P.bytes > ws_bytes) return CURID_NO_WORKSPACE;
  adj_plan<real>(ctx, m, n, k, ws, &P);
  ctx.status = P.status;
  CURID_CUDA(cudaMemsetAsync(P.status, 0, sizeof(StatusBlock), ctx.stream));
  const int64_t nk = n - k;
  const real one(1), zero(0), mone(-1);
  auto mm = [&](bool ta, bool tb, int64_t M, int64_t N, int64_t Kd, real alpha, const real* X,
                int64_t ldx, const real* Y, int64_t ldy, real beta, real* Z, int64_t ldz) {
    return gemm<real>(ctx, ta, tb, M, N, Kd, alpha, X, ldx, Y, ldy, beta, Z, ldz, P.partial,
                      P.partial_cap);
  };

  // R = L_R Q_R (Cholesky QR of R's rows); L_R = R Q_R^T
  CURID_TRY(gather_rows<real>(ctx, A, m, n, lda, I, k, P.R1, n));
  real* Qr = P.R1;
  real* Rraw = P.R2;
  CURID_TRY(chol_qr_rows<real>(ctx, &Qr, &Rraw, k, n, n, P.G, P.partial, P.partial_cap));
  CURID_TRY(gather_rows<real>(ctx, A, m, n, lda, I, k, Rraw, n));
  CURID_TRY(mm(false, true, k, k, n, one, Rraw, n, Qr, n, zero, P.Lr, k));
  // C^T = L_C Q_C^T; L_C = C^T Q_C; C^T itself is kept (gathered again)
  CURID_TRY(gather_cols<real>(ctx, A, m, n, lda, J, k, P.C1, m, true));
  real* Qc = P.C1;
  real* Craw = P.C2;
  CURID_TRY(chol_qr_rows<real>(ctx, &Qc, &Craw, k, m, m, P.G, P.partial, P.partial_cap));
  CURID_TRY(gather_cols<real>(ctx, A, m, n, lda, J, k, Craw, m, true));
  CURID_TRY(mm(false, true, k, k, m, one, Craw, m, Qc, m, zero, P.Lc, k));
  CURID_TRY(tri_solve<real>(ctx, k, P.Lr, k, false, false, nullptr, 0, P.Lri, k, k, nullptr));
  CURID_TRY(tri_solve<real>(ctx, k, P.Lc, k, false, false, nullptr, 0, P.Lci, k, k, nullptr));

  // ---- through U = V* R^+ ----
  CURID_TRY((cast_copy<real, double>(ctx, k, k, Ubar, k, P.Ub)));
  {
    const unsigned g = grid_for((int64_t)k * n, ctx.num_sms);
    assemble_cols_kernel<real><<<g, 256, 0, ctx.stream>>>(k, (int)n, J, 1, T, ldt, P.Vs);
    CURID_LAUNCHED(ctx);
  }
  CURID_TRY(mm(false, true, k, k, n, one, P.Vs, n, Qr, n, zero, P.Nm, k));       // V* Q_R^T
  CURID_TRY(mm(true, false, k, k, k, one, P.Nm, k, P.Ub, k, zero, P.Pm, k));     // P = Q_R M
  CURID_TRY(mm(false, true, k, k, k, one, P.Ub, k, P.Lri, k, zero, P.X1, k));    // Ubar L_R^{-T}
  CURID_TRY(mm(false, false, k, n, k, one, P.X1, k, Qr, n, zero, P.Vsb, n));     // Vsbar
  CURID_TRY(split_s<real>(ctx, P.Vsb, n, J, k, n, P.S11, P.Tb));                 // Tbar
  CURID_TRY(mm(true, false, k, k, k, one, P.Lri, k, P.Lri, k, zero, P.W2, k));   // (R R^T)^{-1}
  CURID_TRY(mm(false, true, k, k, k, one, P.Pm, k, P.Lri, k, zero, P.X1, k));    // P L_R^{-T}
  CURID_TRY(mm(true, false, k, k, k, one, P.Lri, k, P.X1, k, zero, P.W1, k));    // L_R^{-T} P L_R^{-T}
  CURID_TRY(mm(false, true, k, k, k, one, P.W2, k, P.Pm, k, one, P.W1, k));      // + (R R^T)^{-1} P^T
  CURID_TRY(mm(false, true, k, k, k, one, P.W2, k, P.Ub, k, zero, P.G1, k));     // (R R^T)^{-1} Ubar^T
  CURID_TRY((cast_copy<real, real>(ctx, k, n, Rbar, n, P.Rt)));
  CURID_TRY(mm(false, false, k, n, k, one, P.G1, k, P.Vs, n, one, P.Rt, n));
  CURID_TRY(mm(false, false, k, n, k, mone, P.W1, k, Qr, n, one, P.Rt, n));

  // ---- through T = C^+ B ----
  CURID_TRY(mm(true, false, k, k, k, one, P.Lci, k, P.Lci, k, zero, P.Wc, k));   // (C^T C)^{-1}
  CURID_TRY(mm(false, false, k, nk, k, one, P.Wc, k, P.Tb, std::max<int64_t>(1, nk), zero, P.K,
               std::max<int64_t>(1, nk)));
  {
    const unsigned g = grid_for((int64_t)k * n, ctx.num_sms);
    assemble_cols_kernel<real>
        <<<g, 256, 0, ctx.stream>>>(k, (int)n, J, 0, P.K, std::max<int64_t>(1, nk), P.Kf);
    CURID_LAUNCHED(ctx);
  }
  // S = T K^T + K T^T
  CURID_TRY(mm(false, true, k, k, nk, one, T, ldt, P.K, std::max<int64_t>(1, nk), zero, P.S, k));
  if (nk > 0)
    CURID_TRY(mm(false, true, k, k, nk, one, P.K, nk, T, ldt, one, P.S, k));
  // total Cbar = Cbar + A Kf^T - C S
  CURID_TRY((cast_copy<real, real>(ctx, m, k, Cbar, k, P.Ct)));
  CURID_TRY(mm(false, true, m, k, n, one, A, lda, P.Kf, n, one, P.Ct, k));
  CURID_TRY(mm(true, false, m, k, k, mone, Craw, m, P.S, k, one, P.Ct, k));

  // ---- Abar = C Kf, then the scatters ----
  CURID_TRY(mm(true, false, m, n, k, one, Craw, m, P.Kf, n, zero, Abar, ldab));
  scatter_add_cols_kernel<real><<<grid_for(m * k, ctx.num_sms), 256, 0, ctx.stream>>>(
      m, k, (int)n, J, P.Ct, Abar, ldab);
  CURID_LAUNCHED(ctx);
  {
    dim3 g((unsigned)std::min<int64_t>((n + 255) / 256, 64), (unsigned)k);
    scatter_add_rows_kernel<real><<<g, 256, 0, ctx.stream>>>(k, n, m, I, P.Rt, Abar, ldab);
    CURID_LAUNCHED(ctx);
  }
  return CURID_OK;
}

curid_status adjoint_check(curid_handle* h, curid_dtype dt, int64_t m, int64_t n, int k) {
  if (!h) return CURID_INVALID_ARG;
  if (dt != CURID_F32 && dt != CURID_F64) return CURID_INVALID_ARG;
  if (m <= 0 || n <= 0 || m > INT32_MAX || n > INT32_MAX) return CURID_INVALID_ARG;
  if (k < 1 || k > std::min(m, n)) return CURID_INVALID_ARG;
  Ctx ctx{nullptr, h->num_sms, h->smem_optin, nullptr};
  ctx.spin = h->spin;
  ctx.concurrency = h->concurrency;
  const bool fits = dt == CURID_F64
                        ? (tri_solve_fits<double>(ctx, k) && chol_inverse_fits<double>(ctx, k))
                        : (tri_solve_fits<float>(ctx, k) && chol_inverse_fits<float>(ctx, k));
  return fits ? CURID_OK : CURID_UNSUPPORTED;
}

}  // namespace

extern "C" {

curid_status curid_cur_adjoint_workspace_size(curid_handle* handle, curid_dtype dtype, int64_t m,
                                              int64_t n, int k, size_t* bytes) {
  if (!bytes) return CURID_INVALID_ARG;
  CURID_TRY(adjoint_check(handle, dtype, m, n, k));
  Ctx ctx{nullptr, handle->num_sms, handle->smem_optin, nullptr};
  ctx.spin = handle->spin;
  ctx.concurrency = handle->concurrency;
  if (dtype == CURID_F64) {
    AdjPlan<double> P;
    adj_plan<double>(ctx, m, n, k, nullptr, &P);
    *bytes = P.bytes;
  } else {
    AdjPlan<float> P;
    adj_plan<float>(ctx, m, n, k, nullptr, &P);
    *bytes = P.bytes;
  }
  return CURID_OK;
}

curid_status curid_cur_adjoint(curid_handle* handle, curid_dtype dtype, const void* A, int64_t m,
                               int64_t n, int64_t lda, int k, const int32_t* J, const int32_t* I,
                               const void* T, int64_t ldt, const void* Cbar, const double* Ubar,
                               const void* Rbar, void* Abar, int64_t ldab) {
  CURID_TRY(adjoint_check(handle, dtype, m, n, k));
  if (!A || !J || !I || !Abar || lda < n || ldab < n) return CURID_INVALID_ARG;
  if (n > k && (!T || ldt < n - k)) return CURID_INVALID_ARG;
  int prev = -1;
  if (cudaGetDevice(&prev) != cudaSuccess) return CURID_CUDA_ERROR;
  if (prev != handle->device && cudaSetDevice(handle->device) != cudaSuccess)
    return CURID_CUDA_ERROR;
  Ctx ctx{handle->stream, handle->num_sms, handle->smem_optin, nullptr};
  ctx.spin = handle->spin;
  ctx.concurrency = handle->concurrency;
  ctx.launches = handle->profiling ? &handle->launches : nullptr;
  curid_status st;
  if (dtype == CURID_F64)
    st = adjoint_run<double>(ctx, (const double*)A, m, n, lda, k, J, I, (const double*)T,
                             std::max<int64_t>(1, ldt), (const double*)Cbar, Ubar,
                             (const double*)Rbar, (double*)Abar, ldab, handle->ws,
                             handle->ws_bytes);
  else
    st = adjoint_run<float>(ctx, (const float*)A, m, n, lda, k, J, I, (const float*)T,
                            std::max<int64_t>(1, ldt), (const float*)Cbar, Ubar,
                            (const float*)Rbar, (float*)Abar, ldab, handle->ws,
                            handle->ws_bytes);
  if (prev != handle->device) cudaSetDevice(prev);
  return st;
}

}  // extern "C"
