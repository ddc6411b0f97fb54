// C-ABI entry points: argument checks, workspace layout and the order of
// kernels for CPQR -> column ID -> row ID of C -> CUR (Algorithms 1-4).
// Every step of the method runs in this library's kernels; the host only
// validates, carves the caller's workspace and enqueues launches.
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>

#include "kernels.cuh"

using namespace curid;

namespace {

// CurCorrected: CUR-ID with U from the error-corrected system of Eq. (4.3)
enum class Op { IdCol, Tsid, Cur, CurCorrected };

struct DeviceGuard {
  int prev = -1;
  bool ok = true;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) { ok = false; return; }
    if (prev != dev && cudaSetDevice(dev) != cudaSuccess) ok = false;
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

cudaEvent_t take_event(curid_handle* h) {
  if (h->pool_used < h->pool.size()) return h->pool[h->pool_used++];
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  h->pool.push_back(e);
  h->pool_used = h->pool.size();
  return e;
}

// Records CUDA events around one phase of a call when profiling is on.
struct PhaseScope {
  curid_handle* h;
  int phase;
  cudaEvent_t start = nullptr;
  PhaseScope(curid_handle* hh, int ph) : h(hh), phase(ph) {
    if (h && h->profiling) {
      start = take_event(h);
      if (start) cudaEventRecord(start, h->stream);
    }
  }
  ~PhaseScope() {
    if (!start) return;
    cudaEvent_t stop = take_event(h);
    if (!stop) return;
    cudaEventRecord(stop, h->stream);
    h->recs.push_back({phase, start, stop});
  }
};

// Context for sizing (no stream): the handle's settings that shape plans.
Ctx host_ctx(curid_handle* h) {
  Ctx c{nullptr, h->num_sms, h->smem_optin, nullptr};
  c.spin = h->spin;
  c.concurrency = h->concurrency;
  return c;
}

Ctx make_ctx(curid_handle* h) {
  Ctx c{h->stream, h->num_sms, h->smem_optin, nullptr};
  c.launches = h->profiling ? &h->launches : nullptr;
  c.spin = h->spin;
  c.concurrency = h->concurrency;
  return c;
}

// All buffers of one decomposition, carved from the workspace in a fixed
// order.  With a null base the carver only counts bytes.
template <typename real>
struct Plan {
  StatusBlock* status = nullptr;
  // randomized front end
  real* omega = nullptr;  // l x m (when generated)
  real* B[3] = {nullptr, nullptr, nullptr};  // sample-matrix buffers, l x max(m, n)
  real* G = nullptr;      // l x l  (Gram)
  real* Linv = nullptr;   // l x l
  real* Li = nullptr;     // l x pad4(l) (tensor-core orth apply)
  // column CPQR and T
  CpqrScratch cs{};
  real* S = nullptr;      // k x n
  real* S11 = nullptr;    // k x k
  real* S12 = nullptr;    // k x (n - k)
  real* Sinv = nullptr;   // k x k
  real* T = nullptr;      // k x (n - k)
  // row ID of C
  real* Ct = nullptr;     // k x m
  CpqrScratch rs{};
  int32_t* I = nullptr;   // m (when the caller passes none)
  real* SW = nullptr;     // k x m
  real* SW11 = nullptr;   // k x k
  real* SW12 = nullptr;   // k x (m - k)
  real* SWinv = nullptr;  // k x k
  // U = V* R^+
  real* R = nullptr;      // k x n
  real* Rt = nullptr;     // k x n
  real* Q = nullptr;      // k x n
  real* Gu = nullptr;     // k x k
  real* L1 = nullptr;     // k x k
  real* L2 = nullptr;     // k x k
  real* Qsk = nullptr;    // k x k
  real* Qres = nullptr;   // k x (n - k)
  real* M = nullptr;      // k x k
  real* Uh = nullptr;     // k x k
  // error-corrected U (Eq. (4.3)): Q_C with C^T = L Q_C, K = Q_C C, Q_C A
  real* Xc[2] = {nullptr, nullptr};  // k x pad4(m)
  real* Bq = nullptr;     // k x pad4(n)
  real* Bq2 = nullptr;    // k x pad4(n) (TF32: the product with the low part of Q_C)
  real* Kc = nullptr;     // k x k
  real* Mp = nullptr;     // k x k
  real* partial = nullptr;
  size_t partial_cap = 0;
  // BF16 storage of A: the split sample operand, and the float64 T solve
  void* xsplit = nullptr;
  size_t xsplit_elems = 0;
  double* S11d = nullptr;  // k x k
  double* S12d = nullptr;  // k x (n - k)
  // sparse A: the transposed sample operand and the transposed product
  const SparseA* sp = nullptr;
  real* spX = nullptr;     // max(m, n) x l
  real* spO = nullptr;     // max(m, n) x l
  size_t bytes = 0;
};

inline int64_t pad4(int64_t x) { return (x + 3) & ~int64_t(3); }

struct Dims {
  int64_t m, n, lda;
  int k, l;
  bool randomized;
  int q;
  bool tf32 = false;
  bool bf16 = false;  // A stored as bfloat16 (float32 pipeline, BF16 tensor-core products)
  const SparseA* sp = nullptr;  // A sparse (randomized method only)
};

template <typename real>
curid_status make_plan(const Ctx& ctx, Op op, const Dims& d, bool gen_omega, bool need_I,
                       void* base, Plan<real>* P) {
  Carver cv(base);
  const int64_t m = d.m, n = d.n;
  const int k = d.k, l = d.l;
  P->status = cv.take<StatusBlock>(1);
  P->sp = d.sp;
  if (d.sp) {
    P->spX = cv.take<real>((size_t)std::max(m, n) * l);
    P->spO = cv.take<real>((size_t)std::max(m, n) * l);
  }
  size_t part = 0;
  auto upd = [&](int64_t M, int64_t N, int64_t K) {
    part = std::max(part, gemm_partial_elems<real>(M, N, K, ctx.num_sms));
  };
  if (d.randomized) {
    // Omega is kept with a leading dimension padded to 4 elements (16 bytes,
    // what the tensor-core loads require) when it is generated, or copied
    // when a caller's Omega is misaligned for them.
    if (gen_omega || (d.tf32 && (m & 3))) P->omega = cv.take<real>((size_t)l * pad4(m));
    upd(l, n, m);
    if (d.tf32) {
      part = std::max(part, gemm_tf32_partial_elems(l, n, m, ctx.num_sms));
      part = std::max(part, gemm_tf32_partial_elems(l, m, n, ctx.num_sms));
    }
    if (d.bf16) {
      P->xsplit_elems = gemm_bf16_split_elems(l, std::max(m, n));
      P->xsplit = cv.take<__nv_bfloat16>(P->xsplit_elems);
    }
    if (d.q == 0) {
      P->B[0] = cv.take<real>((size_t)l * pad4(n));
    } else {
      for (int b = 0; b < 3; ++b) P->B[b] = cv.take<real>((size_t)l * pad4(std::max(m, n)));
      P->G = cv.take<real>((size_t)l * l);
      P->Linv = cv.take<real>((size_t)l * l);
      if (sizeof(real) == 4 && (d.tf32 || d.bf16) && !d.sp)
        part = std::max(part, gemm_tf32_partial_elems(std::min<int64_t>(l, 256), l,
                                                      std::max(m, n), ctx.num_sms));
      if (sizeof(real) == 4 && (d.tf32 || d.bf16) && !d.sp) {
        // explicit L^{-1} for the tensor-core apply of the orth
        P->Li = cv.take<real>((size_t)l * pad4(l));
        part = std::max(part, gemm_tf32_partial_elems(std::min<int64_t>(l, 256), std::max(m, n),
                                                      l, ctx.num_sms));
      }
      upd(l, l, n);
      upd(l, l, m);
      upd(l, n, l);
      upd(l, m, l);
      upd(l, m, n);
    }
  }
  const int64_t ly = d.randomized ? l : m;
  int grid;
  size_t smem;
  CURID_TRY(cpqr_plan<real>(ctx, ly, n, &grid, &smem));
  cpqr_carve<real>(cv, ctx, ly, n, &P->cs);
  P->S = cv.take<real>((size_t)k * n);
  P->S11 = cv.take<real>((size_t)k * k);
  P->S12 = cv.take<real>((size_t)k * std::max<int64_t>(1, n - k));
  P->Sinv = cv.take<real>((size_t)k * k);
  P->T = cv.take<real>((size_t)k * std::max<int64_t>(1, n - k));
  if (d.bf16) {
    P->S11d = cv.take<double>((size_t)k * k);
    P->S12d = cv.take<double>((size_t)k * std::max<int64_t>(1, n - k));
  }
  upd(k, n - k, k);
  if (!tri_solve_fits<real>(ctx, k)) return CURID_UNSUPPORTED;
  if (d.randomized && d.q > 0 && !chol_inverse_fits<real>(ctx, l)) return CURID_UNSUPPORTED;
  const bool cur_op = op == Op::Cur || op == Op::CurCorrected;
  if (op == Op::Tsid || cur_op) {
    P->Ct = cv.take<real>((size_t)k * m);
    CURID_TRY(cpqr_plan<real>(ctx, k, m, &grid, &smem));
    cpqr_carve<real>(cv, ctx, k, m, &P->rs);
    if (need_I) P->I = cv.take<int32_t>(m);
    P->SW = cv.take<real>((size_t)k * m);
    P->SW11 = cv.take<real>((size_t)k * k);
    P->SW12 = cv.take<real>((size_t)k * std::max<int64_t>(1, m - k));
    P->SWinv = cv.take<real>((size_t)k * k);
    upd(k, m - k, k);
  }
  if (cur_op) {
    P->R = cv.take<real>((size_t)k * n);
    P->Rt = cv.take<real>((size_t)k * n);
    P->Q = cv.take<real>((size_t)k * n);
    P->Gu = cv.take<real>((size_t)k * k);
    P->L1 = cv.take<real>((size_t)k * k);
    P->L2 = cv.take<real>((size_t)k * k);
    P->Qsk = cv.take<real>((size_t)k * k);
    P->Qres = cv.take<real>((size_t)k * std::max<int64_t>(1, n - k));
    P->M = cv.take<real>((size_t)k * k);
    P->Uh = cv.take<real>((size_t)k * k);
    upd(k, n, k);
    upd(k, k, n);
    upd(k, k, n - k);
    upd(k, k, k);
  }
  if (op == Op::CurCorrected) {
    for (int b = 0; b < 2; ++b) P->Xc[b] = cv.take<real>((size_t)k * pad4(m));
    P->Bq = cv.take<real>((size_t)k * pad4(n));
    if (d.tf32) P->Bq2 = cv.take<real>((size_t)k * pad4(n));
    P->Kc = cv.take<real>((size_t)k * k);
    P->Mp = cv.take<real>((size_t)k * k);
    upd(k, k, m);
    upd(k, m, k);
    upd(k, n, m);
    if (d.tf32) part = std::max(part, gemm_tf32_partial_elems(k, n, m, ctx.num_sms));
  }
  P->partial_cap = part;
  P->partial = part ? cv.take<real>(part) : nullptr;
  P->bytes = cv.used + 256;
  return CURID_OK;
}

// Products that read A (Y = Omega A, Z = Q A^T, Y = Q A): FP32 FMA, FP64 FMA,
// or TF32 tensor cores when requested.
template <typename real>
curid_status a_product(const Ctx& ctx, bool tf32, bool bf16, bool tb, int64_t M, int64_t N,
                       int64_t K, const real* X, int64_t ldx, const void* A, int64_t lda,
                       real* out, int64_t ldo, const Plan<real>& P) {
  if (P.sp) {
    // sparse A: out = X A = ((X A)^T)^T with (X A)^T from the compressed
    // columns; out = X A^T from the compressed rows; X^T is the gathered
    // operand (K x M) and the product comes out transposed (N x M)
    const SparseA& S = *P.sp;
    CURID_TRY(transpose2d<real>(ctx, X, ldx, P.spX, M, M, K));
    if (!tb)
      CURID_TRY(spmm_rows<real>(ctx, N, S.col_ptr, S.row_idx, static_cast<const real*>(S.col_val),
                                S.nnz, K, P.spX, M, M, P.spO, M));
    else
      CURID_TRY(spmm_rows<real>(ctx, N, S.row_ptr, S.col_idx, static_cast<const real*>(S.row_val),
                                S.nnz, K, P.spX, M, M, P.spO, M));
    return transpose2d<real>(ctx, P.spO, M, out, ldo, N, M);
  }
  if constexpr (sizeof(real) == 4) {
    if (bf16)
      return gemm_bf16(ctx, tb, M, N, K, X, ldx, A, lda, out, ldo, P.xsplit, P.xsplit_elems);
    if (tf32)
      return gemm_tf32(ctx, false, tb, M, N, K, X, ldx, static_cast<const real*>(A), lda, out,
                       ldo, P.partial, P.partial_cap);
  }
  return gemm<real>(ctx, false, tb, M, N, K, real(1), X, ldx, static_cast<const real*>(A), lda,
                    real(0), out, ldo, P.partial, P.partial_cap);
}

// Row orthonormalisation without pivoting (Section 5.3) by Cholesky-QR
// passes (chol_qr_rows), the Gram matrix in the plan's l x l buffer.
//
// orth(X) is the Q of X = L Q with L lower triangular, positive diagonal.
// If a product's input is N Q instead (N lower triangular, positive
// diagonal), the product N Q B has the same Q factor as Q B, so every orth
// whose output is multiplied by A and orthonormalised again needs only a
// well-conditioned N: two passes (condition number 1 + O(u kappa_1^2),
// kappa_1 <= 1 / sqrt(shift) after the shifted first pass).  The last orth,
// whose Q forms the Y that is pivoted, takes all three.
//
// With tensor-core products (TF32, or BF16 storage of A) and samples of more
// than 256 rows the orth runs on the TF32 tensor cores at float32 accuracy:
// the Gram matrices (gram_tf32) and the apply X <- L^{-1} X through an
// explicit L^{-1}, each one launch that splits both operands into TF32 parts
// in shared memory (l = 520 rows of 20000: orth 13 -> 10 ms per
// decomposition with the Gram alone).  Samples
// of up to 256 rows go to the tensor cores when several decompositions are
// in flight, where the SIMT products' SM time is what limits throughput;
// one at a time they keep the SIMT Gram and the triangular solve.
// CURID_ORTH_TC=1 / 0 in the environment forces either for small samples
// (for comparisons).
template <typename real>
curid_status orth_rows(const Ctx& ctx, real** X, real** tmp, int64_t r, int64_t c, int64_t ld,
                       const Plan<real>& P, bool final_orth, bool tc) {
  const bool tc_ok = sizeof(real) == 4 && tc && P.Li && !P.sp;
  bool small_tc = tc_ok && r <= 256 && P.Li && ctx.concurrency > 1;
  if (const char* env = std::getenv("CURID_ORTH_TC")) {
    if (std::strcmp(env, "1") == 0) small_tc = tc_ok && r <= 256 && P.Li;
    if (std::strcmp(env, "0") == 0) small_tc = false;
  }
  const bool use_tc = tc_ok && (r > 256 || small_tc);
  return chol_qr_rows<real>(ctx, X, tmp, r, c, ld, P.G, P.partial, P.partial_cap,
                            final_orth ? 3 : 2, use_tc, use_tc ? P.Li : nullptr);
}

// Sample matrix of Algorithm 4 with the power scheme of Section 5.3:
// (2a) Y = Omega A; for i = 1..q: (2c) Y <- orth(Y) A^*, (2d) Y <- orth(Y) A.
// Returns the buffer holding the final Y (l x n, leading dimension
// pad4(n)); Omega has leading dimension ldo.
template <typename real>
curid_status sketch(curid_handle* h, const Ctx& ctx, const Plan<real>& P, const void* A,
                    int64_t m, int64_t n, int64_t lda, int l, int q, bool tf32, bool bf16,
                    const real* Om, int64_t ldo, real** Yout, const int32_t* srft_rows = nullptr,
                    const int8_t* srft_signs = nullptr) {
  const int64_t ldy = pad4(n), ldz = pad4(m);
  auto other = [&](const real* a, const real* b) -> real* {
    for (int i = 0; i < 3; ++i)
      if (P.B[i] != a && P.B[i] != b) return P.B[i];
    return nullptr;
  };
  real* cur = P.B[0];
  {
    PhaseScope ps(h, CURID_PHASE_SKETCH);
    if (srft_rows) {
      // structured Omega of Eq. (5.2) applied by the fast transform
      if (bf16) return CURID_UNSUPPORTED;
      CURID_TRY(srft_apply<real>(ctx, static_cast<const real*>(A), m, n, lda, l, srft_rows,
                                 srft_signs, cur, ldy));
    } else {
      CURID_TRY(a_product<real>(ctx, tf32, bf16, false, l, n, m, Om, ldo, A, lda, cur, ldy, P));
    }
  }
  for (int i = 0; i < q; ++i) {
    real* t = other(cur, nullptr);
    {
      PhaseScope ps(h, CURID_PHASE_ORTH);
      CURID_TRY(orth_rows<real>(ctx, &cur, &t, l, n, ldy, P, false, tf32 || bf16));
    }
    real* z = other(cur, nullptr);
    {
      PhaseScope ps(h, CURID_PHASE_SKETCH);
      CURID_TRY(a_product<real>(ctx, tf32, bf16, true, l, m, n, cur, ldy, A, lda, z, ldz, P));
    }
    real* zt = other(z, nullptr);
    {
      PhaseScope ps(h, CURID_PHASE_ORTH);
      CURID_TRY(orth_rows<real>(ctx, &z, &zt, l, m, ldz, P, i == q - 1, tf32 || bf16));
    }
    real* y = other(z, nullptr);
    {
      PhaseScope ps(h, CURID_PHASE_SKETCH);
      CURID_TRY(a_product<real>(ctx, tf32, bf16, false, l, n, m, z, ldz, A, lda, y, ldy, P));
    }
    cur = y;
  }
  *Yout = cur;
  return CURID_OK;
}

// T = S11^{-1} S12 (Eq. (2.8)) from S (k x n, original column order) and J:
// a blocked back substitution on the n - k columns of S12.
template <typename real>
curid_status t_solve(const Ctx& ctx, const real* S, int64_t n, const int32_t* J, int k,
                     const int* k_eff, real* S11, real* S12, real* T, int64_t ldt) {
  CURID_TRY(split_s<real>(ctx, S, n, J, k, n, S11, S12));
  if (n - k > 0)
    CURID_TRY(tri_solve<real>(ctx, k, S11, k, true, false, S12, n - k, T, ldt, n - k, k_eff));
  return CURID_OK;
}

// The same T solve in float64 (the precision form with BF16 storage keeps the
// triangular solve in float64): S11, S12 widened, blocked float64 back
// substitution in place, T rounded to the working precision.
template <typename real>
curid_status t_solve64(const Ctx& ctx, const real* S, int64_t n, const int32_t* J, int k,
                       const int* k_eff, real* S11, real* S12, double* S11d, double* S12d,
                       real* T, int64_t ldt) {
  CURID_TRY(split_s<real>(ctx, S, n, J, k, n, S11, S12));
  if (n - k <= 0) return CURID_OK;
  CURID_TRY((convert2d<real, double>(ctx, S11, k, S11d, k, k, k)));
  CURID_TRY((convert2d<real, double>(ctx, S12, n - k, S12d, n - k, k, n - k)));
  CURID_TRY(tri_solve<double>(ctx, k, S11d, k, true, false, S12d, n - k, S12d, n - k, n - k,
                              k_eff));
  return convert2d<double, real>(ctx, S12d, n - k, T, ldt, k, n - k);
}

struct Outputs {
  int32_t* J;
  void* T;
  int64_t ldt;
  int32_t* I;
  void* TW;
  int64_t ldtw;
  double* U;
  void* C;
  void* R;
};

template <typename real>
curid_status run(curid_handle* h, Op op, const void* Araw, const Dims& d, double tol,
                 const curid_sketch& sk, const Outputs& o, char* ws, size_t ws_bytes) {
  // BF16 storage: A is read only by the tensor-core products and the gathers
  const real* A = d.bf16 ? nullptr : static_cast<const real*>(Araw);
  const __nv_bfloat16* Ab = d.bf16 ? static_cast<const __nv_bfloat16*>(Araw) : nullptr;
  if (d.bf16 && (reinterpret_cast<uintptr_t>(Araw) & 15)) return CURID_UNSUPPORTED;
  Ctx ctx = make_ctx(h);
  Plan<real> P;
  const bool structured = d.randomized && sk.srft_rows != nullptr;
  const bool gen_omega = d.randomized && sk.omega == nullptr && !structured;
  const bool need_I = o.I == nullptr;
  CURID_TRY(make_plan<real>(ctx, op, d, gen_omega, need_I, nullptr, &P));
  if (ws == nullptr || P.bytes > ws_bytes) return CURID_NO_WORKSPACE;
  CURID_TRY(make_plan<real>(ctx, op, d, gen_omega, need_I, ws, &P));
  ctx.status = P.status;
  const int64_t m = d.m, n = d.n, lda = d.lda;
  const int k = d.k, l = d.l;
  CURID_CUDA(cudaMemsetAsync(P.status, 0, sizeof(StatusBlock), ctx.stream));

  // ---- sample matrix (Algorithm 4 lines 1-2; Section 5.3 steps 2a-2e) ----
  const real* Y = A;
  int64_t ly = m, ldy = lda;
  if (d.randomized) {
    const real* Om = static_cast<const real*>(sk.omega);
    int64_t ldo = m;
    if (gen_omega) {
      PhaseScope ps(h, CURID_PHASE_OMEGA);
      CURID_TRY(gaussian_fill<real>(ctx, l, m, sk.seed, P.omega, pad4(m)));
      Om = P.omega;
      ldo = pad4(m);
    } else if (P.omega && !structured) {
      CURID_TRY(copy2d<real>(ctx, Om, m, P.omega, pad4(m), l, m));
      Om = P.omega;
      ldo = pad4(m);
    }
    real* Yr;
    CURID_TRY(sketch<real>(h, ctx, P, Araw, m, n, lda, l, d.q, sk.tf32 != 0, d.bf16, Om, ldo,
                           &Yr, structured ? sk.srft_rows : nullptr,
                           structured ? sk.srft_signs : nullptr));
    Y = Yr;
    ly = l;
    ldy = pad4(n);
  }

  // ---- truncated CPQR and T (Algorithm 1 / 4) ----
  {
    PhaseScope ps(h, CURID_PHASE_CPQR_COL);
    CURID_TRY(cpqr_run<real>(ctx, Y, ly, n, ldy, k, tol, o.J, P.S, n, P.cs, 0));
  }
  const bool cur_op = op == Op::Cur || op == Op::CurCorrected;
  real* T = (o.T && !cur_op) ? static_cast<real*>(o.T) : P.T;
  int64_t ldt = (T == P.T) ? std::max<int64_t>(1, n - k) : o.ldt;
  {
    PhaseScope ps(h, CURID_PHASE_T);
    if (sizeof(real) == 4 && d.bf16)
      CURID_TRY(t_solve64<real>(ctx, P.S, n, o.J, k, &P.status->k_eff, P.S11, P.S12, P.S11d,
                                P.S12d, T, ldt));
    else
      CURID_TRY(t_solve<real>(ctx, P.S, n, o.J, k, &P.status->k_eff, P.S11, P.S12, T, ldt));
    if (o.T && T == P.T)
      CURID_TRY(copy2d<real>(ctx, P.T, ldt, static_cast<real*>(o.T), o.ldt, k, n - k));
  }
  if (op == Op::IdCol) return CURID_OK;

  // ---- row ID of C (Algorithm 2, Eq. (2.11)): full k-step CPQR of C^T ----
  int32_t* I = o.I ? o.I : P.I;
  {
    PhaseScope ps(h, CURID_PHASE_GATHER);
    if constexpr (sizeof(real) == 4) {
      if (d.bf16) {
        CURID_TRY((gather_cols_as<__nv_bfloat16, real>(ctx, Ab, m, n, lda, o.J, k, P.Ct, m, true)));
        if (o.C)
          CURID_TRY((gather_cols_as<__nv_bfloat16, __nv_bfloat16>(
              ctx, Ab, m, n, lda, o.J, k, static_cast<__nv_bfloat16*>(o.C), k, false)));
      }
    }
    if (d.sp) {
      CURID_TRY(scatter_lists<real>(ctx, o.J, k, n, d.sp->col_ptr, d.sp->row_idx,
                                    static_cast<const real*>(d.sp->col_val), m, P.Ct, m,
                                    static_cast<real*>(o.C), k));
    } else if (!d.bf16) {
      CURID_TRY(gather_cols<real>(ctx, A, m, n, lda, o.J, k, P.Ct, m, true));
      if (o.C)
        CURID_TRY(gather_cols<real>(ctx, A, m, n, lda, o.J, k, static_cast<real*>(o.C), k, false));
    }
  }
  {
    PhaseScope ps(h, CURID_PHASE_CPQR_ROW);
    CURID_TRY(cpqr_run<real>(ctx, P.Ct, k, m, m, k, 0.0, I, P.SW, m, P.rs, 1));
  }
  PhaseScope ps_u(h, CURID_PHASE_U);
  if (o.TW) {
    CURID_TRY(t_solve<real>(ctx, P.SW, m, I, k, &P.status->k_row, P.SW11, P.SW12,
                            static_cast<real*>(o.TW), o.ldtw));
  } else {
    CURID_TRY(split_s<real>(ctx, P.SW, m, I, k, m, P.SW11, P.SW12));
  }
  if (cur_op)
    CURID_TRY(upper_tri_inverse<real>(ctx, P.SW11, k, &P.status->k_row, P.SWinv));
  if (op == Op::Tsid) return CURID_OK;

  // ---- U = V* R^+ (Eq. (3.5), Algorithm 3 line 3) ----
  // R = A(I[:k], :) = S_W11^T Q_W^T-structured; R~ = S_W11^{-T} R has a small
  // condition number, so its Cholesky QR R~ = L Q is accurate in the working
  // precision; then U = (V* Q^T) L^{-1} S_W11^{-T}, whose last product is
  // accumulated in float64.
  {
    PhaseScope ps(h, CURID_PHASE_GATHER);
    if constexpr (sizeof(real) == 4) {
      if (d.bf16) {
        CURID_TRY((gather_rows_as<__nv_bfloat16, real>(ctx, Ab, m, n, lda, I, k, P.R, n)));
        if (o.R)
          CURID_TRY((convert2d<real, __nv_bfloat16>(ctx, P.R, n,
                                                     static_cast<__nv_bfloat16*>(o.R), n, k, n)));
      }
    }
    if (d.sp) {
      CURID_TRY(scatter_lists<real>(ctx, I, k, m, d.sp->row_ptr, d.sp->col_idx,
                                    static_cast<const real*>(d.sp->row_val), n, P.R, n, nullptr,
                                    0));
      if (o.R) CURID_TRY(copy2d<real>(ctx, P.R, n, static_cast<real*>(o.R), n, k, n));
    } else if (!d.bf16) {
      CURID_TRY(gather_rows<real>(ctx, A, m, n, lda, I, k, P.R, n));
      if (o.R) CURID_TRY(copy2d<real>(ctx, P.R, n, static_cast<real*>(o.R), n, k, n));
    }
  }
  CURID_TRY(gemm<real>(ctx, true, false, k, n, k, real(1), P.SWinv, k, P.R, n, real(0), P.Rt, n,
                       P.partial, P.partial_cap));
  CURID_TRY(gemm<real>(ctx, false, true, k, k, n, real(1), P.Rt, n, P.Rt, n, real(0), P.Gu, k,
                       P.partial, P.partial_cap));
  CURID_TRY(chol_inverse<real>(ctx, P.Gu, k, 0.0, P.L1));
  CURID_TRY(gemm<real>(ctx, false, false, k, n, k, real(1), P.L1, k, P.Rt, n, real(0), P.Q, n,
                       P.partial, P.partial_cap));
  CURID_TRY(gemm<real>(ctx, false, true, k, k, n, real(1), P.Q, n, P.Q, n, real(0), P.Gu, k,
                       P.partial, P.partial_cap));
  CURID_TRY(chol_inverse<real>(ctx, P.Gu, k, 0.0, P.L2));
  CURID_TRY(gemm<real>(ctx, false, false, k, n, k, real(1), P.L2, k, P.Q, n, real(0), P.Rt, n,
                       P.partial, P.partial_cap));
  if (op == Op::CurCorrected) {
    // Eq. (4.3): U R = V* + C^+ E with E = A - C V*, i.e. U = C^+ A R^+.
    // C^T = L Q_C (three Cholesky-QR passes); C^+ = K^{-1} Q_C with
    // K = Q_C C (= L^T, upper triangular to rounding, solved as such); so
    // M = C^+ A Q^T = K^{-1} (Q_C A) Q^T, and U = M L^{-1} S_W11^{-T} below.
    const int64_t ldx = pad4(m);
    CURID_TRY(copy2d<real>(ctx, P.Ct, m, P.Xc[0], ldx, k, m));
    real* qc = P.Xc[0];
    real* qt = P.Xc[1];
    CURID_TRY(chol_qr_rows<real>(ctx, &qc, &qt, k, m, ldx, P.Gu, P.partial, P.partial_cap, 3));
    CURID_TRY(gemm<real>(ctx, false, true, k, k, m, real(1), qc, ldx, P.Ct, m, real(0), P.Kc, k,
                         P.partial, P.partial_cap));
    // Q_C A must be accurate to the working precision (C^+ is applied to
    // it exactly, unlike a sketch operand): with TF32 products Q_C is split
    // into its TF32 part and the remainder, two products with A (each with
    // A split hi + lo) summed.
    bool split_done = false;
    if constexpr (sizeof(real) == 4) {
      if (sk.tf32 && !d.bf16 && !d.sp) {
        CURID_TRY(split_tf32(ctx, qc, ldx, qc, ldx, qt, ldx, k, m));
        CURID_TRY(a_product<real>(ctx, true, false, false, k, n, m, qc, ldx, Araw, lda, P.Bq,
                                  pad4(n), P));
        CURID_TRY(a_product<real>(ctx, true, false, false, k, n, m, qt, ldx, Araw, lda, P.Bq2,
                                  pad4(n), P));
        CURID_TRY(add2d<real>(ctx, P.Bq2, pad4(n), P.Bq, pad4(n), k, n));
        split_done = true;
      }
    }
    if (!split_done)
      CURID_TRY(a_product<real>(ctx, sk.tf32 != 0, d.bf16, false, k, n, m, qc, ldx, Araw, lda,
                                P.Bq, pad4(n), P));
    CURID_TRY(gemm<real>(ctx, false, true, k, k, n, real(1), P.Bq, pad4(n), P.Rt, n, real(0),
                         P.Mp, k, P.partial, P.partial_cap));
    CURID_TRY(tri_solve<real>(ctx, k, P.Kc, k, true, false, P.Mp, k, P.M, k, k,
                              &P.status->k_row));
  } else {
    // M = V* Q^T = Q(:, J[:k])^T + T Q(:, J[k:])^T
    CURID_TRY(split_s<real>(ctx, P.Rt, n, o.J, k, n, P.Qsk, P.Qres));
    if (n - k > 0) {
      CURID_TRY(gemm<real>(ctx, false, true, k, k, n - k, real(1), T, ldt, P.Qres, n - k,
                           real(0), P.M, k, P.partial, P.partial_cap));
    } else {
      CURID_CUDA(cudaMemsetAsync(P.M, 0, (size_t)k * k * sizeof(real), ctx.stream));
    }
    CURID_TRY(add_transpose<real>(ctx, P.Qsk, k, P.M, k, k, k));
  }
  CURID_TRY(gemm<real>(ctx, false, false, k, k, k, real(1), P.M, k, P.L2, k, real(0), P.Uh, k,
                       P.partial, P.partial_cap));
  CURID_TRY(gemm<real>(ctx, false, false, k, k, k, real(1), P.Uh, k, P.L1, k, real(0), P.M, k,
                       P.partial, P.partial_cap));
  CURID_TRY(gemm_nt_f64acc<real>(ctx, k, k, k, P.M, k, P.SWinv, k, o.U, k));
  return CURID_OK;
}

curid_status check_common(curid_handle* h, curid_dtype dt, const void* A, int64_t m, int64_t n,
                          int64_t lda, int k, double tol, const curid_sketch& sk, Dims* d) {
  if (!h) return CURID_INVALID_ARG;
  if (dt != CURID_F32 && dt != CURID_F64 && dt != CURID_BF16) return CURID_INVALID_ARG;
  if (!A || m <= 0 || n <= 0 || lda < n) return CURID_INVALID_ARG;
  if (m > INT32_MAX || n > INT32_MAX) return CURID_INVALID_ARG;
  if (k < 0 || tol < 0) return CURID_INVALID_ARG;
  if (k == 0) return tol > 0 ? CURID_UNSUPPORTED : CURID_INVALID_ARG;
  if (k > std::min(m, n)) return CURID_INVALID_ARG;
  if (sk.q < 0) return CURID_INVALID_ARG;
  if (sk.tf32 && dt != CURID_F32) return CURID_INVALID_ARG;
  if (sk.srft_rows || sk.srft_signs) {
    // the structured Omega replaces omega and seed; it needs both arrays
    if (!sk.srft_rows || !sk.srft_signs || sk.omega || sk.p < 0) return CURID_INVALID_ARG;
    if (dt == CURID_BF16) return CURID_UNSUPPORTED;
  }
  if (dt == CURID_BF16) {
    // the randomized method only: the products run on the tensor cores from
    // 16-byte aligned rows of A
    if (sk.p < 0 || (lda & 7)) return CURID_UNSUPPORTED;
  }
  d->bf16 = dt == CURID_BF16;
  d->m = m;
  d->n = n;
  d->lda = lda;
  d->k = k;
  d->randomized = sk.p >= 0;
  d->l = d->randomized ? k + sk.p : (int)m;
  d->q = sk.q;
  d->tf32 = sk.tf32 != 0;
  if (d->randomized && d->l > std::min(m, n)) return CURID_INVALID_ARG;
  if (!d->randomized && sk.q > 0) return CURID_INVALID_ARG;
  return CURID_OK;
}

template <typename F>
curid_status dispatch(curid_handle* h, F&& f) {
  DeviceGuard g(h->device);
  if (!g.ok) return CURID_CUDA_ERROR;
  return f();
}

// Adaptive rank of the deterministic decompositions (the tolerance stop of
// Section 3): the truncated CPQR of A runs with the stop ||A - C V*||_F <=
// tol ||A||_F (curid_cpqr, S placed after its scratch in the workspace), the
// stream is synchronised once to read the rank reached, and the caller then
// runs the fixed-rank pipeline at that rank (its CPQR repeats the same pivots:
// the tolerance only decides when to stop).  Rank 0 (the tolerance met by no
// column, e.g. A = 0): J comes back from this call and the caller fills I.
curid_status adaptive_rank(curid_handle* h, curid_dtype dt, const void* A, int64_t m, int64_t n,
                           int64_t lda, double tol, int32_t* J, int* k_out) {
  const int64_t kmax = std::min(m, n);
  const size_t esz = dt == CURID_F64 ? 8 : 4;
  Ctx ctx = host_ctx(h);
  Carver cv(nullptr);
  cv.take<StatusBlock>(1);
  CpqrScratch cs;
  if (dt == CURID_F64) cpqr_carve<double>(cv, ctx, m, n, &cs);
  else cpqr_carve<float>(cv, ctx, m, n, &cs);
  const size_t off = (cv.used + 255) & ~size_t(255);
  if (!h->ws || off + (size_t)kmax * n * esz > h->ws_bytes) return CURID_NO_WORKSPACE;
  CURID_TRY(curid_cpqr(h, dt, A, m, n, lda, 0, tol, J, h->ws + off));
  StatusBlock sb;
  DeviceGuard g(h->device);
  if (!g.ok) return CURID_CUDA_ERROR;
  if (cudaStreamSynchronize(h->stream) != cudaSuccess) return CURID_CUDA_ERROR;
  if (cudaMemcpy(&sb, h->ws, sizeof(sb), cudaMemcpyDeviceToHost) != cudaSuccess)
    return CURID_CUDA_ERROR;
  if (sb.flags & FLAG_TIMEOUT) return CURID_TIMEOUT;
  if (sb.flags & FLAG_NONFINITE) return CURID_NONFINITE;
  *k_out = sb.k_done;
  return CURID_OK;
}

// First sample size of the adaptive randomized search, and its cap (the
// largest order of the dense factorisations of the l x l Gram matrices).
constexpr int64_t kAdaptiveL0 = 64;
constexpr int64_t kAdaptiveLMax = kMaxDenseOrder;

inline int64_t adaptive_l_cap(int64_t m, int64_t n) {
  return std::min<int64_t>(std::min(m, n), kAdaptiveLMax);
}

// Adaptive rank with a sketch (Algorithm 4 with the tolerance stop of
// Section 3): the rank sets the sample size l = k + p, so l is searched.
// Starting at l = max(64, p + 1) (capped by min(m, n, 4096)), the sample
// Y = Omega_l A (A^* A)^q is formed and its CPQR runs with at most l - p
// steps and the stop ||Y - Q_j Q_j^T Y||_F <= tol ||Y||_F; if the stop
// comes before l - p steps its step count is the rank, else l doubles.
// Omega is drawn from the seed, and the rows of a smaller Omega are the
// leading rows of a larger one, so the fixed-rank run that follows (rank k,
// p' = l - k) samples with exactly the Y searched.  The stop is tested on the
// sample: for q = 0 the squared residual ratio of Y estimates A's without
// bias (E||Omega E||_F^2 = l ||E||_F^2 for Gaussian Omega); power steps
// weight the dominant directions and make it optimistic.  At the cap the rank
// is l - p whether or not the tolerance was met.
curid_status adaptive_rank_randomized(curid_handle* h, curid_dtype dt, const void* A, int64_t m,
                                      int64_t n, int64_t lda, double tol, curid_sketch* sk,
                                      int32_t* J, int* k_out) {
  // the sample grows: Omega comes from the seed
  if (sk->omega || sk->srft_rows || sk->srft_signs) return CURID_UNSUPPORTED;
  const int64_t cap = adaptive_l_cap(m, n);
  if (sk->p < 0 || sk->p >= cap) return CURID_INVALID_ARG;
  int64_t l = std::min<int64_t>(cap, std::max<int64_t>(kAdaptiveL0, sk->p + 1));
  while (true) {
    const int kmax = (int)(l - sk->p);
    Dims d;
    CURID_TRY(check_common(h, dt, A, m, n, lda, kmax, 0.0, *sk, &d));
    Outputs o{J, nullptr, 0, nullptr, nullptr, 0, nullptr, nullptr, nullptr};
    CURID_TRY(dispatch(h, [&]() -> curid_status {
      if (dt == CURID_F64)
        return run<double>(h, Op::IdCol, (const double*)A, d, tol, *sk, o, h->ws, h->ws_bytes);
      return run<float>(h, Op::IdCol, A, d, tol, *sk, o, h->ws, h->ws_bytes);
    }));
    StatusBlock sb;
    DeviceGuard g(h->device);
    if (!g.ok) return CURID_CUDA_ERROR;
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) return CURID_CUDA_ERROR;
    if (cudaMemcpy(&sb, h->ws, sizeof(sb), cudaMemcpyDeviceToHost) != cudaSuccess)
      return CURID_CUDA_ERROR;
    if (sb.flags & FLAG_TIMEOUT) return CURID_TIMEOUT;
    if (sb.flags & FLAG_NONFINITE) return CURID_NONFINITE;
    if (sb.flags & FLAG_BREAKDOWN) return CURID_BREAKDOWN;
    if (sb.k_done < kmax || l >= cap) {
      *k_out = sb.k_done;
      sk->p = (int)(l - sb.k_done);
      return CURID_OK;
    }
    l = std::min<int64_t>(cap, 2 * l);
  }
}

// Decides between the fixed rank k and the adaptive rank (k == 0, tol > 0);
// on return *k is the rank to run, or 0 when the tolerance is met by no
// column (J already written).  With a sketch, sk->p becomes the oversampling
// of the sample size the search settled on.
curid_status resolve_rank(curid_handle* h, curid_dtype dt, const void* A, int64_t m, int64_t n,
                          int64_t lda, int* k, double tol, curid_sketch* sk, int32_t* J) {
  if (*k != 0) return CURID_OK;
  if (!h || !A || !J || m <= 0 || n <= 0 || lda < n || !(tol > 0)) return CURID_INVALID_ARG;
  int kout = 0;
  if (sk->p >= 0) {
    CURID_TRY(adaptive_rank_randomized(h, dt, A, m, n, lda, tol, sk, J, &kout));
  } else {
    if (dt == CURID_BF16) return CURID_UNSUPPORTED;  // BF16 storage: randomized method only
    CURID_TRY(adaptive_rank(h, dt, A, m, n, lda, tol, J, &kout));
  }
  *k = kout;
  return CURID_OK;
}

__global__ void iota_kernel(int32_t* x, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    x[i] = (int32_t)i;
}

// Rank 0: I = 0..m-1 (nothing is selected); the status block records k = 0.
curid_status rank_zero_rows(curid_handle* h, int32_t* I, int64_t m) {
  DeviceGuard g(h->device);
  if (!g.ok) return CURID_CUDA_ERROR;
  if (I) {
    iota_kernel<<<(unsigned)std::min<int64_t>((m + 255) / 256, 1024), 256, 0, h->stream>>>(I, m);
    CURID_CUDA(cudaGetLastError());
  }
  return CURID_OK;
}

// Regularised T (Section 4.1: Eq. (4.1) with a Tikhonov term):
// T = argmin ||S11 T - S12||^2 + lam^2 ||T||^2 is the least-squares solution
// of [S11; lam I] T = [S12; 0].  With W = [S11; lam I] = Q_a R_a (the rows of
// W^T = [S11^T | lam I] orthonormalised by three Cholesky-QR passes, Q = Q_a^T
// k x 2k), T = R_a^{-1} Q(:, :k) S12 and R_a = Q W (upper triangular to
// rounding, solved as such).  No normal equations: cond(W) <= ||S11|| / lam.
template <typename real>
struct TikPlan {
  StatusBlock* status = nullptr;
  real* S11 = nullptr;   // k x k
  real* S12 = nullptr;   // k x (n - k)
  real* W[3] = {nullptr, nullptr, nullptr};  // k x 2k: two passes' buffers, W^T kept
  real* G = nullptr;     // k x k
  real* K = nullptr;     // k x k
  real* Z = nullptr;     // k x (n - k)
  real* partial = nullptr;
  size_t partial_cap = 0;
  size_t bytes = 0;
};

template <typename real>
void tik_plan(const Ctx& ctx, int64_t n, int k, void* base, TikPlan<real>* P) {
  Carver cv(base);
  const int64_t r = std::max<int64_t>(1, n - k);
  P->status = cv.take<StatusBlock>(1);
  P->S11 = cv.take<real>((size_t)k * k);
  P->S12 = cv.take<real>((size_t)k * r);
  for (int b = 0; b < 3; ++b) P->W[b] = cv.take<real>((size_t)k * 2 * k);
  P->G = cv.take<real>((size_t)k * k);
  P->K = cv.take<real>((size_t)k * k);
  P->Z = cv.take<real>((size_t)k * r);
  const size_t part = std::max(gemm_partial_elems<real>(k, k, 2 * k, ctx.num_sms),
                               gemm_partial_elems<real>(k, r, k, ctx.num_sms));
  P->partial_cap = part;
  P->partial = part ? cv.take<real>(part) : nullptr;
  P->bytes = cv.used + 256;
}

template <typename real>
curid_status tikhonov_run(curid_handle* h, const real* S, int64_t lds, const int32_t* J,
                          int64_t n, int k, double lam, real* T, int64_t ldt) {
  Ctx ctx = make_ctx(h);
  TikPlan<real> P;
  tik_plan<real>(ctx, n, k, nullptr, &P);
  if (!h->ws || P.bytes > h->ws_bytes) return CURID_NO_WORKSPACE;
  tik_plan<real>(ctx, n, k, h->ws, &P);
  if (!tri_solve_fits<real>(ctx, k) || !chol_inverse_fits<real>(ctx, k)) return CURID_UNSUPPORTED;
  ctx.status = P.status;
  PhaseScope ps(h, CURID_PHASE_T);
  CURID_CUDA(cudaMemsetAsync(P.status, 0, sizeof(StatusBlock), ctx.stream));
  CURID_TRY(split_s<real>(ctx, S, lds, J, k, n, P.S11, P.S12));
  const int64_t lw = 2LL * k;
  CURID_TRY(aug_transpose<real>(ctx, P.S11, k, k, (real)lam, P.W[2], lw));
  CURID_TRY(copy2d<real>(ctx, P.W[2], lw, P.W[0], lw, k, lw));
  real* x = P.W[0];
  real* t = P.W[1];
  CURID_TRY(chol_qr_rows<real>(ctx, &x, &t, k, lw, lw, P.G, P.partial, P.partial_cap, 3));
  CURID_TRY(gemm<real>(ctx, false, true, k, k, lw, real(1), x, lw, P.W[2], lw, real(0), P.K, k,
                       P.partial, P.partial_cap));
  if (n - k <= 0) return CURID_OK;
  CURID_TRY(gemm<real>(ctx, false, false, k, n - k, k, real(1), x, lw, P.S12, n - k, real(0),
                       P.Z, n - k, P.partial, P.partial_cap));
  return tri_solve<real>(ctx, k, P.K, k, true, false, P.Z, n - k, T, ldt, n - k, nullptr);
}

// Complex A (the paper works over C): the real pipeline on the embedding
// E(A) (2m x 2n, rank 2k, sample 2(k + p) rows from E(Omega) with a complex
// Gaussian Omega), then the complex J, I, T, U read off the real results
// (complex.cu).  The real plan occupies the start of the workspace (its
// status block is the handle's), the embedding buffers follow it.
template <typename real>
struct ComplexPlan {
  Dims d;
  size_t run_bytes = 0;
  real* E = nullptr;     // 2m x 2n
  real* Ge = nullptr;    // l x 2m: Gaussian (re, im) pairs
  real* Om = nullptr;    // 2l x 2m
  int32_t* Jp = nullptr;
  int32_t* Ip = nullptr;
  double* Up = nullptr;  // 2k x 2k
  real* Tp = nullptr;    // 2k x 2(n - k)
  size_t bytes = 0;
};

template <typename real>
curid_status complex_plan(const Ctx& ctx, int64_t m, int64_t n, int k, const curid_sketch& sk,
                          char* base, ComplexPlan<real>* P) {
  Dims& d = P->d;
  d.m = 2 * m;
  d.n = 2 * n;
  d.lda = 2 * n;
  d.k = 2 * k;
  d.randomized = sk.p >= 0;
  d.l = d.randomized ? 2 * (k + sk.p) : (int)(2 * m);
  d.q = sk.q;
  d.tf32 = sk.tf32 != 0;
  d.bf16 = false;
  Plan<real> rp;
  CURID_TRY(make_plan<real>(ctx, Op::Cur, d, false, false, nullptr, &rp));
  P->run_bytes = (rp.bytes + 255) & ~size_t(255);
  Carver cv(base ? base + P->run_bytes : nullptr);
  P->E = cv.take<real>((size_t)4 * m * n);
  if (d.randomized) {
    const int64_t l = k + sk.p;
    P->Ge = cv.take<real>((size_t)l * 2 * m);
    P->Om = cv.take<real>((size_t)4 * l * m);
  }
  P->Jp = cv.take<int32_t>((size_t)2 * n);
  P->Ip = cv.take<int32_t>((size_t)2 * m);
  P->Up = cv.take<double>((size_t)4 * k * k);
  P->Tp = cv.take<real>((size_t)2 * k * std::max<int64_t>(1, 2 * (n - k)));
  P->bytes = P->run_bytes + cv.used + 256;
  return CURID_OK;
}

template <typename real>
curid_status cur_complex_run(curid_handle* h, const real* A, int64_t m, int64_t n, int64_t lda,
                             int k, const curid_sketch& sk, int32_t* J, int32_t* I, double* U,
                             real* T, int64_t ldt) {
  Ctx ctx = make_ctx(h);
  ComplexPlan<real> P;
  CURID_TRY(complex_plan<real>(ctx, m, n, k, sk, nullptr, &P));
  if (!h->ws || P.bytes > h->ws_bytes) return CURID_NO_WORKSPACE;
  CURID_TRY(complex_plan<real>(ctx, m, n, k, sk, h->ws, &P));
  CURID_TRY(embed_complex<real>(ctx, A, m, n, lda, P.E, 2 * n));
  curid_sketch sk2 = sk;
  if (P.d.randomized) {
    const int64_t l = k + sk.p;
    CURID_TRY(gaussian_fill<real>(ctx, l, 2 * m, sk.seed, P.Ge, 2 * m));
    CURID_TRY(embed_complex<real>(ctx, P.Ge, l, m, m, P.Om, 2 * m));
    sk2.p = 2 * sk.p;
    sk2.omega = P.Om;
  }
  const int64_t ldtp = std::max<int64_t>(1, 2 * (n - k));
  Outputs o{P.Jp, P.Tp, ldtp, P.Ip, nullptr, 0, P.Up, nullptr, nullptr};
  CURID_TRY(run<real>(h, Op::Cur, P.E, P.d, 0.0, sk2, o, h->ws, P.run_bytes));
  ctx.status = reinterpret_cast<StatusBlock*>(h->ws);
  CURID_TRY(extract_pivots(ctx, P.Jp, k, n, J, true));
  CURID_TRY(extract_pivots(ctx, P.Ip, k, m, I, false));
  CURID_TRY(extract_u(ctx, P.Up, P.Jp, P.Ip, k, U));
  if (T && n - k > 0) CURID_TRY(extract_t<real>(ctx, P.Tp, ldtp, P.Jp, k, n - k, T, ldt));
  return CURID_OK;
}

// Truncated-SVD T (Section 4.1): S11 = U diag(sigma) V^T by one-sided
// Jacobi, singular values below rtol * sigma_1 dropped, T = V D^+ U^T S12.
// With the Jacobi output W^T = diag(sigma) U^T (rows), B = W^T S12 has rows
// sigma_i u_i^T S12; scaling row i by 1 / sigma_i^2 (or 0) and multiplying by
// V gives T.
template <typename real>
struct TsvdPlan {
  StatusBlock* status = nullptr;
  real* S11 = nullptr;   // k x k
  real* S12 = nullptr;   // k x (n - k)
  real* Wt = nullptr;    // k x k
  real* Vt = nullptr;    // k x k
  real* B = nullptr;     // k x (n - k)
  real* f = nullptr;     // k
  int* rot = nullptr;    // sweep counters
  real* partial = nullptr;
  size_t partial_cap = 0;
  size_t bytes = 0;
};

template <typename real>
void tsvd_plan(const Ctx& ctx, int64_t n, int k, void* base, TsvdPlan<real>* P) {
  Carver cv(base);
  const int64_t r = std::max<int64_t>(1, n - k);
  P->status = cv.take<StatusBlock>(1);
  P->S11 = cv.take<real>((size_t)k * k);
  P->S12 = cv.take<real>((size_t)k * r);
  P->Wt = cv.take<real>((size_t)k * k);
  P->Vt = cv.take<real>((size_t)k * k);
  P->B = cv.take<real>((size_t)k * r);
  P->f = cv.take<real>((size_t)k);
  P->rot = cv.take<int>(64);
  const size_t part = gemm_partial_elems<real>(k, r, k, ctx.num_sms);
  P->partial_cap = part;
  P->partial = part ? cv.take<real>(part) : nullptr;
  P->bytes = cv.used + 256;
}

template <typename real>
curid_status tsvd_run(curid_handle* h, const real* S, int64_t lds, const int32_t* J, int64_t n,
                      int k, double rtol, real* T, int64_t ldt) {
  Ctx ctx = make_ctx(h);
  if (!jacobi_svd_fits<real>(k)) return CURID_UNSUPPORTED;
  TsvdPlan<real> P;
  tsvd_plan<real>(ctx, n, k, nullptr, &P);
  if (!h->ws || P.bytes > h->ws_bytes) return CURID_NO_WORKSPACE;
  tsvd_plan<real>(ctx, n, k, h->ws, &P);
  ctx.status = P.status;
  PhaseScope ps(h, CURID_PHASE_T);
  CURID_CUDA(cudaMemsetAsync(P.status, 0, sizeof(StatusBlock), ctx.stream));
  CURID_TRY(split_s<real>(ctx, S, lds, J, k, n, P.S11, P.S12));
  CURID_TRY(transpose2d<real>(ctx, P.S11, k, P.Wt, k, k, k));
  CURID_TRY(identity_fill<real>(ctx, P.Vt, k));
  CURID_TRY(jacobi_svd<real>(ctx, k, P.Wt, P.Vt, P.rot));
  if (n - k <= 0) return CURID_OK;
  CURID_TRY(tsvd_filter<real>(ctx, k, P.Wt, rtol, P.f));
  CURID_TRY(gemm<real>(ctx, false, false, k, n - k, k, real(1), P.Wt, k, P.S12, n - k, real(0),
                       P.B, n - k, P.partial, P.partial_cap));
  CURID_TRY(scale_rows<real>(ctx, P.B, n - k, k, n - k, P.f));
  return gemm<real>(ctx, true, false, k, n - k, k, real(1), P.Vt, k, P.B, n - k, real(0), T, ldt,
                    P.partial, P.partial_cap);
}

}  // namespace

extern "C" {

curid_status curid_create(curid_handle** handle, int device) {
  if (!handle) return CURID_INVALID_ARG;
  *handle = nullptr;
  int count = 0;
  if (cudaGetDeviceCount(&count) != cudaSuccess) return CURID_CUDA_ERROR;
  if (device < 0 || device >= count) return CURID_INVALID_ARG;
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) return CURID_CUDA_ERROR;
  if (!prop.cooperativeLaunch) return CURID_UNSUPPORTED;
  curid_handle* h = new (std::nothrow) curid_handle();
  if (!h) return CURID_INVALID_ARG;
  h->device = device;
  h->num_sms = prop.multiProcessorCount;
  h->smem_optin = prop.sharedMemPerBlockOptin;
  *handle = h;
  return CURID_OK;
}

curid_status curid_destroy(curid_handle* handle) {
  if (handle) {
    for (cudaEvent_t e : handle->pool) cudaEventDestroy(e);
  }
  delete handle;
  return CURID_OK;
}

curid_status curid_profile(curid_handle* handle, int enable) {
  if (!handle) return CURID_INVALID_ARG;
  handle->profiling = enable ? 1 : 0;
  handle->recs.clear();
  handle->pool_used = 0;
  handle->launches = 0;
  return CURID_OK;
}

curid_status curid_profile_read(curid_handle* handle, double* ms, int* calls,
                                long long* launches) {
  if (!handle) return CURID_INVALID_ARG;
  DeviceGuard g(handle->device);
  if (!g.ok) return CURID_CUDA_ERROR;
  if (cudaStreamSynchronize(handle->stream) != cudaSuccess) return CURID_CUDA_ERROR;
  for (int p = 0; p < CURID_NUM_PHASES; ++p) {
    if (ms) ms[p] = 0.0;
    if (calls) calls[p] = 0;
  }
  for (const curid_phase_rec& r : handle->recs) {
    float t = 0.f;
    if (cudaEventElapsedTime(&t, r.start, r.stop) != cudaSuccess) return CURID_CUDA_ERROR;
    if (r.phase >= 0 && r.phase < CURID_NUM_PHASES) {
      if (ms) ms[r.phase] += t;
      if (calls) calls[r.phase] += 1;
    }
  }
  if (launches) *launches = handle->launches;
  handle->recs.clear();
  handle->pool_used = 0;
  handle->launches = 0;
  return CURID_OK;
}

curid_status curid_set_stream(curid_handle* handle, void* stream) {
  if (!handle) return CURID_INVALID_ARG;
  handle->stream = static_cast<cudaStream_t>(stream);
  return CURID_OK;
}

curid_status curid_set_timeout(curid_handle* handle, long long cycles) {
  if (!handle || cycles < 0) return CURID_INVALID_ARG;
  handle->spin = cycles > 0 ? cycles : kSpinBudget;
  return CURID_OK;
}

curid_status curid_set_concurrency(curid_handle* handle, int inflight) {
  if (!handle || inflight < 1) return CURID_INVALID_ARG;
  handle->concurrency = inflight;
  return CURID_OK;
}

curid_status curid_set_workspace(curid_handle* handle, void* ptr, size_t bytes) {
  if (!handle) return CURID_INVALID_ARG;
  if (ptr && (reinterpret_cast<uintptr_t>(ptr) & 255)) return CURID_INVALID_ARG;
  handle->ws = static_cast<char*>(ptr);
  handle->ws_bytes = ptr ? bytes : 0;
  return CURID_OK;
}

curid_status curid_workspace_size(curid_handle* handle, curid_dtype dtype, int64_t m, int64_t n,
                                  int k, curid_sketch sk, size_t* bytes) {
  if (!handle || !bytes) return CURID_INVALID_ARG;
  // adaptive rank (k == 0): room for every rank up to min(m, n), or with a
  // sketch for the largest sample the search may reach (l = min(m, n, 4096))
  if (k == 0 && m > 0 && n > 0) {
    if (sk.p >= 0) {
      if (sk.omega || sk.srft_rows || sk.srft_signs) return CURID_UNSUPPORTED;
      const int64_t cap = adaptive_l_cap(m, n);
      if (sk.p >= cap) return CURID_INVALID_ARG;
      k = (int)(cap - sk.p);
    } else {
      if (dtype == CURID_BF16) return CURID_UNSUPPORTED;
      k = (int)std::min<int64_t>(m, n);
    }
  }
  Dims d;
  int dummy = 1;
  CURID_TRY(check_common(handle, dtype, &dummy, m, n, n, k, 0.0, sk, &d));
  Ctx ctx = host_ctx(handle);
  const bool gen = d.randomized && sk.omega == nullptr && sk.srft_rows == nullptr;
  Dims dt;
  const bool row_ok = check_common(handle, dtype, &dummy, n, m, m, k, 0.0, sk, &dt) == CURID_OK;
  auto size_for = [&](auto tag) -> curid_status {
    using real = decltype(tag);
    Plan<real> P;
    CURID_TRY(make_plan<real>(ctx, Op::CurCorrected, d, gen, true, nullptr, &P));
    size_t b = P.bytes;
    if (row_ok) {
      Plan<real> Pt;
      if (make_plan<real>(ctx, Op::IdCol, dt, gen, true, nullptr, &Pt) == CURID_OK)
        b = std::max(b, (((size_t)m * n * sizeof(real) + 255) & ~size_t(255)) + Pt.bytes);
    }
    *bytes = b;
    return CURID_OK;
  };
  if (dtype == CURID_F64) return size_for(double{});
  return size_for(float{});
}

curid_status curid_last_status(curid_handle* handle, int* k_out) {
  if (!handle) return CURID_INVALID_ARG;
  if (!handle->ws) return CURID_NO_WORKSPACE;
  DeviceGuard g(handle->device);
  if (!g.ok) return CURID_CUDA_ERROR;
  StatusBlock sb;
  if (cudaStreamSynchronize(handle->stream) != cudaSuccess) return CURID_CUDA_ERROR;
  if (cudaMemcpy(&sb, handle->ws, sizeof(sb), cudaMemcpyDeviceToHost) != cudaSuccess)
    return CURID_CUDA_ERROR;
  if (k_out) *k_out = sb.k_eff;
  if (sb.flags & FLAG_TIMEOUT) return CURID_TIMEOUT;
  if (sb.flags & FLAG_NONFINITE) return CURID_NONFINITE;
  if (sb.flags & FLAG_BREAKDOWN) return CURID_BREAKDOWN;
  if (sb.flags & FLAG_RANK_DEFICIENT) return CURID_RANK_DEFICIENT;
  return CURID_OK;
}

curid_status curid_gaussian(curid_handle* handle, curid_dtype dtype, int64_t rows, int64_t cols,
                            uint64_t seed, void* out) {
  if (!handle || !out || rows < 0 || cols < 0) return CURID_INVALID_ARG;
  return dispatch(handle, [&]() -> curid_status {
    Ctx ctx = make_ctx(handle);
    PhaseScope ps(handle, CURID_PHASE_OMEGA);
    if (dtype == CURID_F64)
      return gaussian_fill<double>(ctx, rows, cols, seed, (double*)out, cols);
    if (dtype == CURID_F32) return gaussian_fill<float>(ctx, rows, cols, seed, (float*)out, cols);
    return CURID_INVALID_ARG;
  });
}

curid_status curid_srft_omega(curid_handle* handle, curid_dtype dtype, int64_t m, int64_t l,
                              const int32_t* rows, const int8_t* signs, void* omega,
                              int64_t ldo) {
  if (!handle || !rows || !signs || !omega || m < 1 || l < 1 || ldo < m)
    return CURID_INVALID_ARG;
  return dispatch(handle, [&]() -> curid_status {
    Ctx ctx = make_ctx(handle);
    PhaseScope ps(handle, CURID_PHASE_OMEGA);
    if (dtype == CURID_F64)
      return srft_fill<double>(ctx, m, l, rows, signs, static_cast<double*>(omega), ldo);
    if (dtype == CURID_F32)
      return srft_fill<float>(ctx, m, l, rows, signs, static_cast<float*>(omega), ldo);
    return CURID_UNSUPPORTED;
  });
}

curid_status curid_srft_draw(curid_handle* handle, int64_t m, int64_t l, uint64_t seed,
                             int32_t* rows, int8_t* signs) {
  if (!handle || !rows || !signs || m < 1 || l < 1 || l > m) return CURID_INVALID_ARG;
  return dispatch(handle, [&]() -> curid_status {
    Ctx ctx = make_ctx(handle);
    PhaseScope ps(handle, CURID_PHASE_OMEGA);
    return srft_draw(ctx, m, l, seed, rows, signs);
  });
}

curid_status curid_srft_sketch(curid_handle* handle, curid_dtype dtype, const void* A,
                               int64_t m, int64_t n, int64_t lda, int64_t l,
                               const int32_t* rows, const int8_t* signs, void* Y, int64_t ldy) {
  if (!handle || !A || !rows || !signs || !Y || m < 1 || n < 1 || l < 1 || lda < n || ldy < n)
    return CURID_INVALID_ARG;
  return dispatch(handle, [&]() -> curid_status {
    Ctx ctx = make_ctx(handle);
    PhaseScope ps(handle, CURID_PHASE_SKETCH);
    switch (dtype) {
      case CURID_F64:
        return srft_apply<double>(ctx, static_cast<const double*>(A), m, n, lda, l, rows, signs,
                                  static_cast<double*>(Y), ldy);
      case CURID_F32:
        return srft_apply<float>(ctx, static_cast<const float*>(A), m, n, lda, l, rows, signs,
                                 static_cast<float*>(Y), ldy);
      default:
        return CURID_UNSUPPORTED;
    }
  });
}

curid_status curid_sketch_matrix(curid_handle* handle, curid_dtype dtype, const void* A,
                                 int64_t m, int64_t n, int64_t lda, int l, int q, int tf32,
                                 const void* omega, void* Y) {
  if (!handle || !A || !omega || !Y || m <= 0 || n <= 0 || lda < n || l <= 0 || q < 0)
    return CURID_INVALID_ARG;
  if (l > std::min(m, n)) return CURID_INVALID_ARG;
  if (tf32 && dtype != CURID_F32) return CURID_INVALID_ARG;
  const bool bf16 = dtype == CURID_BF16;
  if (bf16 && ((lda & 7) || (reinterpret_cast<uintptr_t>(A) & 15))) return CURID_UNSUPPORTED;
  return dispatch(handle, [&]() -> curid_status {
    Ctx ctx = make_ctx(handle);
    Dims d{m, n, lda, 1, l, true, q, tf32 != 0, bf16};
    auto go = [&](auto tag) -> curid_status {
      using real = decltype(tag);
      Plan<real> P;
      CURID_TRY(make_plan<real>(ctx, Op::IdCol, d, false, false, nullptr, &P));
      if (!handle->ws || P.bytes > handle->ws_bytes) return CURID_NO_WORKSPACE;
      CURID_TRY(make_plan<real>(ctx, Op::IdCol, d, false, false, handle->ws, &P));
      ctx.status = P.status;
      CURID_CUDA(cudaMemsetAsync(P.status, 0, sizeof(StatusBlock), ctx.stream));
      const real* Om = static_cast<const real*>(omega);
      int64_t ldo = m;
      if (tf32 && (m & 3)) {
        // caller's Omega rows are not 16-byte aligned: copy with a padded stride
        CURID_TRY(copy2d<real>(ctx, Om, m, P.omega, pad4(m), l, m));
        Om = P.omega;
        ldo = pad4(m);
      }
      real* cur;
      CURID_TRY(sketch<real>(handle, ctx, P, A, m, n, lda, l, q, tf32 != 0, bf16, Om, ldo,
                             &cur));
      return copy2d<real>(ctx, cur, pad4(n), static_cast<real*>(Y), n, l, n);
    };
    if (dtype == CURID_F64) return go(double{});
    if (dtype == CURID_F32 || bf16) return go(float{});
    return CURID_INVALID_ARG;
  });
}

curid_status curid_cpqr(curid_handle* handle, curid_dtype dtype, const void* Y, int64_t l,
                        int64_t n, int64_t ldy, int k, double tol, int32_t* J, void* S) {
  if (!handle || !Y || !J || !S || l <= 0 || n <= 0 || ldy < n || k < 0 || tol < 0)
    return CURID_INVALID_ARG;
  if (k == 0 && !(tol > 0)) return CURID_INVALID_ARG;
  if (k > std::min(l, n)) return CURID_INVALID_ARG;
  const int k_max = k > 0 ? k : (int)std::min(l, n);
  return dispatch(handle, [&]() -> curid_status {
    Ctx ctx = make_ctx(handle);
    auto go = [&](auto tag) -> curid_status {
      using real = decltype(tag);
      int grid;
      size_t smem;
      CURID_TRY(cpqr_plan<real>(ctx, l, n, &grid, &smem));
      Carver cv(nullptr);
      StatusBlock* st = cv.take<StatusBlock>(1);
      CpqrScratch cs;
      cpqr_carve<real>(cv, ctx, l, n, &cs);
      if (!handle->ws || cv.used > handle->ws_bytes) return CURID_NO_WORKSPACE;
      Carver cw(handle->ws);
      st = cw.take<StatusBlock>(1);
      cpqr_carve<real>(cw, ctx, l, n, &cs);
      ctx.status = st;
      CURID_CUDA(cudaMemsetAsync(st, 0, sizeof(StatusBlock), ctx.stream));
      PhaseScope ps(handle, CURID_PHASE_CPQR_COL);
      return cpqr_run<real>(ctx, static_cast<const real*>(Y), l, n, ldy, k_max, k > 0 ? 0.0 : tol,
                            J, static_cast<real*>(S), n, cs, 0);
    };
    if (dtype == CURID_F64) return go(double{});
    if (dtype == CURID_F32) return go(float{});
    return CURID_INVALID_ARG;
  });
}

curid_status curid_id_col(curid_handle* handle, curid_dtype dtype, const void* A, int64_t m,
                          int64_t n, int64_t lda, int k, double tol, curid_sketch sk, int32_t* J,
                          void* T, int64_t ldt) {
  CURID_TRY(resolve_rank(handle, dtype, A, m, n, lda, &k, tol, &sk, J));
  if (k == 0 && tol > 0) return CURID_OK;
  Dims d;
  CURID_TRY(check_common(handle, dtype, A, m, n, lda, k, tol, sk, &d));
  if (!J || !T || ldt < std::max<int64_t>(1, n - k)) return CURID_INVALID_ARG;
  Outputs o{J, T, ldt, nullptr, nullptr, 0, nullptr, nullptr, nullptr};
  return dispatch(handle, [&]() -> curid_status {
    if (dtype == CURID_F64)
      return run<double>(handle, Op::IdCol, (const double*)A, d, 0.0, sk, o, handle->ws,
                         handle->ws_bytes);
    return run<float>(handle, Op::IdCol, (const float*)A, d, 0.0, sk, o, handle->ws,
                      handle->ws_bytes);
  });
}

curid_status curid_id_row(curid_handle* handle, curid_dtype dtype, const void* A, int64_t m,
                          int64_t n, int64_t lda, int k, double tol, curid_sketch sk, int32_t* I,
                          void* TW, int64_t ldtw) {
  // Row ID = column ID of A^* (Remark 2.1): A^T is formed in the workspace
  // (n x m, leading dimension m) and the column-ID pipeline runs on it.
  Dims d0;
  CURID_TRY(check_common(handle, dtype, A, m, n, lda, k, tol, sk, &d0));
  if (dtype == CURID_BF16) return CURID_UNSUPPORTED;
  Dims d;
  CURID_TRY(check_common(handle, dtype, A, n, m, m, k, tol, sk, &d));
  if (!I || !TW || ldtw < std::max<int64_t>(1, m - k)) return CURID_INVALID_ARG;
  Outputs o{I, TW, ldtw, nullptr, nullptr, 0, nullptr, nullptr, nullptr};
  return dispatch(handle, [&]() -> curid_status {
    Ctx ctx = make_ctx(handle);
    auto go = [&](auto tag) -> curid_status {
      using real = decltype(tag);
      // the pipeline's buffers (status block first) at the start, A^T after them
      Plan<real> P;
      CURID_TRY(make_plan<real>(ctx, Op::IdCol, d, d.randomized && sk.omega == nullptr, true,
                                nullptr, &P));
      const size_t off = (P.bytes + 255) & ~size_t(255);
      if (!handle->ws || off + (size_t)m * n * sizeof(real) > handle->ws_bytes)
        return CURID_NO_WORKSPACE;
      real* At = reinterpret_cast<real*>(handle->ws + off);
      CURID_TRY(transpose2d<real>(ctx, static_cast<const real*>(A), lda, At, m, m, n));
      return run<real>(handle, Op::IdCol, At, d, 0.0, sk, o, handle->ws, off);
    };
    if (dtype == CURID_F64) return go(double{});
    return go(float{});
  });
}

curid_status curid_tsid(curid_handle* handle, curid_dtype dtype, const void* A, int64_t m,
                        int64_t n, int64_t lda, int k, double tol, curid_sketch sk, int32_t* J,
                        void* T, int64_t ldt, int32_t* I, void* TW, int64_t ldtw) {
  CURID_TRY(resolve_rank(handle, dtype, A, m, n, lda, &k, tol, &sk, J));
  if (k == 0 && tol > 0) return rank_zero_rows(handle, I, m);
  Dims d;
  CURID_TRY(check_common(handle, dtype, A, m, n, lda, k, tol, sk, &d));
  if (!J || !T || !I || !TW || ldt < std::max<int64_t>(1, n - k) ||
      ldtw < std::max<int64_t>(1, m - k))
    return CURID_INVALID_ARG;
  Outputs o{J, T, ldt, I, TW, ldtw, nullptr, nullptr, nullptr};
  return dispatch(handle, [&]() -> curid_status {
    if (dtype == CURID_F64)
      return run<double>(handle, Op::Tsid, (const double*)A, d, 0.0, sk, o, handle->ws,
                         handle->ws_bytes);
    return run<float>(handle, Op::Tsid, (const float*)A, d, 0.0, sk, o, handle->ws,
                      handle->ws_bytes);
  });
}

curid_status curid_cur(curid_handle* handle, curid_dtype dtype, const void* A, int64_t m,
                       int64_t n, int64_t lda, int k, double tol, curid_sketch sk, int32_t* J,
                       int32_t* I, double* U, void* C, void* R, void* T, int64_t ldt, void* TW,
                       int64_t ldtw) {
  CURID_TRY(resolve_rank(handle, dtype, A, m, n, lda, &k, tol, &sk, J));
  if (k == 0 && tol > 0) return rank_zero_rows(handle, I, m);
  Dims d;
  CURID_TRY(check_common(handle, dtype, A, m, n, lda, k, tol, sk, &d));
  if (!J || !I || !U) return CURID_INVALID_ARG;
  if (T && ldt < std::max<int64_t>(1, n - k)) return CURID_INVALID_ARG;
  if (TW && ldtw < std::max<int64_t>(1, m - k)) return CURID_INVALID_ARG;
  Outputs o{J, T, ldt, I, TW, ldtw, U, C, R};
  return dispatch(handle, [&]() -> curid_status {
    if (dtype == CURID_F64)
      return run<double>(handle, Op::Cur, (const double*)A, d, 0.0, sk, o, handle->ws,
                         handle->ws_bytes);
    return run<float>(handle, Op::Cur, (const float*)A, d, 0.0, sk, o, handle->ws,
                      handle->ws_bytes);
  });
}

curid_status curid_cur_corrected(curid_handle* handle, curid_dtype dtype, const void* A,
                                 int64_t m, int64_t n, int64_t lda, int k, double tol,
                                 curid_sketch sk, int32_t* J, int32_t* I, double* U, void* C,
                                 void* R, void* T, int64_t ldt, void* TW, int64_t ldtw) {
  CURID_TRY(resolve_rank(handle, dtype, A, m, n, lda, &k, tol, &sk, J));
  if (k == 0 && tol > 0) return rank_zero_rows(handle, I, m);
  Dims d;
  CURID_TRY(check_common(handle, dtype, A, m, n, lda, k, tol, sk, &d));
  if (!J || !I || !U) return CURID_INVALID_ARG;
  if (T && ldt < std::max<int64_t>(1, n - k)) return CURID_INVALID_ARG;
  if (TW && ldtw < std::max<int64_t>(1, m - k)) return CURID_INVALID_ARG;
  Outputs o{J, T, ldt, I, TW, ldtw, U, C, R};
  return dispatch(handle, [&]() -> curid_status {
    if (dtype == CURID_F64)
      return run<double>(handle, Op::CurCorrected, (const double*)A, d, 0.0, sk, o, handle->ws,
                         handle->ws_bytes);
    return run<float>(handle, Op::CurCorrected, (const float*)A, d, 0.0, sk, o, handle->ws,
                      handle->ws_bytes);
  });
}

// Sparse A: Dims of the randomized CUR-ID (fixed rank, p >= 0; the
// products run on the CUDA cores, so the tf32 flag is not used).
static curid_status sparse_dims(curid_handle* h, curid_dtype dt, int64_t m, int64_t n,
                                const curid_sparse* A, int k, const curid_sketch& sk,
                                SparseA* sa, Dims* d) {
  if (!h || !A || (dt != CURID_F32 && dt != CURID_F64)) return CURID_INVALID_ARG;
  if (m <= 0 || n <= 0 || m > INT32_MAX || n > INT32_MAX || A->nnz < 0) return CURID_INVALID_ARG;
  if (!A->row_ptr || !A->col_ptr || (A->nnz > 0 && (!A->col_idx || !A->row_val || !A->row_idx ||
                                                    !A->col_val)))
    return CURID_INVALID_ARG;
  if (sk.p < 0 || sk.q < 0 || k < 1 || k + (int64_t)sk.p > std::min(m, n))
    return CURID_INVALID_ARG;
  if (sk.srft_rows || sk.srft_signs) return CURID_UNSUPPORTED;
  *sa = SparseA{A->nnz, A->row_ptr, A->col_idx, A->row_val, A->col_ptr, A->row_idx, A->col_val};
  d->m = m;
  d->n = n;
  d->lda = n;
  d->k = k;
  d->l = k + sk.p;
  d->randomized = true;
  d->q = sk.q;
  d->tf32 = false;
  d->bf16 = false;
  d->sp = sa;
  return CURID_OK;
}

curid_status curid_sparse_workspace_size(curid_handle* handle, curid_dtype dtype, int64_t m,
                                         int64_t n, int k, curid_sketch sk, size_t* bytes) {
  if (!bytes) return CURID_INVALID_ARG;
  const int64_t ptr0 = 0;
  curid_sparse dummy{0, &ptr0, nullptr, nullptr, &ptr0, nullptr, nullptr};
  SparseA sa;
  Dims d;
  CURID_TRY(sparse_dims(handle, dtype, m, n, &dummy, k, sk, &sa, &d));
  Ctx ctx = host_ctx(handle);
  const bool gen = sk.omega == nullptr;
  if (dtype == CURID_F64) {
    Plan<double> P;
    CURID_TRY(make_plan<double>(ctx, Op::CurCorrected, d, gen, true, nullptr, &P));
    *bytes = P.bytes;
  } else {
    Plan<float> P;
    CURID_TRY(make_plan<float>(ctx, Op::CurCorrected, d, gen, true, nullptr, &P));
    *bytes = P.bytes;
  }
  return CURID_OK;
}

curid_status curid_cur_sparse(curid_handle* handle, curid_dtype dtype, int64_t m, int64_t n,
                              const curid_sparse* A, int k, curid_sketch sk, int corrected,
                              int32_t* J, int32_t* I, double* U, void* C, void* R, void* T,
                              int64_t ldt, void* TW, int64_t ldtw) {
  SparseA sa;
  Dims d;
  CURID_TRY(sparse_dims(handle, dtype, m, n, A, k, sk, &sa, &d));
  if (!J || !I || !U) return CURID_INVALID_ARG;
  if (T && ldt < std::max<int64_t>(1, n - k)) return CURID_INVALID_ARG;
  if (TW && ldtw < std::max<int64_t>(1, m - k)) return CURID_INVALID_ARG;
  sk.tf32 = 0;
  Outputs o{J, T, ldt, I, TW, ldtw, U, C, R};
  const Op op = corrected ? Op::CurCorrected : Op::Cur;
  return dispatch(handle, [&]() -> curid_status {
    if (dtype == CURID_F64)
      return run<double>(handle, op, nullptr, d, 0.0, sk, o, handle->ws, handle->ws_bytes);
    return run<float>(handle, op, nullptr, d, 0.0, sk, o, handle->ws, handle->ws_bytes);
  });
}

static curid_status complex_check(curid_handle* h, curid_dtype dt, int64_t m, int64_t n,
                                  int k, const curid_sketch& sk) {
  if (!h || (dt != CURID_F32 && dt != CURID_F64)) return CURID_INVALID_ARG;
  if (m <= 0 || n <= 0 || 2 * m > INT32_MAX || 2 * n > INT32_MAX) return CURID_INVALID_ARG;
  if (k < 1 || k > std::min(m, n) || sk.q < 0) return CURID_INVALID_ARG;
  if (sk.p >= 0 && k + (int64_t)sk.p > std::min(m, n)) return CURID_INVALID_ARG;
  if (sk.p < 0 && sk.q > 0) return CURID_INVALID_ARG;
  if (sk.tf32 && dt != CURID_F32) return CURID_INVALID_ARG;
  // the sample is drawn from the seed
  if (sk.omega || sk.srft_rows || sk.srft_signs) return CURID_UNSUPPORTED;
  return CURID_OK;
}

curid_status curid_complex_workspace_size(curid_handle* handle, curid_dtype dtype, int64_t m,
                                          int64_t n, int k, curid_sketch sk, size_t* bytes) {
  if (!bytes) return CURID_INVALID_ARG;
  CURID_TRY(complex_check(handle, dtype, m, n, k, sk));
  Ctx ctx = host_ctx(handle);
  if (dtype == CURID_F64) {
    ComplexPlan<double> P;
    CURID_TRY(complex_plan<double>(ctx, m, n, k, sk, nullptr, &P));
    *bytes = P.bytes;
  } else {
    ComplexPlan<float> P;
    CURID_TRY(complex_plan<float>(ctx, m, n, k, sk, nullptr, &P));
    *bytes = P.bytes;
  }
  return CURID_OK;
}

curid_status curid_cur_complex(curid_handle* handle, curid_dtype dtype, const void* A, int64_t m,
                               int64_t n, int64_t lda, int k, curid_sketch sk, int32_t* J,
                               int32_t* I, double* U, void* T, int64_t ldt) {
  CURID_TRY(complex_check(handle, dtype, m, n, k, sk));
  if (!A || !J || !I || !U || lda < n) return CURID_INVALID_ARG;
  if (T && ldt < std::max<int64_t>(1, n - k)) return CURID_INVALID_ARG;
  return dispatch(handle, [&]() -> curid_status {
    if (dtype == CURID_F64)
      return cur_complex_run<double>(handle, static_cast<const double*>(A), m, n, lda, k, sk, J,
                                     I, U, static_cast<double*>(T), ldt);
    return cur_complex_run<float>(handle, static_cast<const float*>(A), m, n, lda, k, sk, J, I, U,
                                  static_cast<float*>(T), ldt);
  });
}

curid_status curid_interp_tsvd_workspace_size(curid_handle* handle, curid_dtype dtype, int64_t n,
                                              int k, size_t* bytes) {
  if (!handle || !bytes || n < 1 || k < 1 || k > n) return CURID_INVALID_ARG;
  Ctx ctx = host_ctx(handle);
  if (dtype == CURID_F64) {
    TsvdPlan<double> P;
    tsvd_plan<double>(ctx, n, k, nullptr, &P);
    *bytes = P.bytes;
  } else if (dtype == CURID_F32) {
    TsvdPlan<float> P;
    tsvd_plan<float>(ctx, n, k, nullptr, &P);
    *bytes = P.bytes;
  } else {
    return CURID_UNSUPPORTED;
  }
  return CURID_OK;
}

curid_status curid_interp_tsvd(curid_handle* handle, curid_dtype dtype, const void* S,
                               int64_t lds, const int32_t* J, int64_t n, int k, double rtol,
                               void* T, int64_t ldt) {
  if (!handle || !S || !J || !T || n < 1 || k < 1 || k > n || lds < n || !(rtol >= 0) ||
      !(rtol < 1) || ldt < std::max<int64_t>(1, n - k))
    return CURID_INVALID_ARG;
  return dispatch(handle, [&]() -> curid_status {
    if (dtype == CURID_F64)
      return tsvd_run<double>(handle, static_cast<const double*>(S), lds, J, n, k, rtol,
                              static_cast<double*>(T), ldt);
    if (dtype == CURID_F32)
      return tsvd_run<float>(handle, static_cast<const float*>(S), lds, J, n, k, rtol,
                             static_cast<float*>(T), ldt);
    return CURID_UNSUPPORTED;
  });
}

curid_status curid_interp_tikhonov_workspace_size(curid_handle* handle, curid_dtype dtype,
                                                  int64_t n, int k, size_t* bytes) {
  if (!handle || !bytes || n < 1 || k < 1 || k > n) return CURID_INVALID_ARG;
  Ctx ctx = host_ctx(handle);
  if (dtype == CURID_F64) {
    TikPlan<double> P;
    tik_plan<double>(ctx, n, k, nullptr, &P);
    *bytes = P.bytes;
  } else if (dtype == CURID_F32) {
    TikPlan<float> P;
    tik_plan<float>(ctx, n, k, nullptr, &P);
    *bytes = P.bytes;
  } else {
    return CURID_UNSUPPORTED;
  }
  return CURID_OK;
}

curid_status curid_interp_tikhonov(curid_handle* handle, curid_dtype dtype, const void* S,
                                   int64_t lds, const int32_t* J, int64_t n, int k, double lam,
                                   void* T, int64_t ldt) {
  if (!handle || !S || !J || !T || n < 1 || k < 1 || k > n || lds < n || !(lam > 0) ||
      !std::isfinite(lam) || ldt < std::max<int64_t>(1, n - k))
    return CURID_INVALID_ARG;
  return dispatch(handle, [&]() -> curid_status {
    if (dtype == CURID_F64)
      return tikhonov_run<double>(handle, static_cast<const double*>(S), lds, J, n, k, lam,
                                  static_cast<double*>(T), ldt);
    if (dtype == CURID_F32)
      return tikhonov_run<float>(handle, static_cast<const float*>(S), lds, J, n, k, lam,
                                 static_cast<float*>(T), ldt);
    return CURID_UNSUPPORTED;
  });
}

}  // extern "C"
