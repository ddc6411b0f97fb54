// Internal interfaces between the C-ABI layer (curid_api.cu) and the
// kernels.  Nothing here is exported from the shared library.
#pragma once

#include <algorithm>

#include <cuda_bf16.h>

#include "common.cuh"

namespace curid {

struct Ctx {
  cudaStream_t stream;
  int num_sms;
  size_t smem_optin;
  StatusBlock* status;          // device
  long long* launches = nullptr;  // host counter of kernel launches (profiling)
  long long spin = kSpinBudget;   // bound of inter-block waits, SM clock cycles
  int concurrency = 1;            // decompositions the caller keeps in flight
};

// After a kernel launch: report a launch error, count the launch.
#define CURID_LAUNCHED(ctx)                                  \
  do {                                                       \
    CURID_CUDA(cudaGetLastError());                          \
    if ((ctx).launches) ++*(ctx).launches;                   \
  } while (0)

// ---- dense products (gemm_simt.cu) ----------------------------------------
template <typename real>
int gemm_splits(int64_t M, int64_t N, int64_t K, int num_sms);
template <typename real>
size_t gemm_partial_elems(int64_t M, int64_t N, int64_t K, int num_sms);
template <typename real>
curid_status gemm(const Ctx& ctx, bool ta, bool tb, int64_t M, int64_t N, int64_t K,
                  real alpha, const real* A, int64_t lda, const real* B, int64_t ldb,
                  real beta, real* C, int64_t ldc, real* partial, size_t partial_cap);

// ---- tensor-core products (gemm_tc.cu): TF32 inputs, FP32 accumulation ----
// C[M x N] = op(A) op(B) with the same op convention as gemm(); returns
// CURID_UNSUPPORTED for shapes or alignments the kernel does not take.
// split_x: the left operand is split into TF32 high and low parts too (three
// MMAs per K step, float32 accuracy for both operands).
curid_status gemm_tf32(const Ctx& ctx, bool ta, bool tb, int64_t M, int64_t N, int64_t K,
                       const float* A, int64_t lda, const float* B, int64_t ldb, float* C,
                       int64_t ldc, float* partial, size_t partial_cap, bool split_x = false);
size_t gemm_tf32_partial_elems(int64_t M, int64_t N, int64_t K, int num_sms);
// BF16 A (gemm_bf16.cu): C[M x N] = X A (tb false; A K x N) or X A^T (tb
// true; A N x K), X float32 (M x K) split into BF16 high and low parts in
// `split` (gemm_bf16_split_elems(M, K) bfloat16 values); A's rows 16-byte
// aligned (lda a multiple of 8).
size_t gemm_bf16_split_elems(int64_t M, int64_t K);
curid_status gemm_bf16(const Ctx& ctx, bool tb, int64_t M, int64_t N, int64_t K, const float* X,
                       int64_t ldx, const void* A, int64_t lda, float* C, int64_t ldc,
                       void* split, size_t split_elems);

// ---- truncated CPQR (cpqr.cu) -----------------------------------------------
// Scratch for one CPQR launch (carved from the workspace).
struct CpqrScratch {
  void* slots;       // 2 * G slot records
  void* slot_data;   // 2 * G * l reals
  void* overflow;    // column groups beyond shared memory and registers (or null)
  int* counts;       // G
  int* abort_flag;   // 1
  int grid;          // G
};
template <typename real>
curid_status cpqr_plan(const Ctx& ctx, int64_t l, int64_t n, int* grid, size_t* smem);
template <typename real>
void cpqr_carve(Carver& cv, const Ctx& ctx, int64_t l, int64_t n, CpqrScratch* s);
// which: 0 = column CPQR (status k_done/k_eff), 1 = row CPQR (status k_row)
template <typename real>
curid_status cpqr_run(const Ctx& ctx, const real* Y, int64_t l, int64_t n, int64_t ldy,
                      int k_max, double tol, int32_t* J, real* S, int64_t lds,
                      const CpqrScratch& s, int which);

// ---- small dense factorizations (dense_small.cu) ---------------------------
// Orders up to the one-CTA limits (256 float32, 192 float64) run in one CTA
// with the matrix in shared memory; larger orders, up to kMaxDenseOrder, are
// blocked over diagonal blocks of that size with GEMM updates in between.
constexpr int kMaxDenseOrder = 4096;
template <typename real>
constexpr int kCholBlock() { return sizeof(real) == 4 ? 256 : 192; }
// Inverse of the leading triangle of S (k x k, columns gathered by J) for the
// T solve; rows/columns at and after *k_eff are zeroed.
template <typename real>
curid_status upper_tri_inverse(const Ctx& ctx, const real* S11, int k, const int* k_eff,
                               real* X);
template <typename real>
bool upper_tri_inverse_fits(const Ctx& ctx, int k);
// Cholesky of G + shift*I (shift = rel_shift * trace(G)); the lower factor
// L overwrites G.  Breakdown -> FLAG_BREAKDOWN.
template <typename real>
curid_status cholesky(const Ctx& ctx, real* G, int l, double rel_shift);
// cholesky() then Linv = L^{-1} (l x l, lower triangular); G holds L after.
template <typename real>
curid_status chol_inverse(const Ctx& ctx, real* G, int l, double rel_shift, real* Linv);
// Solve op(T) X = B (T k x k row-major with leading dimension ldt, upper or
// lower, op = transpose when trans) for N columns; B == nullptr means the
// identity (X = op(T)^{-1}).  Rows/columns at or after *kk (if given) are
// an identity block with zero right-hand side.  X may be B itself (same
// pointer and leading dimension) but must not alias T.  Orders above one
// CTA's limit are solved blockwise (trans == false only).
template <typename real>
curid_status tri_solve(const Ctx& ctx, int k, const real* T, int64_t ldt, bool upper, bool trans,
                       const real* B, int64_t ldb, real* X, int64_t ldx, int64_t N,
                       const int* kk);
template <typename real>
bool tri_solve_fits(const Ctx& ctx, int k);
template <typename real>
bool chol_inverse_fits(const Ctx& ctx, int l);
// Row orthonormalisation without pivoting (Section 5.3) by Cholesky-QR
// passes: G = X X^T, G + shift I = L L^T, X <- L^{-1} X, the first pass
// shifted (float32: 1e-5 trace(G), float64: 1e-13 trace(G)).  Three passes
// give rows orthonormal to working precision; two give a lower-triangular
// multiple of them with condition number near 1, which is all a product
// whose result is orthonormalised again needs.  X is r x c with leading
// dimension ld; each pass writes out of place, and on return *X points at
// the result and *tmp at the other buffer.  G: r x r scratch.
// With tc_gram (float32 only) each Gram matrix is formed on the TF32 tensor
// cores at float32 accuracy (gram_tf32); with li as well (r x pad4(r)
// scratch) the apply X <- L^{-1} X runs on the tensor cores too, through an
// explicit L^{-1}.
template <typename real>
curid_status chol_qr_rows(const Ctx& ctx, real** X, real** tmp, int64_t r, int64_t c, int64_t ld,
                          real* G, real* partial, size_t partial_cap, int passes = 3,
                          bool tc_gram = false, real* li = nullptr);
// G (r x r, leading dimension r) = X X^T on the TF32 tensor cores, both
// operands split into TF32 parts and float32 remainders in shared memory.
curid_status gram_tf32(const Ctx& ctx, const float* X, int64_t r, int64_t c, int64_t ld, float* G,
                       float* partial, size_t partial_cap);
// C (float64) = A B^T with float64 accumulation; A M x K, B N x K.
template <typename real>
curid_status gemm_nt_f64acc(const Ctx& ctx, int64_t M, int64_t N, int64_t K, const real* A,
                            int64_t lda, const real* B, int64_t ldb, double* C, int64_t ldc);

// ---- gathers and copies (gather.cu) ------------------------------------------
template <typename real>
curid_status gather_cols(const Ctx& ctx, const real* A, int64_t m, int64_t n, int64_t lda,
                         const int32_t* J, int k, real* out, int64_t ldo, bool transpose);
template <typename real>
curid_status gather_rows(const Ctx& ctx, const real* A, int64_t m, int64_t n, int64_t lda,
                         const int32_t* I, int k, real* out, int64_t ldo);
// the same gathers and a 2-D copy with a change of element type (instantiated
// for bfloat16 -> float / bfloat16, float -> bfloat16 / double, double -> float)
template <typename S, typename D>
curid_status gather_cols_as(const Ctx& ctx, const S* A, int64_t m, int64_t n, int64_t lda,
                            const int32_t* J, int k, D* out, int64_t ldo, bool transpose);
template <typename S, typename D>
curid_status gather_rows_as(const Ctx& ctx, const S* A, int64_t m, int64_t n, int64_t lda,
                            const int32_t* I, int k, D* out, int64_t ldo);
template <typename S, typename D>
curid_status convert2d(const Ctx& ctx, const S* src, int64_t lds, D* dst, int64_t ldd,
                       int64_t rows, int64_t cols);
// S11[i][t] = S[i][J[t]] (t < k); S12[i][c] = S[i][J[k+c]] (c < n-k)
template <typename real>
curid_status split_s(const Ctx& ctx, const real* S, int64_t lds, const int32_t* J, int k,
                     int64_t n, real* S11, real* S12);
template <typename real>
curid_status copy2d(const Ctx& ctx, const real* src, int64_t lds, real* dst, int64_t ldd,
                    int64_t rows, int64_t cols);
// dst (cols x rows, leading dimension ldd) = src^T (src rows x cols)
template <typename real>
curid_status transpose2d(const Ctx& ctx, const real* src, int64_t lds, real* dst, int64_t ldd,
                         int64_t rows, int64_t cols);
// dst (k x 2k) = [S11^T | lam I]
template <typename real>
curid_status aug_transpose(const Ctx& ctx, const real* S11, int64_t lds, int k, real lam,
                           real* dst, int64_t ldd);
// dst += src (rows x cols)
template <typename real>
curid_status add2d(const Ctx& ctx, const real* src, int64_t lds, real* dst, int64_t ldd,
                   int64_t rows, int64_t cols);
// x (rows x cols) -> its TF32 part into hi (may be x), the float32 remainder
// into lo
curid_status split_tf32(const Ctx& ctx, const float* x, int64_t ldx, float* hi, int64_t ldh,
                        float* lo, int64_t ldl, int64_t rows, int64_t cols);
// dst[i][t] = src[t][i] (k x k transpose-add): dst += src^T
template <typename real>
curid_status add_transpose(const Ctx& ctx, const real* src, int64_t lds, real* dst,
                           int64_t ldd, int64_t rows, int64_t cols);

// ---- Jacobi SVD of a k x k triangle (svd.cu) ------------------------------------
// W^T (k x k, row i = column i of the matrix) is rotated in place into
// U diag(sigma) (as rows), V^T (k x k, identity on entry) into V^T; k <= 256;
// rotations: device scratch of 40 ints.
template <typename real>
bool jacobi_svd_fits(int k);
template <typename real>
curid_status jacobi_svd(const Ctx& ctx, int k, real* Wt, real* Vt, int* rotations);
// X (k x k) = I
template <typename real>
curid_status identity_fill(const Ctx& ctx, real* X, int k);
// f[i] = 1 / sigma_i^2 (sigma_i = ||row i of W^T||) above rtol * max sigma, else 0
template <typename real>
curid_status tsvd_filter(const Ctx& ctx, int k, const real* Wt, double rtol, real* f);
// row r of B (rows x cols, ldb) times f[r]
template <typename real>
curid_status scale_rows(const Ctx& ctx, real* B, int64_t ldb, int64_t rows, int64_t cols,
                        const real* f);

// ---- complex A through its real embedding (complex.cu) -------------------------
// E (2m x 2n, lde) = the real 2 x 2 blocks [[x, -y], [y, x]] of A (m x n
// complex, interleaved, lda in complex entries)
template <typename real>
curid_status embed_complex(const Ctx& ctx, const real* A, int64_t m, int64_t n, int64_t lda,
                           real* E, int64_t lde);
// J (n) from the real pivots Jp (2n): pairs -> complex indices; a broken
// pair sets FLAG_BREAKDOWN; halve_ranks halves the status block's ranks
curid_status extract_pivots(const Ctx& ctx, const int32_t* Jp, int k, int64_t n, int32_t* J,
                            bool halve_ranks);
// T (k x cols complex, ldt complex entries) from the real Tp (2k x 2 cols)
template <typename real>
curid_status extract_t(const Ctx& ctx, const real* Tp, int64_t ldtp, const int32_t* Jp, int k,
                       int64_t cols, real* T, int64_t ldt);
// U (k x k complex float64) from the real Up (2k x 2k float64)
curid_status extract_u(const Ctx& ctx, const double* Up, const int32_t* Jp, const int32_t* Ip,
                       int k, double* U);

// ---- sparse A (sparse.cu) ---------------------------------------------------
// A m x n with its stored entries in compressed rows (row_ptr [m + 1],
// col_idx, row_val) and compressed columns (col_ptr [n + 1], row_idx,
// col_val): the same values twice, no duplicate entries.
struct SparseA {
  int64_t nnz;
  const int64_t* row_ptr;
  const int32_t* col_idx;
  const void* row_val;
  const int64_t* col_ptr;
  const int32_t* row_idx;
  const void* col_val;
};
// out (R x L, ldo) = for each list r: sum of val[e] * in[idx[e], :] over its
// entries (nnz in all lists); in is nrows_in x L (ldi).
template <typename real>
curid_status spmm_rows(const Ctx& ctx, int64_t R, const int64_t* ptr, const int32_t* idx,
                       const real* val, int64_t nnz, int64_t nrows_in, const real* in,
                       int64_t ldi, int64_t L, real* out, int64_t ldo);
// dst (k x cols, ldd) row t = list sel[t] scattered densely (zeros elsewhere);
// dst2 (cols x k, ld2), if non-null, the same as columns.
template <typename real>
curid_status scatter_lists(const Ctx& ctx, const int32_t* sel, int k, int64_t lists,
                           const int64_t* ptr, const int32_t* idx, const real* val, int64_t cols,
                           real* dst, int64_t ldd, real* dst2, int64_t ld2);

// ---- random numbers (philox.cu) --------------------------------------------
template <typename real>
curid_status gaussian_fill(const Ctx& ctx, int64_t rows, int64_t cols, uint64_t seed, real* out,
                           int64_t ld);

// ---- structured sampling matrix (srft.cu) -------------------------------------
// Omega = sqrt(m/l) R F D of Eq. (5.2), real form (DCT-II, sign flips), l x m
// into out (leading dimension ld >= m) from the l sampled rows and m signs.
// Its random choices from a seed (philox.cu): m signs, l distinct rows in [0, m).
curid_status srft_draw(const Ctx& ctx, int64_t m, int64_t l, uint64_t seed, int32_t* rows,
                       int8_t* signs);
template <typename real>
curid_status srft_fill(const Ctx& ctx, int64_t m, int64_t l, const int32_t* rows,
                       const int8_t* signs, real* out, int64_t ld);
// Y = Omega A (l x n, leading dimension ldy) for the same Omega without
// forming it: one pass over A, a fast DCT of its columns in shared memory.
// UNSUPPORTED when m has a prime factor above 7 or its columns do not fit.
template <typename real>
curid_status srft_apply(const Ctx& ctx, const real* A, int64_t m, int64_t n, int64_t lda,
                        int64_t l, const int32_t* rows, const int8_t* signs, real* Y,
                        int64_t ldy);

}  // namespace curid
