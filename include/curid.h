/*
 * curid.h -- C ABI of the GB300 (sm_103a) CUR / interpolative decomposition
 * library.  Method: Voronin & Martinsson, "Efficient Algorithms for CUR and
 * Interpolative Matrix Decompositions" (arXiv:1412.8447).
 *
 * Conventions shared by every entry point
 * ----------------------------------------
 *  - Matrices are dense, row-major, real (float64 or float32), with an
 *    explicit leading dimension (elements between consecutive rows).  The
 *    paper's A^* is the transpose.  Sparse A (curid_cur_sparse) comes in
 *    compressed rows and columns; complex A (curid_cur_complex) as
 *    interleaved (re, im) pairs, its A^* the conjugate transpose.
 *  - Every matrix / index pointer passed to a compute entry point is DEVICE
 *    memory on the handle's device, owned by the caller; the library never
 *    frees or keeps it after the call's work has finished on the stream.
 *  - Indices are 0-based int32.  A pivot vector J of length n lists the k
 *    skeleton columns in selection order, then the other n-k columns in
 *    ascending index order.  Among exactly equal pivot norms the smallest
 *    column index wins.
 *  - T (k x (n-k), leading dimension ldt) holds the interpolation
 *    coefficients; its column c belongs to original column J[k + c].
 *  - Work is enqueued on the handle's stream and runs asynchronously.  A
 *    compute call returns CURID_OK once its work is enqueued, or an error
 *    found on the host (bad argument, workspace too small, launch failure).
 *    Conditions found on the device (rank deficiency, non-finite input, a
 *    timed-out inter-block wait, Cholesky breakdown) are recorded in the
 *    handle's device status word and read with curid_last_status().
 *  - The library allocates no device memory: scratch comes from the
 *    workspace the caller attaches with curid_set_workspace(), sized by
 *    curid_workspace_size() (or the *_workspace_size call beside an entry
 *    point that has its own).
 *  - Errors are returned, never trapped; no kernel of this library faults
 *    or spins without a bound.
 */
#ifndef CURID_H
#define CURID_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  CURID_OK = 0,
  CURID_INVALID_ARG = 1,     /* a size, pointer or leading dimension is invalid */
  CURID_RANK_DEFICIENT = 2,  /* S11 numerically singular: k_out < k (Section 2.3) */
  CURID_BREAKDOWN = 3,       /* row orthonormalisation failed (non-positive Gram pivot),
                                or a complex pivot pair was split (curid_cur_complex) */
  CURID_NONFINITE = 4,       /* NaN or Inf found in the input */
  CURID_TIMEOUT = 5,         /* an inter-block wait exceeded its bound */
  CURID_CUDA_ERROR = 6,      /* a CUDA runtime call failed */
  CURID_NO_WORKSPACE = 7,    /* attached workspace smaller than required */
  CURID_UNSUPPORTED = 8,     /* valid request outside what this build implements */
  CURID_TOL_NOT_MET = 9      /* batched ID, per block: k_max steps left the
                                residual above tol */
} curid_status;

/* Element type of A.  CURID_BF16 (bfloat16 storage; the precision form of
 * the method): only the randomized decompositions (p >= 0) of curid_id_col,
 * curid_tsid and curid_cur, with lda a multiple of 8 and A 16-byte aligned
 * (else CURID_UNSUPPORTED).  The products with A run as BF16 tensor-core
 * MMAs with float32 accumulation, the sample operand split into two BF16
 * parts (about 16 significant bits); every other step runs in float32 and
 * the T solve (Eq. (2.8)) in float64.  Outputs: T and TW float32, C and R
 * bfloat16 (exact copies of A's entries), U float64. */
typedef enum { CURID_F64 = 0, CURID_F32 = 1, CURID_BF16 = 2 } curid_dtype;

/* Randomized front end (Section 5, Algorithm 4 and the power scheme of
 * Section 5.3).
 *   p < 0 : deterministic method, CPQR runs on A itself (Algorithms 1-3).
 *   p >= 0: randomized method with l = k + p sample rows,
 *           Y = Omega A (A^* A)^q, with row orthonormalisation between the
 *           products (Section 5.3, steps 2a-2e).
 *   omega : optional DEVICE matrix l x m (row-major, leading dimension m,
 *           same dtype as A) used as Omega; when NULL the library draws
 *           Omega from its Philox4x32-10 + Box-Muller generator with `seed`.
 *   tf32  : for CURID_F32 only: 1 = the three kinds of sketch product run on
 *           the tensor cores in TF32 with FP32 accumulation; 0 = FP32 FMA.
 *   srft_rows, srft_signs : optional DEVICE arrays (int32 [l], int8 [m]):
 *           Omega is the structured matrix of Section 5.2, Eq. (5.2), with
 *           these sampled rows and signs (see curid_srft_omega), and the
 *           first product Omega A is the fast transform of curid_srft_sketch
 *           (Omega is never formed; the power steps, if any, are the usual
 *           products).  Both or neither; omega must then be NULL and p >= 0;
 *           dtype CURID_F32 or CURID_F64 (BF16: CURID_UNSUPPORTED), and m
 *           within curid_srft_sketch's limits.  Not for the sparse and
 *           complex decompositions nor the adaptive rank (UNSUPPORTED). */
typedef struct {
  int p;
  int q;
  uint64_t seed;
  const void* omega;
  int tf32;
  const int32_t* srft_rows;
  const int8_t* srft_signs;
} curid_sketch;

typedef struct curid_handle curid_handle;

/* Handle: binds a device, a stream (default: the legacy default stream) and
 * a caller-owned workspace.  create/destroy are not thread safe with respect
 * to the same handle; one handle serves one stream at a time. */
curid_status curid_create(curid_handle** handle, int device);
curid_status curid_destroy(curid_handle* handle);
/* stream: a cudaStream_t passed as void* (NULL = default stream). */
curid_status curid_set_stream(curid_handle* handle, void* stream);
/* ptr: device memory of `bytes` bytes, 256-byte aligned, owned by the
 * caller and kept alive while work that uses it is in flight. */
curid_status curid_set_workspace(curid_handle* handle, void* ptr, size_t bytes);
/* Bound of every wait between the blocks of a persistent kernel (the CPQR
 * pivot exchange), in SM clock cycles; 0 restores the default (4e9, about
 * 2 s).  A wait that runs out ends the kernel without fault: the call's
 * status becomes CURID_TIMEOUT (curid_last_status) and the handle stays
 * usable.  Not part of the paper's method (failure handling for the
 * persistent kernels).  Errors: INVALID_ARG (null handle, cycles < 0). */
curid_status curid_set_timeout(curid_handle* handle, long long cycles);
/* How many decompositions the caller keeps in flight on this GPU at once
 * (each with its own handle, stream and workspace; default 1).  With 1 the
 * persistent CPQR kernel runs one block per SM, the lowest latency per
 * factorization; with more it runs on the fewest SMs that hold the matrix
 * (about a third for the sample matrix of an 8000 x 6000 decomposition at
 * k = 200), a little slower on its own but leaving the other SMs to the
 * other decompositions.  Results do not depend on it beyond rounding.
 * Set it before sizing the workspace.  Errors: INVALID_ARG (null handle,
 * inflight < 1). */
curid_status curid_set_concurrency(curid_handle* handle, int inflight);

/* Workspace bytes needed by curid_cur / curid_tsid / curid_id_col /
 * curid_id_row for an m x n matrix of dtype `dtype` at rank k with sketch
 * parameters `sk`.  k = 0 asks for the adaptive-rank size: every rank up to
 * min(m, n) for the deterministic method (sk.p < 0, FP32/FP64), or the
 * largest sample the randomized search may reach, l = min(m, n, 4096)
 * (sk.p >= 0, sk.omega NULL; else CURID_UNSUPPORTED).  Host-only. */
curid_status curid_workspace_size(curid_handle* handle, curid_dtype dtype,
                                  int64_t m, int64_t n,
                                  int k, curid_sketch sk, size_t* bytes);

/* Synchronises the handle's stream and returns the status recorded on the
 * device by the last compute call (CURID_OK, CURID_RANK_DEFICIENT,
 * CURID_NONFINITE, CURID_TIMEOUT, CURID_BREAKDOWN), or CURID_CUDA_ERROR.
 * *k_out (may be NULL) receives the rank actually produced. */
curid_status curid_last_status(curid_handle* handle, int* k_out);

/* ----- profiling -------------------------------------------------------
 * With profiling enabled, every compute call records a CUDA event pair on
 * the handle's stream around each phase below and counts the kernels it
 * launches.  curid_profile_read() synchronises the stream, returns the
 * summed milliseconds and the number of timed intervals per phase (arrays
 * of CURID_NUM_PHASES entries, either may be NULL) and the launch count
 * since the last read, then resets them.  Events come from a pool owned by
 * the handle (no device memory is allocated). */
enum {
  CURID_PHASE_OMEGA = 0,     /* Gaussian Omega (Algorithm 4 line 1) */
  CURID_PHASE_SKETCH = 1,    /* products with A: Omega A, Q A^T, Q A (Section 5.3) */
  CURID_PHASE_ORTH = 2,      /* row orthonormalisation between power steps */
  CURID_PHASE_CPQR_COL = 3,  /* truncated CPQR of Y (or A) */
  CURID_PHASE_T = 4,         /* T = S11^{-1} S12 */
  CURID_PHASE_GATHER = 5,    /* C = A(:, J), R = A(I, :) */
  CURID_PHASE_CPQR_ROW = 6,  /* full-rank CPQR of C^T (row ID of C) */
  CURID_PHASE_U = 7,         /* T_W and U = V* R^+ */
  CURID_NUM_PHASES = 8
};
curid_status curid_profile(curid_handle* handle, int enable);
curid_status curid_profile_read(curid_handle* handle, double* ms, int* calls,
                                long long* launches);

/* ----- building blocks ----------------------------------------------- */

/* i.i.d. N(0,1) matrix (Algorithm 4, line 1): rows x cols, row-major,
 * leading dimension cols, dtype `dtype`, written to device `out`.
 * Element e = r*cols + c comes from Philox4x32-10 (Salmon et al., SC'11)
 * with key (seed low 32 bits, seed high 32 bits) and counter
 * (e/4, 0, 0, 0), word e%4, mapped to (0,1] and paired by Box-Muller. */
curid_status curid_gaussian(curid_handle* handle, curid_dtype dtype,
                            int64_t rows, int64_t cols, uint64_t seed,
                            void* out);

/* Structured sampling matrix of the accelerated randomized scheme
 * (Section 5.2, Eq. (5.2)): Omega = sqrt(m/l) R F D, l x m, written
 * row-major to device `omega` with leading dimension ldo >= m, dtype
 * CURID_F32 or CURID_F64 (for BF16 storage of A the sample is float32).
 * Real form of the paper's complex construction: D = diag(signs) with
 * signs[t] < 0 read as -1 and anything else as +1 (random signs replace
 * the unit-circle entries), F is the orthonormal DCT-II,
 * F(f, t) = c_f cos(pi f (2t+1) / (2m)), c_0 = sqrt(1/m), c_f = sqrt(2/m),
 * and R keeps the rows listed in `rows` (l entries, frequencies in [0, m),
 * drawn without replacement by the caller; other values give rows of the
 * periodic extension of F).  rows (int32, [l]) and signs (int8, [m]) are
 * device memory owned by the caller; nothing is allocated.  The result is
 * passed to the decompositions as curid_sketch.omega with p = l - k
 * (l = 2k suffices in practice, Section 5.2).  Errors: INVALID_ARG for
 * null pointers, m < 1, l < 1 or ldo < m; UNSUPPORTED for m > about 900000
 * (angle tables in shared memory) or another dtype. */
curid_status curid_srft_omega(curid_handle* handle, curid_dtype dtype,
                              int64_t m, int64_t l, const int32_t* rows,
                              const int8_t* signs, void* omega, int64_t ldo);

/* Y = Omega A for the structured Omega of curid_srft_omega (Section 5.2,
 * Eq. (5.2), same reading, rows and signs) without forming Omega: the fast
 * application the paper gives the structured matrix for.  Each column of
 * D A is transformed by a DCT-II computed through a mixed-radix FFT in
 * shared memory (cost O(m log m) per column, A read once), and the l rows
 * listed in `rows` are kept and scaled; a row outside [0, m) is read from
 * the periodic extension of F as in curid_srft_omega.  A is m x n (lda, row
 * major), Y is l x n (ldy), both device memory of dtype CURID_F32 or
 * CURID_F64 owned by the caller; rows (int32, [l]) and signs (int8, [m])
 * are device arrays; nothing is allocated.  Agrees with curid_srft_omega
 * followed by the product Omega A up to rounding (float32: about 1e-6 of
 * the largest |Y|).  Errors: INVALID_ARG for null pointers, m, n or l < 1,
 * lda < n or ldy < n; UNSUPPORTED for another dtype, for m with a prime
 * factor above 7, or for m beyond one SM's shared memory (m complex values:
 * m <= 29000 in float32, 14500 in float64 on a GPU with 227 KB per CTA). */
curid_status curid_srft_sketch(curid_handle* handle, curid_dtype dtype,
                               const void* A, int64_t m, int64_t n,
                               int64_t lda, int64_t l, const int32_t* rows,
                               const int8_t* signs, void* Y, int64_t ldy);

/* The random choices of Eq. (5.2) drawn on the device from `seed`: signs
 * (int8, [m], each -1 or +1) for D and rows (int32, [l]) for R, l distinct
 * values in [0, m) ("drawn randomly without replacement").  Signs come from
 * Philox4x32-10 (top bit of word t % 4 at counter (t / 4, 0, 1, 0), key as
 * in curid_gaussian); rows[i] = pi(i) for the permutation pi of [0, m) given
 * by a four-round Feistel network with a Philox round function, restricted
 * to [0, m) by cycle walking.  Device buffers owned by the caller; nothing
 * is allocated.  INVALID_ARG for null pointers, m < 1, l < 1 or l > m;
 * UNSUPPORTED for m > 2^30. */
curid_status curid_srft_draw(curid_handle* handle, int64_t m, int64_t l,
                             uint64_t seed, int32_t* rows, int8_t* signs);

/* Sample matrix Y = Omega A (A^* A)^q (Eq. (5.1); Section 5.3 with orth):
 * A m x n (lda), omega l x m (leading dimension m, device, required),
 * Y l x n written with leading dimension n.  With CURID_BF16, A is
 * bfloat16 (lda a multiple of 8, 16-byte aligned) and omega and Y are
 * float32. */
curid_status curid_sketch_matrix(curid_handle* handle, curid_dtype dtype,
                                 const void* A, int64_t m, int64_t n,
                                 int64_t lda, int l, int q, int tf32,
                                 const void* omega, void* Y);

/* Truncated column-pivoted QR (Section 2.2, Eq. (2.4)-(2.5)) of Y (l x n,
 * leading dimension ldy): k > 0 steps, or (k == 0, tol > 0) until the
 * residual ||Y(:,J) - Q1 S1||_F <= tol ||Y||_F.
 * Outputs: J (n), S (k_max x n, leading dimension n, row i = S1(i, :) with
 * columns in ORIGINAL column order, i.e. S[i*n + J[t]] = S1(i, t)).  Only
 * the first k_out rows of S are written. */
curid_status curid_cpqr(curid_handle* handle, curid_dtype dtype,
                        const void* Y, int64_t l, int64_t n, int64_t ldy,
                        int k, double tol, int32_t* J, void* S);

/* Regularised interpolation matrix (Section 4.1: the least-squares form
 * Eq. (4.1) of T = S11^{-1} S12, amended by a Tikhonov term):
 * T = argmin ||S11 T - S12||_F^2 + lam^2 ||T||_F^2, lam > 0, for an S11 too
 * ill-conditioned for the back substitution of Eq. (2.8).  Inputs are what
 * curid_cpqr returns: S (k x n, leading dimension lds >= n, columns in
 * ORIGINAL order) and J (n; J[:k] the pivots).  Output T (k x (n-k),
 * leading dimension ldt >= n-k; column c belongs to J[k + c]).  Computed
 * without normal equations: the rows of [S11^T | lam I] are orthonormalised
 * by three Cholesky-QR passes (Q, k x 2k), R_a = Q [S11; lam I] and
 * T = R_a^{-1} Q(:, :k) S12.  Scratch from the handle's workspace
 * (curid_interp_tikhonov_workspace_size); CURID_F32 or CURID_F64;
 * k <= 4096.  Errors: INVALID_ARG (null pointers, lam <= 0 or not finite,
 * bad sizes), NO_WORKSPACE, UNSUPPORTED; a Cholesky breakdown is recorded
 * in the device status. */
curid_status curid_interp_tikhonov_workspace_size(curid_handle* handle,
                                                  curid_dtype dtype, int64_t n,
                                                  int k, size_t* bytes);
curid_status curid_interp_tikhonov(curid_handle* handle, curid_dtype dtype,
                                   const void* S, int64_t lds,
                                   const int32_t* J, int64_t n, int k,
                                   double lam, void* T, int64_t ldt);

/* Truncated-SVD interpolation matrix (Section 4.1: a stabilised
 * pseudo-inverse of S11 from its SVD with the small singular values
 * dropped): S11 = U diag(sigma) V^T, T = V diag(1/sigma_i : sigma_i >
 * rtol sigma_1, else 0) U^T S12, 0 <= rtol < 1.  Inputs and output as
 * curid_interp_tikhonov (S and J from curid_cpqr; T k x (n-k), ldt).  The
 * SVD is a one-sided Jacobi iteration (cyclic round-robin pairs, one
 * cooperative launch, at most 40 sweeps), k <= 256.  Scratch from the
 * handle's workspace (curid_interp_tsvd_workspace_size); CURID_F32 or
 * CURID_F64.  Errors: INVALID_ARG (null pointers, rtol outside [0, 1), bad
 * sizes), NO_WORKSPACE, UNSUPPORTED (k > 256 or another dtype). */
curid_status curid_interp_tsvd_workspace_size(curid_handle* handle,
                                              curid_dtype dtype, int64_t n,
                                              int k, size_t* bytes);
curid_status curid_interp_tsvd(curid_handle* handle, curid_dtype dtype,
                               const void* S, int64_t lds, const int32_t* J,
                               int64_t n, int k, double rtol, void* T,
                               int64_t ldt);

/* Truncated CPQR exactly as curid_cpqr, for callers that cannot allocate
 * device memory when they factor: a service that reserves all of its GPU
 * memory at start-up and must not fail on an allocation later, code running
 * inside a framework or memory pool that owns every device allocation and
 * has no scratch buffer to lend, a plug-in with no access to the caller's
 * allocator.  There is no counterpart in the paper; this is an interface
 * convenience around the same kernel.
 *   - No handle, no workspace, no cudaMalloc/cudaFree: the kernel's scratch
 *     is a 4 MiB static device array that every GPU loading this library
 *     keeps until the process exits.  Requests whose scratch exceeds it
 *     (about 256 + 2 G (32 + 16 l) bytes for float64, 2 G (32 + 8 l) for
 *     float32, G = min(number of SMs, n): on a 152-SM GPU l up to about
 *     860 rows in float64, 1720 in float32) return CURID_NO_WORKSPACE
 *     before any work is enqueued.
 *   - The first call on a device (with that device current) looks up the
 *     array's device address; with lazy module loading that call is also
 *     where the array is reserved (and can fail for lack of memory), so make
 *     it before reserving the rest of device memory, and before any stream
 *     capture.
 *   - Every call reuses the same array, so calls whose work overlaps on the
 *     GPU (other streams, other host threads) race: serialise them.
 *   - stream: a cudaStream_t passed as void*; Y, J, S as in curid_cpqr on
 *     the current device; info (optional, device, 3 ints): status flags
 *     (1 rank deficient, 2 breakdown, 4 non-finite input, 8 timed-out wait),
 *     the number of steps taken, and the numerical rank. */
curid_status curid_cpqr_static(void* stream, curid_dtype dtype,
                               const void* Y, int64_t l, int64_t n,
                               int64_t ldy, int k, double tol, int32_t* J,
                               void* S, int* info);

/* ----- the decompositions -------------------------------------------- */

/* Rank selection of the decompositions below: k > 0 is a fixed rank
 * (1 <= k <= min(m, n); randomized: k + p <= min(m, n)).  k == 0 with
 * tol > 0 is the adaptive rank of Section 3 for the deterministic method
 * (p < 0) of curid_id_col, curid_tsid and curid_cur: the smallest k with
 * ||A - A(:, J[:k]) V*||_F <= tol ||A||_F.  The call then synchronises the
 * stream once (to read that rank; not for graph capture), runs the
 * decomposition at that rank, and curid_last_status reports it as k_out.
 * Output buffers must hold the largest rank, min(m, n): T and TW are written
 * with the caller's ldt / ldtw, U (k_out x k_out) and C (m x k_out) packed
 * with leading dimension k_out, R with leading dimension n.  k_out == 0
 * (the tolerance met with no column, e.g. A = 0): J and I ascending, nothing
 * else written.  With a sketch (p >= 0) the sample size l = k + p depends
 * on the rank, so it is searched: l = max(64, p + 1), doubling up to
 * min(m, n, 4096); each sample Y = Omega_l A (A^* A)^q (Omega from
 * sk.seed, whose first rows do not depend on l; sk.omega must be NULL, else
 * CURID_UNSUPPORTED) is factored by a CPQR of at most l - p steps with the
 * stop ||Y - Q_j Q_j^T Y||_F <= tol ||Y||_F; the first stop before l - p
 * steps gives the rank, which is then decomposed with p' = l - k on the same
 * sample (at the cap, k = l - p).  The test is on the sample: for q = 0 its
 * squared residual ratio estimates A's without bias; power steps make it
 * optimistic.  One synchronisation per sample size.  curid_id_row answers
 * CURID_UNSUPPORTED for k == 0.
 *
 * Order limits: the k x k triangular solves (T, the row ID, U) and the
 * l x l Gram factorisations between power steps (q >= 1, l = k + p) run in
 * one CTA with the matrix in shared memory up to order 256 (CURID_F32) /
 * 192 (CURID_F64) and blockwise above that, up to 4096; larger k or l return
 * CURID_UNSUPPORTED before any work is queued. */

/* Column ID (Algorithm 1; randomized: Algorithm 4):
 * A ~ A(:, J[:k]) [I T] P^*.  A m x n (lda).  Outputs J (n) and
 * T (k x (n-k), leading dimension ldt >= n-k; rows at and after k_out are
 * zero when rank deficient). */
curid_status curid_id_col(curid_handle* handle, curid_dtype dtype,
                          const void* A, int64_t m, int64_t n, int64_t lda,
                          int k, double tol, curid_sketch sk, int32_t* J,
                          void* T, int64_t ldt);

/* Row ID (Remark 2.1): A ~ W A(I[:k], :), W = P [I; T_W^*], computed as
 * the column ID of A^*.  Outputs I (m), TW (k x (m-k), leading dimension
 * ldtw).  With a sketch, Omega is that of the column ID of A^*: sk.omega
 * is l x n, and sk.srft_signs has n entries. */
curid_status curid_id_row(curid_handle* handle, curid_dtype dtype,
                          const void* A, int64_t m, int64_t n, int64_t lda,
                          int k, double tol, curid_sketch sk, int32_t* I,
                          void* TW, int64_t ldtw);

/* Two-sided ID (Algorithm 2, Eq. (2.12)): column ID of A (or of its sketch),
 * then the full rank-k ID of C^* (Eq. (2.11)).  Outputs J, T, I, TW as in
 * curid_id_col / curid_id_row. */
curid_status curid_tsid(curid_handle* handle, curid_dtype dtype,
                        const void* A, int64_t m, int64_t n, int64_t lda,
                        int k, double tol, curid_sketch sk, int32_t* J,
                        void* T, int64_t ldt, int32_t* I, void* TW,
                        int64_t ldtw);

/* CUR-ID (Algorithm 3): C = A(:, J[:k]), R = A(I[:k], :), U = V* R^+
 * (Eq. (3.1), (3.5)).  Outputs J (n), I (m) and U (k x k, leading
 * dimension k, ALWAYS float64: U carries the conditioning of the skeleton,
 * its entries reach 1/sigma_k, and rounding U alone to float32 moves
 * ||A - CUR||_F / ||A||_F by about 1e-5 on the 8000 x 6000, k = 200
 * workload); optional (NULL = not written): C (m x k, leading dimension k),
 * R (k x n, leading dimension n), T (k x (n-k), ldt), TW (k x (m-k), ldtw),
 * in the dtype of A. */
curid_status curid_cur(curid_handle* handle, curid_dtype dtype,
                       const void* A, int64_t m, int64_t n, int64_t lda,
                       int k, double tol, curid_sketch sk, int32_t* J,
                       int32_t* I, double* U, void* C, void* R, void* T,
                       int64_t ldt, void* TW, int64_t ldtw);

/* CUR-ID with U from the error-corrected system of Section 4.3, Eq. (4.3):
 * A = C V* + E gives U R = V* + C^+ E, whose least-squares solution is
 * U = C^+ A R^+ (the U that minimises ||A - C U R||_F for the chosen C and
 * R).  With the deterministic column ID (p < 0) C^+ E = 0 (E lies in the
 * complement of range(C)) and U equals curid_cur's up to rounding; with a
 * sketch (p >= 0), especially without power steps, it is more accurate.
 * Cost over curid_cur: three Cholesky-QR passes over C^T (C^T = L Q_C), one
 * more product with A (Q_C A, on the tensor cores when tf32 is set) and
 * k x k work; C^+ = K^{-1} Q_C with K = Q_C C solved as upper triangular.
 * Arguments, outputs, statuses and workspace exactly as curid_cur
 * (curid_workspace_size covers both). */
curid_status curid_cur_corrected(curid_handle* handle, curid_dtype dtype,
                                 const void* A, int64_t m, int64_t n,
                                 int64_t lda, int k, double tol,
                                 curid_sketch sk, int32_t* J, int32_t* I,
                                 double* U, void* C, void* R, void* T,
                                 int64_t ldt, void* TW, int64_t ldtw);

/* ----- sparse A ------------------------------------------------------- */

/* A sparse m x n matrix (Section 1: the case CUR is made for, as C and R
 * keep A's sparsity), given twice, in compressed rows and in compressed
 * columns, with the same stored values and no duplicate entries.  All
 * arrays are device memory owned by the caller; values have the dtype of
 * the call (float32 or float64); indices 0-based.  Entries whose index is
 * out of range are skipped by the gathers and read row 0 in the products;
 * the pointer arrays must be non-decreasing from 0 to nnz. */
typedef struct {
  int64_t nnz;
  const int64_t* row_ptr;  /* [m + 1] */
  const int32_t* col_idx;  /* [nnz], column of each entry in row order */
  const void* row_val;     /* [nnz] */
  const int64_t* col_ptr;  /* [n + 1] */
  const int32_t* row_idx;  /* [nnz], row of each entry in column order */
  const void* col_val;     /* [nnz] */
} curid_sparse;

/* Randomized CUR-ID of a sparse A (Algorithms 3 and 4): the products of the
 * sketch and the power steps (Omega A, Q A^T, Q A) are sparse-times-dense
 * products (the sample operand transposed, one warp per output row
 * gathering l-wide rows, on the CUDA cores; sk.tf32 is not used); C and R are
 * gathered from the compressed columns and rows; the rest is the dense
 * pipeline of curid_cur.  Fixed rank only (k >= 1, p >= 0, k + p <=
 * min(m, n)); corrected != 0 takes U from Eq. (4.3) as curid_cur_corrected.
 * Outputs as curid_cur: J, I, U (float64), optional dense C (m x k) and
 * R (k x n), T, TW.  Workspace: curid_sparse_workspace_size. */
curid_status curid_sparse_workspace_size(curid_handle* handle, curid_dtype dtype,
                                         int64_t m, int64_t n, int k,
                                         curid_sketch sk, size_t* bytes);
curid_status curid_cur_sparse(curid_handle* handle, curid_dtype dtype,
                              int64_t m, int64_t n, const curid_sparse* A,
                              int k, curid_sketch sk, int corrected,
                              int32_t* J, int32_t* I, double* U, void* C,
                              void* R, void* T, int64_t ldt, void* TW,
                              int64_t ldtw);

/* ----- complex A -------------------------------------------------------- */

/* CUR-ID of a complex A (the paper works over C): A is m x n complex,
 * interleaved (re, im) pairs of dtype CURID_F32 (complex64) or CURID_F64
 * (complex128), leading dimension lda in complex entries.  Computed by the
 * real pipeline on the embedding E(A) (each entry x + iy as the 2 x 2 block
 * [[x, -y], [y, x]]; 2m x 2n, rank 2k; with a sketch, E(Omega) for a complex
 * Gaussian Omega drawn from sk.seed, l = 2(k + p) real rows; sk.omega must
 * be NULL): greedy pivoting on E takes each complex column as a pair of
 * real ones, and T, U are read off the real results.  Outputs: J (n), I
 * (m) as for curid_cur, U (k x k complex float64, interleaved), T
 * (optional, k x (n-k) complex of A's dtype, ldt in complex entries).  A
 * pair broken by a tie in the pivot norms within rounding sets
 * CURID_BREAKDOWN (curid_last_status); the ranks reported there count
 * complex pivots.  Scratch: curid_complex_workspace_size (the real pipeline
 * for the embedding plus the embedded A, about 4 m n reals). */
curid_status curid_complex_workspace_size(curid_handle* handle, curid_dtype dtype,
                                          int64_t m, int64_t n, int k,
                                          curid_sketch sk, size_t* bytes);
curid_status curid_cur_complex(curid_handle* handle, curid_dtype dtype,
                               const void* A, int64_t m, int64_t n, int64_t lda,
                               int k, curid_sketch sk, int32_t* J, int32_t* I,
                               double* U, void* T, int64_t ldt);

/* ----- adjoint with frozen skeletons ----------------------------------- */

/* Reverse-mode derivative of the deterministic CUR-ID (p < 0) with the index
 * sets held fixed.  The paper does not differentiate the decomposition; the
 * map follows from its definitions: with J and I fixed, C = A(:, J[:k]),
 * R = A(I[:k], :), T = S11^{-1} S12, which equals the least-squares
 * solution C^+ A(:, J[k:]) (Section 2.3, Eq. (2.8)), and U = V* R^+ with
 * V* = [I T] P^* (Eq. (3.5)).  Given cotangents of the outputs C, U, R,
 * the call writes Abar = the gradient with respect to A of
 * <Cbar, C> + <Ubar, U> + <Rbar, R>.
 *
 * A m x n (lda); k, J (n) and I (m, only I[:k] read), T (k x (n-k), ldt;
 * may be NULL when n == k) exactly as returned by curid_cur with p < 0 on
 * this A.  Cotangents, each NULL for zero: Cbar m x k (leading dimension k)
 * and Rbar k x n (leading dimension n) in the dtype of A, Ubar k x k
 * float64 (leading dimension k, like U).  Output Abar m x n (ldab),
 * overwritten.  All pointers are device memory owned by the caller; the
 * scratch (curid_cur_adjoint_workspace_size bytes) is the attached
 * workspace.  k <= 4096, else CURID_UNSUPPORTED.  R or C numerically rank
 * deficient: Cholesky breakdown, reported by curid_last_status as
 * CURID_BREAKDOWN (Abar then undefined). */
curid_status curid_cur_adjoint_workspace_size(curid_handle* handle,
                                              curid_dtype dtype, int64_t m,
                                              int64_t n, int k,
                                              size_t* bytes);
curid_status curid_cur_adjoint(curid_handle* handle, curid_dtype dtype,
                               const void* A, int64_t m, int64_t n,
                               int64_t lda, int k, const int32_t* J,
                               const int32_t* I, const void* T, int64_t ldt,
                               const void* Cbar, const double* Ubar,
                               const void* Rbar, void* Abar, int64_t ldab);

/* ----- batched adaptive-rank column ID --------------------------------- */

/* Column IDs of nb independent blocks A_b (m_b x n_b) in one persistent
 * launch: per block, the truncated column-pivoted QR of Algorithm 1 with the
 * tolerance stop of Section 3 -- stop at the smallest j with
 * ||A_b - A_b(:, J[:j]) V*||_F <= tol ||A_b||_F, i.e. the root of the sum
 * of the unselected residual column norms squared (tol == 0: exactly
 * min(m_b, n_b, k_max) steps) -- then T_b = S11^{-1} S12 (Eq. (2.8)).
 * Pivot ties, the order of J[k:] and the rank-deficiency rule are those of
 * curid_cpqr.
 *
 * Every array argument is DEVICE memory with nb entries: A (pointers to
 * row-major blocks), lda, m, n, J (pointers to n_b int32 each), T (pointers
 * to k_max x n_b entries each; T_b is written with leading dimension n_b,
 * its first k_out[b] rows and n_b - k_out[b] columns meaningful), k_out
 * (ranks); block_status (curid_status per block: OK, RANK_DEFICIENT,
 * NONFINITE or TOL_NOT_MET) and order (a permutation of 0..nb-1 giving the
 * processing order; largest blocks first balances the launch) may be NULL.
 * max_m, max_n (host) bound every m_b, n_b: the workspace
 * (curid_id_col_batched_workspace_size) holds one max_m x max_n scratch
 * matrix per resident CTA.  Limits: k_max <= 128, max_n <= 2048, and the
 * reflector, S11 and column flags (max_m + k_max^2 reals + max_n ints) fit
 * one SM's shared memory; else CURID_UNSUPPORTED.  dtype is that of every
 * block and T.  The call enqueues two memsets and one kernel on the handle's
 * stream and performs no host synchronisation or allocation, so it can be
 * captured into a CUDA graph once the workspace is attached. */
curid_status curid_id_col_batched_workspace_size(curid_handle* handle,
                                                 curid_dtype dtype, int max_m,
                                                 int max_n, int k_max,
                                                 size_t* bytes);
curid_status curid_id_col_batched(curid_handle* handle, curid_dtype dtype,
                                  int nb, const void* const* A,
                                  const int64_t* lda, const int* m,
                                  const int* n, const int* order, int max_m,
                                  int max_n, double tol, int k_max,
                                  int32_t* const* J, void* const* T,
                                  int* k_out, int* block_status);

/* Autotuner for curid_id_col_batched: runs the batch (same arguments, same
 * outputs) once per feasible launch shape (threads per CTA x CTAs per SM),
 * times each with CUDA events, and keeps the fastest shape for this dtype on
 * the handle; later curid_id_col_batched calls use it.  Reports the chosen
 * shape in threads / ctas_per_sm (may be NULL).  Synchronises the stream:
 * call it outside graph capture. */
curid_status curid_id_col_batched_autotune(curid_handle* handle,
                                           curid_dtype dtype, int nb,
                                           const void* const* A,
                                           const int64_t* lda, const int* m,
                                           const int* n, const int* order,
                                           int max_m, int max_n, double tol,
                                           int k_max, int32_t* const* J,
                                           void* const* T, int* k_out,
                                           int* block_status, int* threads,
                                           int* ctas_per_sm);

#ifdef __cplusplus
}
#endif

#endif /* CURID_H */
