// Batched adaptive-rank column ID of many independent small matrices
// (Algorithm 1 per block with the tolerance stop of Section 3): for every
// block A_b (m_b x n_b) a truncated column-pivoted Householder QR that stops
// at the first step j with ||A_b - C V*||_F, the root of the sum of the
// unselected residual norms squared, <= tol ||A_b||_F, then
// T_b = S11^{-1} S12 by back substitution (Eq. (2.8)).
//
// One persistent launch: each CTA takes blocks from a global counter (in the
// caller's order; largest first balances the tail) and factors one block at
// a time.  The block is copied row-major into the CTA's shared memory when
// it fits there (the launch gives each CTA its share of the SM's shared
// memory: blocks of up to about 52K float32 elements at one CTA per SM),
// else into the CTA's global scratch (L2); the two cases are instantiations
// of their own, so an on-chip block uses shared-memory addressing only.
// Thread t
// owns columns t, t + blockDim, ... (at most kColsPerThread), so applying a
// reflector is two coalesced sweeps down the rows: w = v^T X for every
// column, then X -= tau v w^T fused with the new column norms, recomputed
// from the updated entries (no downdating).  The pivot choice (largest norm,
// smallest index on ties) and the pivot column's norm are CTA reductions:
// a step needs no exchange between CTAs.  The reflector sits in shared
// memory; S stays in the scratch's top rows.
#include <cfloat>
#include <climits>

#include "kernels.cuh"

using namespace curid;

namespace {

constexpr int kBatchKCap = 128;    // largest k_max (S11 of the T solve in shared memory)
constexpr int kColsPerThread = 4;  // n_b <= 4 x threads per CTA
constexpr int kMaxBlockDim = 512;
constexpr int kRowBatch = 16;     // loads in flight per thread in a row sweep

template <typename real>
struct BatchParams {
  int nb;
  const real* const* A;
  const int64_t* lda;
  const int* m;
  const int* n;
  const int* order;   // processing order (nullable)
  real tol;
  int k_max;
  int32_t* const* J;
  real* const* T;     // k_max x n_b each, leading dimension n_b
  int* k_out;
  int* block_status;  // nullable
  real* scratch;      // gridDim.x x scratch_stride
  int64_t scratch_stride;
  int64_t xcap;       // elements of a block that fit the CTA's shared memory
  int max_n;
  int max_m;
  int* counter;
  StatusBlock* status;
};

// CTA-wide argmax of (value, index): largest value, smallest index on ties.
template <typename real>
__device__ void cta_argmax(real v, int idx, real* s_val, int* s_idx, real* out_v, int* out_i) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const real ov = __shfl_xor_sync(0xffffffffu, v, o);
    const int oi = __shfl_xor_sync(0xffffffffu, idx, o);
    if (ov > v || (ov == v && oi < idx)) {
      v = ov;
      idx = oi;
    }
  }
  if (lane == 0) {
    s_val[warp] = v;
    s_idx[warp] = idx;
  }
  __syncthreads();
  if (warp == 0) {
    v = lane < nw ? s_val[lane] : real(-1);
    idx = lane < nw ? s_idx[lane] : INT_MAX;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const real ov = __shfl_xor_sync(0xffffffffu, v, o);
      const int oi = __shfl_xor_sync(0xffffffffu, idx, o);
      if (ov > v || (ov == v && oi < idx)) {
        v = ov;
        idx = oi;
      }
    }
    if (lane == 0) {
      s_val[0] = v;
      s_idx[0] = idx;
    }
  }
  __syncthreads();
  *out_v = s_val[0];
  *out_i = s_idx[0];
  __syncthreads();
}

template <typename real>
__device__ real cta_sum(real v, real* s_red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  v = warp_sum(v);
  if (lane == 0) s_red[warp] = v;
  __syncthreads();
  if (warp == 0) {
    v = lane < nw ? s_red[lane] : real(0);
    v = warp_sum(v);
    if (lane == 0) s_red[0] = v;
  }
  __syncthreads();
  const real r = s_red[0];
  __syncthreads();
  return r;
}

template <typename real>
size_t batched_smem(int max_m, int max_n, int k_max) {
  return ((size_t)((max_m + 3) & ~3) + (size_t)k_max * k_max) * sizeof(real) +
         (size_t)((max_n + 3) & ~3) * sizeof(int);
}

// Factor block b (m x n), row-major with leading dimension n, held whole in
// the CTA's shared memory (SH: X points there) or in its global scratch.
// (Holding the first rows on chip and the rest in L2 measured no faster than
// the whole block in L2: the L2 rows set the pace of every sweep.)  Every
// thread of the CTA calls it.
template <typename real, bool SH>
__device__ __forceinline__ void factor_block(const BatchParams<real>& P, int b, int m, int n,
                                             real* X, real* v, real* S11, int* active,
                                             real* s_val, int* s_idx) {
  const int tid = threadIdx.x, nt = blockDim.x;
  const int kk = P.k_max;
  const real eps = sizeof(real) == 8 ? real(DBL_EPSILON) : real(FLT_EPSILON);
  const int64_t lda = P.lda[b];
  const real* A = P.A[b];
  const int kcap = min(min(m, n), kk);
  int32_t* Jb = P.J[b];

  // copy A_b into X (row-major, leading dimension n)
  for (int r = tid / 32; r < m; r += nt / 32)
    for (int c = tid & 31; c < n; c += 32) X[(int64_t)r * n + c] = A[r * lda + c];
  for (int c = tid; c < n; c += nt) active[c] = 1;
  __syncthreads();
  // column norms of the owned columns
  real nu2[kColsPerThread];
  real local2 = real(0);
#pragma unroll
  for (int u = 0; u < kColsPerThread; ++u) {
    nu2[u] = real(0);
    const int c = tid + u * nt;
    if (c < n) {
      for (int r0 = 0; r0 < m; r0 += kRowBatch) {
        real xv[kRowBatch];
#pragma unroll
        for (int q = 0; q < kRowBatch; ++q)
          xv[q] = r0 + q < m ? X[(int64_t)(r0 + q) * n + c] : real(0);
#pragma unroll
        for (int q = 0; q < kRowBatch; ++q) nu2[u] += xv[q] * xv[q];
      }
    }
    local2 += nu2[u];
  }
  const real norm2 = cta_sum(local2, s_val);
  const real normA = sqrt(norm2);
  real resid2 = norm2;
  bool nonfinite = !isfinite(norm2);
  int k = 0, k_eff = -1;
  real nu_first = real(0);

  while (!nonfinite && k < kcap) {
    if (P.tol > real(0) && sqrt(resid2) <= P.tol * normA) break;
    // (1) pivot: the largest residual norm among the active columns
    real best = real(-1);
    int bi = INT_MAX;
#pragma unroll
    for (int u = 0; u < kColsPerThread; ++u) {
      const int c = tid + u * nt;
      if (c < n && active[c]) {
        const real nu = sqrt(nu2[u]);
        if (nu > best || (nu == best && c < bi)) {
          best = nu;
          bi = c;
        }
      }
    }
    real pnu;
    int p;
    cta_argmax<real>(best, bi, s_val, s_idx, &pnu, &p);
    if (p < 0 || p >= n) break;
    if (k == 0) nu_first = pnu;
    if (k_eff < 0 && (pnu == real(0) || pnu <= real(2) * sqrt(real(m)) * eps * nu_first))
      k_eff = k;
    // (2) Householder reflector H = I - tau v v^T of X[k:m, p], v(k) = 1,
    // H X[k:m, p] = beta e_k
    for (int r = k + tid; r < m; r += nt) v[r] = X[(int64_t)r * n + p];
    __syncthreads();
    const real alpha = v[k];
    real sig = real(0);
    for (int r = k + 1 + tid; r < m; r += nt) sig += v[r] * v[r];
    sig = cta_sum(sig, s_val);
    real beta, tau, scale;
    if (sig == real(0)) {
      beta = alpha;
      tau = real(0);
      scale = real(0);
    } else {
      const real nrm = sqrt(alpha * alpha + sig);
      beta = alpha >= real(0) ? -nrm : nrm;
      tau = (beta - alpha) / beta;
      scale = real(1) / (alpha - beta);
    }
    for (int r = k + 1 + tid; r < m; r += nt) v[r] *= scale;
    if (tid == 0) {
      v[k] = real(1);
      X[(int64_t)k * n + p] = beta;
      Jb[k] = p;
      active[p] = 0;
    }
    __syncthreads();
    // (3) w = tau v^T X[k:m, c]; X[k:m, c] -= w v; norm of rows k+1..m-1.
    // Rows go in batches of kRowBatch loads issued before their use, so
    // each thread keeps that many L2 requests in flight.
    real loc = real(0);
#pragma unroll
    for (int u = 0; u < kColsPerThread; ++u) {
      const int c = tid + u * nt;
      if (c < n && active[c]) {
        real w = real(0);
        for (int r0 = k; r0 < m; r0 += kRowBatch) {
          real xv[kRowBatch];
#pragma unroll
          for (int q = 0; q < kRowBatch; ++q) {
            const int r = r0 + q;
            xv[q] = r < m ? X[(int64_t)r * n + c] : real(0);
          }
#pragma unroll
          for (int q = 0; q < kRowBatch; ++q)
            if (r0 + q < m) w += v[r0 + q] * xv[q];
        }
        w *= tau;
        real s2 = real(0);
        for (int r0 = k; r0 < m; r0 += kRowBatch) {
          real xv[kRowBatch];
#pragma unroll
          for (int q = 0; q < kRowBatch; ++q) {
            const int r = r0 + q;
            xv[q] = r < m ? X[(int64_t)r * n + c] : real(0);
          }
#pragma unroll
          for (int q = 0; q < kRowBatch; ++q) {
            const int r = r0 + q;
            if (r < m) {
              const real x = xv[q] - w * v[r];
              X[(int64_t)r * n + c] = x;
              if (r > k) s2 += x * x;
            }
          }
        }
        nu2[u] = s2;
        loc += s2;
      }
    }
    resid2 = cta_sum(loc, s_val);
    if (!isfinite(resid2)) nonfinite = true;
    ++k;
  }
  // J[k:] = the unselected columns in ascending order
  if (tid == 0) {
    int pos = k;
    for (int c = 0; c < n; ++c)
      if (active[c]) Jb[pos++] = c;
  }
  __syncthreads();
  const int ke = k_eff < 0 ? k : k_eff;
  for (int e = tid; e < ke * ke; e += nt) {
    const int i = e / ke, t = e % ke;
    S11[i * kk + t] = i <= t ? X[(int64_t)i * n + Jb[t]] : real(0);
  }
  __syncthreads();
  // T (k x (n - k), leading dimension n), one column per thread; rows at
  // and after the numerical rank are zero (Section 2.3)
  real* Tb = P.T[b];
  for (int c = tid; c < n - k; c += nt) {
    const int col = Jb[k + c];
    for (int i = k - 1; i >= ke; --i) Tb[(int64_t)i * n + c] = real(0);
    for (int i = ke - 1; i >= 0; --i) {
      real s = X[(int64_t)i * n + col];
      for (int t = i + 1; t < ke; ++t) s -= S11[i * kk + t] * Tb[(int64_t)t * n + c];
      Tb[(int64_t)i * n + c] = s / S11[i * kk + i];
    }
  }
  if (tid == 0) {
    P.k_out[b] = k;
    int st = CURID_OK;
    if (nonfinite) st = CURID_NONFINITE;
    else if (k_eff >= 0) st = CURID_RANK_DEFICIENT;
    else if (P.tol > real(0) && k == kcap && sqrt(resid2) > P.tol * normA) st = CURID_TOL_NOT_MET;
    if (P.block_status) P.block_status[b] = st;
    if (st == CURID_NONFINITE) set_flag(&P.status->flags, FLAG_NONFINITE);
    if (st == CURID_RANK_DEFICIENT) set_flag(&P.status->flags, FLAG_RANK_DEFICIENT);
  }
}

template <typename real>
__global__ void __launch_bounds__(kMaxBlockDim) batched_id_kernel(BatchParams<real> P) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  real* v = reinterpret_cast<real*>(smem_raw);                 // reflector, max_m
  real* S11 = v + ((P.max_m + 3) & ~3);                         // k_max x k_max
  int* active = reinterpret_cast<int*>(S11 + (size_t)P.k_max * P.k_max);  // max_n
  real* Xs = reinterpret_cast<real*>(active + ((P.max_n + 3) & ~3));     // xcap elements
  __shared__ real s_val[32];
  __shared__ int s_idx[32];
  __shared__ int s_blk;
  const int tid = threadIdx.x;
  real* Xg = P.scratch + (int64_t)blockIdx.x * P.scratch_stride;

  for (;;) {
    if (tid == 0) s_blk = atomicAdd(P.counter, 1);
    __syncthreads();
    int b = s_blk;
    __syncthreads();
    if (b >= P.nb) break;
    if (P.order) b = P.order[b];
    const int m = P.m[b], n = P.n[b];
    if ((int64_t)m * n <= P.xcap)
      factor_block<real, true>(P, b, m, n, Xs, v, S11, active, s_val, s_idx);
    else
      factor_block<real, false>(P, b, m, n, Xg, v, S11, active, s_val, s_idx);
    __syncthreads();
  }
}

struct BatchArgs {
  int nb;
  const void* const* A;
  const int64_t* lda;
  const int* m;
  const int* n;
  const int* order;
  int max_m, max_n;
  double tol;
  int k_max;
  int32_t* const* J;
  void* const* T;
  int* k_out;
  int* block_status;
};

// Launch shapes the autotuner chooses among: threads per CTA x CTAs per SM.
constexpr int kShapes[][2] = {{512, 1}, {256, 1}, {256, 2}, {128, 2}, {128, 4}};
constexpr int kNumShapes = sizeof(kShapes) / sizeof(kShapes[0]);

// A launch shape's grid, dynamic shared memory and on-chip block capacity:
// each CTA gets its share of the SM's shared memory for a block.
template <typename real>
bool shape_ok(const curid_handle* h, const BatchArgs& a, int s, int* grid, size_t* smem_out,
              int64_t* xcap_out) {
  const int threads = kShapes[s][0], per_sm = kShapes[s][1];
  if (a.max_n > kColsPerThread * threads) return false;
  const size_t base = batched_smem<real>(a.max_m, a.max_n, a.k_max);
  if (base > h->smem_optin) return false;
  int per_sm_bytes = 0;
  if (cudaDeviceGetAttribute(&per_sm_bytes, cudaDevAttrMaxSharedMemoryPerMultiprocessor,
                             h->device) != cudaSuccess)
    return false;
  // per CTA: 1 KB reserved by the system and the kernel's static variables
  const int64_t share = (int64_t)per_sm_bytes / per_sm - 2048;
  int64_t xbytes = std::min<int64_t>(share - (int64_t)base, (int64_t)h->smem_optin - (int64_t)base);
  xbytes = std::max<int64_t>(0, xbytes) & ~int64_t(1023);
  for (;; xbytes -= 1024) {
    if (xbytes < 0) return false;
    const size_t smem = base + (size_t)xbytes;
    if (cudaFuncSetAttribute(batched_id_kernel<real>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem) != cudaSuccess)
      return false;
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, batched_id_kernel<real>, threads,
                                                      smem) != cudaSuccess)
      return false;
    if (occ >= per_sm) {
      *smem_out = smem;
      *xcap_out = xbytes / (int64_t)sizeof(real);
      break;
    }
  }
  *grid = h->num_sms * per_sm;
  return true;
}

template <typename real>
size_t batched_ws(const curid_handle* h, const BatchArgs& a) {
  Carver cv(nullptr);
  cv.take<StatusBlock>(1);
  cv.take<int>(1);
  int max_per_sm = 1;
  for (int s = 0; s < kNumShapes; ++s) max_per_sm = std::max(max_per_sm, kShapes[s][1]);
  cv.take<real>((size_t)h->num_sms * max_per_sm * a.max_m * a.max_n);
  return cv.used;
}

template <typename real>
curid_status batched_launch(curid_handle* h, const BatchArgs& a, int shape) {
  int grid = 0;
  size_t smem = 0;
  int64_t xcap = 0;
  if (!shape_ok<real>(h, a, shape, &grid, &smem, &xcap)) return CURID_UNSUPPORTED;
  if (!h->ws || batched_ws<real>(h, a) > h->ws_bytes) return CURID_NO_WORKSPACE;
  Carver cv(h->ws);
  StatusBlock* st = cv.take<StatusBlock>(1);
  int* counter = cv.take<int>(1);
  const int64_t stride = (int64_t)a.max_m * a.max_n;
  real* scratch = cv.take<real>((size_t)grid * stride);
  CURID_CUDA(cudaMemsetAsync(st, 0, sizeof(StatusBlock), h->stream));
  CURID_CUDA(cudaMemsetAsync(counter, 0, sizeof(int), h->stream));
  BatchParams<real> P;
  P.nb = a.nb;
  P.A = reinterpret_cast<const real* const*>(a.A);
  P.lda = a.lda;
  P.m = a.m;
  P.n = a.n;
  P.order = a.order;
  P.tol = (real)a.tol;
  P.k_max = a.k_max;
  P.J = a.J;
  P.T = reinterpret_cast<real* const*>(a.T);
  P.k_out = a.k_out;
  P.block_status = a.block_status;
  P.scratch = scratch;
  P.scratch_stride = stride;
  P.max_m = a.max_m;
  P.max_n = a.max_n;
  P.xcap = xcap;
  P.counter = counter;
  P.status = st;
  batched_id_kernel<real><<<grid, kShapes[shape][0], smem, h->stream>>>(P);
  CURID_CUDA(cudaGetLastError());
  if (h->profiling) ++h->launches;
  return CURID_OK;
}

curid_status batched_check(curid_handle* h, curid_dtype dt, const BatchArgs& a) {
  if (!h) return CURID_INVALID_ARG;
  if (dt != CURID_F32 && dt != CURID_F64) return CURID_INVALID_ARG;
  if (a.nb < 0 || a.max_m <= 0 || a.max_n <= 0) return CURID_INVALID_ARG;
  if (a.k_max < 1 || !(a.tol >= 0)) return CURID_INVALID_ARG;
  if (a.k_max > kBatchKCap) return CURID_UNSUPPORTED;
  if (a.max_n > kColsPerThread * kMaxBlockDim) return CURID_UNSUPPORTED;
  if (a.nb > 0 && (!a.A || !a.lda || !a.m || !a.n || !a.J || !a.T || !a.k_out))
    return CURID_INVALID_ARG;
  return CURID_OK;
}

int tuned_shape(const curid_handle* h, curid_dtype dt) {
  const int s = h->batch_shape[dt == CURID_F64 ? 0 : 1];
  return s >= 0 && s < kNumShapes ? s : -1;
}

template <typename real>
curid_status batched_default(curid_handle* h, curid_dtype dt, const BatchArgs& a) {
  int s = tuned_shape(h, dt);
  if (s >= 0) return batched_launch<real>(h, a, s);
  int grid;
  size_t smem;
  int64_t xcap;
  for (s = 0; s < kNumShapes; ++s)
    if (shape_ok<real>(h, a, s, &grid, &smem, &xcap)) return batched_launch<real>(h, a, s);
  return CURID_UNSUPPORTED;
}

// Times every feasible launch shape on this batch (two runs each, the
// second timed) and keeps the fastest for later calls on the handle.
template <typename real>
curid_status batched_tune(curid_handle* h, curid_dtype dt, const BatchArgs& a, int* chosen) {
  cudaEvent_t e0, e1;
  CURID_CUDA(cudaEventCreate(&e0));
  CURID_CUDA(cudaEventCreate(&e1));
  float best = 1e30f;
  int best_s = -1;
  curid_status result = CURID_OK;
  for (int s = 0; s < kNumShapes && result == CURID_OK; ++s) {
    int grid;
    size_t smem;
    int64_t xcap;
    if (!shape_ok<real>(h, a, s, &grid, &smem, &xcap)) continue;
    for (int rep = 0; rep < 2 && result == CURID_OK; ++rep) {
      if (cudaEventRecord(e0, h->stream) != cudaSuccess) { result = CURID_CUDA_ERROR; break; }
      result = batched_launch<real>(h, a, s);
      if (result != CURID_OK) break;
      if (cudaEventRecord(e1, h->stream) != cudaSuccess ||
          cudaEventSynchronize(e1) != cudaSuccess) {
        result = CURID_CUDA_ERROR;
        break;
      }
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) { result = CURID_CUDA_ERROR; break; }
      if (rep == 1 && ms < best) {
        best = ms;
        best_s = s;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (result != CURID_OK) return result;
  if (best_s < 0) return CURID_UNSUPPORTED;
  h->batch_shape[dt == CURID_F64 ? 0 : 1] = best_s;
  if (chosen) *chosen = best_s;
  return CURID_OK;
}

struct DevSwitch {
  int prev = -1;
  bool ok = true;
  explicit DevSwitch(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) { ok = false; return; }
    if (prev != dev && cudaSetDevice(dev) != cudaSuccess) ok = false;
  }
  ~DevSwitch() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

}  // namespace

extern "C" {

curid_status curid_id_col_batched_workspace_size(curid_handle* handle, curid_dtype dtype,
                                                 int max_m, int max_n, int k_max,
                                                 size_t* bytes) {
  if (!bytes) return CURID_INVALID_ARG;
  BatchArgs a{};
  a.max_m = max_m;
  a.max_n = max_n;
  a.k_max = k_max;
  CURID_TRY(batched_check(handle, dtype, a));
  *bytes = dtype == CURID_F64 ? batched_ws<double>(handle, a) : batched_ws<float>(handle, a);
  return CURID_OK;
}

curid_status curid_id_col_batched(curid_handle* handle, curid_dtype dtype, int nb,
                                  const void* const* A, const int64_t* lda, const int* m,
                                  const int* n, const int* order, int max_m, int max_n,
                                  double tol, int k_max, int32_t* const* J, void* const* T,
                                  int* k_out, int* block_status) {
  BatchArgs a{nb, A, lda, m, n, order, max_m, max_n, tol, k_max, J, T, k_out, block_status};
  CURID_TRY(batched_check(handle, dtype, a));
  if (nb == 0) return CURID_OK;
  DevSwitch g(handle->device);
  if (!g.ok) return CURID_CUDA_ERROR;
  if (dtype == CURID_F64) return batched_default<double>(handle, dtype, a);
  return batched_default<float>(handle, dtype, a);
}

curid_status curid_id_col_batched_autotune(curid_handle* handle, curid_dtype dtype, int nb,
                                           const void* const* A, const int64_t* lda,
                                           const int* m, const int* n, const int* order,
                                           int max_m, int max_n, double tol, int k_max,
                                           int32_t* const* J, void* const* T, int* k_out,
                                           int* block_status, int* threads, int* ctas_per_sm) {
  BatchArgs a{nb, A, lda, m, n, order, max_m, max_n, tol, k_max, J, T, k_out, block_status};
  CURID_TRY(batched_check(handle, dtype, a));
  if (nb == 0) return CURID_INVALID_ARG;
  DevSwitch g(handle->device);
  if (!g.ok) return CURID_CUDA_ERROR;
  int s = -1;
  CURID_TRY(dtype == CURID_F64 ? batched_tune<double>(handle, dtype, a, &s)
                               : batched_tune<float>(handle, dtype, a, &s));
  if (threads) *threads = kShapes[s][0];
  if (ctas_per_sm) *ctas_per_sm = kShapes[s][1];
  return CURID_OK;
}

}  // extern "C"
