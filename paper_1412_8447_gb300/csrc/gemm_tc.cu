// Products with the data matrix A on the 5th-generation tensor cores
// (tcgen05, TMEM accumulators, TMA loads): C = X A or C = X A^T, where X is
// the l x K sketch operand (Omega, or an orthonormal basis Q, Section 5.3)
// and A the m x n data matrix.
//
// Precision: A is split in shared memory into an exactly-truncated TF32 high
// part and the FP32 remainder, A = A_hi + A_lo, and each K-step issues two
// TF32 MMAs, X A_hi + X A_lo, with FP32 accumulation.  X itself is read as
// TF32.  Rounding A to TF32 alone adds a noise floor of about 2^-11 |A| to
// every singular direction and costs the skeleton up to 8 % in residual on
// the sigma_j = j^-2 workload; the split keeps the sample matrix at FP32
// quality (an orthonormal or Gaussian X rounded to TF32 only perturbs
// directions that the sample already spans).  Where X is not a sketch
// operand (the Gram matrices and the L^{-1} apply of the orthonormalisation,
// split_x) X is split the same way in shared memory and a third MMA,
// X_lo A_hi, joins each K step: both operands at FP32 accuracy in one launch.
//
// Tiling: the transposed product D = C^T is computed, so the MMA's M = 128
// rows are 128 output columns and its N = l (<= 256, rounded up to 16) is
// the whole sample: one CTA holds a 128 x l accumulator in TMEM and streams
// its 128 columns of A exactly once over its K range.  Larger samples run in
// equal row chunks of at most 256, one per CTA, the chunks of a column tile
// neighbouring CTAs so that they stream the same tiles of A together.  K is
// split across CTAs when the tiles alone cannot fill the SMs the caller can
// expect; partial tiles are summed in a fixed order.  Warp 0 issues TMA loads, warp 1 the MMAs,
// warps 4-7 split A into hi/lo per stage and run the epilogue
// (TMEM -> registers -> coalesced stores of C).  Both MMA operands are
// K-major: for C = X A, where A's rows run along K, the TMA brings an
// MN-major tile and the same warps transpose it into K-major hi/lo tiles
// while splitting.  Every mbarrier wait is
// bounded; a timeout raises FLAG_TIMEOUT and the CTA drains and returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <mutex>

#include "kernels.cuh"
#include "tcgen05.cuh"

namespace curid {

namespace {

constexpr int kBM = 128;            // MMA M: output columns per CTA
constexpr int kBK = 32;             // K per stage: 32 FP32 = one 128-byte swizzle row
constexpr int kStages = 3;
constexpr int kTcThreads = 256;
constexpr int kAtileBytes = kBM * kBK * 4;  // 16 KB
constexpr int kTmemCols = 256;

struct TcParams {
  int M;         // rows of C (= l)
  int NP;        // rows of a chunk of C (<= 256, a multiple of 16): the MMA's N
  int nch;       // chunks of rows; chunk = blockIdx.x % nch (neighbouring CTAs)
  int N;         // columns of C
  int K;
  int kchunk;    // K per split, multiple of kBK
  int mn_major;  // 1: C = X A (A read MN-major); 0: C = X A^T (K-major)
  int split_x;   // 1: X split in shared memory too (X_hi A_hi + X_hi A_lo + X_lo A_hi)
  int stages;    // pipeline stages (<= kStages)
  float* C;
  int64_t ldc;
  float* partial;  // [splits][M][N] when K is split
  StatusBlock* status;
  uint32_t idesc;
};

__global__ void __launch_bounds__(kTcThreads, 1)
tc_sketch_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmX,
                 TcParams P) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  const uintptr_t base = (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023);
  const int xbytes = ((P.NP * 128 + 1023) / 1024) * 1024;
  const int S = P.stages;
  unsigned char* Ahi[kStages];
  unsigned char* Alo[kStages];
  unsigned char* Xs[kStages];
  unsigned char* Xl[kStages];
  unsigned char* p = reinterpret_cast<unsigned char*>(base);
  for (int s = 0; s < S; ++s) {
    Ahi[s] = p;
    Alo[s] = p + kAtileBytes;
    Xs[s] = p + 2 * kAtileBytes;
    Xl[s] = Xs[s] + xbytes;
    p += 2 * kAtileBytes + (P.split_x ? 2 : 1) * xbytes;
  }
  uint64_t* bars = reinterpret_cast<uint64_t*>(p);  // full[S], conv[S], empty[S], acc
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 3 * kStages + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  auto full = [&](int s) { return smem_u32(bars + s); };
  auto conv = [&](int s) { return smem_u32(bars + kStages + s); };
  auto empty = [&](int s) { return smem_u32(bars + 2 * kStages + s); };
  const uint32_t acc_bar = smem_u32(bars + 3 * kStages);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // the row chunks of one column tile are neighbouring CTAs: they stream the
  // same tiles of A at the same time, so A comes from HBM about once
  const int row0 = (int)(blockIdx.x % P.nch) * P.NP;
  const int n0 = (int)(blockIdx.x / P.nch) * kBM;
  const int kbeg = blockIdx.y * P.kchunk;
  const int kend = min(P.K, kbeg + P.kchunk);
  const int nk = (kend - kbeg + kBK - 1) / kBK;
  const uint32_t xtile_bytes = (uint32_t)P.NP * 128u;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(full(s), 1);
      mbar_init(conv(s), 128);
      mbar_init(empty(s), 1);
    }
    mbar_init(acc_bar, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    __syncwarp();
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  if (warp == 0 && lane == 0) {
    // ---- producer: TMA loads of A and X per stage ----
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmA)) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmX)) : "memory");
    int issued = 0;
    for (int i = 0; i < nk; ++i) {
      const int s = i % S;
      const uint32_t ph = (uint32_t)(i / S) & 1u;
      if (i >= S && !mbar_wait(empty(s), ph ^ 1u)) {
        *abort_flag = 1;
        atomicCAS(&P.status->timeout_site, 0, (1 << 24) | (s << 16) | i);
        break;
      }
      if (*abort_flag) break;
      mbar_expect_tx(full(s), (uint32_t)kAtileBytes + xtile_bytes);
      const int k = kbeg + i * kBK;
      if (P.mn_major) {
        // raw MN-major tile into the lo buffer; the converter transposes it
#pragma unroll
        for (int j = 0; j < 4; ++j)
          tma_load_2d(smem_u32(Alo[s] + j * 4096), &tmA, n0 + 32 * j, k, full(s));
      } else {
        tma_load_2d(smem_u32(Ahi[s]), &tmA, k, n0, full(s));
      }
      tma_load_2d(smem_u32(Xs[s]), &tmX, k, row0, full(s));
      issued = i + 1;
    }
    if (*abort_flag) {
      // let every load this thread issued land before the CTA can exit
      for (int i = max(0, issued - S); i < issued; ++i)
        mbar_wait(full(i % S), (uint32_t)(i / S) & 1u);
    }
  } else if (warp == 1 && lane == 0) {
    // ---- MMA issuer ----
    for (int i = 0; i < nk; ++i) {
      const int s = i % S;
      const uint32_t ph = (uint32_t)(i / S) & 1u;
      if (!mbar_wait(conv(s), ph) || *abort_flag) {
        *abort_flag = 1;
        atomicCAS(&P.status->timeout_site, 0, (2 << 24) | (s << 16) | i);
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t ah = smem_u32(Ahi[s]), al = smem_u32(Alo[s]), xb = smem_u32(Xs[s]);
      const uint32_t xlb = smem_u32(Xl[s]);
#pragma unroll
      for (int kk = 0; kk < kBK / 8; ++kk) {
        // K-major tiles: 128 rows of 128 bytes, 8 K elements = 32 bytes per MMA
        const uint64_t dh = smem_desc(ah + kk * 32, 16, 1024);
        const uint64_t dl = smem_desc(al + kk * 32, 16, 1024);
        const uint64_t dx = smem_desc(xb + kk * 32, 16, 1024);
        mma_tf32(tmem, dh, dx, P.idesc, (i > 0 || kk > 0) ? 1u : 0u);
        mma_tf32(tmem, dl, dx, P.idesc, 1u);
        if (P.split_x) mma_tf32(tmem, dh, smem_desc(xlb + kk * 32, 16, 1024), P.idesc, 1u);
      }
      mma_commit(empty(s));
    }
    mma_commit(acc_bar);
  } else if (warp >= 4) {
    // ---- split A into hi / lo, then the epilogue ----
    const int t = threadIdx.x - 128;
    for (int i = 0; i < nk; ++i) {
      const int s = i % S;
      const uint32_t ph = (uint32_t)(i / S) & 1u;
      if (!mbar_wait(full(s), ph) || *abort_flag) {
        *abort_flag = 1;
        atomicCAS(&P.status->timeout_site, 0, (3 << 24) | (s << 16) | i);
        break;
      }
      if (P.mn_major) {
        // The TMA tile is MN-major: four 4 KB boxes, box j holding columns
        // 32j..32j+31 as 32 K rows of 128 swizzled bytes.  Thread t takes
        // output column t: it gathers its 32 K values into registers, then
        // (after all 128 threads have read the raw tile, which is reused for
        // the low part) writes the row t of the K-major hi and lo tiles.
        const unsigned char* raw = Alo[s];
        float v[kBK];
#pragma unroll
        for (int k = 0; k < kBK; ++k) {
          const int off = (t >> 5) * 4096 + k * 128 + ((((t & 31) >> 2) ^ (k & 7)) << 4) + ((t & 3) << 2);
          v[k] = *reinterpret_cast<const float*>(raw + off);
        }
        asm volatile("bar.sync 1, 128;" ::: "memory");
#pragma unroll
        for (int c = 0; c < kBK / 4; ++c) {
          float4 h, w;
          h.x = __uint_as_float(__float_as_uint(v[4 * c + 0]) & 0xFFFFE000u);
          h.y = __uint_as_float(__float_as_uint(v[4 * c + 1]) & 0xFFFFE000u);
          h.z = __uint_as_float(__float_as_uint(v[4 * c + 2]) & 0xFFFFE000u);
          h.w = __uint_as_float(__float_as_uint(v[4 * c + 3]) & 0xFFFFE000u);
          w = make_float4(v[4 * c + 0] - h.x, v[4 * c + 1] - h.y, v[4 * c + 2] - h.z,
                          v[4 * c + 3] - h.w);
          const int off = t * 128 + ((c ^ (t & 7)) << 4);
          *reinterpret_cast<float4*>(Ahi[s] + off) = h;
          *reinterpret_cast<float4*>(Alo[s] + off) = w;
        }
      } else {
        // K-major tile: split in place (hi over the loaded data, lo beside it)
        float4* hi = reinterpret_cast<float4*>(Ahi[s]);
        float4* lo = reinterpret_cast<float4*>(Alo[s]);
#pragma unroll
        for (int q = 0; q < kAtileBytes / 16 / 128; ++q) {
          const int idx = t + 128 * q;
          const float4 v = hi[idx];
          float4 h;
          h.x = __uint_as_float(__float_as_uint(v.x) & 0xFFFFE000u);
          h.y = __uint_as_float(__float_as_uint(v.y) & 0xFFFFE000u);
          h.z = __uint_as_float(__float_as_uint(v.z) & 0xFFFFE000u);
          h.w = __uint_as_float(__float_as_uint(v.w) & 0xFFFFE000u);
          hi[idx] = h;
          lo[idx] = make_float4(v.x - h.x, v.y - h.y, v.z - h.z, v.w - h.w);
        }
      }
      if (P.split_x) {
        // the X tile: NP rows of 128 bytes, split elementwise in place (the
        // swizzle is a permutation within each 1024-byte atom, the same for
        // the low buffer)
        float4* xh = reinterpret_cast<float4*>(Xs[s]);
        float4* xl = reinterpret_cast<float4*>(Xl[s]);
        for (int idx = t; idx < P.NP * 8; idx += 128) {
          const float4 v = xh[idx];
          float4 h;
          h.x = __uint_as_float(__float_as_uint(v.x) & 0xFFFFE000u);
          h.y = __uint_as_float(__float_as_uint(v.y) & 0xFFFFE000u);
          h.z = __uint_as_float(__float_as_uint(v.z) & 0xFFFFE000u);
          h.w = __uint_as_float(__float_as_uint(v.w) & 0xFFFFE000u);
          xh[idx] = h;
          xl[idx] = make_float4(v.x - h.x, v.y - h.y, v.z - h.z, v.w - h.w);
        }
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      mbar_arrive(conv(s));
    }
    // warp-uniform decision before the warp-collective TMEM loads
    int ok = 0;
    if (lane == 0) {
      ok = mbar_wait(acc_bar, 0) ? 1 : 0;
      if (!ok) {
        *abort_flag = 1;
        atomicCAS(&P.status->timeout_site, 0, 4 << 24);
      }
      ok = ok && !*abort_flag;
    }
    ok = __shfl_sync(0xffffffffu, ok, 0);
    __syncwarp();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (ok) {
      const int q = warp - 4;             // TMEM lanes 32q .. 32q+31
      const int col = n0 + q * 32 + lane;  // output column of this thread
      float* dst = P.partial ? P.partial + (size_t)blockIdx.y * P.M * P.N : P.C;
      const int64_t ld = P.partial ? P.N : P.ldc;
      const int rows = min(P.NP, P.M - row0);
      for (int c0 = 0; c0 < P.NP; c0 += 32) {
        uint32_t r[32];
        tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)c0, r);
        if (col < P.N) {
#pragma unroll
          for (int j = 0; j < 32; ++j)
            if (c0 + j < rows) dst[(int64_t)(row0 + c0 + j) * ld + col] = __uint_as_float(r[j]);
        }
      }
    }
  }
  __syncthreads();
  if (*abort_flag && threadIdx.x == 0) set_flag(&P.status->flags, FLAG_TIMEOUT);
  if (warp == 1) {
    __syncwarp();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(kTmemCols)
                 : "memory");
  }
}

__global__ void tc_reduce_kernel(int M, int N, int splits, const float* __restrict__ partial,
                                 float* __restrict__ C, int64_t ldc) {
  const int64_t total = (int64_t)M * N;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    float s = 0.f;
    for (int z = 0; z < splits; ++z) s += partial[(int64_t)z * total + e];
    C[(e / N) * ldc + e % N] = s;
  }
}

// 2-D FP32 tensor map, 128-byte swizzle, box {32, rows}
bool make_map(CUtensorMap* map, const float* ptr, uint64_t inner, uint64_t outer, int64_t ld,
              uint32_t box_rows) {
  const cuuint64_t dims[2] = {inner, outer};
  const cuuint64_t strides[1] = {(cuuint64_t)ld * sizeof(float)};
  const cuuint32_t box[2] = {32, box_rows};
  const cuuint32_t estr[2] = {1, 1};
  return tma_encoder()(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(ptr), dims, strides,
                  box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int tc_splits(int64_t N, int64_t K, int num_sms) {
  const int64_t tiles = (N + kBM - 1) / kBM;
  int64_t s = std::max<int64_t>(1, num_sms / std::max<int64_t>(1, tiles));
  s = std::min<int64_t>(s, std::max<int64_t>(1, K / (8 * kBK)));
  return (int)s;
}

size_t tc_smem(int NP, int stages, bool split_x) {
  const int xbytes = ((NP * 128 + 1023) / 1024) * 1024;
  return 1024 + (size_t)stages * (2 * kAtileBytes + (split_x ? 2 : 1) * xbytes) +
         (3 * kStages + 1) * 8 + 16;
}

}  // namespace

size_t gemm_tf32_partial_elems(int64_t M, int64_t N, int64_t K, int num_sms) {
  const int s = tc_splits(N, K, num_sms);
  return s > 1 ? (size_t)s * M * N : 0;
}

curid_status gemm_tf32(const Ctx& ctx, bool ta, bool tb, int64_t M, int64_t N, int64_t K,
                       const float* X, int64_t ldx, const float* A, int64_t lda, float* C,
                       int64_t ldc, float* partial, size_t partial_cap, bool split_x) {
  if (ta || M <= 0 || N <= 0 || K <= 0 || M > (int64_t)INT32_MAX / 2) return CURID_UNSUPPORTED;
  if ((reinterpret_cast<uintptr_t>(X) & 15) || (reinterpret_cast<uintptr_t>(A) & 15) ||
      (ldx & 3) || (lda & 3))
    return CURID_UNSUPPORTED;
  if (!tma_encoder()) return CURID_CUDA_ERROR;
  // rows in chunks of at most 256 (the MMA's N), equal up to rounding to 16
  const int nch = (int)((M + 255) / 256);
  const int NP = (int)(((M + nch - 1) / nch + 15) / 16 * 16);
  CUtensorMap mapA, mapX;
  const bool mn = !tb;
  // C = X A: A is K x N (rows k, columns n), box {32 columns, 32 rows};
  // C = X A^T: A is N x K, box {32 K, 128 rows}.
  if (!(mn ? make_map(&mapA, A, (uint64_t)N, (uint64_t)K, lda, 32)
           : make_map(&mapA, A, (uint64_t)K, (uint64_t)N, lda, kBM)))
    return CURID_CUDA_ERROR;
  if (!make_map(&mapX, X, (uint64_t)K, (uint64_t)M, ldx, (uint32_t)NP)) return CURID_CUDA_ERROR;
  // K is split to fill the SMs this caller's decomposition can expect to
  // have: all of them one at a time, a share of them with several in flight
  int splits = tc_splits(N, K, std::max(1, ctx.num_sms / std::max(1, ctx.concurrency) / nch));
  if (splits > 1 && (!partial || (size_t)splits * M * N > partial_cap)) splits = 1;
  const int kchunk = (int)(((K + splits - 1) / splits + kBK - 1) / kBK * kBK);
  splits = (int)((K + kchunk - 1) / kchunk);
  TcParams P;
  P.M = (int)M;
  P.NP = NP;
  P.nch = nch;
  P.N = (int)N;
  P.K = (int)K;
  P.kchunk = kchunk;
  P.mn_major = mn ? 1 : 0;
  P.split_x = split_x ? 1 : 0;
  P.C = C;
  P.ldc = ldc;
  P.partial = splits > 1 ? partial : nullptr;
  P.status = ctx.status;
  // instruction descriptor: FP32 accumulator, TF32 A and B, both K-major,
  // N >> 3, M >> 4
  P.idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(NP >> 3) << 17) |
            ((uint32_t)(kBM >> 4) << 24);
  int stages = kStages;
  while (stages > 2 && tc_smem(NP, stages, split_x) > ctx.smem_optin) --stages;
  const size_t smem = tc_smem(NP, stages, split_x);
  if (smem > ctx.smem_optin) return CURID_UNSUPPORTED;
  P.stages = stages;
  CURID_CUDA(cudaFuncSetAttribute(tc_sketch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem));
  dim3 grid((unsigned)(nch * ((N + kBM - 1) / kBM)), (unsigned)splits);
  tc_sketch_kernel<<<grid, kTcThreads, smem, ctx.stream>>>(mapA, mapX, P);
  CURID_LAUNCHED(ctx);
  if (splits > 1) {
    const int64_t total = M * N;
    const unsigned blocks =
        (unsigned)std::min<int64_t>((total + 255) / 256, 8LL * ctx.num_sms);
    tc_reduce_kernel<<<blocks, 256, 0, ctx.stream>>>((int)M, (int)N, splits, partial, C, ldc);
    CURID_LAUNCHED(ctx);
  }
  return CURID_OK;
}

}  // namespace curid
