// Products with a BF16 data matrix A on the tcgen05 tensor cores:
// C = X A or C = X A^T with X the FP32 sketch operand (Omega, or an
// orthonormal basis between power steps, Section 5.3), FP32 accumulation in
// TMEM.
//
// Precision: A is stored in BF16, so its values enter the MMA exactly.  X is
// split once, before the product, into X = X_hi + X_lo with X_hi the BF16
// rounding of X and X_lo the BF16 rounding of the remainder (about 16
// significant bits together), and each K step issues two BF16 MMAs,
// A X_hi^T and A X_lo^T.  A BF16-rounded X alone would perturb every sample
// row by 2^-9 relative.
//
// Tiling as in the TF32 kernel: D = C^T, the MMA's M = 128 output columns of
// C, its N = a chunk of the sample's rows (<= 256; l > 256 is cut into
// equal chunks, since a 128-lane accumulator holds at most 512 FP32 columns
// of TMEM).  The chunks of one column tile are neighbouring CTAs (the chunk
// is the grid's fastest index), so they stream the same A tiles at the same
// time and A comes from HBM about once.  Operands use the 128-byte swizzle:
// for C = X A^T the rows of A are K-major and come by TMA as they are; for
// C = X A the TMA brings MN-major 64 x 64 boxes and the MMA reads them as an
// MN-major operand (kind::f16 allows either major-ness for 16-bit types), so
// no thread touches A.  Warp 0 issues TMA, warp 1 the MMAs, warps 4-7 run
// the epilogue.  Every mbarrier wait is bounded.
#include <cuda_bf16.h>

#include "kernels.cuh"
#include "tcgen05.cuh"

namespace curid {

namespace {

constexpr int kBM = 128;               // output columns per CTA (MMA M)
constexpr int kBK = 64;                // K per stage: 64 BF16 = one 128-byte swizzle row
constexpr int kATile = kBM * kBK * 2;  // 16 KB
constexpr int kMaxStages = 3;
constexpr int kThreads = 256;
constexpr int kTmemCols = 256;

struct Bf16Params {
  int M;          // rows of C (sample rows)
  int N;          // columns of C
  int K;
  int chunk;      // sample rows per grid row (multiple of 16, <= 256)
  int mn_major;   // 1: C = X A (A tiles MN-major, transposed in shared memory)
  int stages;
  float* C;
  int64_t ldc;
  StatusBlock* status;
  uint32_t idesc;
};

size_t bf16_stage_bytes(int chunk) { return (size_t)kATile + 2 * (size_t)chunk * 128; }

size_t bf16_smem(int chunk, int stages) {
  return 1024 + (size_t)stages * bf16_stage_bytes(chunk) + (2 * kMaxStages + 1) * 8 + 16;
}

__global__ void __launch_bounds__(kThreads, 1)
tc_bf16_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmXh,
               const __grid_constant__ CUtensorMap tmXl, Bf16Params P) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  const uintptr_t base = (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023);
  const bool mn = P.mn_major != 0;
  const int S = P.stages;
  const uint32_t xbytes = (uint32_t)P.chunk * 128u;
  unsigned char* Ak[kMaxStages];  // A tile: K-major 128 rows, or two MN-major 64 x 64 boxes
  unsigned char* Xh[kMaxStages];
  unsigned char* Xl[kMaxStages];
  unsigned char* p = reinterpret_cast<unsigned char*>(base);
  for (int s = 0; s < S; ++s) {
    Ak[s] = p;
    p += kATile;
    Xh[s] = p;
    Xl[s] = p + xbytes;
    p += 2 * xbytes;
  }
  uint64_t* bars = reinterpret_cast<uint64_t*>(p);  // full[S], empty[S], acc
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * kMaxStages + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  auto full = [&](int s) { return smem_u32(bars + s); };
  auto empty = [&](int s) { return smem_u32(bars + kMaxStages + s); };
  const uint32_t acc_bar = smem_u32(bars + 2 * kMaxStages);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int row0 = blockIdx.x * P.chunk;  // chunk fastest: a column tile's chunks run together
  const int n0 = blockIdx.y * kBM;
  const int nk = (P.K + kBK - 1) / kBK;

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(full(s), 1);
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
    // ---- producer ----
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmA)) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmXh)) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmXl)) : "memory");
    int issued = 0;
    for (int i = 0; i < nk; ++i) {
      const int s = i % S;
      const uint32_t ph = (uint32_t)(i / S) & 1u;
      if (i >= S && !mbar_wait(empty(s), ph ^ 1u)) {
        *abort_flag = 1;
        atomicCAS(&P.status->timeout_site, 0, (5 << 24) | (s << 16) | i);
        break;
      }
      if (*abort_flag) break;
      mbar_expect_tx(full(s), (uint32_t)kATile + 2 * xbytes);
      const int k = i * kBK;
      if (mn) {
        tma_load_2d(smem_u32(Ak[s]), &tmA, n0, k, full(s));
        tma_load_2d(smem_u32(Ak[s] + kATile / 2), &tmA, n0 + 64, k, full(s));
      } else {
        tma_load_2d(smem_u32(Ak[s]), &tmA, k, n0, full(s));
      }
      tma_load_2d(smem_u32(Xh[s]), &tmXh, k, row0, full(s));
      tma_load_2d(smem_u32(Xl[s]), &tmXl, k, row0, full(s));
      issued = i + 1;
    }
    if (*abort_flag) {
      for (int i = max(0, issued - S); i < issued; ++i)
        mbar_wait(full(i % S), (uint32_t)(i / S) & 1u);
    }
  } else if (warp == 1 && lane == 0) {
    // ---- MMA issuer: per 16-element K step, A X_hi^T then A X_lo^T ----
    for (int i = 0; i < nk; ++i) {
      const int s = i % S;
      const uint32_t ph = (uint32_t)(i / S) & 1u;
      if (!mbar_wait(full(s), ph) || *abort_flag) {
        *abort_flag = 1;
        atomicCAS(&P.status->timeout_site, 0, (6 << 24) | (s << 16) | i);
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t a = smem_u32(Ak[s]), xh = smem_u32(Xh[s]), xl = smem_u32(Xl[s]);
#pragma unroll
      for (int kk = 0; kk < kBK / 16; ++kk) {
        // K-major: 16 K values are 32 bytes along each 128-byte row; MN-major:
        // two 8-row K groups (1024 bytes apart, the stride byte offset), the
        // second 64 columns 8 KB on (the leading byte offset)
        const uint64_t da = mn ? smem_desc(a + kk * 2048, kATile / 2, 1024)
                               : smem_desc(a + kk * 32, 16, 1024);
        const uint64_t dh = smem_desc(xh + kk * 32, 16, 1024);
        const uint64_t dl = smem_desc(xl + kk * 32, 16, 1024);
        mma_f16(tmem, da, dh, P.idesc, (i > 0 || kk > 0) ? 1u : 0u);
        mma_f16(tmem, da, dl, P.idesc, 1u);
      }
      mma_commit(empty(s));
    }
    mma_commit(acc_bar);
  } else if (warp >= 4) {
    // ---- epilogue: TMEM -> registers -> C ----
    int ok = 0;
    if (lane == 0) {
      ok = mbar_wait(acc_bar, 0) ? 1 : 0;
      if (!ok) {
        *abort_flag = 1;
        atomicCAS(&P.status->timeout_site, 0, 8 << 24);
      }
      ok = ok && !*abort_flag;
    }
    ok = __shfl_sync(0xffffffffu, ok, 0);
    __syncwarp();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (ok) {
      const int q = warp - 4;
      const int col = n0 + q * 32 + lane;
      const int rows = min(P.chunk, P.M - row0);
      for (int c0 = 0; c0 < P.chunk; c0 += 32) {
        uint32_t r[32];
        tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)c0, r);
        if (col < P.N) {
#pragma unroll
          for (int j = 0; j < 32; ++j)
            if (c0 + j < rows) P.C[(int64_t)(row0 + c0 + j) * P.ldc + col] = __uint_as_float(r[j]);
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

// X (rows x K, ldx, float) -> hi, lo (rows_pad x kpad, bfloat16): hi = bf16(x),
// lo = bf16(x - hi); zero outside rows x K.
__global__ void split_bf16_kernel(const float* __restrict__ X, int64_t ldx, int rows, int K,
                                  int rows_pad, int kpad, __nv_bfloat16* __restrict__ hi,
                                  __nv_bfloat16* __restrict__ lo) {
  const int64_t total = (int64_t)rows_pad * kpad;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / kpad, k = e % kpad;
    const float x = (r < rows && k < K) ? X[r * ldx + k] : 0.f;
    const __nv_bfloat16 h = __float2bfloat16_rn(x);
    hi[e] = h;
    lo[e] = __float2bfloat16_rn(x - __bfloat162float(h));
  }
}

// 2-D BF16 tensor map, 128-byte swizzle, box {64, box_rows}
bool make_map_bf16(CUtensorMap* map, const void* ptr, uint64_t inner, uint64_t outer, int64_t ld,
                   uint32_t box_rows) {
  const cuuint64_t dims[2] = {inner, outer};
  const cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
  const cuuint32_t box[2] = {64, box_rows};
  const cuuint32_t estr[2] = {1, 1};
  return tma_encoder()(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(ptr), dims,
                       strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                       CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                       CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

void bf16_chunking(int64_t M, int* chunk, int* nchunks) {
  const int nc = (int)((M + 255) / 256);
  const int per = (int)((M + nc - 1) / nc);
  *chunk = (per + 15) / 16 * 16;
  *nchunks = nc;
}

}  // namespace

size_t gemm_bf16_split_elems(int64_t M, int64_t K) {
  int chunk, nch;
  bf16_chunking(M, &chunk, &nch);
  const int64_t kpad = (K + 7) / 8 * 8;
  return 2 * (size_t)chunk * nch * kpad;
}

curid_status gemm_bf16(const Ctx& ctx, bool tb, int64_t M, int64_t N, int64_t K, const float* X,
                       int64_t ldx, const void* A, int64_t lda, float* C, int64_t ldc,
                       void* split, size_t split_elems) {
  if (M <= 0 || N <= 0 || K <= 0) return CURID_UNSUPPORTED;
  if ((reinterpret_cast<uintptr_t>(A) & 15) || (lda & 7) || (reinterpret_cast<uintptr_t>(split) & 15))
    return CURID_UNSUPPORTED;
  if (split_elems < gemm_bf16_split_elems(M, K)) return CURID_NO_WORKSPACE;
  if (!tma_encoder()) return CURID_CUDA_ERROR;
  int chunk, nch;
  bf16_chunking(M, &chunk, &nch);
  const int rows_pad = chunk * nch;
  const int kpad = (int)((K + 7) / 8 * 8);
  __nv_bfloat16* hi = static_cast<__nv_bfloat16*>(split);
  __nv_bfloat16* lo = hi + (size_t)rows_pad * kpad;
  {
    const int64_t total = (int64_t)rows_pad * kpad;
    const unsigned g = (unsigned)std::max<int64_t>(1, std::min<int64_t>((total + 255) / 256,
                                                                        16LL * ctx.num_sms));
    split_bf16_kernel<<<g, 256, 0, ctx.stream>>>(X, ldx, (int)M, (int)K, rows_pad, kpad, hi, lo);
    CURID_LAUNCHED(ctx);
  }
  const bool mn = !tb;
  CUtensorMap mapA, mapH, mapL;
  // C = X A: A is K x N (rows k), boxes {64 columns, 64 rows};
  // C = X A^T: A is N x K, box {64 K, 128 rows}.
  if (!(mn ? make_map_bf16(&mapA, A, (uint64_t)N, (uint64_t)K, lda, kBK)
           : make_map_bf16(&mapA, A, (uint64_t)K, (uint64_t)N, lda, kBM)))
    return CURID_CUDA_ERROR;
  if (!make_map_bf16(&mapH, hi, (uint64_t)kpad, (uint64_t)rows_pad, kpad, (uint32_t)chunk) ||
      !make_map_bf16(&mapL, lo, (uint64_t)kpad, (uint64_t)rows_pad, kpad, (uint32_t)chunk))
    return CURID_CUDA_ERROR;
  int stages = kMaxStages;
  while (stages > 1 && bf16_smem(chunk, stages) > ctx.smem_optin) --stages;
  if (stages < 2) return CURID_UNSUPPORTED;
  Bf16Params P;
  P.M = (int)M;
  P.N = (int)N;
  P.K = (int)K;
  P.chunk = chunk;
  P.mn_major = mn ? 1 : 0;
  P.stages = stages;
  P.C = C;
  P.ldc = ldc;
  P.status = ctx.status;
  // instruction descriptor (kind::f16): FP32 accumulator, BF16 A and B, A
  // MN-major (bit 15) for C = X A else K-major, B K-major, N >> 3, M >> 4
  P.idesc = (1u << 4) | (1u << 7) | (1u << 10) | (mn ? 1u << 15 : 0u) |
            ((uint32_t)(chunk >> 3) << 17) | ((uint32_t)(kBM >> 4) << 24);
  const size_t smem = bf16_smem(chunk, stages);
  CURID_CUDA(cudaFuncSetAttribute(tc_bf16_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem));
  dim3 grid((unsigned)nch, (unsigned)((N + kBM - 1) / kBM));
  tc_bf16_kernel<<<grid, kThreads, smem, ctx.stream>>>(mapA, mapH, mapL, P);
  CURID_LAUNCHED(ctx);
  return CURID_OK;
}

}  // namespace curid
