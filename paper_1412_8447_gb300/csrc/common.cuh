// Shared definitions of the CUR / ID library: handle, workspace carving,
// device status flags, small device helpers.
#pragma once

#include <cuda_runtime.h>
#include <cstddef>
#include <cstdint>

#include "../../include/curid.h"

namespace curid {

// Device status flags (OR-ed by kernels into the status block).
enum : int {
  FLAG_RANK_DEFICIENT = 1,
  FLAG_BREAKDOWN = 2,
  FLAG_NONFINITE = 4,
  FLAG_TIMEOUT = 8,
};

// Status block at the start of every workspace: written by kernels,
// read back by curid_last_status().
struct StatusBlock {
  int flags;      // OR of FLAG_*
  int k_done;     // CPQR steps taken by the column CPQR
  int k_eff;      // numerical rank (k_out reported to the caller)
  int k_row;      // rank found by the row CPQR (row ID of C)
  int timeout_site;  // first wait that timed out: (role << 24) | (stage << 16) | iteration
  int pad[59];
};
static_assert(sizeof(StatusBlock) == 256, "status block is 256 bytes");

// Bump allocator over the caller's workspace.  With base == nullptr it only
// counts, which is how curid_workspace_size() sizes a request.
struct Carver {
  char* base;
  size_t used = 0;
  explicit Carver(void* b) : base(static_cast<char*>(b)) {}
  template <typename T>
  T* take(size_t count) {
    size_t off = (used + 255) & ~size_t(255);
    used = off + count * sizeof(T);
    return base ? reinterpret_cast<T*>(base + off) : nullptr;
  }
};

inline size_t dtype_size(curid_dtype dt) { return dt == CURID_F64 ? 8 : 4; }

// Spin budget for inter-block waits, in SM clock cycles (about 2 s).
constexpr long long kSpinBudget = 4000000000LL;

__device__ __forceinline__ void set_flag(int* flags, int f) { atomicOr(flags, f); }

template <typename real>
__device__ __forceinline__ real warp_sum(real v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Loads and stores between CTAs of one GPU: relaxed at GPU scope (performed
// in L2, never from a stale L1 line).  Volatile accesses would be
// system-scope, which on a GPU whose memory the CPU caches coherently costs
// more per access.
__device__ __forceinline__ unsigned long long ld_gpu_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ int ld_gpu_i32(const int* p) {
  int v;
  asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_gpu_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

}  // namespace curid

#include <vector>

// One timed phase of a call: CUDA events recorded on the handle's stream.
struct curid_phase_rec {
  int phase;
  cudaEvent_t start, stop;
};

struct curid_handle {
  int device = 0;
  cudaStream_t stream = nullptr;
  char* ws = nullptr;
  size_t ws_bytes = 0;
  int num_sms = 0;
  size_t smem_optin = 0;
  // profiling (curid_profile / curid_profile_read)
  int profiling = 0;
  long long launches = 0;
  std::vector<curid_phase_rec> recs;
  std::vector<cudaEvent_t> pool;
  size_t pool_used = 0;
  // batched column ID: launch shape chosen by the autotuner ([0] float64,
  // [1] float32; -1 = not tuned)
  int batch_shape[2] = {-1, -1};
  // bound of every inter-block wait in SM clock cycles (curid_set_timeout)
  long long spin = curid::kSpinBudget;
  // decompositions the caller keeps in flight on this GPU (curid_set_concurrency)
  int concurrency = 1;
};

#define CURID_CUDA(call)                                \
  do {                                                  \
    cudaError_t e_ = (call);                            \
    if (e_ != cudaSuccess) return CURID_CUDA_ERROR;     \
  } while (0)

#define CURID_TRY(call)                                 \
  do {                                                  \
    curid_status s_ = (call);                           \
    if (s_ != CURID_OK) return s_;                      \
  } while (0)
