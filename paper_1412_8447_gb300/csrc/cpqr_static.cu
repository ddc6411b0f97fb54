// curid_cpqr_static: the truncated column-pivoted QR without any device
// allocation and without a handle or workspace.
//
// Who needs it: code that may not call cudaMalloc (or ask a framework's
// caching allocator for memory) at the point where it factors a matrix --
// for example a solver step running inside a memory pool whose budget is
// fixed up front, an embedded or real-time service that reserves all of its
// device memory at start-up and must not fail later on an allocation, or a
// plug-in called from a host framework that owns every device allocation
// and offers no scratch buffer.  Such a caller still provides the input Y
// and the outputs J, S (and optionally info); the scratch the CPQR kernel
// needs for its inter-block exchange lives in a fixed array below.
//
// The scratch is a file-scope __device__ array of kStaticScratchBytes
// (4 MiB); every GPU that loads this library keeps it until the process
// exits.  With CUDA's lazy module loading the array is reserved when this
// module is first used on a device, which is this entry point's first call
// there: that call is the one point where the reservation can fail, so make
// it before reserving the rest of device memory.  Host code may not use the
// array's name as a device address (on the host it is only a stand-in
// object), so the first call on each device, with that device current,
// looks the address up with cudaGetSymbolAddress and caches it; make that
// first call before any stream capture too.  All calls share the one array and it
// keeps the previous call's contents, so each call clears the parts that
// must start at zero; two calls whose work overlaps on the GPU (different
// streams, or different host threads) race on the array and must be
// serialised by the caller.
#include <cstddef>
#include <mutex>

#include "kernels.cuh"

using namespace curid;

namespace {

constexpr size_t kStaticScratchBytes = size_t(4) << 20;
static __device__ __align__(256) unsigned char g_cpqr_scratch[kStaticScratchBytes];

constexpr int kMaxDevices = 64;
struct StaticDevice {
  bool ready;
  void* base;  // device address of g_cpqr_scratch on this device
  int num_sms;
  size_t smem_optin;
};
StaticDevice g_devices[kMaxDevices];
std::mutex g_setup_mutex;

// One-time set-up for the current device: resolve the scratch address and
// read the device limits the kernel plan needs.
curid_status setup_current_device(int dev, StaticDevice** out) {
  if (dev < 0 || dev >= kMaxDevices) return CURID_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  StaticDevice& d = g_devices[dev];
  if (!d.ready) {
    void* base = nullptr;
    if (cudaGetSymbolAddress(&base, g_cpqr_scratch) != cudaSuccess || base == nullptr)
      return CURID_CUDA_ERROR;
    int sms = 0, optin = 0, coop = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) !=
            cudaSuccess ||
        cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess)
      return CURID_CUDA_ERROR;
    if (!coop) return CURID_UNSUPPORTED;
    d.base = base;
    d.num_sms = sms;
    d.smem_optin = (size_t)optin;
    d.ready = true;
  }
  *out = &d;
  return CURID_OK;
}

template <typename real>
curid_status run_static(const StaticDevice& d, cudaStream_t stream, const real* Y, int64_t l,
                        int64_t n, int64_t ldy, int k_max, double tol, int32_t* J, real* S,
                        int* info) {
  Ctx ctx{stream, d.num_sms, d.smem_optin, nullptr};
  int grid;
  size_t smem;
  CURID_TRY(cpqr_plan<real>(ctx, l, n, &grid, &smem));
  Carver count(nullptr);
  count.take<StatusBlock>(1);
  CpqrScratch cs;
  cpqr_carve<real>(count, ctx, l, n, &cs);
  if (count.used > kStaticScratchBytes) return CURID_NO_WORKSPACE;
  Carver cv(d.base);
  StatusBlock* st = cv.take<StatusBlock>(1);
  cpqr_carve<real>(cv, ctx, l, n, &cs);
  ctx.status = st;
  CURID_CUDA(cudaMemsetAsync(st, 0, sizeof(StatusBlock), stream));
  CURID_TRY(cpqr_run<real>(ctx, Y, l, n, ldy, k_max, tol, J, S, n, cs, 0));
  // info = the status block's first three words (flags, steps, rank)
  static_assert(offsetof(StatusBlock, flags) == 0 && offsetof(StatusBlock, k_done) == 4 &&
                    offsetof(StatusBlock, k_eff) == 8,
                "info copies flags, k_done and k_eff in this order");
  if (info) CURID_CUDA(cudaMemcpyAsync(info, st, 3 * sizeof(int), cudaMemcpyDeviceToDevice, stream));
  return CURID_OK;
}

}  // namespace

extern "C" curid_status curid_cpqr_static(void* stream, curid_dtype dtype, const void* Y,
                                          int64_t l, int64_t n, int64_t ldy, int k, double tol,
                                          int32_t* J, void* S, int* info) {
  if (!Y || !J || !S || l <= 0 || n <= 0 || ldy < n || k < 0 || tol < 0)
    return CURID_INVALID_ARG;
  if (k == 0 && !(tol > 0)) return CURID_INVALID_ARG;
  if (k > std::min(l, n)) return CURID_INVALID_ARG;
  if (dtype != CURID_F32 && dtype != CURID_F64) return CURID_INVALID_ARG;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return CURID_CUDA_ERROR;
  StaticDevice* d = nullptr;
  CURID_TRY(setup_current_device(dev, &d));
  const int k_max = k > 0 ? k : (int)std::min(l, n);
  const double t = k > 0 ? 0.0 : tol;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (dtype == CURID_F64)
    return run_static<double>(*d, s, static_cast<const double*>(Y), l, n, ldy, k_max, t, J,
                              static_cast<double*>(S), info);
  return run_static<float>(*d, s, static_cast<const float*>(Y), l, n, ldy, k_max, t, J,
                           static_cast<float*>(S), info);
}
