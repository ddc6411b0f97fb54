// Tensor-core (tcgen05, TF32 operands, FP32 accumulation) products of the
// randomized front end.  Placeholder until the kernel lands: reports the
// request as unsupported so callers that ask for TF32 get a clear status.
#include "kernels.cuh"

namespace curid {

curid_status gemm_tf32(const Ctx&, bool, bool, int64_t, int64_t, int64_t, const float*, int64_t,
                       const float*, int64_t, float*, int64_t, float*, size_t) {
  return CURID_UNSUPPORTED;
}

size_t gemm_tf32_partial_elems(int64_t, int64_t, int64_t, int) { return 0; }

}  // namespace curid
