// tcgen05 tensor-core GEMMs (placeholder until the kernel lands).
#include <cuda_bf16.h>

#include "common.cuh"

namespace apgb {
size_t tc_similarity_pad_rows() { return 128; }
int32_t tc_similarity_bf16(const __nv_bfloat16*, const float*, int, int, float*, int64_t,
                           cudaStream_t) {
    return AP_ERR_UNSUPPORTED;
}
}  // namespace apgb
