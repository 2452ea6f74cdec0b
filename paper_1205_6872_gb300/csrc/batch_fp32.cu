// Batched kernel instantiations of the FP32 form (M = 2 and 3, every launch shape).
#include "batch_kernel.cuh"

namespace quapi {
namespace batchk {

cudaError_t launch_batch_fp32(BatchLaunch& L, cudaStream_t st, bool prep) {
    return launch_batch_form<QUAPI_FP32>(L, st, prep);
}

}  // namespace batchk
}  // namespace quapi
