// Batched kernel instantiations of the DF64 form (M = 2 and 3, every launch shape).
#include "batch_kernel.cuh"

namespace quapi {
namespace batchk {

cudaError_t launch_batch_df64(BatchLaunch& L, cudaStream_t st, bool prep) {
    return launch_batch_form<QUAPI_DF64>(L, st, prep);
}

}  // namespace batchk
}  // namespace quapi
