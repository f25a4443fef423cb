// k_tc.cu -- tensor-core engine for fused k = 5, 6 blocks (complex64).
#include "hq_internal.cuh"

namespace hq {

hq_status launch_tc_block(void *, int, int, const int *, const double *, int64_t, int, cudaStream_t)
{
    return HQ_ERR_ARG;
}

}  // namespace hq
