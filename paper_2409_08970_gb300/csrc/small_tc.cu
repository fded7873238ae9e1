// Tensor-core (tcgen05) kernel for n <= 64. Placeholder: not yet enabled.
#include "internal.cuh"

namespace dctplus {

dctplus_status setup_small_tc(dctplus_plan_t) { return DCTPLUS_OK; }

bool small_tc_available(dctplus_plan_t) { return false; }

bool group_tc_available(dctplus_group_t) { return false; }

dctplus_status launch_small_tc(dctplus_plan_t, const float*, int64_t, float*, int64_t, int64_t,
                               cudaStream_t) {
    return DCTPLUS_ERR_UNSUPPORTED;
}

dctplus_status launch_group_tc(dctplus_group_t, const float*, float*, cudaStream_t) {
    return DCTPLUS_ERR_UNSUPPORTED;
}

}  // namespace dctplus
