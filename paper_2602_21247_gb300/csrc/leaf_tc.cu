// leaf_tc.cu -- A2..A4 on the tcgen05 tensor cores (byte data, exact BF16 Gram).
#include "internal.cuh"

namespace pipnn {

int leaf_pick_tc(const void *, uint64_t, uint32_t, int, const int32_t *, const uint64_t *, const uint32_t *,
                 uint64_t, const uint32_t *, const uint64_t *, uint32_t, uint32_t *, uint32_t *, float *,
                 Workspace &, cudaEvent_t, cudaEvent_t, uint32_t *) {
    return set_error(PIPNN_EUNSUPPORTED, "tensor-core leaf engine not built");
}

}  // namespace pipnn
