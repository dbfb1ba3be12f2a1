// Batch class kernels with 8 omnigram groups per scan step (classes of 1024-thread tiles).
#include "fim_batch_launch.cuh"

namespace fim {

fim_status batch_class_k8(const BatchClass& c, const BatchClassArgs* a, int* occ, cudaStream_t stream) {
    return batch_class_dispatch<8>(c, a, occ, stream);
}

fim_status read_and_clear_batch_k8_status() { return read_and_clear_unit_status(); }

}  // namespace fim
