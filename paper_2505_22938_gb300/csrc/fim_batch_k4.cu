// Batch class kernels with 4 omnigram groups per scan step (classes of the small-CTA tiles of
// small kernels).
#include "fim_batch_launch.cuh"

namespace fim {

fim_status batch_class_k4(const BatchClass& c, const BatchClassArgs* a, int* occ, cudaStream_t stream) {
    return batch_class_dispatch<4>(c, a, occ, stream);
}

fim_status read_and_clear_batch_k4_status() { return read_and_clear_unit_status(); }

}  // namespace fim
