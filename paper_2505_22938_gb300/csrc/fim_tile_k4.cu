// Single-image launches with 4 omnigram groups per scan step (the small-CTA tiles of small
// kernels, where scans are short).
#include "fim_tile_launch.cuh"

namespace fim {

fim_status launch_tile_kernel_k4(Plan& p, cudaStream_t stream) { return launch_tile_kernel_ks<4>(p, stream); }

fim_status launch_tile_kernel_fixed_k4(Plan& p, unsigned char* scratch, size_t capacity, cudaStream_t stream,
                                       bool launch) {
    return launch_tile_kernel_fixed_ks<4>(p, scratch, capacity, stream, launch);
}

fim_status read_and_clear_k4_status() { return read_and_clear_unit_status(); }

}  // namespace fim
