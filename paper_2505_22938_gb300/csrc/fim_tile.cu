// Single-image launches with 8 omnigram groups per scan step (the 1024-thread tiles of large
// kernels) and the dispatch between the sets of kernels.
#include "fim_tile_launch.cuh"

namespace fim {

fim_status launch_tile_kernel(Plan& p, cudaStream_t stream) {
    if (p.rank_map != nullptr) return launch_tile_kernel_map(p, stream);
    if (p.model != nullptr || p.samples != nullptr || p.stats != nullptr || p.nranks > 1 || p.multi)
        return launch_tile_kernel_extras(p, stream);
    return p.scan_groups == 4 ? launch_tile_kernel_k4(p, stream) : launch_tile_kernel_ks<8>(p, stream);
}

fim_status launch_tile_kernel_fixed(Plan& p, unsigned char* scratch, size_t capacity, cudaStream_t stream,
                                    bool launch) {
    return p.scan_groups == 4 ? launch_tile_kernel_fixed_k4(p, scratch, capacity, stream, launch)
                              : launch_tile_kernel_fixed_ks<8>(p, scratch, capacity, stream, launch);
}

fim_status read_and_clear_device_status(cudaStream_t stream) {
    if (cudaStreamSynchronize(stream) != cudaSuccess) return FIM_ERR_CUDA;
    // every translation unit with device code has its own status word: report the first error
    const fim_status a = read_and_clear_unit_status();
    const fim_status b = read_and_clear_k4_status();
    const fim_status c = read_and_clear_batch_k8_status();
    const fim_status c4 = read_and_clear_batch_k4_status();
    const fim_status d = read_and_clear_extras_status();
    const fim_status e = read_and_clear_map_status();
    for (fim_status x : {a, b, c, c4, d, e})
        if (x != FIM_OK) return x;
    return FIM_OK;
}

}  // namespace fim
