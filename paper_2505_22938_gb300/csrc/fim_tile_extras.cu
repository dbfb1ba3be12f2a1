// Single-image launches with the extras compiled in: the learned rank bracket, training-row
// output and seed statistics (fim_median_learned, fim_collect_seed_samples), and several
// target ranks from one ordinal transform (fim_percentiles).
#include "fim_tile_launch.cuh"

namespace fim {

fim_status launch_tile_kernel_extras(Plan& p, cudaStream_t stream) {
    // the 1024-thread tiles of large kernels (where the learned bracket is meant to help) get a
    // compile-time scan width; other plans read it at run time
    return p.scan_groups == 8 ? launch_tile_kernel_ks<8, 1>(p, stream) : launch_tile_kernel_ks<0, 1>(p, stream);
}

fim_status read_and_clear_extras_status() { return read_and_clear_unit_status(); }

}  // namespace fim
