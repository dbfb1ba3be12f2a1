// Single-image launches with the extras compiled in: the learned rank bracket, training-row
// output and seed statistics (fim_median_learned, fim_collect_seed_samples). The scan-step
// width is read from the plan at run time.
#include "fim_tile_launch.cuh"

namespace fim {

fim_status launch_tile_kernel_extras(Plan& p, cudaStream_t stream) { return launch_tile_kernel_ks<0, 1>(p, stream); }

fim_status read_and_clear_extras_status() { return read_and_clear_unit_status(); }

}  // namespace fim
