// Single-image launches with a target rank per output pixel (fim_percentile_map, Fig. 14):
// the only kernels that read a rank image, so the others carry none of its code; and the
// pre-pass that turns a percentile map into that rank image.
#include "fim_tile_launch.cuh"

namespace fim {

fim_status launch_tile_kernel_map(Plan& p, cudaStream_t stream) {
    // one kernel set with the scan width read at run time keeps this unit quick to compile
    return launch_tile_kernel_ks<0, 2>(p, stream);
}

fim_status read_and_clear_map_status() { return read_and_clear_unit_status(); }

namespace {

// Rank of each percentile (Fig. 14): clamped to [0, 100] (NaN counts as 0), then
// floor(p / 100 * (n - 1) + 1/2) in fp64 with every operation rounded on its own (no fused
// multiply-add), the same arithmetic as the host's rank for a single percentile.
__global__ void percentile_rank_kernel(const float* __restrict__ pct, long long pitch, int w, int h, int n,
                                       int* __restrict__ ranks) {
    const long long total = (long long)w * h;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int y = (int)(i / w), x = (int)(i - (long long)y * w);
        const float* row = reinterpret_cast<const float*>(reinterpret_cast<const char*>(pct) + y * pitch);
        const float p = fminf(fmaxf(__ldg(row + x), 0.f), 100.f);
        const double t = __dadd_rn(__dmul_rn(__ddiv_rn((double)p, 100.0), (double)(n - 1)), 0.5);
        ranks[i] = min((int)floor(t), n - 1);
    }
}

}  // namespace

fim_status launch_percentile_ranks(const float* pct, long long pct_pitch, int w, int h, int n, int* ranks,
                                   cudaStream_t stream) {
    int sms = 0, dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return FIM_ERR_CUDA;
    const long long total = (long long)w * h;
    const int grid = (int)std::min<long long>((total + 255) / 256, (long long)sms * 8);
    percentile_rank_kernel<<<grid, 256, 0, stream>>>(pct, pct_pitch, w, h, n, ranks);
    return cudaGetLastError() == cudaSuccess ? FIM_OK : FIM_ERR_CUDA;
}

}  // namespace fim
