#pragma once
// Single-image launches of the tile pipeline, for one number KS of omnigram groups per scan
// step: each CTA takes Tx x Ty output tiles from a device-side queue and filters them one
// after the other (Sec. 3.3, Sec. 4.2). Included by one translation unit per KS, so that the
// two sets of kernels compile in parallel.
#include "fim_tile_pipeline.cuh"

namespace fim {
namespace {

// Persistent CTAs: each takes tiles from the queue counter in the scratch header until none are
// left. The counter is zeroed on the stream before every launch.
template <int DT, int SHAPE, int W, int OG, int KS, int XT>
__global__ void __launch_bounds__(1024, 1) tile_median_kernel(const __grid_constant__ Plan P) {
    __shared__ int s_tile;
    const int tid = threadIdx.x;
    unsigned char* gslice = P.scratch + 256 + (size_t)blockIdx.x * (size_t)P.scratch_per_cta;
    load_tables(P);
    unsigned int* counter = reinterpret_cast<unsigned int*>(P.scratch);
    const Grp G{tid, tid & 31, tid >> 5, (int)blockDim.x, 0, 0};
    // the footprint copies' mbarrier (scan scratch words 34-35), initialised before the first tile
    extern __shared__ __align__(16) unsigned char smem_dyn[];
    TmaState tma{0u, 0};
    if (P.use_tma && tid == 0) mbar_init(reinterpret_cast<uint64_t*>(smem_dyn + P.off_misc + 34 * 4));
    for (;;) {
        if (tid == 0) s_tile = (int)atomicAdd(counter, 1u);
        __syncthreads();
        const int tile = s_tile;
        if (tile >= P.ntiles) break;
        stamp(P, tile, 0, G);
        process_tile<DT, SHAPE, W, OG, KS, XT>(P, P.tile0 + tile, gslice, G, &tma);
    }
}

template <int DT, int SHAPE, int W, int OG, int KS, int XT>
fim_status launch_typed(Plan& p, cudaStream_t stream) {
    auto fn = tile_median_kernel<DT, SHAPE, W, OG, KS, XT>;
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, p.smem_bytes) != cudaSuccess) {
        cudaGetLastError();
        return FIM_ERR_CUDA;
    }
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, p.threads, p.smem_bytes) != cudaSuccess || occ < 1) {
        cudaGetLastError();
        return FIM_ERR_UNSUPPORTED;
    }
    const long long tiles = p.tile_count > 0 ? (long long)p.tile_count : (long long)p.tiles_x * p.tiles_y;
    if (tiles > 0x7fffffffLL) return FIM_ERR_UNSUPPORTED;
    p.ntiles = (int)tiles;
    const int grid = (int)std::min<long long>(tiles, (long long)occ * device_sm_count());
    unsigned char* scratch = nullptr;
    fim_status s = get_scratch(stream, 256 + (size_t)grid * (size_t)p.scratch_per_cta, &scratch);
    if (s != FIM_OK) return s;
    p.scratch = scratch;
    attach_tma(p);
    if (cudaMemsetAsync(scratch, 0, 16, stream) != cudaSuccess) return FIM_ERR_CUDA;
    fn<<<grid, p.threads, p.smem_bytes, stream>>>(p);
    if (cudaGetLastError() != cudaSuccess) return FIM_ERR_CUDA;
    return FIM_OK;
}

// Same launch, but on a caller-provided workspace of fixed capacity (no allocation). Returns
// FIM_ERR_UNSUPPORTED when this launch would need more workspace than `capacity` bytes. With
// `launch` false it only answers that question (FIM_OK: it fits) and launches nothing.
template <int DT, int SHAPE, int W, int OG, int KS>
fim_status launch_typed_fixed(Plan& p, unsigned char* scratch, size_t capacity, cudaStream_t stream, bool launch) {
    auto fn = tile_median_kernel<DT, SHAPE, W, OG, KS, 0>;
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, p.smem_bytes) != cudaSuccess) {
        cudaGetLastError();
        return FIM_ERR_CUDA;
    }
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, p.threads, p.smem_bytes) != cudaSuccess || occ < 1) {
        cudaGetLastError();
        return FIM_ERR_UNSUPPORTED;
    }
    const long long tiles = (long long)p.tiles_x * p.tiles_y;
    if (tiles > 0x7fffffffLL) return FIM_ERR_UNSUPPORTED;
    p.ntiles = (int)tiles;
    const int grid = (int)std::min<long long>(tiles, (long long)occ * device_sm_count());
    if (256 + (unsigned long long)grid * (unsigned long long)p.scratch_per_cta > capacity) return FIM_ERR_UNSUPPORTED;
    if (!launch) return FIM_OK;
    p.scratch = scratch;
    attach_tma(p);
    if (cudaMemsetAsync(scratch, 0, 16, stream) != cudaSuccess) return FIM_ERR_CUDA;  // tile queue counter
    fn<<<grid, p.threads, p.smem_bytes, stream>>>(p);
    if (cudaGetLastError() != cudaSuccess) return FIM_ERR_CUDA;
    return FIM_OK;
}

template <int DT, int SHAPE, int KS>
fim_status launch_w_fixed(Plan& p, unsigned char* scratch, size_t capacity, cudaStream_t stream, bool launch) {
    if (p.wide) return launch_typed_fixed<DT, SHAPE, 1, 1, KS>(p, scratch, capacity, stream, launch);
    return p.loc_om < 0 ? launch_typed_fixed<DT, SHAPE, 0, 1, KS>(p, scratch, capacity, stream, launch)
                        : launch_typed_fixed<DT, SHAPE, 0, 0, KS>(p, scratch, capacity, stream, launch);
}

template <int DT, int SHAPE, int KS, int XT>
fim_status launch_w(Plan& p, cudaStream_t stream) {
    if (p.wide) return launch_typed<DT, SHAPE, 1, 1, KS, XT>(p, stream);
    return p.loc_om < 0 ? launch_typed<DT, SHAPE, 0, 1, KS, XT>(p, stream)
                        : launch_typed<DT, SHAPE, 0, 0, KS, XT>(p, stream);
}


template <int KS, int XT = 0>
fim_status launch_tile_kernel_ks(Plan& p, cudaStream_t stream) {
    const bool disk = p.shape == kShapeDisk;
    switch (p.dtype) {
        case FIM_U8:
            return disk ? launch_w<FIM_U8, kShapeDisk, KS, XT>(p, stream)
                        : launch_w<FIM_U8, kShapeSpans, KS, XT>(p, stream);
        case FIM_U16:
            return disk ? launch_w<FIM_U16, kShapeDisk, KS, XT>(p, stream)
                        : launch_w<FIM_U16, kShapeSpans, KS, XT>(p, stream);
        case FIM_F32:
            return disk ? launch_w<FIM_F32, kShapeDisk, KS, XT>(p, stream)
                        : launch_w<FIM_F32, kShapeSpans, KS, XT>(p, stream);
    }
    return FIM_ERR_INVALID_ARG;
}

template <int KS>
fim_status launch_tile_kernel_fixed_ks(Plan& p, unsigned char* scratch, size_t capacity, cudaStream_t stream,
                                       bool launch) {
    const bool disk = p.shape == kShapeDisk;
    switch (p.dtype) {
        case FIM_U8:
            return disk ? launch_w_fixed<FIM_U8, kShapeDisk, KS>(p, scratch, capacity, stream, launch)
                        : launch_w_fixed<FIM_U8, kShapeSpans, KS>(p, scratch, capacity, stream, launch);
        case FIM_U16:
            return disk ? launch_w_fixed<FIM_U16, kShapeDisk, KS>(p, scratch, capacity, stream, launch)
                        : launch_w_fixed<FIM_U16, kShapeSpans, KS>(p, scratch, capacity, stream, launch);
        case FIM_F32:
            return disk ? launch_w_fixed<FIM_F32, kShapeDisk, KS>(p, scratch, capacity, stream, launch)
                        : launch_w_fixed<FIM_F32, kShapeSpans, KS>(p, scratch, capacity, stream, launch);
    }
    return FIM_ERR_INVALID_ARG;
}

}  // namespace
}  // namespace fim
