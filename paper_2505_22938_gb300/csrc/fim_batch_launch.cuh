#pragma once
// Batched persistent launch (device side): one persistent kernel per class of jobs that share a
// tile-pipeline instantiation (dtype, kernel shape, omnigram encoding and home, scan width) and a
// CTA size. A class kernel's CTAs take tiles from the class's device-side queue, which runs over
// the tiles of all its jobs in the order the host sorted them (decreasing cost per tile), and
// reload the plan of a tile's job when it changes. Each class kernel is the same specialised
// pipeline as the single-image kernel of that class, at the CTA size its plans ask for. Included
// by one translation unit per scan width, so that the two sets compile in parallel.
#include "fim_tile_pipeline.cuh"

namespace fim {
namespace {

// The job of class-local tile t: the last j with tile_start[j] <= t (tile_start is increasing,
// tile_start[0] = 0, njobs entries).
__device__ __forceinline__ int batch_job_of(const int* __restrict__ tile_start, int njobs, int t) {
    int lo = 0, hi = njobs - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(tile_start + mid) <= t)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

template <int DT, int SHAPE, int W, int OG, int KS>
__global__ void __launch_bounds__(1024, 1) batch_class_kernel(const __grid_constant__ BatchClassArgs A) {
    __shared__ int s_tile, s_job;
    // the current job's plan scalars (everything before the tables); the tables go to the
    // dynamic shared memory as in the single-image kernel
    __shared__ __align__(16) unsigned char s_plan[kPlanScalarBytes];
    // the footprint copies' mbarrier, one for the CTA's whole run (the jobs' tensor maps stay in
    // the plan array in global memory)
    __shared__ __align__(8) uint64_t s_bar;
    const int tid = threadIdx.x;
    unsigned char* gslice = A.scratch + (size_t)blockIdx.x * (size_t)A.scratch_per_cta;
    const Grp G{tid, tid & 31, tid >> 5, (int)blockDim.x, 0, 0};
    TmaState tma{0u, 0};
    if (tid == 0) mbar_init(&s_bar);  // visible after the loop's first barrier
    int cur = -1;
    for (;;) {
        if (tid == 0) {
            const int t = (int)atomicAdd(A.counter, 1u);
            s_tile = t;
            s_job = t < A.total_tiles ? batch_job_of(A.tile_start, A.njobs, t) : -1;
        }
        __syncthreads();
        const int t = s_tile, job = s_job;
        if (t >= A.total_tiles) break;
        if (job != cur) {  // every thread is past the previous tile's last barrier
            const Plan* gp = A.plans + job;
            load_tables(*gp);
            const uint32_t* src = reinterpret_cast<const uint32_t*>(gp);
            uint32_t* dst = reinterpret_cast<uint32_t*>(s_plan);
            for (int i = tid; i < (int)(kPlanScalarBytes / 4); i += blockDim.x) dst[i] = src[i];
            __syncthreads();
            cur = job;
        }
        const Plan& P = *reinterpret_cast<const Plan*>(s_plan);
        process_tile<DT, SHAPE, W, OG, KS, 0, 2>(P, t - __ldg(A.tile_start + job), gslice, G, &tma, &s_bar,
                                                 &A.plans[job].tmap);
    }
}

template <int DT, int SHAPE, int W, int OG, int KS>
fim_status batch_class_typed(const BatchClassArgs* a, int threads, int smem, int* occ, cudaStream_t stream,
                             int grid) {
    auto fn = batch_class_kernel<DT, SHAPE, W, OG, KS>;
    if (a == nullptr) {  // set-up: shared-memory opt-in and the resident CTAs per SM
        if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, fn, threads, smem) != cudaSuccess) {
            cudaGetLastError();
            return FIM_ERR_CUDA;
        }
        return *occ >= 1 ? FIM_OK : FIM_ERR_UNSUPPORTED;
    }
    fn<<<grid, threads, smem, stream>>>(*a);
    return cudaGetLastError() == cudaSuccess ? FIM_OK : FIM_ERR_CUDA;
}

template <int DT, int SHAPE, int KS>
fim_status batch_class_w(const BatchClass& c, const BatchClassArgs* a, int* occ, cudaStream_t stream) {
    if (c.wide) return batch_class_typed<DT, SHAPE, 1, 1, KS>(a, c.threads, c.smem, occ, stream, c.grid);
    return c.og ? batch_class_typed<DT, SHAPE, 0, 1, KS>(a, c.threads, c.smem, occ, stream, c.grid)
                : batch_class_typed<DT, SHAPE, 0, 0, KS>(a, c.threads, c.smem, occ, stream, c.grid);
}

// a == nullptr: set-up (fills *occ); otherwise launches the class kernel with c.grid CTAs.
template <int KS>
fim_status batch_class_dispatch(const BatchClass& c, const BatchClassArgs* a, int* occ, cudaStream_t stream) {
    const bool disk = c.shape == kShapeDisk;
    switch (c.dtype) {
        case FIM_U8:
            return disk ? batch_class_w<FIM_U8, kShapeDisk, KS>(c, a, occ, stream)
                        : batch_class_w<FIM_U8, kShapeSpans, KS>(c, a, occ, stream);
        case FIM_U16:
            return disk ? batch_class_w<FIM_U16, kShapeDisk, KS>(c, a, occ, stream)
                        : batch_class_w<FIM_U16, kShapeSpans, KS>(c, a, occ, stream);
        case FIM_F32:
            return disk ? batch_class_w<FIM_F32, kShapeDisk, KS>(c, a, occ, stream)
                        : batch_class_w<FIM_F32, kShapeSpans, KS>(c, a, occ, stream);
    }
    return FIM_ERR_INVALID_ARG;
}

}  // namespace
}  // namespace fim
