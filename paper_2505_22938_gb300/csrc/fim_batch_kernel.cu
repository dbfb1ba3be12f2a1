// Batched persistent launch (device side): the tile pipeline of every job of a batch in one
// kernel launch.
#include "fim_tile_pipeline.cuh"

namespace fim {
namespace {

// ---- batched persistent launch ---------------------------------------------------------------
// Every CTA visits the jobs in order (sorted by decreasing cost per tile on the host, so the
// long tiles start first). For a job, it loads the job's plan scalars and tables into shared
// memory, then each of its tile groups takes tiles of that job from the job's counter on its
// own, with no CTA-wide barrier between tiles; when the job has no tiles left the CTA moves on.
// The per-type pipelines are inlined into the kernel: behind a call boundary they spill.
template <int DT, int SHAPE, int W, int OG, int KS = 0>
__device__ __forceinline__ void batch_tile(const Plan* P, int tile, unsigned char* gslice, const Grp G) {
    process_tile<DT, SHAPE, W, OG, KS>(*P, tile, gslice, G);
}

__device__ __forceinline__ void dispatch_tile(const Plan* P, int tile, unsigned char* gslice, const Grp G) {
    const int cls = P->wide ? 2 : (P->loc_om < 0 ? 1 : 0);
    const bool disk = P->shape == kShapeDisk;
#define FIM_CASE(DT)                                                                   \
    if (disk) {                                                                        \
        if (cls == 0 && P->scan_groups == 8) batch_tile<DT, kShapeDisk, 0, 0, 8>(P, tile, gslice, G); \
        else if (cls == 0) batch_tile<DT, kShapeDisk, 0, 0>(P, tile, gslice, G);      \
        else if (cls == 1) batch_tile<DT, kShapeDisk, 0, 1>(P, tile, gslice, G);      \
        else batch_tile<DT, kShapeDisk, 1, 1>(P, tile, gslice, G);                    \
    } else {                                                                           \
        if (cls == 0) batch_tile<DT, kShapeSpans, 0, 0>(P, tile, gslice, G);          \
        else if (cls == 1) batch_tile<DT, kShapeSpans, 0, 1>(P, tile, gslice, G);     \
        else batch_tile<DT, kShapeSpans, 1, 1>(P, tile, gslice, G);                   \
    }
    switch (P->dtype) {
        case FIM_U8: FIM_CASE(FIM_U8) break;
        case FIM_U16: FIM_CASE(FIM_U16) break;
        default: FIM_CASE(FIM_F32) break;
    }
#undef FIM_CASE
}


__global__ void __launch_bounds__(1024, 1) batch_median_kernel(const __grid_constant__ BatchArgs A) {
    __shared__ int s_left;                   // the current job still has tiles
    __shared__ int s_job;                    // the current job (re-read after each tile)
    __shared__ int s_tile[kMaxBatchGroups];  // each group's next tile
    // the current job's plan scalars (everything before the tables), so that the tile pipeline
    // reads them from shared memory rather than global memory
    __shared__ __align__(16) unsigned char s_plan[kPlanScalarBytes];
    const int tid = threadIdx.x;
    unsigned int* counters = reinterpret_cast<unsigned int*>(A.scratch);
    for (int job = 0; job < A.njobs; ++job) {
        const Plan* Gp = A.plans + job;
        if (tid == 0) {
            s_left = *reinterpret_cast<volatile unsigned int*>(counters + job) < (unsigned)Gp->ntiles;
            s_job = job;
        }
        __syncthreads();
        const int left = s_left;
        __syncthreads();  // everyone has read the flag before thread 0 rewrites it
        if (!left) continue;
        load_tables(*Gp);
        {
            const uint32_t* src = reinterpret_cast<const uint32_t*>(Gp);
            uint32_t* dst = reinterpret_cast<uint32_t*>(s_plan);
            for (int i = tid; i < (int)(kPlanScalarBytes / 4); i += blockDim.x) dst[i] = src[i];
        }
        __syncthreads();
        const Plan* P = reinterpret_cast<const Plan*>(s_plan);
        const int T = P->threads;
        const int g = tid / T;
        if (g < P->groups) {
            const int lt = tid - g * T;
            const Grp G{lt, lt & 31, lt >> 5, T, T == (int)blockDim.x ? 0 : 1 + g, g * P->group_bytes};
            for (;;) {
                if (lt == 0) s_tile[g] = (int)atomicAdd(counters + s_job, 1u);
                G.sync();
                const int tile = s_tile[g];
                if (tile >= P->ntiles) break;
                {   // rebuilt from shared memory and special registers: little stays live across
                    // the inlined pipeline, which needs every register it can get
                    const int t2 = threadIdx.x, T2 = P->threads, g2 = t2 / T2, l2 = t2 - g2 * T2;
                    const Grp G2{l2, l2 & 31, l2 >> 5, T2, T2 == (int)blockDim.x ? 0 : 1 + g2, g2 * P->group_bytes};
                    unsigned char* gs2 = A.scratch + A.header_bytes +
                                         ((size_t)blockIdx.x * A.max_groups + g2) * (size_t)A.scratch_per_cta;
                    dispatch_tile(P, tile, gs2, G2);  // ends with a group barrier
                }
            }
        }
        __syncthreads();  // the next job reloads the tables and plan scalars
    }
}

}  // namespace

fim_status batch_prepare(int smem) {
    if (cudaFuncSetAttribute(batch_median_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess) {
        cudaGetLastError();
        return FIM_ERR_CUDA;
    }
    return FIM_OK;
}

fim_status batch_grid(int threads, int smem, long long total_tiles, int* grid) {
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, batch_median_kernel, threads, smem) != cudaSuccess ||
        occ < 1) {
        cudaGetLastError();
        return FIM_ERR_UNSUPPORTED;
    }
    *grid = (int)std::min<long long>(total_tiles, (long long)occ * device_sm_count());
    return FIM_OK;
}

fim_status batch_launch(const BatchArgs& a, int grid, int threads, int smem, cudaStream_t stream) {
    if (cudaMemsetAsync(a.scratch, 0, (size_t)a.header_bytes, stream) != cudaSuccess) return FIM_ERR_CUDA;
    batch_median_kernel<<<grid, threads, smem, stream>>>(a);
    if (cudaGetLastError() != cudaSuccess) return FIM_ERR_CUDA;
    return FIM_OK;
}

fim_status read_and_clear_batch_status() {
    int v = 0;
    if (cudaMemcpyFromSymbol(&v, g_status, sizeof(int)) != cudaSuccess) return FIM_ERR_CUDA;
    const int zero = 0;
    if (v != 0 && cudaMemcpyToSymbol(g_status, &zero, sizeof(int)) != cudaSuccess) return FIM_ERR_CUDA;
    return (fim_status)v;
}

}  // namespace fim
