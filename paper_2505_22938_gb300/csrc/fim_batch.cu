// Batched persistent launch (host side): many images of any size, dtype and kernel in one
// kernel launch. The batch object owns its device-side plans (sorted by decreasing cost per
// tile) and its workspace, whose header holds one tile counter per job; fim_batch_run() only
// zeroes the header and launches: both are stream operations and can be captured in a CUDA
// graph.
#include <string.h>

#include <algorithm>
#include <iterator>
#include <new>
#include <numeric>
#include <vector>

#include "fim_internal.h"

using namespace fim;

struct fim_batch {
    int njobs = 0;
    int total_tiles = 0, max_groups = 1, header_bytes = 256;
    int grid = 0, threads = 0, smem = 0;
    long long scratch_per_cta = 0;
    Plan* d_plans = nullptr;
    unsigned char* scratch = nullptr;
    int device = 0;
};

namespace {

int esize(int dtype) { return dtype == FIM_U8 ? 1 : (dtype == FIM_U16 ? 2 : 4); }

// Relative cost of one tile, used only to start the expensive tiles first.
double tile_cost(const Plan& p) {
    const double px = (double)p.Tx * p.Ty;
    const double sort = p.sort == kSortRadix ? 12.0 : (p.sort == kSortRadix16 ? 8.0 : 3.0);
    return p.N * sort + px * (2.0 * p.ncols + 80.0) + (double)p.RB * p.G * p.n * 2.0;
}

// Byte range [lo, hi) an image of one job occupies.
struct Span {
    uintptr_t lo, hi;
};

Span image_span(const void* base, const fim_job& j) {
    const uintptr_t lo = (uintptr_t)base;
    return Span{lo, lo + j.pitch_bytes * (size_t)(j.h - 1) + (size_t)j.w * (size_t)esize(j.dtype)};
}

// All jobs of a batch run in one launch, so no output may overlap another output or any input
// (its own job's included): a tile would read pixels another tile has already overwritten.
// Several jobs may read one input. O(n log n): sort the outputs, check neighbours, then look up
// each input among them.
bool batch_aliases(const fim_job* jobs, int count) {
    std::vector<Span> outs((size_t)count);
    for (int i = 0; i < count; ++i) outs[i] = image_span(jobs[i].out, jobs[i]);
    std::sort(outs.begin(), outs.end(), [](const Span& a, const Span& b) { return a.lo < b.lo; });
    for (int i = 1; i < count; ++i)
        if (outs[i].lo < outs[i - 1].hi) return true;
    for (int i = 0; i < count; ++i) {
        const Span in = image_span(jobs[i].in, jobs[i]);
        // the last output starting below the input's end is the only one that can reach into it
        auto it = std::lower_bound(outs.begin(), outs.end(), in.hi,
                                   [](const Span& s, uintptr_t v) { return s.lo < v; });
        if (it != outs.begin() && std::prev(it)->hi > in.lo) return true;
    }
    return false;
}

void free_batch(fim_batch* b) {
    if (!b) return;
    cudaDeviceSynchronize();
    if (b->d_plans) cudaFree(b->d_plans);
    if (b->scratch) cudaFree(b->scratch);
    delete b;
}

}  // namespace

extern "C" {

fim_status fim_batch_create(const fim_job* jobs, int count, fim_batch** out) {
    if (!out || !jobs || count <= 0) return FIM_ERR_INVALID_ARG;
    *out = nullptr;
    constexpr int kCta = 1024;  // every batch CTA; jobs with smaller configurations run several groups
    std::vector<Plan> plans((size_t)count);
    for (int i = 0; i < count; ++i) {
        const fim_job& j = jobs[i];
        if (!j.in || !j.out || !j.kernel || j.w <= 0 || j.h <= 0) return FIM_ERR_INVALID_ARG;
        if (j.dtype != FIM_U8 && j.dtype != FIM_U16 && j.dtype != FIM_F32) return FIM_ERR_INVALID_ARG;
        const size_t es = (size_t)esize(j.dtype);
        if (j.pitch_bytes < (size_t)j.w * es || j.pitch_bytes % es != 0) return FIM_ERR_INVALID_ARG;
        if (!(j.percentile < 0.0 || j.percentile <= 100.0)) return FIM_ERR_INVALID_ARG;
    }
    if (batch_aliases(jobs, count)) return FIM_ERR_INVALID_ARG;
    const int limit = device_smem_limit();
    if (limit <= 0) return FIM_ERR_CUDA;
    for (int i = 0; i < count; ++i) {
        const fim_job& j = jobs[i];
        TileShape ts;
        fim_status s = choose_tile(j.kernel, j.dtype, limit, &ts);
        if (s != FIM_OK) return s;
        const int n = j.kernel->n;
        int rank = (n - 1) / 2;
        if (j.percentile >= 0.0) rank = std::min(std::max((int)(j.percentile / 100.0 * (n - 1) + 0.5), 0), n - 1);
        Plan& p = plans[i];
        s = make_plan(j.kernel, j.dtype, rank, j.w, j.h, ts, limit, &p);
        if (s != FIM_OK) return s;
        p.in = j.in;
        p.out = j.out;
        p.pitch = (long long)j.pitch_bytes;
        p.ntiles = p.tiles_x * p.tiles_y;
        // as many groups as fit the CTA and shared memory, but no more than the job has tiles
        int groups = std::min(kCta / p.threads, kMaxBatchGroups);
        while (groups > 1 && p.tab_bytes + (size_t)groups * p.group_bytes > (size_t)limit) --groups;
        p.groups = std::max(1, std::min(groups, p.ntiles));
    }
    std::vector<int> order((size_t)count);
    std::iota(order.begin(), order.end(), 0);
    // the CTAs visit the jobs in this order: expensive tiles first, cheap ones fill the tail
    std::stable_sort(order.begin(), order.end(),
                     [&](int a, int b) { return tile_cost(plans[a]) > tile_cost(plans[b]); });
    std::vector<Plan> sorted((size_t)count);
    long long tiles = 0, spc = 0;
    int smem = 0, max_groups = 1;
    for (int i = 0; i < count; ++i) {
        Plan& p = sorted[i];
        p = plans[order[i]];
        tiles += p.ntiles;
        spc = std::max(spc, p.scratch_per_cta);
        smem = std::max(smem, p.tab_bytes + p.groups * p.group_bytes);
        max_groups = std::max(max_groups, p.groups);
    }
    if (tiles > 0x7fffffffLL) return FIM_ERR_UNSUPPORTED;
    fim_batch* b = new (std::nothrow) fim_batch();
    if (!b) return FIM_ERR_OOM;
    cudaGetDevice(&b->device);
    b->njobs = count;
    b->total_tiles = (int)tiles;
    b->max_groups = max_groups;
    b->scratch_per_cta = spc;
    b->threads = kCta;
    b->smem = smem;
    b->header_bytes = (int)((((size_t)count * 4) + 255) & ~(size_t)255);
    fim_status s = batch_prepare(smem);
    if (s == FIM_OK) s = batch_grid(b->threads, b->smem, tiles, &b->grid);
    if (s != FIM_OK) {
        free_batch(b);
        return s;
    }
    const size_t scratch_bytes = (size_t)b->header_bytes + (size_t)b->grid * (size_t)max_groups * (size_t)spc;
    if (cudaMalloc(&b->d_plans, sizeof(Plan) * (size_t)count) != cudaSuccess ||
        cudaMalloc(&b->scratch, scratch_bytes) != cudaSuccess) {
        cudaGetLastError();
        free_batch(b);
        return FIM_ERR_OOM;
    }
    if (cudaMemcpy(b->d_plans, sorted.data(), sizeof(Plan) * (size_t)count, cudaMemcpyHostToDevice) != cudaSuccess) {
        free_batch(b);
        return FIM_ERR_CUDA;
    }
    *out = b;
    return FIM_OK;
}

fim_status fim_batch_run(fim_batch* b, void* stream) {
    if (!b) return FIM_ERR_INVALID_ARG;
    BatchArgs a;
    a.plans = b->d_plans;
    a.njobs = b->njobs;
    a.header_bytes = b->header_bytes;
    a.max_groups = b->max_groups;
    a.scratch = b->scratch;
    a.scratch_per_cta = b->scratch_per_cta;
    return batch_launch(a, b->grid, b->threads, b->smem, (cudaStream_t)stream);
}

fim_status fim_batch_info(const fim_batch* b, int* total_tiles, int* grid, int* threads, int* smem_bytes) {
    if (!b) return FIM_ERR_INVALID_ARG;
    if (total_tiles) *total_tiles = b->total_tiles;
    if (grid) *grid = b->grid;
    if (threads) *threads = b->threads;
    if (smem_bytes) *smem_bytes = b->smem;
    return FIM_OK;
}

void fim_batch_destroy(fim_batch* b) { free_batch(b); }

fim_status fim_median_batch(const fim_job* jobs, int count, void* stream) {
    fim_batch* b = nullptr;
    fim_status s = fim_batch_create(jobs, count, &b);
    if (s != FIM_OK) return s;
    s = fim_batch_run(b, stream);
    if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess && s == FIM_OK) s = FIM_ERR_CUDA;
    fim_batch_destroy(b);
    return s;
}

}  // extern "C"
