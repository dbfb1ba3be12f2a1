// Batched persistent launch (host side): many images of any size, dtype and kernel. The jobs are
// grouped into classes that share a tile-pipeline instantiation and CTA size; each class runs as
// one persistent kernel whose device-side queue spans the tiles of all its jobs (sorted by
// decreasing cost per tile), and the class kernels run side by side on forked streams, so the
// tail of one class overlaps the others. The batch object owns its device-side plans, queues and
// workspace and its side streams; fim_batch_run() only zeroes the queue counters and launches,
// all stream operations, so a run can be captured in a CUDA graph.
#include <string.h>

#include <algorithm>
#include <iterator>
#include <new>
#include <numeric>
#include <tuple>
#include <vector>

#include "fim_internal.h"

using namespace fim;

struct fim_batch {
    int njobs = 0;
    int total_tiles = 0;
    std::vector<BatchClass> classes;          // in launch order (largest estimated cost first)
    std::vector<BatchClassArgs> args;         // one per class
    Plan* d_plans = nullptr;                  // every plan, grouped by class
    int* d_tile_start = nullptr;              // per class, its jobs' tile prefix sums
    unsigned int* d_counters = nullptr;       // one queue counter per class
    unsigned char* scratch = nullptr;         // per class, grid * scratch_per_cta bytes
    std::vector<cudaStream_t> side;           // classes after the first run on these
    std::vector<cudaEvent_t> ev;              // fork event, then one join event per side stream
    // per class (launch order): a one-job class runs the single-image kernel on its plan (kept
    // here) over the class's workspace, whose first 256 bytes then hold that kernel's queue
    std::vector<char> solo;
    std::vector<Plan> solo_plan;
    std::vector<unsigned char*> cls_scratch;
    std::vector<size_t> cls_bytes;
    int device = 0;
};

namespace {

int esize(int dtype) { return dtype == FIM_U8 ? 1 : (dtype == FIM_U16 ? 2 : 4); }

// Relative cost of one tile, used only to start the expensive tiles first.
double tile_cost(const Plan& p) {
    const double px = (double)p.Tx * p.Ty;
    const double sort = p.sort == kSortRadix ? 12.0 : (p.sort == kSortRadix16 ? 8.0 : (p.sort == kSortCount16x2 ? 6.0 : 3.0));
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
    if (b->d_tile_start) cudaFree(b->d_tile_start);
    if (b->d_counters) cudaFree(b->d_counters);
    if (b->scratch) cudaFree(b->scratch);
    for (cudaStream_t st : b->side) cudaStreamDestroy(st);
    for (cudaEvent_t e : b->ev) cudaEventDestroy(e);
    delete b;
}

fim_status class_kernel(const BatchClass& c, const BatchClassArgs* a, int* occ, cudaStream_t st) {
    return c.ks == 4 ? batch_class_k4(c, a, occ, st) : batch_class_k8(c, a, occ, st);
}

}  // namespace

extern "C" {

fim_status fim_batch_create(const fim_job* jobs, int count, fim_batch** out) {
    if (!out || !jobs || count <= 0) return FIM_ERR_INVALID_ARG;
    *out = nullptr;
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
        // a batch fills the GPU with the tiles of all its jobs: the shapes tuned for large images
        fim_status s = choose_tile(j.kernel, j.dtype, limit, &ts, 0, 0);
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
        attach_tma(p);  // the class kernels stage interior footprints like the single-image kernel
    }
    // classes: the instantiation a plan runs on and its CTA size
    auto key = [&](const Plan& p) {
        return std::make_tuple(p.dtype, p.shape, p.wide, p.loc_om < 0 ? 1 : 0, p.scan_groups == 4 ? 4 : 8, p.threads);
    };
    std::vector<int> order((size_t)count);
    std::iota(order.begin(), order.end(), 0);
    // grouped by class; inside a class the CTAs start on the expensive tiles, cheap ones fill the tail
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        if (key(plans[a]) != key(plans[b])) return key(plans[a]) < key(plans[b]);
        return tile_cost(plans[a]) > tile_cost(plans[b]);
    });
    std::vector<Plan> sorted((size_t)count);
    std::vector<int> tile_start((size_t)count);
    std::vector<BatchClass> classes;
    std::vector<int> first_job;  // per class, its first plan in `sorted`
    std::vector<double> cost;    // per class, estimated total cost
    long long tiles = 0;
    for (int i = 0; i < count; ++i) {
        const Plan& p = plans[order[i]];
        sorted[i] = p;
        if (i == 0 || key(p) != key(plans[order[i - 1]])) {
            BatchClass c{};
            c.dtype = p.dtype;
            c.shape = p.shape;
            c.wide = p.wide;
            c.og = p.loc_om < 0 ? 1 : 0;
            c.ks = p.scan_groups == 4 ? 4 : 8;
            c.threads = p.threads;
            classes.push_back(c);
            first_job.push_back(i);
            cost.push_back(0.0);
        }
        BatchClass& c = classes.back();
        tile_start[i] = c.total_tiles;
        if ((long long)c.total_tiles + p.ntiles > 0x7fffffffLL) return FIM_ERR_UNSUPPORTED;
        c.total_tiles += p.ntiles;
        c.njobs += 1;
        c.smem = std::max(c.smem, p.smem_bytes);
        c.scratch_per_cta = std::max(c.scratch_per_cta, p.scratch_per_cta);
        cost.back() += tile_cost(p) * p.ntiles;
        tiles += p.ntiles;
    }
    if (tiles > 0x7fffffffLL) return FIM_ERR_UNSUPPORTED;
    fim_batch* b = new (std::nothrow) fim_batch();
    if (!b) return FIM_ERR_OOM;
    cudaGetDevice(&b->device);
    b->njobs = count;
    b->total_tiles = (int)tiles;
    const int ncls = (int)classes.size();
    size_t scratch_bytes = 0;
    std::vector<size_t> scratch_off((size_t)ncls);
    for (int c = 0; c < ncls; ++c) {
        BatchClass& k = classes[c];
        int occ = 0;
        fim_status s = class_kernel(k, nullptr, &occ, nullptr);
        if (s != FIM_OK) {
            free_batch(b);
            return s;
        }
        k.grid = (int)std::min<long long>(k.total_tiles, (long long)occ * device_sm_count());
        scratch_off[c] = scratch_bytes;
        scratch_bytes += 256 + (((size_t)k.grid * (size_t)k.scratch_per_cta + 255) & ~(size_t)255);
    }
    if (cudaMalloc(&b->d_plans, sizeof(Plan) * (size_t)count) != cudaSuccess ||
        cudaMalloc(&b->d_tile_start, sizeof(int) * (size_t)count) != cudaSuccess ||
        cudaMalloc(&b->d_counters, 256 * (size_t)ncls) != cudaSuccess ||
        (scratch_bytes > 0 && cudaMalloc(&b->scratch, scratch_bytes) != cudaSuccess)) {
        cudaGetLastError();
        free_batch(b);
        return FIM_ERR_OOM;
    }
    if (cudaMemcpy(b->d_plans, sorted.data(), sizeof(Plan) * (size_t)count, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(b->d_tile_start, tile_start.data(), sizeof(int) * (size_t)count, cudaMemcpyHostToDevice) !=
            cudaSuccess) {
        free_batch(b);
        return FIM_ERR_CUDA;
    }
    // launch order: the classes with the most work first, so that the small ones fill the tail
    std::vector<int> lorder((size_t)ncls);
    std::iota(lorder.begin(), lorder.end(), 0);
    std::stable_sort(lorder.begin(), lorder.end(), [&](int a, int c) { return cost[a] > cost[c]; });
    for (int c : lorder) {
        const BatchClass& k = classes[c];
        BatchClassArgs a;
        a.plans = b->d_plans + first_job[c];
        a.tile_start = b->d_tile_start + first_job[c];
        a.njobs = k.njobs;
        a.total_tiles = k.total_tiles;
        a.counter = reinterpret_cast<unsigned int*>(reinterpret_cast<unsigned char*>(b->d_counters) +
                                                    256 * b->classes.size());
        a.scratch = b->scratch ? b->scratch + scratch_off[c] + 256 : nullptr;
        a.scratch_per_cta = k.scratch_per_cta;
        b->classes.push_back(k);
        b->args.push_back(a);
        // A class of one job runs the single-image kernel (its plan as the kernel parameter, no
        // job lookup), where that kernel's grid fits the class's workspace.
        const size_t bytes = 256 + (((size_t)k.grid * (size_t)k.scratch_per_cta + 255) & ~(size_t)255);
        Plan solo = sorted[first_job[c]];
        const bool one = k.njobs == 1 && b->scratch != nullptr &&
                         launch_tile_kernel_fixed(solo, nullptr, bytes, nullptr, false) == FIM_OK;
        b->solo.push_back(one ? 1 : 0);
        b->solo_plan.push_back(solo);
        b->cls_scratch.push_back(b->scratch ? b->scratch + scratch_off[c] : nullptr);
        b->cls_bytes.push_back(bytes);
    }
    for (int c = 1; c < ncls; ++c) {
        cudaStream_t st;
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
            free_batch(b);
            return FIM_ERR_CUDA;
        }
        b->side.push_back(st);
    }
    for (int e = 0; e < ncls; ++e) {
        cudaEvent_t ev;
        if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
            free_batch(b);
            return FIM_ERR_CUDA;
        }
        b->ev.push_back(ev);
    }
    *out = b;
    return FIM_OK;
}

fim_status fim_batch_run(fim_batch* b, void* stream) {
    if (!b) return FIM_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const int ncls = (int)b->classes.size();
    if (cudaMemsetAsync(b->d_counters, 0, 256 * (size_t)ncls, st) != cudaSuccess) return FIM_ERR_CUDA;
    // fork: the side streams wait for the counters, run their classes, and the caller's stream
    // waits for all of them
    if (ncls > 1 && cudaEventRecord(b->ev[0], st) != cudaSuccess) return FIM_ERR_CUDA;
    for (int c = 0; c < ncls; ++c) {
        cudaStream_t cs = c == 0 ? st : b->side[c - 1];
        if (c > 0 && cudaStreamWaitEvent(cs, b->ev[0], 0) != cudaSuccess) return FIM_ERR_CUDA;
        fim_status s;
        if (b->solo[c]) {
            Plan p = b->solo_plan[c];
            s = launch_tile_kernel_fixed(p, b->cls_scratch[c], b->cls_bytes[c], cs, true);
        } else {
            s = class_kernel(b->classes[c], &b->args[c], nullptr, cs);
        }
        if (s != FIM_OK) return s;
        if (c > 0 && cudaEventRecord(b->ev[c], cs) != cudaSuccess) return FIM_ERR_CUDA;
    }
    for (int c = 1; c < ncls; ++c)
        if (cudaStreamWaitEvent(st, b->ev[c], 0) != cudaSuccess) return FIM_ERR_CUDA;
    return FIM_OK;
}

fim_status fim_batch_info(const fim_batch* b, int* total_tiles, int* grid, int* threads, int* smem_bytes) {
    if (!b) return FIM_ERR_INVALID_ARG;
    int g = 0, t = 0, sm = 0;
    for (const BatchClass& c : b->classes) {
        g += c.grid;
        t = std::max(t, c.threads);
        sm = std::max(sm, c.smem);
    }
    if (total_tiles) *total_tiles = b->total_tiles;
    if (grid) *grid = g;
    if (threads) *threads = t;
    if (smem_bytes) *smem_bytes = sm;
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
