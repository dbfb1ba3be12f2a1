// fim_median_noalloc: the median filter for callers that must not allocate device memory.
//
// Some callers cannot call cudaMalloc: code running while a CUDA stream is being captured into a
// graph (allocation is not a stream operation), callers whose device memory is owned by an
// external pool or framework allocator that forbids side allocations, and real-time or
// safety-critical services that allocate everything once at start-up. fim_median lazily grows a
// workspace with cudaMalloc; this entry point instead uses one fixed array of device memory that
// is part of the library image, so it never allocates.
//
// The array is a file-scope __device__ variable. Host code cannot use its name as an address, so
// the first call on each device looks the address up with cudaGetSymbolAddress (with that device
// current) and caches it. Every call, on every stream, shares the one array; calls whose work
// overlaps on the GPU therefore race and must be serialised by the caller (one stream, or events).
#include <mutex>
#include <new>

#include "fim_internal.h"

namespace {

// Workspace of every fim_median_noalloc call on this device: a 256-byte header (the tile queue
// counter, cleared before each launch) followed by the per-CTA buffers of large kernels.
static __device__ __align__(256) unsigned char g_noalloc_workspace[FIM_NOALLOC_WORKSPACE_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char* g_addr[kMaxDevices] = {nullptr};

// Address of the workspace on the current device (looked up once per device).
fim_status workspace_address(unsigned char** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return FIM_ERR_CUDA;
    if (dev < 0 || dev >= kMaxDevices) return FIM_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> g(g_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_workspace) != cudaSuccess || !p) {
            cudaGetLastError();
            return FIM_ERR_CUDA;
        }
        g_addr[dev] = static_cast<unsigned char*>(p);
    }
    *out = g_addr[dev];
    return FIM_OK;
}

// The library's default tile choice (its shapes in its order of preference by kernel extent,
// small kernels on 32x32 tiles in small CTAs first, and its two exceptions past the first valid
// shape: a later shape of at least 64x64 that keeps the omnigram in shared memory where the
// first one spills it, and for 16-bit data the first exact-rank shape of at least 64x64; then
// the smaller shapes of small images), without the autotuner's cache, whose lookup allocates. A candidate is valid when it fits shared memory and its launch
// fits the fixed array (per-CTA buffers of large kernels times the resident CTAs). Trial plans
// and the chosen one are built in the caller's storage.
fim_status pick_plan(const fim_kernel* k, int dtype, int w, int h, int limit, fim::Plan* plan) {
    static const fim::TileShape cands[] = {{32, 32, 2, 1}, {32, 32, 4, 1}, {64, 128, 8, 2}, {64, 64, 8, 2},
                                           {32, 64, 8, 2}, {32, 32, 8, 2}, {32, 16, 8, 2}};
    const int ncands = (int)(sizeof(cands) / sizeof(cands[0]));
    const int extent = (k->xmax - k->xmin > k->ymax - k->ymin ? k->xmax - k->xmin : k->ymax - k->ymin) + 1;
    const int first = extent <= 33 ? 0 : (extent <= 45 ? 1 : (extent >= 65 ? 2 : 3));
    auto valid = [&](int i) {
        return fim::make_plan(k, dtype, (k->n - 1) / 2, w, h, cands[i], limit, plan) == FIM_OK &&
               plan->smem_bytes <= limit &&
               fim::launch_tile_kernel_fixed(*plan, nullptr, FIM_NOALLOC_WORKSPACE_BYTES, nullptr, false) == FIM_OK;
    };
    int i0 = -1;
    for (int i = first; i < ncands && i0 < 0; ++i)
        if (valid(i)) i0 = i;
    if (i0 < 0) return FIM_ERR_UNSUPPORTED;
    const bool om_smem = plan->loc_om >= 0;
    const int n0 = plan->N;
    int pick = i0;
    if (!om_smem)
        for (int i = i0 + 1; i < ncands; ++i)
            if (valid(i) && plan->loc_om >= 0 && cands[i].Tx * cands[i].Ty >= 4096) {
                pick = i;
                break;
            }
    if (pick == i0 && dtype == FIM_U16 && n0 > 65535)
        for (int i = i0 + 1; i < ncands; ++i)
            if (valid(i) && plan->N <= 65535) {
                pick = cands[i].Tx * cands[i].Ty < 4096 ? i0 : i;
                break;
            }
    fim::TileShape small;  // and the library's small-image rule, where its shape also fits the array
    if (fim::small_image_shape(k, dtype, w, h, limit, 0, false, cands[pick], plan, &small) &&
        fim::make_plan(k, dtype, (k->n - 1) / 2, w, h, small, limit, plan) == FIM_OK && plan->smem_bytes <= limit &&
        fim::launch_tile_kernel_fixed(*plan, nullptr, FIM_NOALLOC_WORKSPACE_BYTES, nullptr, false) == FIM_OK)
        return FIM_OK;
    return valid(pick) ? FIM_OK : FIM_ERR_UNSUPPORTED;
}

bool overlap(const void* a, const void* b, size_t bytes) {
    const uintptr_t pa = (uintptr_t)a, pb = (uintptr_t)b;
    return pa < pb + bytes && pb < pa + bytes;
}

}  // namespace

extern "C" fim_status fim_median_noalloc(const void* in, void* out, int w, int h, size_t pitch_bytes,
                                         fim_dtype dtype, const fim_kernel* k, fim_border border, void* stream) {
    if (!in || !out || !k || w <= 0 || h <= 0) return FIM_ERR_INVALID_ARG;
    if (dtype != FIM_U8 && dtype != FIM_U16 && dtype != FIM_F32) return FIM_ERR_INVALID_ARG;
    if (border != FIM_BORDER_CLAMP) return FIM_ERR_INVALID_ARG;
    const size_t es = dtype == FIM_U8 ? 1 : (dtype == FIM_U16 ? 2 : 4);
    if (pitch_bytes < (size_t)w * es || pitch_bytes % es != 0) return FIM_ERR_INVALID_ARG;
    if (overlap(in, out, pitch_bytes * (size_t)(h - 1) + (size_t)w * es)) return FIM_ERR_INVALID_ARG;
    const int limit = fim::device_smem_limit();
    if (limit <= 0) return FIM_ERR_CUDA;
    unsigned char* ws = nullptr;
    fim_status s = workspace_address(&ws);
    if (s != FIM_OK) return s;
    // the plan lives in this thread's storage: no heap allocation on the call path
    static thread_local fim::Plan plan;
    s = pick_plan(k, dtype, w, h, limit, &plan);
    if (s != FIM_OK) return s;  // no tile shape fits the fixed array: FIM_ERR_UNSUPPORTED
    plan.in = in;
    plan.out = out;
    plan.pitch = (long long)pitch_bytes;
    // rejects (FIM_ERR_UNSUPPORTED) a call that would need more than the fixed workspace
    return fim::launch_tile_kernel_fixed(plan, ws, FIM_NOALLOC_WORKSPACE_BYTES, (cudaStream_t)stream);
}
