// Host side of libfim: kernel shapes, tile planning, argument checks and the C ABI.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <new>
#include <vector>

#include "fim_internal.h"

namespace fim {
namespace {

int64_t isqrt64(int64_t v) {
    if (v <= 0) return 0;
    int64_t r = (int64_t)sqrt((double)v);
    while (r * r > v) --r;
    while ((r + 1) * (r + 1) <= v) ++r;
    return r;
}

// Fills the column runs from the row spans; fails unless every column is a single run and
// every row is non-empty (the shape is convex along both axes).
fim_status finish_kernel(fim_kernel* k) {
    const int rows = (int)k->rlo.size();
    if (rows <= 0) return FIM_ERR_INVALID_ARG;
    int xmin = k->rlo[0], xmax = k->rhi[0];
    int64_t n = 0;
    for (int i = 0; i < rows; ++i) {
        if (k->rlo[i] > k->rhi[i]) return FIM_ERR_INVALID_ARG;
        xmin = std::min(xmin, k->rlo[i]);
        xmax = std::max(xmax, k->rhi[i]);
        n += k->rhi[i] - k->rlo[i] + 1;
    }
    k->xmin = xmin;
    k->xmax = xmax;
    k->ymax = k->ymin + rows - 1;
    if (xmax - xmin + 1 > FIM_MAX_KERNEL_EXTENT || rows > FIM_MAX_KERNEL_EXTENT) return FIM_ERR_UNSUPPORTED;
    const int cols = xmax - xmin + 1;
    k->ctop.assign(cols, 0);
    k->cbot.assign(cols, 0);
    for (int j = 0; j < cols; ++j) {
        const int dx = xmin + j;
        int first = -1, last = -1;
        for (int i = 0; i < rows; ++i) {
            const bool in = k->rlo[i] <= dx && dx <= k->rhi[i];
            if (in) {
                if (first < 0) first = i;
                else if (last != i - 1) return FIM_ERR_INVALID_ARG;  // second run in this column
                last = i;
            }
        }
        if (first < 0) return FIM_ERR_INVALID_ARG;  // empty column inside the bounding box
        k->ctop[j] = k->ymin + first;
        k->cbot[j] = k->ymin + last;
    }
    k->n = (int)n;
    return FIM_OK;
}

fim_status new_kernel(fim_kernel** out, fim_kernel** k) {
    if (!out) return FIM_ERR_INVALID_ARG;
    *out = nullptr;
    *k = new (std::nothrow) fim_kernel();
    return *k ? FIM_OK : FIM_ERR_OOM;
}

fim_status publish(fim_kernel* k, fim_kernel** out) {
    fim_status s = finish_kernel(k);
    if (s != FIM_OK) {
        delete k;
        return s;
    }
    *out = k;
    return FIM_OK;
}

fim_status disk_kernel(int64_t limit, fim_kernel** out) {
    fim_kernel* k;
    fim_status s = new_kernel(out, &k);
    if (s != FIM_OK) return s;
    const int r = (int)isqrt64(limit);
    k->shape = kShapeDisk;
    k->r2 = limit;
    k->ymin = -r;
    for (int dy = -r; dy <= r; ++dy) {
        const int half = (int)isqrt64(limit - (int64_t)dy * dy);
        k->rlo.push_back(-half);
        k->rhi.push_back(half);
    }
    return publish(k, out);
}

}  // namespace

int device_sm_count() {
    static int cached[64] = {0};
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) return 1;
    if (dev < 64 && cached[dev] > 0) return cached[dev];
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) return 1;
    if (dev < 64) cached[dev] = v;
    return v;
}

namespace {
// Global scratch of the tile kernels, cached per (device, stream). Launches on one stream run
// in order, so they can share one buffer; a buffer is only replaced after its stream drained.
struct ScratchBuf {
    void* ptr = nullptr;
    size_t bytes = 0;
};
std::mutex g_scratch_mu;
std::map<std::pair<int, uintptr_t>, ScratchBuf>& scratch_map() {
    static std::map<std::pair<int, uintptr_t>, ScratchBuf> m;
    return m;
}
}  // namespace

fim_status get_scratch(cudaStream_t stream, size_t bytes, unsigned char** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return FIM_ERR_CUDA;
    std::lock_guard<std::mutex> g(g_scratch_mu);
    ScratchBuf& b = scratch_map()[{dev, (uintptr_t)stream}];
    if (b.bytes < bytes) {
        if (b.ptr) {
            if (cudaStreamSynchronize(stream) != cudaSuccess) return FIM_ERR_CUDA;
            cudaFree(b.ptr);
            b.ptr = nullptr;
            b.bytes = 0;
        }
        const size_t want = std::max(bytes, (size_t)1 << 20);
        if (cudaMalloc(&b.ptr, want) != cudaSuccess) {
            cudaGetLastError();
            b.ptr = nullptr;
            return FIM_ERR_OOM;
        }
        b.bytes = want;
    }
    *out = static_cast<unsigned char*>(b.ptr);
    return FIM_OK;
}

fim_status release_scratch() {
    std::lock_guard<std::mutex> g(g_scratch_mu);
    if (cudaDeviceSynchronize() != cudaSuccess) return FIM_ERR_CUDA;
    int cur = 0;
    cudaGetDevice(&cur);
    for (auto& kv : scratch_map()) {
        if (kv.second.ptr) {
            cudaSetDevice(kv.first.first);
            cudaFree(kv.second.ptr);
        }
    }
    scratch_map().clear();
    cudaSetDevice(cur);
    return FIM_OK;
}

int device_smem_per_sm() {
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess) return 0;
    return v;
}

namespace {
// cuTensorMapEncodeTiled from the driver, found through the runtime (no driver library link)
using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                 const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiled encode_tiled() {
    static EncodeTiled fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPoint("cuTensorMapEncodeTiled", &f, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiled>(f);
        cudaGetLastError();
    });
    return fn;
}
}  // namespace

void attach_tma(Plan& p) {
    p.use_tma = 0;
    if (p.loc_stage < 0 || getenv("FIM_NO_TMA")) return;
    if (((uintptr_t)p.in & 15) != 0 || (p.pitch & 15) != 0) return;
    EncodeTiled enc = encode_tiled();
    if (!enc) return;
    const CUtensorMapDataType t = p.dtype == FIM_U8 ? CU_TENSOR_MAP_DATA_TYPE_UINT8
                                  : (p.dtype == FIM_U16 ? CU_TENSOR_MAP_DATA_TYPE_UINT16
                                                        : CU_TENSOR_MAP_DATA_TYPE_FLOAT32);
    const cuuint64_t dims[2] = {(cuuint64_t)p.w, (cuuint64_t)p.h};
    const cuuint64_t strides[1] = {(cuuint64_t)p.pitch};
    const cuuint32_t box[2] = {(cuuint32_t)p.stage_bw, (cuuint32_t)p.SH};
    const cuuint32_t estr[2] = {1, 1};
    if (enc(&p.tmap, t, 2, const_cast<void*>(p.in), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS)
        p.use_tma = 1;
}

int device_smem_limit() {
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) return 0;
    return v - 1024;  // dynamic shared memory; the kernels' static shared variables need the rest
}

static size_t align16(size_t v) { return (v + 15) & ~(size_t)15; }
fim_status layout_plan(Plan* p, int smem_limit, bool stage_model = false);

static int span_lo_host(int s) { return (int)(int16_t)(s & 0xffff); }

static int elem_size(int dtype) { return dtype == FIM_U8 ? 1 : (dtype == FIM_U16 ? 2 : 4); }

fim_status make_plan(const fim_kernel* k, int dtype, int rank, int w, int h, const TileShape& ts, int smem_limit,
                     Plan* p, int cta_threads, bool exact_ranks) {
    memset(p, 0, sizeof(*p));
    p->dtype = dtype;
    p->w = w;
    p->h = h;
    p->Tx = ts.Tx;
    p->Ty = ts.Ty;
    p->txshift = 0;
    while ((1 << p->txshift) < ts.Tx) ++p->txshift;
    if ((1 << p->txshift) != ts.Tx || ts.Tx % 32 != 0 || ts.Ty % ts.RB != 0 || ts.Tx % ts.G != 0 ||
        ts.Ty / ts.RB < 1 || ts.Tx / ts.G < 2)
        return FIM_ERR_UNSUPPORTED;
    p->RB = ts.RB;
    p->G = ts.G;
    p->vthreads = 2 * ts.Tx * ts.RB;
    p->threads = std::max(p->vthreads, cta_threads);
    // Scans are short in the small tiles of small kernels (4 groups per step) and long in the
    // large tiles (8): measured on the 4096^2 photo-like workload, each within 2 % of the best.
    p->scan_groups = p->vthreads < 1024 ? 4 : 8;
    p->nwarps = p->threads / 32;
    if (p->threads > 1024 || p->threads % 32 != 0) return FIM_ERR_UNSUPPORTED;  // 2 x Tx x bands threads
    p->shape = k->shape;
    p->r2 = (int)k->r2;
    p->xmin = k->xmin;
    p->xmax = k->xmax;
    p->ymin = k->ymin;
    p->ymax = k->ymax;
    p->nrows = k->ymax - k->ymin + 1;
    p->ncols = k->xmax - k->xmin + 1;
    p->n = k->n;
    p->rank = rank;
    p->nranks = 1;
    p->ranks[0] = rank;
    // Small kernels: a warp's 32 chains drawn from every band even out the per-warp work of the
    // vertical sweep (scan lengths follow the image content of a band); large kernels prefer the
    // shorter per-step divergence of 32 adjacent columns of one band (measured on the 4096^2
    // photo-like workload: mixing gains 4-13 % up to r = 16, loses 2-4 % from r = 32 on).
    p->vmix = std::max(k->xmax - k->xmin, k->ymax - k->ymin) + 1 <= 40 ? 1 : 0;
    p->S = ts.Tx + (k->xmax - k->xmin);
    p->SH = ts.Ty + (k->ymax - k->ymin);
    if (p->S > kMaxSide || p->SH > kMaxSide) return FIM_ERR_UNSUPPORTED;
    p->SP = (p->S + 1) & ~1;
    if ((p->SP / 2) % 2 == 0) p->SP += 2;  // odd number of 32-bit words per row: no bank aliasing
    p->tiles_x = (w + ts.Tx - 1) / ts.Tx;
    p->tiles_y = (h + ts.Ty - 1) / ts.Ty;
    const int Tx = ts.Tx, Ty = ts.Ty, S = p->S, SP = p->SP;
    // Footprint: the union of the kernel over the tile's output pixels, row by row (Fig. 10).
    int64_t N = 0;
    for (int v = 0; v < p->SH; ++v) {
        const int i0 = std::max(0, v - Ty + 1), i1 = std::min(p->nrows - 1, v);
        int lo = 1 << 30, hi = -(1 << 30);
        for (int i = i0; i <= i1; ++i) {
            lo = std::min(lo, k->rlo[i]);
            hi = std::max(hi, k->rhi[i]);
        }
        const int fl = lo - k->xmin, fr = Tx - 1 + hi - k->xmin;
        p->frow[v] = (int)((uint32_t)(fl & 0xffff) | ((uint32_t)fr << 16));
        N += fr - fl + 1;
    }
    // Footprints beyond 65535 pixels keep 16-bit ordinal ranks relative to the tile's feasible
    // median ranks [rank, N - n + rank] (Fig. 10), which is all a pivot ever takes; callers whose
    // targets vary per pixel or per kernel (exact_ranks) need N <= 65535.
    p->rank_base = 0;
    if (N > 65535) {
        if (exact_ranks || N > (1 << 20)) return FIM_ERR_UNSUPPORTED;
        p->rank_base = std::max(0, rank - 1);
        if (N - k->n + rank - p->rank_base > 65535) return FIM_ERR_UNSUPPORTED;
    }
    p->N = (int)N;
    // 8-bit coordinates (u - S/2, v - SH/2) reach (-128, -128), the mark of the padding entries,
    // only at box position (0, 0) of a 256 x 256 box; they serve unless that corner belongs to the
    // footprint (then it would be a real entry, and a member of some window).
    const bool corner = span_lo_host(p->frow[0]) == 0;
    p->wide = (p->S > 256 || p->SH > 256 || (p->S == 256 && p->SH == 256 && corner)) ? 1 : 0;
    p->cx0 = S / 2;
    p->cy0 = p->SH / 2;
    p->div_magic = (unsigned)(((1ull << 32) + (unsigned)S - 1) / (unsigned)S);
    int hs = 0;
    while (((p->N - 1) >> hs) >= kSeedBins) ++hs;
    p->hist_shift = hs;
    // Seeds: the omnigram walk reads about N/2 entries, the histogram n pixels with a shared-memory
    // atomic each; the walk wins where the footprint is small against the kernel (measured on the
    // 4096^2 photo-like workload: walk +1 % at r = 64, +8 % at r = 96; histogram ahead up to r = 48).
    p->seed_mode = p->N < 4 * p->n ? kSeedWalk : kSeedHistogram;
    if (p->rank_base > 0) p->seed_mode = kSeedWalk;  // the histogram bins the ordinal image's ranks
    if (const char* e = getenv("FIM_SEEDS"))  // experiments: 0 histogram, 1 walk, 2 count at the middle
        if (*e >= '0' && *e <= '2' && e[1] == 0) p->seed_mode = *e - '0';
    for (int j = 0; j < p->ncols; ++j) {
        const int dx = k->xmin + j;
        p->vtab[2 * j] = k->ctop[j] * SP + dx;
        p->vtab[2 * j + 1] = (k->cbot[j] + 1) * SP + dx;
    }
    for (int i = 0; i < p->nrows; ++i) {
        const int dy = k->ymin + i;
        p->htab[2 * i] = dy * SP + k->rlo[i];
        p->htab[2 * i + 1] = dy * SP + k->rhi[i] + 1;
        p->spans[i] = (int)((uint32_t)(k->rlo[i] & 0xffff) | ((uint32_t)k->rhi[i] << 16));
    }
    p->sort = dtype == FIM_U8 ? kSortCount8 : (dtype == FIM_U16 ? kSortCount16 : kSortRadix);
    // The 65536 bins of the 16-bit counting sort (128 KiB) leave room for one CTA per SM, which
    // only a full 1024-thread CTA uses well; smaller CTAs sort 16-bit data by two radix passes.
    if (dtype == FIM_U16 && p->threads < 1024) p->sort = kSortRadix;
    // Float keys in full CTAs: the 65536 bins sort the low half of the key in one pass, which
    // replaces two of the four 8-bit passes (the layout falls back to four when they do not fit).
    if (dtype == FIM_F32 && p->threads >= 1024) p->sort = kSortRadix16;
    // more than 65535 footprint pixels overflow the packed 16-bit counters of the 65536 bins:
    // 16-bit data in full CTAs counts in two rounds of 32-bit bins, and so does the float keys'
    // 16-bit pass (f32 8192^2 r = 100: 1.79 -> 2.02 Gpix/s against four 8-bit passes); smaller
    // CTAs take 8-bit passes
    if (p->N > 65535 && p->sort != kSortCount8 && p->sort != kSortRadix16)
        p->sort = dtype == FIM_U16 && p->threads >= 1024 ? kSortCount16x2 : kSortRadix;
    // Placement. Tables, the ordinal image, medians and histograms always live in shared memory;
    // the omnigram, the radix keys and the radix position lists go to the CTA's global scratch
    // slice when shared memory cannot hold them (large kernels).
    return layout_plan(p, smem_limit);
}

fim_status plan_stage_model(Plan* p, int smem_limit) {
    if (p->model == nullptr) return FIM_OK;
    // Stage the parameters only where they fit beside everything the plain layout keeps in shared
    // memory: moving the omnigram or a sort list to global memory costs far more than reading
    // the parameters from global memory (measured: 3x the sort time at r = 64).
    const int om = p->loc_om, keys = p->loc_keys, a = p->loc_a, b = p->loc_b;
    if (layout_plan(p, smem_limit, true) == FIM_OK &&
        (p->loc_om >= 0) == (om >= 0) && (p->loc_keys >= 0) == (keys >= 0) && (p->loc_a >= 0) == (a >= 0) &&
        (p->loc_b >= 0) == (b >= 0))
        return FIM_OK;
    return layout_plan(p, smem_limit, false);
}

fim_status layout_plan(Plan* p, int smem_limit, bool stage_model) {
    const int Tx = p->Tx, Ty = p->Ty, SP = p->SP;
    const size_t omb = p->wide ? 4 : 2;      // omnigram entry / position bytes
    const size_t om_bytes = align16((size_t)p->N * omb);
    const size_t ord_bytes = align16((size_t)SP * p->SH * 2);
    const size_t med_bytes = align16((size_t)Tx * Ty * 2);
    // one coarse histogram per concurrently solved seed; seeds that walk the omnigram need none
    // (the learned seeds keep one histogram's room for the MLP's shared pre-activations)
    const size_t shist_bytes =
        (size_t)kSeedBins * (p->seed_mode == kSeedHistogram ? std::min(p->nwarps, p->RB * p->G) : 1) * 4;
    const size_t solve_bytes = ord_bytes + med_bytes + shist_bytes;
    size_t tab = 0;
    auto take_tab = [&](int* field, size_t bytes) {
        *field = (int)tab;
        tab += align16(bytes);
    };
    take_tab(&p->off_vtab, (size_t)p->ncols * 8);
    take_tab(&p->off_htab, (size_t)p->nrows * 8);
    take_tab(&p->off_spans, (size_t)p->nrows * 4);
    take_tab(&p->off_frow, (size_t)p->SH * 4);
    p->off_model = -1;
    if (stage_model) take_tab(&p->off_model, (size_t)kMlpParams * 2);
    if (p->xtab_words > 0) take_tab(&p->off_xtab, (size_t)p->xtab_words * 4);
    p->tab_bytes = (int)tab;  // everything from here on belongs to one tile group
    p->off_misc = (int)tab;
    tab += 256;
    auto gloc = [](size_t off) { return -(int)off - 1; };
    p->loc_bins = p->loc_keys = p->loc_a = p->loc_b = p->loc_hist = 0;
    p->loc_dig = -1;
    size_t glob = 0;
    auto take_glob = [&](size_t bytes) {
        const size_t o = glob;
        glob += (bytes + 255) & ~(size_t)255;
        return gloc(o);
    };
    size_t smem = 0;
    if (p->sort == kSortCount8 || p->sort == kSortCount16 || p->sort == kSortCount16x2) {
        const size_t bins = p->sort == kSortCount8 ? 256 * 4 : 32768 * 4;
        const size_t uni = std::max(bins, solve_bytes);
        const bool om_smem = !p->wide && tab + om_bytes + uni <= (size_t)smem_limit;
        size_t off = tab;
        if (om_smem) {
            p->loc_om = (int)off;
            off += om_bytes;
        } else {
            p->loc_om = take_glob(om_bytes);
        }
        p->loc_bins = (int)off;
        p->loc_ord = (int)off;
        p->loc_med = (int)(off + ord_bytes);
        p->loc_shist = (int)(off + ord_bytes + med_bytes);
        smem = off + uni;
    } else {
        const size_t keys_bytes = align16((size_t)p->S * p->SH * 4);
        const size_t dig_bytes = align16((size_t)p->S * p->SH);
        const size_t hist_bytes = align16((size_t)p->nwarps * (kSortBins + 1) * 4);
        // try: (0) everything in shared memory; (1) keys in global; (2) keys and both lists in
        // global. Float keys in (1) and (2) keep list A in global memory too and give the stable
        // passes their digit of every box position in a shared byte array: two stable passes
        // gathering keys from L2 one at a time made the whole sort cost 1.8x as much (f32 r = 64:
        // 429k against 233k cycles per tile). 16-bit data (one stable pass, small footprints)
        // keeps the gathers. The 16-bit first pass's bins alias the region of list A (or the
        // digits) and the histograms, which are only used after it.
        const bool use_dig = p->dtype == FIM_F32;
        int mode = 0;
        for (;;) {
            const size_t bins_bytes = p->sort == kSortRadix16 ? 32768 * 4 : 0;
            for (mode = 0; mode < 3; ++mode) {
                if (mode < 2 && p->wide) continue;  // 32-bit lists of a wide box never fit
                size_t need = tab;
                if (mode < 2) need += om_bytes;  // B / omnigram
                const size_t list_a = mode == 0 ? om_bytes : (use_dig ? dig_bytes : (mode == 1 ? om_bytes : 0));
                const size_t sort_part = (mode == 0 ? keys_bytes : 0) + std::max(list_a + hist_bytes, bins_bytes);
                need += std::max(sort_part, solve_bytes);
                if (need <= (size_t)smem_limit) break;
            }
            if (mode < 3 || p->sort != kSortRadix16) break;
            p->sort = kSortRadix;  // no room for the 65536 bins: four 8-bit passes
        }
        if (mode == 3) return FIM_ERR_UNSUPPORTED;
        size_t off = tab;
        if (mode < 2) {
            p->loc_b = (int)off;
            off += om_bytes;
        } else {
            p->loc_b = take_glob(om_bytes);
        }
        p->loc_om = p->loc_b;  // the sorted positions are turned into the omnigram in place
        const size_t uni = off;
        if (mode == 0) {
            p->loc_keys = (int)off;
            off += keys_bytes;
        } else {
            p->loc_keys = take_glob(keys_bytes);
        }
        if (mode == 0 || (mode == 1 && !use_dig)) {
            p->loc_a = (int)off;
            off += om_bytes;
            p->loc_bins = p->loc_a;  // start of list A's and the histograms' region
        } else {
            p->loc_a = take_glob(om_bytes);
            p->loc_bins = (int)off;  // start of the digits' (if any) and the histograms' region
            if (use_dig) {
                p->loc_dig = (int)off;
                off += dig_bytes;
            }
        }
        p->loc_hist = (int)off;
        off += hist_bytes;
        if (p->sort == kSortRadix16) off = std::max(off, (size_t)p->loc_bins + 32768 * 4);
        p->loc_ord = (int)uni;
        p->loc_med = (int)(uni + ord_bytes);
        p->loc_shist = (int)(uni + ord_bytes + med_bytes);
        smem = std::max(off, uni + solve_bytes);
    }
    if (smem > (size_t)smem_limit) return FIM_ERR_UNSUPPORTED;
    // Staging region for the footprint copies of interior tiles (128 bytes of slack let the kernel
    // align it to 128 bytes): only where the box is a valid copy (at most 256 x 256 elements, rows
    // a multiple of 16 bytes) and the region fits beside everything else without costing the SM a
    // resident CTA.
    p->loc_stage = -1;
    p->stage_bw = 0;
    p->use_tma = 0;
    {
        const int es = elem_size(p->dtype), A = 16 / es;
        const int bw = (p->S + A - 1 + A - 1) / A * A;
        const size_t off = (smem + 127) & ~(size_t)127;
        const size_t end = off + (size_t)bw * p->SH * es + 128;
        const int per_sm = device_smem_per_sm();
        auto ctas = [&](size_t bytes) {  // resident CTAs per SM by shared memory and registers
            const int by_regs = 65536 / (p->threads * 64);
            return per_sm > 0 ? std::min(by_regs, per_sm / (int)(align16(bytes) + 1024)) : 0;
        };
        if (bw <= 256 && p->SH <= 256 && end <= (size_t)smem_limit && per_sm > 0 && ctas(end) >= ctas(smem) &&
            ctas(end) >= 1) {
            p->loc_stage = (int)off;
            p->stage_bw = bw;
            smem = end;
        }
    }
    p->smem_bytes = (int)align16(smem);
    p->group_bytes = p->smem_bytes - p->tab_bytes;
    p->groups = 1;
    p->scratch_per_cta = (long long)glob;
    return FIM_OK;
}

// CTAs of a plan resident per SM: its threads at 64 registers each (the kernels' cap), its
// shared memory plus the 1 KiB the runtime reserves per CTA.
static int resident_ctas(const Plan& p) {
    const int per_sm = device_smem_per_sm();
    const int by_regs = 65536 / (p.threads * 64);
    const int by_smem = per_sm > 0 ? per_sm / (p.smem_bytes + 1024) : 1;
    return std::max(1, std::min(std::min(by_regs, by_smem), std::min(2048 / p.threads, 32)));
}

bool small_image_shape(const fim_kernel* k, int dtype, int w, int h, int smem_limit, int cta_threads,
                       bool exact_ranks, const TileShape& def, Plan* scratch, TileShape* out) {
    if ((long long)w * h <= 0) return false;
    const int extent = std::max(k->xmax - k->xmin, k->ymax - k->ymin) + 1;
    const int sms = device_sm_count();
    auto tiles = [&](const TileShape& c) { return (long long)((w + c.Tx - 1) / c.Tx) * ((h + c.Ty - 1) / c.Ty); };
    if (make_plan(k, dtype, 0, 1, 1, def, smem_limit, scratch, cta_threads, exact_ranks) != FIM_OK) return false;
    if (2 * tiles(def) >= (long long)sms * resident_ctas(*scratch)) return false;
    // kernels up to 65 pixels across: 32-wide tiles with 1-row bands first; larger kernels:
    // 8 bands of 2 or 4 rows (u8 256^2 r = 40 / 64 / 96: 35 / 49 / 70 us per call on 32x16
    // against 142 / 181 / 388 on the defaults; 512^2: 58 / 75 / 107 on 64x32 against 139 /
    // 196 / 441)
    static const TileShape small[] = {{32, 8, 4, 1}, {32, 16, 4, 1}, {32, 8, 2, 1}};
    static const TileShape large[] = {{32, 16, 8, 2}, {64, 32, 8, 2}};
    const bool big = extent > 65;
    const TileShape* list = big ? large : small;
    const int nlist = big ? 2 : 3;
    for (int i = 0; i < nlist; ++i) {
        const TileShape& c = list[i];
        if (make_plan(k, dtype, 0, 1, 1, c, smem_limit, scratch, cta_threads, exact_ranks) != FIM_OK ||
            scratch->smem_bytes > smem_limit)
            continue;
        if (tiles(c) <= (long long)sms * resident_ctas(*scratch)) {
            *out = c;
            return true;
        }
    }
    return false;
}

static bool parse_tile_env(TileShape* ts) {
    const char* e = getenv("FIM_TILE");
    if (!e || !*e) return false;
    int a, b, c, d;
    if (sscanf(e, "%d,%d,%d,%d", &a, &b, &c, &d) != 4) return false;
    *ts = TileShape{a, b, c, d};
    return true;
}

fim_status choose_tile(const fim_kernel* k, int dtype, int smem_limit, TileShape* ts, int w, int h,
                       int cta_threads, bool exact_ranks) {
    static const TileShape cands[] = {{32, 32, 2, 1}, {32, 32, 4, 1}, {64, 128, 8, 2}, {64, 64, 8, 2},
                                      {32, 64, 8, 2}, {32, 32, 8, 2}, {32, 16, 8, 2}};
    TileShape forced;
    if (parse_tile_env(&forced)) {  // explicit override (experiments, tuning)
        Plan* p = new (std::nothrow) Plan;
        if (!p) return FIM_ERR_OOM;
        fim_status s = make_plan(k, dtype, 0, 1, 1, forced, smem_limit, p, cta_threads, exact_ranks);
        const int bytes = p->smem_bytes;
        delete p;
        if (s != FIM_OK) return s;
        if (bytes > smem_limit) return FIM_ERR_UNSUPPORTED;
        *ts = forced;
        return FIM_OK;
    }
    TileShape tuned;
    // configuration chosen by fim_autotune: for this CTA size first, then for any size
    const int sc = size_class(w, h);
    if ((cta_threads > 0 && tuned_lookup(k, dtype, &tuned, sc, cta_threads)) || tuned_lookup(k, dtype, &tuned, sc, 0)) {
        Plan* p = new (std::nothrow) Plan;
        if (!p) return FIM_ERR_OOM;
        fim_status s = make_plan(k, dtype, 0, 1, 1, tuned, smem_limit, p, cta_threads, exact_ranks);
        delete p;
        if (s == FIM_OK) {
            *ts = tuned;
            return FIM_OK;
        }
    }
    // Defaults measured on the 4096^2 photo-like workload. Kernels up to 33 pixels across: 32x32
    // tiles with two bands in 128-thread CTAs, many per SM (the footprint, and so every
    // refinement scan, shrinks with the tile; 16-bit data then sorts by radix passes); up to 45
    // across: the same tiles with four bands; up to 64 across: 64x64 tiles in 1024-thread CTAs;
    // beyond: taller 64x128 tiles, which halve the seed and seed-row work per pixel.
    const int extent = std::max(k->xmax - k->xmin, k->ymax - k->ymin) + 1;
    const int first = extent <= 33 ? 0 : (extent <= 45 ? 1 : (extent >= 65 ? 2 : 3));
    // Beyond the first valid shape, two measured exceptions (4096^2 photo-like u16, 4096^2 u8,
    // 8192^2 f32):
    // (1) where its omnigram spills to global scratch, a later shape of at least 64x64 whose
    //     omnigram stays in shared memory wins (u16 r = 80: 5.04 Gpix/s on 64x64 against 3.37
    //     on 64x128);
    // (2) for 16-bit data, whose footprints beyond 65535 pixels (ranks relative to the feasible
    //     range) count in two rounds and seed by walks, the first exact-rank shape wins unless
    //     its tile is under 64x64 (r = 96: 3.01 on 64x64 against 2.82 on 64x128; r = 112: 2.31
    //     on 64x128 against 0.88 on the exact-rank 32x64). 8-bit
    //     data (256 bins) and float keys (radix passes on global lists at these sizes) keep the
    //     larger tile (u8 r = 96: 4.30 on 64x128 against 3.43; f32 r = 100: 1.75 against 1.67).
    struct Info {
        bool ok;
        int n;
        bool om_smem;
    };
    auto probe = [&](const TileShape& c, Info* inf) {
        inf->ok = false;
        Plan* p = new (std::nothrow) Plan;
        if (!p) return FIM_ERR_OOM;
        const fim_status s = make_plan(k, dtype, 0, 1, 1, c, smem_limit, p, cta_threads, exact_ranks);
        inf->ok = s == FIM_OK && p->smem_bytes <= smem_limit;
        inf->n = p->N;
        inf->om_smem = p->loc_om >= 0;
        delete p;
        return FIM_OK;
    };
    const int ncands = (int)(sizeof(cands) / sizeof(cands[0]));
    int i0 = -1;
    Info f{};
    for (int i = first; i < ncands && i0 < 0; ++i) {
        if (probe(cands[i], &f) != FIM_OK) return FIM_ERR_OOM;
        if (f.ok) i0 = i;
    }
    if (i0 < 0) return FIM_ERR_UNSUPPORTED;
    Info g{};
    int pick = i0;
    if (!f.om_smem)
        for (int i = i0 + 1; i < ncands && pick == i0; ++i) {
            if (probe(cands[i], &g) != FIM_OK) return FIM_ERR_OOM;
            if (g.ok && g.om_smem && cands[i].Tx * cands[i].Ty >= 4096) pick = i;
        }
    if (pick == i0 && dtype == FIM_U16 && f.n > 65535)
        for (int i = i0 + 1; i < ncands; ++i) {
            if (probe(cands[i], &g) != FIM_OK) return FIM_ERR_OOM;
            if (g.ok && g.n <= 65535) {
                if (cands[i].Tx * cands[i].Ty >= 4096) pick = i;
                break;
            }
        }
    *ts = cands[pick];
    // Small images, whose tiles would fill under half the GPU's resident CTAs: the first of the
    // smaller shapes that fits them all in one wave (measured, u8 256^2 r = 4 / 16 / 32: 58 /
    // 50 / 134 us per call on the default tiles against 23 / 26 / 33 on 32x8 tiles with 4 bands;
    // 512^2: 63 / 63 / 160 against 36 / 40 / 54 on 32x16; at 1024^2 the defaults stay ahead).
    Plan* p = new (std::nothrow) Plan;
    if (!p) return FIM_ERR_OOM;
    TileShape small;
    if (small_image_shape(k, dtype, w, h, smem_limit, cta_threads, exact_ranks, *ts, p, &small)) *ts = small;
    delete p;
    return FIM_OK;
}

}  // namespace fim

namespace fim {
namespace {
std::mutex g_diag_mu;
unsigned long long* g_phase_buf = nullptr;
int g_phase_tiles = 0;
}  // namespace

void set_phase_clock_buffer(unsigned long long* buf, int tiles) {
    std::lock_guard<std::mutex> g(g_diag_mu);
    g_phase_buf = buf;
    g_phase_tiles = buf ? tiles : 0;
}

void get_phase_clock_buffer(unsigned long long** buf, int* tiles) {
    std::lock_guard<std::mutex> g(g_diag_mu);
    *buf = g_phase_buf;
    *tiles = g_phase_tiles;
}
}  // namespace fim

using namespace fim;

namespace {

struct Hostbufs {
    void* d_in = nullptr;
    void* d_out = nullptr;
    size_t bytes = 0;
    ~Hostbufs() {
        if (d_in) cudaFree(d_in);
        if (d_out) cudaFree(d_out);
    }
};

// Streams and events of the banded host pipeline (one set per host thread).
constexpr int kHostBands = 8;
struct HostPipe {
    cudaStream_t in = nullptr, out = nullptr, comp[2] = {nullptr, nullptr};
    cudaEvent_t start = nullptr, done = nullptr, in_ev[kHostBands] = {}, comp_ev[kHostBands] = {};
    bool ready = false;
    bool init() {
        if (ready) return true;
        bool ok = cudaStreamCreateWithFlags(&in, cudaStreamNonBlocking) == cudaSuccess &&
                  cudaStreamCreateWithFlags(&out, cudaStreamNonBlocking) == cudaSuccess &&
                  cudaStreamCreateWithFlags(&comp[0], cudaStreamNonBlocking) == cudaSuccess &&
                  cudaStreamCreateWithFlags(&comp[1], cudaStreamNonBlocking) == cudaSuccess &&
                  cudaEventCreateWithFlags(&start, cudaEventDisableTiming) == cudaSuccess &&
                  cudaEventCreateWithFlags(&done, cudaEventDisableTiming) == cudaSuccess;
        for (int b = 0; ok && b < kHostBands; ++b)
            ok = cudaEventCreateWithFlags(&in_ev[b], cudaEventDisableTiming) == cudaSuccess &&
                 cudaEventCreateWithFlags(&comp_ev[b], cudaEventDisableTiming) == cudaSuccess;
        if (!ok) cudaGetLastError();
        ready = ok;
        return ok;
    }
};

bool ranges_overlap(const void* a, const void* b, size_t bytes) {
    const uintptr_t pa = (uintptr_t)a, pb = (uintptr_t)b;
    return pa < pb + bytes && pb < pa + bytes;
}

fim_status check_image_args(const void* in, const void* out, int w, int h, size_t pitch, int dtype,
                            const fim_kernel* k, int border) {
    if (!in || !out || !k || w <= 0 || h <= 0) return FIM_ERR_INVALID_ARG;
    if (dtype != FIM_U8 && dtype != FIM_U16 && dtype != FIM_F32) return FIM_ERR_INVALID_ARG;
    if (border != FIM_BORDER_CLAMP) return FIM_ERR_INVALID_ARG;
    const size_t es = (size_t)elem_size(dtype);
    if (pitch < (size_t)w * es || pitch % es != 0) return FIM_ERR_INVALID_ARG;
    const size_t span = pitch * (size_t)(h - 1) + (size_t)w * es;
    if (ranges_overlap(in, out, span)) return FIM_ERR_INVALID_ARG;
    return FIM_OK;
}

fim_status filter_rank(const void* in, void* out, int w, int h, size_t pitch, int dtype, const fim_kernel* k,
                       int rank, cudaStream_t stream) {
    static thread_local int smem_limit = -1;
    if (smem_limit < 0) smem_limit = device_smem_limit();
    if (smem_limit <= 0) return FIM_ERR_CUDA;
    TileShape ts;
    fim_status s = choose_tile(k, dtype, smem_limit, &ts, w, h);
    if (s != FIM_OK) return s;
    Plan* p = new (std::nothrow) Plan;
    if (!p) return FIM_ERR_OOM;
    s = make_plan(k, dtype, rank, w, h, ts, smem_limit, p);
    if (s == FIM_OK) {
        p->in = in;
        p->out = out;
        p->pitch = (long long)pitch;
        get_phase_clock_buffer(&p->phase_clock, &p->phase_tiles);
        s = launch_tile_kernel(*p, stream);
    }
    delete p;
    return s;
}

}  // namespace

extern "C" {

fim_status fim_create_kernel_circle(int radius, fim_kernel** out) {
    if (!out || radius < 0 || radius > 128) return FIM_ERR_INVALID_ARG;
    return disk_kernel((int64_t)radius * radius, out);
}

fim_status fim_create_kernel_disk_limit(int64_t limit, fim_kernel** out) {
    if (!out || limit < 0 || isqrt64(limit) > 128) return FIM_ERR_INVALID_ARG;
    return disk_kernel(limit, out);
}

fim_status fim_create_kernel_ellipse(int a, int b, fim_kernel** out) {
    if (!out || a < 0 || b < 0 || a > 128 || b > 128) return FIM_ERR_INVALID_ARG;
    fim_kernel* k;
    fim_status s = new_kernel(out, &k);
    if (s != FIM_OK) return s;
    k->shape = kShapeSpans;
    k->r2 = 0;
    const int64_t A = a, B = b;
    if (b == 0) {
        k->ymin = 0;
        k->rlo.push_back(-a);
        k->rhi.push_back(a);
    } else {
        k->ymin = -b;
        for (int dy = -b; dy <= b; ++dy) {
            const int64_t rest = A * A * B * B - (int64_t)dy * dy * A * A;  // >= 0
            const int half = (int)isqrt64(rest / (B * B));
            k->rlo.push_back(-half);
            k->rhi.push_back(half);
        }
    }
    return publish(k, out);
}

fim_status fim_create_kernel_polygon(const double* xy, int nverts, fim_kernel** out) {
    if (!out || !xy || nverts < 3 || nverts > 4096) return FIM_ERR_INVALID_ARG;
    const double eps = 1e-9;
    double area2 = 0.0;
    double xlo = xy[0], xhi = xy[0], ylo = xy[1], yhi = xy[1];
    for (int i = 0; i < nverts; ++i) {
        const double ax = xy[2 * i], ay = xy[2 * i + 1];
        const double bx = xy[2 * ((i + 1) % nverts)], by = xy[2 * ((i + 1) % nverts) + 1];
        const double cx = xy[2 * ((i + 2) % nverts)], cy = xy[2 * ((i + 2) % nverts) + 1];
        if (!isfinite(ax) || !isfinite(ay)) return FIM_ERR_INVALID_ARG;
        area2 += ax * by - bx * ay;
        if ((bx - ax) * (cy - by) - (by - ay) * (cx - bx) < -eps) return FIM_ERR_INVALID_ARG;  // reflex turn
        xlo = std::min(xlo, ax);
        xhi = std::max(xhi, ax);
        ylo = std::min(ylo, ay);
        yhi = std::max(yhi, ay);
    }
    if (area2 <= 0.0) return FIM_ERR_INVALID_ARG;
    if (xhi - xlo > 2.0 * FIM_MAX_KERNEL_EXTENT || yhi - ylo > 2.0 * FIM_MAX_KERNEL_EXTENT) return FIM_ERR_UNSUPPORTED;
    fim_kernel* k;
    fim_status s = new_kernel(out, &k);
    if (s != FIM_OK) return s;
    k->shape = kShapeSpans;
    k->r2 = 0;
    const int x0 = (int)floor(xlo) - 1, x1 = (int)ceil(xhi) + 1;
    const int y0 = (int)floor(ylo) - 1, y1 = (int)ceil(yhi) + 1;
    bool started = false;
    for (int dy = y0; dy <= y1; ++dy) {
        int lo = 1 << 30, hi = -(1 << 30);
        for (int dx = x0; dx <= x1; ++dx) {
            bool inside = true;
            for (int i = 0; i < nverts && inside; ++i) {
                const double ax = xy[2 * i], ay = xy[2 * i + 1];
                const double bx = xy[2 * ((i + 1) % nverts)], by = xy[2 * ((i + 1) % nverts) + 1];
                inside = (bx - ax) * (dy - ay) - (by - ay) * (dx - ax) >= -eps;
            }
            if (inside) {
                lo = std::min(lo, dx);
                hi = std::max(hi, dx);
            }
        }
        if (lo <= hi) {
            if (!started) {
                k->ymin = dy;
                started = true;
            }
            k->rlo.push_back(lo);
            k->rhi.push_back(hi);
        } else if (started) {
            break;
        }
    }
    if (!started) {
        delete k;
        return FIM_ERR_INVALID_ARG;
    }
    return publish(k, out);
}

fim_status fim_create_kernel_spans(const int* lo, const int* hi, int dy0, int rows, fim_kernel** out) {
    if (!out || !lo || !hi || rows <= 0 || rows > FIM_MAX_KERNEL_EXTENT) return FIM_ERR_INVALID_ARG;
    if (dy0 < -4 * FIM_MAX_KERNEL_EXTENT || dy0 > 4 * FIM_MAX_KERNEL_EXTENT) return FIM_ERR_INVALID_ARG;
    for (int i = 0; i < rows; ++i)
        if (lo[i] < -4 * FIM_MAX_KERNEL_EXTENT || hi[i] > 4 * FIM_MAX_KERNEL_EXTENT) return FIM_ERR_INVALID_ARG;
    fim_kernel* k;
    fim_status s = new_kernel(out, &k);
    if (s != FIM_OK) return s;
    k->shape = kShapeSpans;
    k->r2 = 0;
    k->ymin = dy0;
    k->rlo.assign(lo, lo + rows);
    k->rhi.assign(hi, hi + rows);
    return publish(k, out);
}

fim_status fim_kernel_info(const fim_kernel* k, int* ntaps, int* xmin, int* xmax, int* ymin, int* ymax) {
    if (!k) return FIM_ERR_INVALID_ARG;
    if (ntaps) *ntaps = k->n;
    if (xmin) *xmin = k->xmin;
    if (xmax) *xmax = k->xmax;
    if (ymin) *ymin = k->ymin;
    if (ymax) *ymax = k->ymax;
    return FIM_OK;
}

void fim_destroy_kernel(fim_kernel* k) { delete k; }

fim_status fim_median(const void* in, void* out, int w, int h, size_t pitch_bytes, fim_dtype dtype,
                      const fim_kernel* k, fim_border border, void* stream) {
    fim_status s = check_image_args(in, out, w, h, pitch_bytes, dtype, k, border);
    if (s != FIM_OK) return s;
    return filter_rank(in, out, w, h, pitch_bytes, dtype, k, (k->n - 1) / 2, (cudaStream_t)stream);
}

fim_status fim_percentile(const void* in, void* out, int w, int h, size_t pitch_bytes, fim_dtype dtype,
                          const fim_kernel* k, double percentile, fim_border border, void* stream) {
    fim_status s = check_image_args(in, out, w, h, pitch_bytes, dtype, k, border);
    if (s != FIM_OK) return s;
    if (!(percentile >= 0.0 && percentile <= 100.0)) return FIM_ERR_INVALID_ARG;
    const int rank = (int)floor(percentile / 100.0 * (k->n - 1) + 0.5);
    return filter_rank(in, out, w, h, pitch_bytes, dtype, k, std::min(std::max(rank, 0), k->n - 1),
                       (cudaStream_t)stream);
}

fim_status fim_percentiles(const void* in, void* const* outs, const double* percentiles, int count, int w, int h,
                           size_t pitch_bytes, fim_dtype dtype, const fim_kernel* k, fim_border border,
                           void* stream) {
    if (!outs || !percentiles || count < 1 || count > kMaxRanks) return FIM_ERR_INVALID_ARG;
    for (int i = 0; i < count; ++i) {
        fim_status s = check_image_args(in, outs[i], w, h, pitch_bytes, dtype, k, border);
        if (s != FIM_OK) return s;
        if (!(percentiles[i] >= 0.0 && percentiles[i] <= 100.0)) return FIM_ERR_INVALID_ARG;
    }
    static thread_local int smem_limit = -1;
    if (smem_limit < 0) smem_limit = device_smem_limit();
    if (smem_limit <= 0) return FIM_ERR_CUDA;
    TileShape ts;
    fim_status s = choose_tile(k, dtype, smem_limit, &ts, w, h);
    if (s != FIM_OK) return s;
    int ranks[kMaxRanks];
    for (int i = 0; i < count; ++i)
        ranks[i] = std::min(std::max((int)floor(percentiles[i] / 100.0 * (k->n - 1) + 0.5), 0), k->n - 1);
    Plan* p = new (std::nothrow) Plan;
    if (!p) return FIM_ERR_OOM;
    int rmin = ranks[0], rmax = ranks[0];
    for (int i = 1; i < count; ++i) {
        rmin = std::min(rmin, ranks[i]);
        rmax = std::max(rmax, ranks[i]);
    }
    // offset ranks (large footprints) must resolve every target's feasible ranks
    s = make_plan(k, dtype, rmin, w, h, ts, smem_limit, p);
    if (s == FIM_OK && p->N > 65535 && p->N - k->n + rmax - p->rank_base > 65535) s = FIM_ERR_UNSUPPORTED;
    if (s == FIM_OK) {
        p->in = in;
        p->out = outs[0];
        p->pitch = (long long)pitch_bytes;
        p->nranks = count;
        p->rank = ranks[0];
        for (int i = 0; i < count; ++i) {
            p->ranks[i] = ranks[i];
            p->outs[i] = outs[i];
        }
        get_phase_clock_buffer(&p->phase_clock, &p->phase_tiles);
        s = launch_tile_kernel(*p, (cudaStream_t)stream);
    }
    delete p;
    return s;
}

fim_status fim_median_radii(const void* in, void* const* outs, const fim_kernel* const* kernels, int count, int w,
                            int h, size_t pitch_bytes, fim_dtype dtype, fim_border border, void* stream) {
    if (!outs || !kernels || count < 1 || count > kMaxRanks) return FIM_ERR_INVALID_ARG;
    int big = 0;  // the largest disk: its footprint holds every other disk's windows
    for (int i = 0; i < count; ++i) {
        fim_status s = check_image_args(in, outs[i], w, h, pitch_bytes, dtype, kernels[i], border);
        if (s != FIM_OK) return s;
        if (kernels[i]->shape != kShapeDisk) return FIM_ERR_INVALID_ARG;
        if (kernels[i]->r2 > kernels[big]->r2) big = i;
    }
    static thread_local int smem_limit = -1;
    if (smem_limit < 0) smem_limit = device_smem_limit();
    if (smem_limit <= 0) return FIM_ERR_CUDA;
    const fim_kernel* kb = kernels[big];
    TileShape ts;
    // the omnigram is narrowed from disk to disk with exact ranks: no rank offsets
    fim_status s = choose_tile(kb, dtype, smem_limit, &ts, w, h, 0, true);
    if (s != FIM_OK) return s;
    Plan* p = new (std::nothrow) Plan;
    if (!p) return FIM_ERR_OOM;
    s = make_plan(kb, dtype, (kb->n - 1) / 2, w, h, ts, smem_limit, p, 0, true);
    // Targets run largest disk first, so that each footprint holds the next one and the tile can
    // narrow its omnigram from disk to disk. Every disk's tables (per-column vertical-slide
    // offsets, per-row horizontal offsets and spans) are relative to the window centre in the
    // largest disk's footprint box; its footprint rows are in that box's coordinates.
    int order[kMaxRanks];
    for (int q = 0; q < count; ++q) order[q] = q;
    std::stable_sort(order, order + count, [&](int a, int b) { return kernels[a]->r2 > kernels[b]->r2; });
    std::vector<int> xt;
    int rel_v[kMaxRanks], rel_h[kMaxRanks], rel_s[kMaxRanks], rel_f[kMaxRanks];
    if (s == FIM_OK) {
        const int SP = p->SP, SH = p->SH, Tx = p->Tx, Ty = p->Ty;
        for (int q = 0; q < count; ++q) {
            const fim_kernel* k = kernels[order[q]];
            const int nrows = k->ymax - k->ymin + 1, ncols = k->xmax - k->xmin + 1;
            rel_v[q] = (int)xt.size();
            for (int j = 0; j < ncols; ++j) {
                xt.push_back(k->ctop[j] * SP + k->xmin + j);
                xt.push_back((k->cbot[j] + 1) * SP + k->xmin + j);
            }
            rel_h[q] = (int)xt.size();
            for (int i = 0; i < nrows; ++i) {
                xt.push_back((k->ymin + i) * SP + k->rlo[i]);
                xt.push_back((k->ymin + i) * SP + k->rhi[i] + 1);
            }
            rel_s[q] = (int)xt.size();
            for (int i = 0; i < nrows; ++i) xt.push_back((int)((uint32_t)(k->rlo[i] & 0xffff) | ((uint32_t)k->rhi[i] << 16)));
            // this disk's footprint (Fig. 10) in the box: row v holds the columns of the tile's
            // windows whose kernel row i meets box row v
            rel_f[q] = (int)xt.size();
            long long nq = 0;
            for (int v = 0; v < SH; ++v) {
                const int i0 = std::max(0, v + p->ymin - k->ymin - Ty + 1), i1 = std::min(nrows - 1, v + p->ymin - k->ymin);
                int lo = 1 << 14, hi = -(1 << 14);
                for (int i = i0; i <= i1; ++i) {
                    lo = std::min(lo, k->rlo[i] - p->xmin);
                    hi = std::max(hi, k->rhi[i] + Tx - 1 - p->xmin);
                }
                if (lo > hi) lo = 1, hi = 0;  // no pixel of this row
                xt.push_back((int)((uint32_t)(lo & 0xffff) | ((uint32_t)hi << 16)));
                nq += hi - lo + 1;
            }
            if (xt.size() & 1) xt.push_back(0);  // the next disk's int2 tables stay 8-byte aligned
            p->q_r2[q] = (int)k->r2;
            p->q_n[q] = k->n;
            p->q_ymin[q] = k->ymin;
            p->q_nrows[q] = nrows;
            p->q_ncols[q] = ncols;
            p->q_N[q] = (int)nq;
            int hs = 0;
            while (((nq - 1) >> hs) >= kSeedBins) ++hs;
            p->q_hshift[q] = hs;
            p->q_vmix[q] = std::max(k->xmax - k->xmin, k->ymax - k->ymin) + 1 <= 40 ? 1 : 0;
            p->ranks[q] = (k->n - 1) / 2;
            p->outs[q] = outs[order[q]];
        }
        p->xtab_words = (int)xt.size();
        s = layout_plan(p, smem_limit);
    }
    int* dx = nullptr;
    cudaStream_t st = (cudaStream_t)stream;
    if (s == FIM_OK) {
        if (cudaMallocAsync(reinterpret_cast<void**>(&dx), xt.size() * 4, st) != cudaSuccess) {
            cudaGetLastError();
            s = FIM_ERR_OOM;
        } else if (cudaMemcpyAsync(dx, xt.data(), xt.size() * 4, cudaMemcpyHostToDevice, st) != cudaSuccess) {
            s = FIM_ERR_CUDA;
        }
    }
    if (s == FIM_OK) {
        for (int q = 0; q < count; ++q) {
            p->q_vtab[q] = p->off_xtab + 4 * rel_v[q];
            p->q_htab[q] = p->off_xtab + 4 * rel_h[q];
            p->q_spans[q] = p->off_xtab + 4 * rel_s[q];
            p->q_frow[q] = p->off_xtab + 4 * rel_f[q];
        }
        p->multi = 1;
        p->xtab = dx;
        p->in = in;
        p->out = p->outs[0];
        p->rank = p->ranks[0];
        p->pitch = (long long)pitch_bytes;
        p->nranks = count;
        get_phase_clock_buffer(&p->phase_clock, &p->phase_tiles);
        s = launch_tile_kernel(*p, st);
    }
    if (dx && cudaFreeAsync(dx, st) != cudaSuccess && s == FIM_OK) s = FIM_ERR_CUDA;
    delete p;
    return s;
}

fim_status fim_percentile_map(const void* in, void* out, const float* percentiles, size_t pct_pitch_bytes, int w,
                              int h, size_t pitch_bytes, fim_dtype dtype, const fim_kernel* k, fim_border border,
                              void* stream) {
    fim_status s = check_image_args(in, out, w, h, pitch_bytes, dtype, k, border);
    if (s != FIM_OK) return s;
    if (!percentiles || pct_pitch_bytes < (size_t)w * sizeof(float) || pct_pitch_bytes % sizeof(float) != 0)
        return FIM_ERR_INVALID_ARG;
    const size_t map_span = pct_pitch_bytes * (size_t)(h - 1) + (size_t)w * sizeof(float);
    const size_t out_span = pitch_bytes * (size_t)(h - 1) + (size_t)w * (size_t)elem_size(dtype);
    const char* m0 = reinterpret_cast<const char*>(percentiles);
    const char* o0 = static_cast<const char*>(out);
    if (m0 < o0 + out_span && o0 < m0 + map_span) return FIM_ERR_INVALID_ARG;  // the map must outlive the writes
    static thread_local int smem_limit = -1;
    if (smem_limit < 0) smem_limit = device_smem_limit();
    if (smem_limit <= 0) return FIM_ERR_CUDA;
    TileShape ts;
    s = choose_tile(k, dtype, smem_limit, &ts, w, h, 0, true);  // a rank per pixel: exact ranks
    if (s != FIM_OK) return s;
    Plan* p = new (std::nothrow) Plan;
    if (!p) return FIM_ERR_OOM;
    s = make_plan(k, dtype, (k->n - 1) / 2, w, h, ts, smem_limit, p, 0, true);
    if (s == FIM_OK) {
        p->in = in;
        p->out = out;
        p->pitch = (long long)pitch_bytes;
        // the rank image lives in stream-ordered memory: allocated, filled, read by the filter and
        // released in stream order, so the call stays asynchronous
        const cudaStream_t st = (cudaStream_t)stream;
        int* ranks = nullptr;
        if (cudaMallocAsync(reinterpret_cast<void**>(&ranks), (size_t)w * (size_t)h * sizeof(int), st) != cudaSuccess) {
            cudaGetLastError();
            s = FIM_ERR_OOM;
        } else {
            s = launch_percentile_ranks(percentiles, (long long)pct_pitch_bytes, w, h, k->n, ranks, st);
            if (s == FIM_OK) {
                p->rank_map = ranks;
                get_phase_clock_buffer(&p->phase_clock, &p->phase_tiles);
                s = launch_tile_kernel(*p, st);
            }
            if (cudaFreeAsync(ranks, st) != cudaSuccess && s == FIM_OK) s = FIM_ERR_CUDA;
        }
    }
    delete p;
    return s;
}

fim_status fim_median_host(const void* in_host, void* out_host, int w, int h, size_t pitch_bytes,
                           fim_dtype dtype, const fim_kernel* k, fim_border border, void* stream) {
    fim_status s = check_image_args(in_host, out_host, w, h, pitch_bytes, dtype, k, border);
    if (s != FIM_OK) return s;
    static thread_local Hostbufs bufs;
    static thread_local HostPipe pipe;
    const size_t es = (size_t)elem_size(dtype);
    const size_t dpitch = (size_t)w * es;
    const size_t bytes = dpitch * (size_t)h;
    if (bufs.bytes < bytes) {
        if (bufs.d_in) cudaFree(bufs.d_in);
        if (bufs.d_out) cudaFree(bufs.d_out);
        bufs.d_in = bufs.d_out = nullptr;
        bufs.bytes = 0;
        if (cudaMalloc(&bufs.d_in, bytes) != cudaSuccess || cudaMalloc(&bufs.d_out, bytes) != cudaSuccess) {
            cudaGetLastError();
            return FIM_ERR_OOM;
        }
        bufs.bytes = bytes;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const int limit = device_smem_limit();
    if (limit <= 0) return FIM_ERR_CUDA;
    TileShape ts;
    s = choose_tile(k, dtype, limit, &ts, w, h);
    if (s != FIM_OK) return s;
    Plan* p = new (std::nothrow) Plan;
    if (!p) return FIM_ERR_OOM;
    s = make_plan(k, dtype, (k->n - 1) / 2, w, h, ts, limit, p);
    if (s != FIM_OK) {
        delete p;
        return s;
    }
    p->in = bufs.d_in;
    p->out = bufs.d_out;
    p->pitch = (long long)dpitch;
    // Bands of whole tile rows: band b's input rows (its rows plus the kernel's reach below)
    // are copied in, its tiles filtered on one of two compute streams (a band's tail overlaps
    // the next band's start) and its rows copied out, so the copies hide behind the kernels.
    const int rows_per_band = (p->tiles_y + kHostBands - 1) / kHostBands;
    const int bands = (p->tiles_y + rows_per_band - 1) / rows_per_band;
    const char* hin = static_cast<const char*>(in_host);
    char* hout = static_cast<char*>(out_host);
    const char* din = static_cast<const char*>(bufs.d_in);
    const char* dout = static_cast<const char*>(bufs.d_out);
    auto fail = [&]() {
        cudaGetLastError();
        delete p;
        return FIM_ERR_CUDA;
    };
    if (bands < 2 || !pipe.init()) {  // one band: copy in, filter, copy out on the caller's stream
        if (cudaMemcpy2DAsync(bufs.d_in, dpitch, in_host, pitch_bytes, dpitch, h, cudaMemcpyHostToDevice, st) !=
            cudaSuccess)
            return fail();
        s = launch_tile_kernel(*p, st);
        if (s == FIM_OK && cudaMemcpy2DAsync(out_host, pitch_bytes, bufs.d_out, dpitch, dpitch, h,
                                             cudaMemcpyDeviceToHost, st) != cudaSuccess)
            return fail();
    } else {
        if (cudaEventRecord(pipe.start, st) != cudaSuccess || cudaStreamWaitEvent(pipe.in, pipe.start, 0) != cudaSuccess)
            return fail();
        int copied = 0;  // input rows already on the device
        for (int b = 0; b < bands && s == FIM_OK; ++b) {
            const int tr0 = b * rows_per_band, tr1 = std::min(p->tiles_y, tr0 + rows_per_band);
            const int y0 = tr0 * p->Ty, y1 = std::min(h, tr1 * p->Ty);
            const int need = std::min(h, y1 + p->ymax);  // rows [0, need) feed this band
            if (need > copied) {
                if (cudaMemcpy2DAsync((void*)(din + (size_t)copied * dpitch), dpitch,
                                      hin + (size_t)copied * pitch_bytes, pitch_bytes, dpitch, need - copied,
                                      cudaMemcpyHostToDevice, pipe.in) != cudaSuccess)
                    return fail();
                copied = need;
            }
            cudaStream_t cs = pipe.comp[b & 1];
            if (cudaEventRecord(pipe.in_ev[b], pipe.in) != cudaSuccess ||
                cudaStreamWaitEvent(cs, pipe.in_ev[b], 0) != cudaSuccess)
                return fail();
            Plan& band = *p;
            band.tile0 = tr0 * p->tiles_x;
            band.tile_count = (tr1 - tr0) * p->tiles_x;
            s = launch_tile_kernel(band, cs);
            if (s != FIM_OK) {  // nothing may still be writing the caller's buffers on return
                cudaStreamSynchronize(pipe.in);
                cudaStreamSynchronize(pipe.comp[0]);
                cudaStreamSynchronize(pipe.comp[1]);
                cudaStreamSynchronize(pipe.out);
                break;
            }
            if (cudaEventRecord(pipe.comp_ev[b], cs) != cudaSuccess ||
                cudaStreamWaitEvent(pipe.out, pipe.comp_ev[b], 0) != cudaSuccess ||
                cudaMemcpy2DAsync(hout + (size_t)y0 * pitch_bytes, pitch_bytes, dout + (size_t)y0 * dpitch, dpitch,
                                  dpitch, y1 - y0, cudaMemcpyDeviceToHost, pipe.out) != cudaSuccess)
                return fail();
        }
        if (s == FIM_OK && (cudaEventRecord(pipe.done, pipe.out) != cudaSuccess ||
                            cudaStreamWaitEvent(st, pipe.done, 0) != cudaSuccess))
            return fail();
    }
    delete p;
    if (s != FIM_OK) return s;
    if (cudaStreamSynchronize(st) != cudaSuccess) return FIM_ERR_CUDA;
    return FIM_OK;
}

fim_status fim_sync_status(void* stream) { return read_and_clear_device_status((cudaStream_t)stream); }

fim_status fim_plan_info(const fim_kernel* k, fim_dtype dtype, int w, int h, int* tile_w, int* tile_h,
                         int* footprint, int* threads, int* smem_bytes) {
    if (!k || w <= 0 || h <= 0 || (dtype != FIM_U8 && dtype != FIM_U16 && dtype != FIM_F32)) return FIM_ERR_INVALID_ARG;
    const int limit = device_smem_limit();
    if (limit <= 0) return FIM_ERR_CUDA;
    TileShape ts;
    fim_status s = choose_tile(k, dtype, limit, &ts, w, h);
    if (s != FIM_OK) return s;
    Plan* p = new (std::nothrow) Plan;
    if (!p) return FIM_ERR_OOM;
    s = make_plan(k, dtype, (k->n - 1) / 2, w, h, ts, limit, p);
    if (s == FIM_OK) {
        if (tile_w) *tile_w = p->Tx;
        if (tile_h) *tile_h = p->Ty;
        if (footprint) *footprint = p->N;
        if (threads) *threads = p->threads;
        if (smem_bytes) *smem_bytes = p->smem_bytes;
    }
    delete p;
    return s;
}

const char* fim_status_string(fim_status s) {
    switch (s) {
        case FIM_OK: return "FIM_OK";
        case FIM_ERR_INVALID_ARG: return "FIM_ERR_INVALID_ARG";
        case FIM_ERR_UNSUPPORTED: return "FIM_ERR_UNSUPPORTED";
        case FIM_ERR_OOM: return "FIM_ERR_OOM";
        case FIM_ERR_CUDA: return "FIM_ERR_CUDA";
        case FIM_ERR_TIMEOUT: return "FIM_ERR_TIMEOUT";
        case FIM_ERR_INTERNAL: return "FIM_ERR_INTERNAL";
    }
    return "FIM_ERR_UNKNOWN";
}

const char* fim_version(void) { return "0.1.0"; }

fim_status fim_release_workspace(void) { return release_scratch(); }

fim_status fim_debug_phase_clocks(void* dev_buf, int tiles) {
    if ((dev_buf == nullptr) != (tiles <= 0)) return FIM_ERR_INVALID_ARG;
    set_phase_clock_buffer((unsigned long long*)dev_buf, tiles);
    return FIM_OK;
}

}  // extern "C"
