// Internal declarations shared by the host and device translation units of libfim.
#pragma once

#include <cuda.h>  // CUtensorMap (the footprint copies' tensor maps)
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <map>
#include <mutex>
#include <vector>

#include "fim.h"

namespace fim {

constexpr int kMaxExtent = 264;   // kernel rows / columns held in a plan (>= FIM_MAX_KERNEL_EXTENT)
constexpr int kMaxSide = 400;     // bounding-box rows of a tile footprint held in a plan
constexpr int kSortBins = 256;    // 8-bit radix digits
constexpr int kSeedBins = 256;    // coarse histogram bins of a seed solve

enum Shape : int { kShapeDisk = 0, kShapeSpans = 1 };

// Target ranks one launch can serve from one ordinal transform (fim_percentiles).
constexpr int kMaxRanks = 8;

// Rank-bracket MLP: kFeatures inputs -> kHidden -> kHidden -> 2 (predicted rank, log scale).
constexpr int kQuantiles = 32;   // footprint value quantiles
constexpr int kNeigh = 9;        // 3x3 neighbourhood ranks of the window centre
constexpr int kFeatures = kQuantiles + kNeigh;
constexpr int kHidden = 64;
constexpr int kMlpParams = kFeatures * kHidden + kHidden + kHidden * kHidden + kHidden + kHidden * 2 + 2;
static_assert(kMlpParams % 2 == 0, "parameters are staged as 32-bit pairs");
// parameter offsets in the flat vector: W1[f][h], b1[h], W2[h][h'], b2[h'], W3[h'][2], b3[2]
constexpr int kOffW1 = 0;
constexpr int kOffB1 = kOffW1 + kFeatures * kHidden;
constexpr int kOffW2 = kOffB1 + kHidden;
constexpr int kOffB2 = kOffW2 + kHidden * kHidden;
constexpr int kOffW3 = kOffB2 + kHidden;
constexpr int kOffB3 = kOffW3 + kHidden * 2;
// seed statistics: seeds, bracket hits, misses below, misses above, omnigram ranks scanned
constexpr int kStatSlots = 5;

// Geometry of one tile configuration: output tile Tx x Ty, 2*Tx*RB threads.
// RB bands of Ty/RB rows; each band's middle row is a seed row with G seeds.
struct TileShape {
    int Tx, Ty;
    int RB;
    int G;
};

// How the plain seed windows are solved (Sec. 4.2: seeds from histograms of the omnigram):
//   kSeedHistogram - a coarse histogram of the window's ranks (shared-memory atomics), scanned to
//                    the target's bin, then a ballot scan of the omnigram from that bin;
//   kSeedWalk      - a walk of the omnigram from rank 0 (or from N) counting the window's members
//                    512 entries a step, which is the histogram of the omnigram, bin by bin;
//   kSeedMidCount  - the window's members below the middle of the feasible ranks counted in the
//                    ordinal image, then the walk from there.
enum SeedMode : int { kSeedHistogram = 0, kSeedWalk = 1, kSeedMidCount = 2 };

enum SortKind : int {
    kSortCount8 = 0,   // 256-bin counting sort (8-bit data)
    kSortCount16 = 1,  // 65536-bin counting sort with packed 16-bit bins (16-bit data, Eq. 5)
    kSortRadix = 2,    // stable LSD radix sort, 8-bit passes (four for float keys, two for 16-bit data)
    kSortRadix16 = 3,  // float keys in 1024-thread CTAs: 65536-bin counting pass on the low 16 bits,
                       // then two stable 8-bit passes
    kSortCount16x2 = 4 // 16-bit data, footprints beyond 65535 pixels, 1024-thread CTAs: the counting
                       // sort in two rounds over the key range with 32768 32-bit bins each
};

// Everything a tile kernel launch needs, passed by value as a __grid_constant__ parameter.
// Scalars are read at static offsets; the tables are copied into shared memory once per CTA.
struct Plan {
    // image
    const void* in;
    void* out;
    long long pitch;  // bytes, input and output
    int w, h;
    int dtype;
    // tiling
    int Tx, Ty, txshift, RB, G;
    int threads, nwarps;    // CTA size (all cooperative loops and per-warp buffers)
    int vthreads;           // 2*Tx*RB: threads of the vertical sweep (the first ones of the CTA)
    int vmix;               // 1: the lanes of a vertical-sweep warp take their columns from all bands
    int scan_groups;        // 128-bit omnigram groups a vertical-sweep lane tests per scan step
    int S, SH;              // footprint bounding box (columns, rows)
    int SP;                 // row pitch (elements) of the ordinal image; SP/2 is odd
    int tiles_x, tiles_y;
    // kernel
    int shape;
    int r2;                 // disk: dx^2 + dy^2 <= r2
    int xmin, xmax, ymin, ymax, nrows, ncols;
    int n;                  // taps
    int rank;               // target 0-based rank ((n-1)/2 for the median)
    int nranks;             // extras kernels: target ranks served by one ordinal transform (1..kMaxRanks)
    int ranks[kMaxRanks];   //   their ranks; entry 0 is taken from `rank`
    void* outs[kMaxRanks];  //   and their outputs (same pitch as the input); entry 0 is taken from `out`
    // several disks from one transform (fim_median_radii): every target has a kernel of its own,
    // nested in the plan's kernel (which sets the footprint); its tables sit in shared memory
    int multi;                          // 1: the q_ arrays below give each target's kernel
    int q_vtab[kMaxRanks], q_htab[kMaxRanks], q_spans[kMaxRanks];  // shared-memory byte offsets
    int q_r2[kMaxRanks], q_n[kMaxRanks], q_ymin[kMaxRanks], q_nrows[kMaxRanks], q_ncols[kMaxRanks];
    int q_frow[kMaxRanks];              // shared-memory byte offset of each disk's footprint rows
    int q_N[kMaxRanks], q_hshift[kMaxRanks];  // its footprint size and seed-histogram shift
    int q_vmix[kMaxRanks];              // its vertical-sweep lane mixing (as `vmix` for its own plan)
    const int* xtab;                    // device: those tables, copied to shared memory at off_xtab
    int xtab_words;                     // their length in 32-bit words
    int off_xtab;
    // footprint
    int N;                  // pixels in the rounded-rectangle footprint
    int rank_base;          // the ordinal image and the medians hold rank - rank_base (16 bits)
    int cx0, cy0;           // omnigram coordinates are stored as (u - cx0, v - cy0), int8 each
    unsigned div_magic;     // ceil(2^32 / S): v = umulhi(pos, magic) = pos / S for pos < 2^32 / S (radix path)
    int hist_shift;         // seed histogram: bin = rank >> hist_shift
    int seed_mode;          // SeedMode of the plain seeds
    int sort;               // SortKind
    int wide;               // 1: footprint box wider than 256: 32-bit omnigram entries and positions
    // learned rank bracket for the seed windows (all optional; null = the plain histogram seeds)
    const uint16_t* model;            // bf16 MLP parameters (kMlpParams), device memory
    float bracket_z;                  // bracket half-width in predicted standard deviations
    unsigned long long* stats;        // kStatSlots counters, device memory
    float* samples;                   // training rows: kFeatures features + 1 label each
    unsigned int* sample_count;       // rows written so far (device counter)
    int sample_cap;                   // capacity of samples in rows
    // spatially varying percentile (extras kernels; null = every pixel takes `rank`)
    const int* rank_map;              // one target rank per output pixel, w x h, dense rows
    // footprint staging by the tensor memory accelerator (single-image launches; set at launch)
    int use_tma;                      // 1: interior tiles copy their footprint box into loc_stage
    int stage_bw;                     // staged row length in elements (a multiple of 16 bytes)
    int loc_stage;                    // shared-memory offset of the staging region (-1: none)
    unsigned long long* phase_clock;  // optional: 8 clock64() stamps per tile (diagnostics)
    int phase_tiles;                  // capacity of phase_clock in tiles
    // Array placement. A location >= 0 is a byte offset into dynamic shared memory; a location
    // < 0 is -(offset + 1) into the CTA's slice of global scratch.
    int off_vtab, off_htab, off_spans, off_frow;   // tables (shared memory, whole kernel)
    int off_model;                                  // bracket MLP parameters in shared memory, or -1
    int tab_bytes;                                  // the tables' extent; a tile group's partition follows
    int off_misc;                                   // 64 words of scan scratch (per group)
    int group_bytes;                                // bytes of one group's partition (smem_bytes - tab_bytes)
    int groups;                                     // batches: tile groups of this job run per CTA
    int loc_om;                                     // omnigram (from the end of the sort on)
    int loc_bins;                                   // counting sorts: bins
    int loc_keys, loc_a, loc_b, loc_hist;           // radix sort: keys, ping-pong lists, histograms
    int loc_dig;                                    // radix sort with keys in global scratch: digit bytes (-1: none)
    int loc_ord, loc_med, loc_shist;                // solve: ordinal image, medians, seed histograms
    int smem_bytes;
    long long scratch_per_cta;  // bytes of global scratch per resident CTA (multiple of 256)
    // persistent grid
    int ntiles;                 // tiles of this launch
    int tile0, tile_count;      // single-image launches: tiles [tile0, tile0 + tile_count) (count 0: all)
    unsigned char* scratch;     // header (256 B: tile counter) + grid * scratch_per_cta
    // tables (copied to shared memory at kernel start)
    int frow[kMaxSide];                   // footprint row v covers u in [lo, hi]: lo | hi << 16
    int vtab[2 * kMaxExtent];             // per column j: top*SP + dx, (bot+1)*SP + dx
    int htab[2 * kMaxExtent];             // per row i: dy*SP + lo, dy*SP + hi + 1
    int spans[kMaxExtent];                // per row i: (lo & 0xffff) | (hi << 16)
    // tensor map of the input image for the footprint copies (valid when use_tma)
    CUtensorMap tmap;  // (the type carries the alignment the copies need)
};

// Bytes of a Plan before its tables: all the tile pipeline reads once the tables are in
// shared memory.
constexpr size_t kPlanScalarBytes = ((offsetof(Plan, frow) + 15) / 16) * 16;
static_assert(offsetof(Plan, frow) % 4 == 0, "plan scalars are copied as 32-bit words");


// One class of a batch: jobs whose plans run on the same tile-pipeline instantiation and CTA size.
struct BatchClass {
    int dtype, shape, wide, og, ks;  // instantiation: element type, kernel shape, omnigram encoding
                                     // and home (global when og), scan groups per step (4 or 8)
    int threads, smem;               // CTA size and dynamic shared memory (the largest of its plans)
    int grid;                        // persistent CTAs
    int njobs, total_tiles;
    long long scratch_per_cta;       // the largest of its plans
};

// Arguments of one class kernel (all pointers are device memory owned by the batch).
struct BatchClassArgs {
    const Plan* plans;          // the class's plans, in the order of their tiles in the queue
    const int* tile_start;      // njobs exclusive prefix sums of the plans' tile counts
    int njobs, total_tiles;
    unsigned int* counter;      // the class's tile queue (zeroed before each run)
    unsigned char* scratch;     // grid * scratch_per_cta bytes of per-CTA buffers
    long long scratch_per_cta;
};

}  // namespace fim

// Public handle (opaque to callers).
struct fim_kernel {
    int shape;
    int64_t r2;
    int xmin, xmax, ymin, ymax;
    int n;
    std::vector<int> rlo, rhi;    // row dy = ymin + i covers dx in [rlo[i], rhi[i]]
    std::vector<int> ctop, cbot;  // column dx = xmin + j covers dy in [ctop[j], cbot[j]]
};

namespace fim {

// Host-side planning (fim_host.cu).
fim_status get_scratch(cudaStream_t stream, size_t bytes, unsigned char** out);
fim_status release_scratch();
int device_sm_count();
// exact_ranks: the plan's targets vary per pixel or per kernel, so its ordinal image must hold
// exact ranks (footprints up to 65535 pixels); otherwise larger footprints hold ranks relative to
// the feasible median ranks of `rank`.
fim_status make_plan(const fim_kernel* k, int dtype, int rank, int w, int h, const TileShape& ts, int smem_limit,
                     Plan* p, int cta_threads = 0, bool exact_ranks = false);
// Re-lays out a plan whose model is set so that the bracket MLP's parameters are staged in
// shared memory; keeps them in device memory (off_model = -1) when they do not fit.
fim_status plan_stage_model(Plan* p, int smem_limit);
// Tile shape for an image of w x h (w or h <= 0: a batch, which fills the GPU like a large image).
fim_status choose_tile(const fim_kernel* k, int dtype, int smem_limit, TileShape* ts, int w, int h,
                       int cta_threads = 0, bool exact_ranks = false);
int device_smem_limit();

// Autotuner cache (fim_tune.cu).
// Image-size classes of the autotuner cache: the best tile shape depends on how many tiles an
// image has against the SMs. 0: up to 1 Mpix, 1: up to 4 Mpix, 2: up to 16 Mpix, 3: larger (and
// batches, whose tiles of all jobs share one queue).
constexpr int kSizeClasses = 4;
inline int size_class(int w, int h) {
    if (w <= 0 || h <= 0) return kSizeClasses - 1;
    const long long px = (long long)w * h;
    return px <= (1ll << 20) ? 0 : (px <= (1ll << 22) ? 1 : (px <= (1ll << 24) ? 2 : 3));
}
bool tuned_lookup(const fim_kernel* k, int dtype, TileShape* ts, int size_cls, int cta_threads = 0);
void tuned_store(const fim_kernel* k, int dtype, const TileShape& ts, int size_cls, int cta_threads = 0);
void tuned_clear();
void tile_candidates(std::vector<TileShape>* out);

// Diagnostics: device buffer that receives per-phase clock64() stamps (may be null).
void set_phase_clock_buffer(unsigned long long* buf, int tiles);
void get_phase_clock_buffer(unsigned long long** buf, int* tiles);

// Encodes the tensor map of the plan's input image for the footprint copies when the plan has a
// staging region and the image allows them (16-byte aligned base and pitch); sets use_tma.
void attach_tma(Plan& p);
// Small images (w x h; 0 x 0: unknown, e.g. batches) whose tiles of the default shape `def`
// would fill under half the GPU's resident CTAs: the first of the smaller shapes (kernels up
// to 65 pixels across: 32x8 with 4 bands, 32x16 with 4, 32x8 with 2; larger kernels: 32x16 and
// 64x32 with 8 bands) whose tiles all fit in one wave of resident CTAs, in *out (true).
// `scratch` is storage for trial plans.
bool small_image_shape(const fim_kernel* k, int dtype, int w, int h, int smem_limit, int cta_threads,
                       bool exact_ranks, const TileShape& def, Plan* scratch, TileShape* out);

// Device launch (fim_tile.cu).
fim_status launch_tile_kernel(Plan& p, cudaStream_t stream);
fim_status read_and_clear_device_status(cudaStream_t stream);

// (fim_tile_k4.cu) the kernels with 4 omnigram groups per scan step, and their status word
fim_status launch_tile_kernel_k4(Plan& p, cudaStream_t stream);
fim_status launch_tile_kernel_fixed_k4(Plan& p, unsigned char* scratch, size_t capacity, cudaStream_t stream,
                                       bool launch);
fim_status read_and_clear_k4_status();
// (fim_tile_extras.cu) the kernels with the learned bracket, training rows and seed statistics
fim_status launch_tile_kernel_extras(Plan& p, cudaStream_t stream);
fim_status read_and_clear_extras_status();
fim_status launch_tile_kernel_map(Plan& p, cudaStream_t stream);
fim_status read_and_clear_map_status();
// Per-pixel target ranks of a percentile map (w x h floats, pitch in bytes) into `ranks`
// (w x h ints, dense rows), on `stream`.
fim_status launch_percentile_ranks(const float* pct, long long pct_pitch, int w, int h, int n, int* ranks,
                                   cudaStream_t stream);
// Launch on a fixed workspace; FIM_ERR_UNSUPPORTED when it needs more than `capacity` bytes. With
// `launch` false, only that check (FIM_OK: it fits).
fim_status launch_tile_kernel_fixed(Plan& p, unsigned char* scratch, size_t capacity, cudaStream_t stream,
                                    bool launch = true);
// Batch class kernels (fim_batch_k8.cu / fim_batch_k4.cu, by c.ks): with a == nullptr, the set-up
// of c's kernel (shared-memory opt-in) and its resident CTAs per SM in *occ; otherwise a launch of
// c.grid CTAs on `stream`.
fim_status batch_class_k8(const BatchClass& c, const BatchClassArgs* a, int* occ, cudaStream_t stream);
fim_status batch_class_k4(const BatchClass& c, const BatchClassArgs* a, int* occ, cudaStream_t stream);
fim_status read_and_clear_batch_k8_status();
fim_status read_and_clear_batch_k4_status();

}  // namespace fim
