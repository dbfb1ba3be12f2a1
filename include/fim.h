/*
 * fim.h - C ABI of libfim, an exact isotropic median / percentile filter for one GPU.
 *
 * The filter is the one of "Fast Isotropic Median Filtering" (arXiv 2505.22938):
 * out(x, y) is the value of 0-based rank k among the n values
 * in(clamp(x+dx, 0, w-1), clamp(y+dy, 0, h-1)) for (dx, dy) in a convex kernel K
 * (Sec. 3.1 pivot/count principle; Eq. 1-3 region membership; Sec. 3.3 method summary).
 * k = (n-1)/2 for the median. Border handling is clamp-to-edge. Output values are always
 * input values, so results are bit-exact for every dtype.
 *
 * Conventions for every call below:
 *   - Image pointers are DEVICE pointers unless the name says "host". The caller owns them.
 *     Rows are `pitch_bytes` apart; the same pitch applies to input and output. The
 *     pitch must be at least w * element size and a multiple of the element size.
 *     Input and output must not overlap (FIM_ERR_INVALID_ARG).
 *   - `stream` is a cudaStream_t passed as void* (NULL = the legacy default stream).
 *     Filter calls are asynchronous on it. Argument errors return synchronously;
 *     errors detected on the device are recorded in a status word that
 *     fim_sync_status() reads.
 *   - Float data is ordered by IEEE 754 totalOrder (-0 < +0). NaN inputs are ordered by
 *     their bit patterns under the same total order; the filter does no arithmetic on
 *     values, so denormals are never flushed.
 *   - Kernel handles are host objects owned by the caller (fim_destroy_kernel).
 *   - All entry points are thread-safe with respect to distinct handles.
 */
#ifndef FIM_H_
#define FIM_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum { FIM_U8 = 0, FIM_U16 = 1, FIM_F32 = 2 } fim_dtype;

typedef enum { FIM_BORDER_CLAMP = 0 } fim_border;

typedef enum {
    FIM_OK = 0,
    FIM_ERR_INVALID_ARG = 1, /* bad pointer, size, pitch, overlap or kernel shape */
    FIM_ERR_UNSUPPORTED = 2, /* valid request this build cannot serve (e.g. kernel too large) */
    FIM_ERR_OOM = 3,         /* device or host allocation failed */
    FIM_ERR_CUDA = 4,        /* a CUDA runtime call failed */
    FIM_ERR_TIMEOUT = 5,     /* a bounded device-side wait gave up (a footprint copy's mbarrier;
                                the output is still exact: the tile read the image instead) */
    FIM_ERR_INTERNAL = 6     /* a device-side consistency check failed */
} fim_status;

typedef struct fim_kernel fim_kernel;

/* Largest kernel extent along x or y (max - min + 1) this build accepts. */
#define FIM_MAX_KERNEL_EXTENT 257

/*
 * Disk kernel, Eq. 3 on the integer lattice: K = {(dx, dy) : dx^2 + dy^2 <= radius^2}.
 * radius in [0, 128]. *out receives a new handle.
 */
fim_status fim_create_kernel_circle(int radius, fim_kernel** out);

/*
 * Disk kernel with an explicit bound: K = {(dx, dy) : dx^2 + dy^2 <= limit}, limit >= 0
 * and floor(sqrt(limit)) <= 128. limit = r*r + r gives the fuller disk whose tap counts
 * match Fig. 3b and Fig. 10 of the paper (21 taps at r = 2).
 */
fim_status fim_create_kernel_disk_limit(int64_t limit, fim_kernel** out);

/*
 * Axis-aligned ellipse with semi-axes a (along x) and b (along y), both in [0, 128]:
 * K = {(dx, dy) : dx^2 b^2 + dy^2 a^2 <= a^2 b^2}, tested exactly in integers.
 */
fim_status fim_create_kernel_ellipse(int a, int b, fim_kernel** out);

/*
 * Convex polygon kernel (Sec. 6.2.3: a polygon replaces the circle test of Eq. 3).
 * xy holds nverts (x, y) pairs, counter-clockwise, in pixel units relative to the output
 * pixel; K is every lattice point inside or on the polygon (edge tolerance 1e-9).
 * Returns FIM_ERR_INVALID_ARG when the polygon is not convex and counter-clockwise or
 * holds no lattice point.
 */
fim_status fim_create_kernel_polygon(const double* xy, int nverts, fim_kernel** out);

/*
 * Kernel given by row spans: row dy0 + i covers dx in [lo[i], hi[i]], i < rows.
 * Every row must be non-empty and the shape must be convex along columns too (each column
 * a single run), else FIM_ERR_INVALID_ARG.
 */
fim_status fim_create_kernel_spans(const int* lo, const int* hi, int dy0, int rows, fim_kernel** out);

/* Tap count n and bounding box of a kernel. Any output pointer may be NULL. */
fim_status fim_kernel_info(const fim_kernel* k, int* ntaps, int* xmin, int* xmax, int* ymin, int* ymax);

/* Frees a handle (NULL is ignored). The caller must not destroy a kernel still in use by a
 * filter call that has not finished on its stream. */
void fim_destroy_kernel(fim_kernel* k);

/*
 * Median filter (Sec. 3.3 steps 1-7). in/out: device images of w x h elements of `dtype`,
 * rows pitch_bytes apart. w, h >= 1. Asynchronous on `stream`. The tile configuration is the
 * autotuned one for the kernel geometry and image-size class where fim_autotune ran, else a
 * default by kernel extent; images too small to fill the GPU with the default tiles take
 * smaller ones that fit in one wave of resident CTAs. Results do not depend on the tiling.
 */
fim_status fim_median(const void* in, void* out, int w, int h, size_t pitch_bytes, fim_dtype dtype,
                      const fim_kernel* k, fim_border border, void* stream);

/*
 * fim_median for callers that must not allocate device memory (no cudaMalloc, cudaFree or any
 * allocating library call on this path): work inside stream capture, services whose device
 * memory belongs to an external pool, real-time code that allocates only at start-up. The paper
 * has no counterpart; it is an API convenience of this library.
 * Same arguments and result as fim_median. Its workspace is one fixed array of
 * FIM_NOALLOC_WORKSPACE_BYTES of device memory inside the library, held by every GPU that loads
 * the library until the process exits. The first call on each device looks up the array's
 * address (cudaGetSymbolAddress) and keeps it for the life of the process; make that first call
 * before any stream capture. A cudaDeviceReset of that device invalidates the kept address: do
 * not call this entry point on the device again in the same process after one. Calls needing
 * more workspace than the array holds (large kernels on large images: the per-CTA buffers of
 * kernels whose footprint does not fit in shared memory) return FIM_ERR_UNSUPPORTED and launch
 * nothing. All calls share the array, so calls whose work overlaps on the GPU (different streams
 * without ordering) race: serialise them.
 */
#define FIM_NOALLOC_WORKSPACE_BYTES (16u << 20)
fim_status fim_median_noalloc(const void* in, void* out, int w, int h, size_t pitch_bytes, fim_dtype dtype,
                              const fim_kernel* k, fim_border border, void* stream);

/*
 * Percentile (rank-order) filter: the same method with target rank
 * rank = round(percentile / 100 * (n - 1)) instead of (n - 1) / 2 (Sec. 6.2.5, Fig. 12-14).
 * percentile in [0, 100].
 */
fim_status fim_percentile(const void* in, void* out, int w, int h, size_t pitch_bytes, fim_dtype dtype,
                          const fim_kernel* k, double percentile, fim_border border, void* stream);

/*
 * Several percentile filters of one image with one kernel, in one launch: each tile's ordinal
 * transform and ordinal image (the sort, Sec. 3.2) are built once and serve every target rank
 * (the seeds, slides and scans run once per rank). outs: `count` (1..8) device pointers, host
 * array, each an output image with the input's pitch; percentiles: `count` values in [0, 100],
 * rank = round(percentile / 100 * (n - 1)) as in fim_percentile. Same argument checks and
 * errors as fim_percentile (no output may overlap the input; outputs that overlap one
 * another race), plus FIM_ERR_INVALID_ARG for count outside 1..8. Asynchronous on `stream`.
 * Sec. 6.2 proposes this extension (several percentiles, e.g. quartiles, from one ordinal
 * transform); the paper's own implementation filters one percentile at a time.
 */
fim_status fim_percentiles(const void* in, void* const* outs, const double* percentiles, int count, int w, int h,
                           size_t pitch_bytes, fim_dtype dtype, const fim_kernel* k, fim_border border, void* stream);

/*
 * Median filters of one image with several disk kernels, in one launch: each tile's ordinal
 * transform and ordinal image are built once, for the footprint of the largest disk, and serve
 * every disk (its seeds, slides and scans run with its own tables and membership test over the
 * same omnigram). Sec. 6.2 proposes filtering several radii (its example: 8, 16, 32) from one
 * transform; the paper's own implementation filters one radius at a time.
 * kernels: `count` (1..8) handles made by fim_create_kernel_circle / _disk_limit (any other
 * shape: FIM_ERR_INVALID_ARG), host array; outs: `count` device pointers, host array, output q
 * receiving the median with kernels[q], each with the input's pitch. The tile shape is the one
 * the largest disk takes. Same argument checks and errors as fim_median for every (out, kernel)
 * pair, plus FIM_ERR_INVALID_ARG for count outside 1..8; outputs that overlap one another race.
 * Asynchronous on `stream`; the per-kernel tables go to stream-ordered device memory
 * (cudaMallocAsync) for the launch's duration.
 */
fim_status fim_median_radii(const void* in, void* const* outs, const fim_kernel* const* kernels, int count, int w,
                            int h, size_t pitch_bytes, fim_dtype dtype, fim_border border, void* stream);

/*
 * Spatially varying percentile (Fig. 14): every output pixel takes its own percentile from a
 * device float32 map. percentiles: w x h values, rows pct_pitch_bytes apart (>= 4 * w, a
 * multiple of 4); read only, owned by the caller, must not overlap the output and must stay
 * valid until the stream has run the call's work. Each value is
 * clamped to [0, 100] (NaN counts as 0) and rounded to a rank as in fim_percentile, in fp64:
 * floor(p / 100 * (n - 1) + 1/2). Slides carry the count at their pivot from one window's
 * rank to the next, so neighbouring pixels may differ by any amount. Same checks and errors
 * as fim_percentile, plus FIM_ERR_INVALID_ARG for a null map, a bad map pitch, or a map that
 * overlaps the output, and FIM_ERR_OOM when the w x h int32 rank image (stream-ordered
 * device memory, released on the stream after the filter) cannot be allocated. Asynchronous
 * on `stream`.
 */
fim_status fim_percentile_map(const void* in, void* out, const float* percentiles, size_t pct_pitch_bytes, int w,
                              int h, size_t pitch_bytes, fim_dtype dtype, const fim_kernel* k, fim_border border,
                              void* stream);

/*
 * fim_median with HOST buffers: copies the input to the device, filters, copies the result
 * back, and returns when the output is in `out_host`. Device buffers (and, for images of
 * several tile rows, three streams and their events) are allocated on first use and cached
 * per thread. The image is processed in up to 8 bands of whole tile rows: a band's input rows
 * (with the kernel's reach) are copied in, its tiles filtered and its rows copied out while
 * the next bands proceed, so the copies overlap the filtering; with pinned host buffers the
 * copies are asynchronous. The caller's stream waits for the whole pipeline before the call
 * returns. Rows are pitch_bytes apart in both host buffers.
 */
fim_status fim_median_host(const void* in_host, void* out_host, int w, int h, size_t pitch_bytes,
                           fim_dtype dtype, const fim_kernel* k, fim_border border, void* stream);

/*
 * Tunes the tile configuration for (current device, dtype, kernel geometry, image-size class):
 * every valid configuration is run on this image (in -> out, which ends up holding the filtered
 * image) and timed with CUDA events; the fastest is kept in a process-wide cache that later
 * fim_median, fim_percentile and related calls with the same dtype, kernel geometry and size
 * class use. Size classes: up to 1, 4 and 16 Mpix, and larger. Batches take the largest
 * class (the tiles of all their jobs share one queue, so they fill the GPU like a large image).
 * cta_threads = 0 tunes over all CTA sizes; 256, 512 or 1024 restricts the search to that CTA
 * size and stores the result separately, for callers that plan with a fixed CTA size.
 * If the environment variable FIM_TUNE_CACHE names a file, the cache is loaded from it on first
 * use and rewritten after each tuning. tile_w / tile_h (may be NULL) receive the chosen tile.
 * The choice depends on the image size (shapes tuned on a 512x512 crop slowed 4096x4096 images at
 * r = 8-48 by up to 30 %), hence the size classes.
 * Synchronous. Not part of the paper: its GPU tiling is fixed by radius (Sec. 4.2).
 */
fim_status fim_autotune(const void* in, void* out, int w, int h, size_t pitch_bytes, fim_dtype dtype,
                        const fim_kernel* k, int cta_threads, void* stream, int* tile_w, int* tile_h);

/* Forgets every tuned configuration of this process (the cache file is left alone). */
fim_status fim_autotune_clear(void);

/*
 * Batched persistent launch. One job is one 2-D image filtered with its own kernel, dtype, size
 * and pitch; percentile < 0 selects the median, otherwise the percentile filter of fim_percentile.
 * The jobs are grouped into classes by the pipeline they run (dtype, kernel shape, omnigram
 * encoding and home, scan width) and CTA size. Each class is one persistent kernel whose CTAs
 * take tiles from one device-side queue over the tiles of all the class's jobs (expensive tiles
 * first); a class of one job runs the single-image kernel on that job. The classes run side by
 * side on the batch's own streams, forked from and joined to the caller's. Not part of the paper.
 */
typedef struct {
    const void* in;      /* device pointer */
    void* out;           /* device pointer, must not overlap any input */
    int w, h;
    size_t pitch_bytes;  /* input and output */
    fim_dtype dtype;
    const fim_kernel* kernel;
    double percentile;   /* < 0: median */
} fim_job;

typedef struct fim_batch fim_batch;

/*
 * Plans a batch: validates every job, picks tile configurations (tuned ones when available),
 * uploads the per-job plans and allocates the batch's workspace. Synchronous. The images are
 * only referenced: they must stay valid while the batch runs. Every job runs in the same launch,
 * so an output may overlap neither another output nor any job's input (its own included):
 * FIM_ERR_INVALID_ARG. Several jobs may share one input.
 */
fim_status fim_batch_create(const fim_job* jobs, int count, fim_batch** out);

/* Runs a batch on `stream`: one memset of the class queue counters, then per class a kernel
 * launch on the caller's stream or one of the batch's streams (event fork and join): stream
 * operations and host-side launch set-up only, so a run can be captured into a CUDA graph.
 * Runs of one batch must not overlap in time. */
fim_status fim_batch_run(fim_batch* b, void* stream);

/* Size of a batch run: total queued tiles, CTAs over all class kernels, and the largest CTA
 * size and shared memory per CTA among them. */
fim_status fim_batch_info(const fim_batch* b, int* total_tiles, int* grid, int* threads, int* smem_bytes);

/* Waits for the device, then frees the batch (NULL is ignored). */
void fim_batch_destroy(fim_batch* b);

/* One-shot: fim_batch_create + fim_batch_run + wait for `stream` + fim_batch_destroy. */
fim_status fim_median_batch(const fim_job* jobs, int count, void* stream);

/*
 * Learned rank bracket for the seed windows (not part of the paper; the paper's seed windows are
 * solved from a low-precision histogram, Sec. 4.2). A small network predicts, from a seed
 * window's features, where its median rank lies; the filter counts the window's members below
 * both ends of the predicted bracket in one pass and scans the omnigram from the nearer end, so
 * a bad prediction only lengthens the scan: results stay bit-identical to fim_median.
 *
 * Network: 41 features (the tile footprint's 32 value quantiles, normalised by their median and
 * 1/8-7/8 spread, and the ranks / N of the 3x3 pixels around the window centre) -> 64 ReLU ->
 * 64 ReLU -> 2 outputs (mu: the median rank as a fraction of the tile's feasible median ranks;
 * s: log of its standard deviation). bf16 weights, fp32 accumulation. Parameters are one flat
 * fp32 vector of fim_model_param_count() values: W1[41][64], b1[64], W2[64][64], b2[64], W3[64][2],
 * b3[2] (row-major, input index first). Training rows are 42 floats: 41 features then the label.
 */
typedef struct fim_model fim_model;

/* Number of parameters of the network. */
int fim_model_param_count(void);

/* New model with He-uniform weights drawn from `seed`. */
fim_status fim_model_create(uint64_t seed, fim_model** out);

/* Frees a model (waits for the device first). NULL is ignored. */
void fim_model_destroy(fim_model* m);

/* Copies the fp32 master parameters and/or their bf16 rounding (as used by every forward
 * pass) to host arrays of fim_model_param_count() elements; either pointer may be NULL. */
fim_status fim_model_get_params(const fim_model* m, float* host_fp32, uint16_t* host_bf16);

/* Replaces the parameters (host fp32 array); the bf16 copy is re-rounded (nearest even). */
fim_status fim_model_set_params(fim_model* m, const float* host_fp32);

/* Bracket half-width in predicted standard deviations (set by fim_model_calibrate). */
float fim_model_bracket_z(const fim_model* m);

/* Forward pass: rows of features (device, row_stride floats apart) -> out[2*i] = mu,
 * out[2*i+1] = s (device). Synchronous. */
fim_status fim_model_forward(const fim_model* m, const float* x, int rows, int row_stride, float* out, void* stream);

/* Mean Gaussian negative log-likelihood 0.5 (y - mu)^2 / sigma^2 + log sigma (sigma = e^s, s
 * clamped to [-8, 2]) of the rows and its gradient with respect to the parameters (as used by
 * the forward pass) into grad_out (device, may be NULL); loss_out (host, may be NULL). */
fim_status fim_model_loss_grad(fim_model* m, const float* x, int rows, int row_stride, const float* y, int y_stride,
                               float* grad_out, float* loss_out, void* stream);

/* Trains on training rows (device) with Adam (beta 0.9 / 0.999), minibatches of `batch`
 * consecutive rows, for `epochs` passes. Synchronous; last_epoch_loss may be NULL. */
fim_status fim_model_train(fim_model* m, const float* rows_xy, int rows, int epochs, int batch, float lr,
                           void* stream, float* last_epoch_loss);

/* Sets the bracket half-width z so that |y - mu| <= z sigma holds for `coverage` of the given
 * rows (held-out training rows, device). */
fim_status fim_model_calibrate(fim_model* m, const float* rows_xy, int rows, double coverage, void* stream,
                               float* z_out);

/* Saves / loads parameters, bracket width and optimiser state (resumable training). */
fim_status fim_model_save(const fim_model* m, const char* path);
fim_status fim_model_load(const char* path, fim_model** out);

/*
 * Runs fim_median (in -> out) and appends one training row per seed window: its features and its
 * exact median rank as a fraction of the tile's feasible median ranks. rows_xy (device) holds
 * `capacity` rows; *count_dev (device counter, zeroed by the caller) is advanced by every seed,
 * even past the capacity (rows beyond it are not written).
 */
fim_status fim_collect_seed_samples(const void* in, void* out, int w, int h, size_t pitch_bytes, fim_dtype dtype,
                                    const fim_kernel* k, float* rows_xy, int capacity, unsigned int* count_dev,
                                    void* stream);

/*
 * fim_median with the learned seed bracket (model may be NULL: the plain seeds). If stats_dev is
 * not NULL (device, 5 counters the caller zeroes) the launch adds: seed windows, bracket hits,
 * misses below the bracket, misses above it, and omnigram ranks the seeds' scans walked.
 */
fim_status fim_median_learned(const void* in, void* out, int w, int h, size_t pitch_bytes, fim_dtype dtype,
                              const fim_kernel* k, const fim_model* m, fim_border border, void* stream,
                              unsigned long long* stats_dev);

/*
 * Waits for `stream`, then returns and clears the device status word: FIM_OK, or the
 * first device-side error recorded since the last call (FIM_ERR_TIMEOUT, FIM_ERR_INTERNAL).
 */
fim_status fim_sync_status(void* stream);

/*
 * Tiling the filter would use for this kernel, dtype and image size on the current device:
 * output tile tile_w x tile_h, footprint pixels per tile, threads per CTA, dynamic shared
 * memory per CTA. Any output pointer may be NULL. The environment variable
 * FIM_TILE="tile_w,tile_h,bands,seeds" overrides the choice (tile_w a power of two and a
 * multiple of 32; FIM_ERR_UNSUPPORTED if it does not fit the device).
 */
fim_status fim_plan_info(const fim_kernel* k, fim_dtype dtype, int w, int h, int* tile_w, int* tile_h,
                         int* footprint, int* threads, int* smem_bytes);

/*
 * The filter keeps one device workspace per (device, stream) it has run on: the tile queue
 * counter and, for kernels whose footprint does not fit in shared memory, per-CTA buffers.
 * It grows on demand and lives until this call, which waits for the device and frees it.
 */
fim_status fim_release_workspace(void);

/* Static, human-readable name of a status code. */
const char* fim_status_string(fim_status s);

/* Version of this library as "major.minor.patch". */
const char* fim_version(void);

/*
 * Diagnostics. Attaches a device buffer of tiles * 8 uint64 that every following filter
 * launch (from any thread) fills with clock64() stamps at its phase boundaries: load, sort,
 * structure build, seeds, seed rows, vertical sweeps (which also write the output), the end of
 * the first thread's own sweep, end of the tile; one row of 8 per tile
 * index below `tiles`. fim_debug_phase_clocks(NULL, 0) detaches it. The buffer stays owned
 * by the caller and must outlive the launches that use it.
 */
fim_status fim_debug_phase_clocks(void* dev_buf, int tiles);

#ifdef __cplusplus
}
#endif

#endif /* FIM_H_ */
