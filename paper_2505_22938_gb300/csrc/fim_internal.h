// Internal declarations shared by the host and device translation units of libfim.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>
#include <vector>

#include "fim.h"

namespace fim {

constexpr int kMaxExtent = 264;   // kernel rows / columns held in a plan (>= FIM_MAX_KERNEL_EXTENT)
constexpr int kMaxSide = 320;     // bounding-box rows of a tile footprint held in a plan
constexpr int kSortBins = 256;    // 8-bit radix digits
constexpr int kSeedBins = 256;    // coarse histogram bins of a seed solve

enum Shape : int { kShapeDisk = 0, kShapeSpans = 1 };

// Geometry of one tile configuration: output tile T x T, 2*T*RB threads.
// RB bands of T/RB rows; each band's middle row is a seed row with G seeds.
struct TileShape {
    int T;
    int RB;
    int G;
};

// Everything a tile kernel launch needs, passed by value as a __grid_constant__ parameter.
struct Plan {
    // image
    const void* in;
    void* out;
    long long pitch;  // bytes, input and output
    int w, h;
    int dtype;
    // tiling
    int T, RB, G, threads, nwarps;
    int S, SH;              // footprint bounding box (columns, rows)
    int tiles_x, tiles_y;
    // kernel
    int shape;
    int r2;                 // disk: dx^2 + dy^2 <= r2
    int xmin, xmax, ymin, ymax, nrows, ncols;
    int n;                  // taps
    int rank;               // target 0-based rank ((n-1)/2 for the median)
    // footprint
    int N;                  // pixels in the rounded-rectangle footprint
    int cx0, cy0;           // omnigram coordinates are stored as (u - cx0, v - cy0), int8 each
    unsigned div_magic;     // ceil(2^32 / S): v = umulhi(pos, magic) for pos < 2^16
    int hist_shift;         // seed histogram: bin = rank >> hist_shift
    // dynamic shared memory layout (byte offsets)
    int off_keys, off_a, off_b, off_h, off_spans, smem_bytes;
    int16_t fl[kMaxSide], fr[kMaxSide];   // footprint row v covers u in [fl[v], fr[v]]
    int vA[kMaxExtent], vB[kMaxExtent];   // per column j: top*S + dx, (bot+1)*S + dx
    int hL[kMaxExtent], hH[kMaxExtent];   // per row i: dy*S + lo, dy*S + hi + 1
    int spans[kMaxExtent];                // per row i: (lo & 0xffff) | (hi << 16)
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
fim_status make_plan(const fim_kernel* k, int dtype, int rank, int w, int h, const TileShape& ts, Plan* p);
fim_status choose_tile(const fim_kernel* k, int dtype, int smem_limit, TileShape* ts);
int device_smem_limit();

// Device launch (fim_tile.cu).
fim_status launch_tile_kernel(const Plan& p, cudaStream_t stream);
fim_status read_and_clear_device_status(cudaStream_t stream);

}  // namespace fim
