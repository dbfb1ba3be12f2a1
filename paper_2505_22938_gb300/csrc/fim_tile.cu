// Per-tile median kernel: one CTA filters one T x T output tile (Sec. 3.3, Sec. 4.2).
//
// Phases, separated by __syncthreads():
//   1. footprint load  - the rounded-rectangle footprint (Fig. 10) with clamp-to-edge reads,
//                        turned into order-preserving integer keys (Sec. 4.1 float key).
//   2. ordinal transform - stable LSD radix sort of {key, location} in shared memory
//                        (8-bit digits, warp match-based ranking); yields the omnigram
//                        Omega (Sec. 3.3) and the exact ordinal image I (Eq. 4).
//   3. seed solve      - RB*G seed windows, one warp each: coarse histogram of I over the
//                        window, then a ballot scan of Omega to the exact median (Sec. 4.2).
//   4. seed rows       - one warp per (seed, direction) slides the window left/right; lanes
//                        split the kernel rows and reduce the count change (Sec. 3.3 step 4).
//   5. vertical sweep  - one thread per (column, band, direction) slides its window up or
//                        down (Fig. 7); the warp then refines its 32 windows one at a time
//                        by ballot scans of Omega (Sec. 4.1 refinement, Eq. 2).
//   6. output          - out = C[m] through the omnigram: the input value at Omega[m].
// Pivots are exact previous medians (Huang's choice, Sec. 3.1): after each solve the count
// below the pivot is exactly the target rank, and a slide only adds the change.
#include <stdint.h>

#include "fim_internal.h"

namespace fim {

__device__ int g_status;  // first device-side error since the last fim_sync_status()

namespace {

constexpr unsigned kFull = 0xffffffffu;

template <int DT>
struct Traits;
template <>
struct Traits<FIM_U8> {
    using T = uint8_t;
    using K = uint8_t;
    static constexpr int kPasses = 1;
    __device__ static K key(T v) { return v; }
};
template <>
struct Traits<FIM_U16> {
    using T = uint16_t;
    using K = uint16_t;
    static constexpr int kPasses = 2;
    __device__ static K key(T v) { return v; }
};
template <>
struct Traits<FIM_F32> {
    using T = float;
    using K = uint32_t;
    static constexpr int kPasses = 4;
    // Sign-magnitude to unsigned order (Sec. 4.1): negative values have all bits flipped,
    // non-negative values only the sign bit, so unsigned comparison is IEEE totalOrder.
    __device__ static K key(T v) {
        const uint32_t b = __float_as_uint(v);
        return b ^ ((uint32_t)((int32_t)b >> 31) | 0x80000000u);
    }
};

__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}
__device__ __forceinline__ uint32_t lanemask_le() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_le;" : "=r"(m));
    return m;
}
__device__ __forceinline__ uint32_t lanemask_ge() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_ge;" : "=r"(m));
    return m;
}

__device__ __forceinline__ void set_status(int code) { atomicCAS(&g_status, 0, code); }

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return min(max(v, lo), hi); }

// Region membership of one omnigram entry (Eq. 2). The entry packs the location as two
// int8 coordinates relative to the footprint centre; (px, py) is the window centre in the
// same frame.
template <int SHAPE>
struct Member;

template <>
struct Member<kShapeDisk> {
    int r2;
    __device__ __forceinline__ bool operator()(uint32_t e, int px, int py) const {
        const int dx = (int)(int8_t)(e & 0xffu) - px;
        const int dy = (int)(int8_t)(e >> 8) - py;
        return dx * dx + dy * dy <= r2;   // Eq. 3 on the lattice
    }
};

template <>
struct Member<kShapeSpans> {
    const int* spans;  // shared memory, per kernel row: lo | hi << 16
    int ymin, nrows;
    __device__ __forceinline__ bool operator()(uint32_t e, int px, int py) const {
        const int i = (int)(int8_t)(e >> 8) - py - ymin;
        if ((unsigned)i >= (unsigned)nrows) return false;
        const int s = spans[i];
        const int dx = (int)(int8_t)(e & 0xffu) - px;
        return dx >= (int)(int16_t)(s & 0xffff) && dx <= (s >> 16);
    }
};

// Exact selection by ballot scans of the omnigram (Sec. 4.1, Sec. 4.2).
// Given a pivot rank p and c = #{window members with rank < p}, returns the rank m of the
// window element with window-rank `target`. All 32 lanes pass the same arguments and get
// the same result; -1 means the counts were inconsistent (never expected).
template <class M>
__device__ __forceinline__ int ballot_select(const uint16_t* __restrict__ om, int N, int p, int c, int target,
                                             int px, int py, const M& member) {
    const int lane = threadIdx.x & 31;
    if (c <= target) {  // the answer is at or above p
        int need = target - c + 1;
        for (int v0 = p; v0 < N; v0 += 32) {
            const int v = v0 + lane;
            const bool in = v < N && member(om[v], px, py);
            const uint32_t mask = __ballot_sync(kFull, in);
            const int cnt = __popc(mask);
            if (cnt >= need) {
                const uint32_t hit = __ballot_sync(kFull, in && __popc(mask & lanemask_le()) == need);
                return v0 + __ffs(hit) - 1;
            }
            need -= cnt;
        }
    } else {  // the answer is below p: walk down, the need-th member met is the answer
        int need = c - target;
        for (int v1 = p; v1 > 0; v1 -= 32) {
            const int v = v1 - 32 + lane;
            const bool in = v >= 0 && member(om[v], px, py);
            const uint32_t mask = __ballot_sync(kFull, in);
            const int cnt = __popc(mask);
            if (cnt >= need) {
                const uint32_t hit = __ballot_sync(kFull, in && __popc(mask & lanemask_ge()) == need);
                return v1 - 32 + __ffs(hit) - 1;
            }
            need -= cnt;
        }
    }
    return -1;
}

template <int DT, int SHAPE>
__global__ void __launch_bounds__(1024, 1) tile_median_kernel(const __grid_constant__ Plan P) {
    using TR = Traits<DT>;
    using V = typename TR::T;
    using K = typename TR::K;
    extern __shared__ __align__(16) unsigned char smem[];

    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int warp = tid >> 5;
    const int nthreads = P.threads;
    const int nwarps = P.nwarps;
    const int S = P.S, SH = P.SH, N = P.N, T = P.T;
    const int tile = blockIdx.x;
    const int tx0 = (tile % P.tiles_x) * T;
    const int ty0 = (tile / P.tiles_x) * T;
    const int gx0 = tx0 + P.xmin;  // global coordinates of bounding-box pixel (0, 0)
    const int gy0 = ty0 + P.ymin;

    K* keys = reinterpret_cast<K*>(smem + P.off_keys);
    uint16_t* ord = reinterpret_cast<uint16_t*>(smem + P.off_keys);  // ordinal image, after the sort
    uint16_t* bufA = reinterpret_cast<uint16_t*>(smem + P.off_a);
    uint16_t* bufB = reinterpret_cast<uint16_t*>(smem + P.off_b);
    uint32_t* hist = reinterpret_cast<uint32_t*>(smem + P.off_h);
    int* spans = reinterpret_cast<int*>(smem + P.off_spans);

    // ---- 1. footprint load (clamp-to-edge), as order-preserving keys ------------------------
    const char* in = static_cast<const char*>(P.in);
    for (int v = warp; v < SH; v += nwarps) {
        const int gy = clampi(gy0 + v, 0, P.h - 1);
        const V* row = reinterpret_cast<const V*>(in + (long long)gy * P.pitch);
        const int lo = P.fl[v], hi = P.fr[v];
        for (int u = lo + lane; u <= hi; u += 32) {
            const int gx = clampi(gx0 + u, 0, P.w - 1);
            keys[v * S + u] = TR::key(__ldg(row + gx));
        }
    }
    for (int i = tid; i < P.nrows; i += nthreads) spans[i] = P.spans[i];
    __syncthreads();

    // ---- 2. ordinal transform: stable LSD radix sort of bounding-box positions by key ----------
    // Pass 0 enumerates the bounding box row-major and skips non-footprint positions, so ties
    // keep row-major order. Each warp owns one contiguous segment of the current order; ranks
    // are (digit, warp)-major exclusive offsets plus the position among equal digits.
    const int area = S * SH;
    const uint16_t* src = nullptr;
    uint16_t* dst = bufA;
    for (int pass = 0; pass < TR::kPasses; ++pass) {
        const int shift = 8 * pass;
        const int len = pass == 0 ? area : N;
        const int seg = ((len + nwarps - 1) / nwarps + 31) & ~31;
        const int s0 = min(len, warp * seg), s1 = min(len, s0 + seg);
        for (int d = lane; d < kSortBins; d += 32) hist[d * nwarps + warp] = 0;
        __syncwarp();
        for (int b = s0; b < s1; b += 32) {
            const int i = b + lane;
            bool valid = i < s1;
            int pos = 0;
            if (valid) {
                if (pass == 0) {
                    const int v = (int)__umulhi((unsigned)i, P.div_magic);
                    const int u = i - v * S;
                    valid = u >= P.fl[v] && u <= P.fr[v];
                    pos = i;
                } else {
                    pos = src[i];
                }
            }
            const int d = valid ? (int)((uint32_t)keys[pos] >> shift) & 0xff : kSortBins + lane;
            const uint32_t peers = __match_any_sync(kFull, d);
            if (valid && lane == __ffs(peers) - 1) atomicAdd(&hist[d * nwarps + warp], (uint32_t)__popc(peers));
        }
        __syncthreads();
        {   // exclusive scan of the (digit, warp) counters, in place
            const int total = kSortBins * nwarps;
            const int per = total / nthreads;  // 8 with 1024 threads, 16 with 512
            uint32_t* h = hist + tid * per;
            uint32_t local = 0;
            for (int j = 0; j < per; ++j) local += h[j];
            uint32_t incl = local;
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t t = __shfl_up_sync(kFull, incl, o);
                if (lane >= o) incl += t;
            }
            __shared__ uint32_t wsum[32];
            if (lane == 31) wsum[warp] = incl;
            __syncthreads();
            if (warp == 0) {
                uint32_t x = lane < nwarps ? wsum[lane] : 0;
                for (int o = 1; o < 32; o <<= 1) {
                    const uint32_t t = __shfl_up_sync(kFull, x, o);
                    if (lane >= o) x += t;
                }
                wsum[lane] = x;
            }
            __syncthreads();
            uint32_t run = incl - local + (warp > 0 ? wsum[warp - 1] : 0);
            for (int j = 0; j < per; ++j) {
                const uint32_t c = h[j];
                h[j] = run;
                run += c;
            }
        }
        __syncthreads();
        for (int b = s0; b < s1; b += 32) {
            const int i = b + lane;
            bool valid = i < s1;
            int pos = 0;
            if (valid) {
                if (pass == 0) {
                    const int v = (int)__umulhi((unsigned)i, P.div_magic);
                    const int u = i - v * S;
                    valid = u >= P.fl[v] && u <= P.fr[v];
                    pos = i;
                } else {
                    pos = src[i];
                }
            }
            const int d = valid ? (int)((uint32_t)keys[pos] >> shift) & 0xff : kSortBins + lane;
            const uint32_t peers = __match_any_sync(kFull, d);
            uint32_t base = 0;
            if (valid) base = hist[d * nwarps + warp];
            __syncwarp();
            if (valid) {
                dst[base + __popc(peers & lanemask_lt())] = (uint16_t)pos;
                if (lane == __ffs(peers) - 1) hist[d * nwarps + warp] = base + __popc(peers);
            }
            __syncwarp();
        }
        __syncthreads();
        src = dst;
        dst = (dst == bufA) ? bufB : bufA;
    }

    // ---- build the ordinal image I (Eq. 4) and the omnigram Omega ------------------------------
    const uint16_t* sorted = src;            // bounding-box positions in ascending key order
    uint16_t* om = dst;                      // the other buffer receives Omega
    for (int v = tid; v < N; v += nthreads) {
        const int pos = sorted[v];
        const int y = (int)__umulhi((unsigned)pos, P.div_magic);
        const int x = pos - y * S;
        om[v] = (uint16_t)(((uint32_t)(uint8_t)(int8_t)(x - P.cx0)) | ((uint32_t)(uint8_t)(int8_t)(y - P.cy0) << 8));
    }
    __syncthreads();  // keys are dead from here on; I overwrites them
    for (int v = tid; v < N; v += nthreads) ord[sorted[v]] = (uint16_t)v;
    uint16_t* med = reinterpret_cast<uint16_t*>(hist);  // T x T exact median ranks
    uint32_t* shist = hist + ((T * T * 2 + 15) & ~15) / 4;  // per-warp seed histograms
    __syncthreads();

    Member<SHAPE> member;
    if constexpr (SHAPE == kShapeDisk) {
        member.r2 = P.r2;
    } else {
        member.spans = spans;
        member.ymin = P.ymin;
        member.nrows = P.nrows;
    }
    const int target = P.rank;
    const int BH = T / P.RB;       // band height
    const int GW = T / P.G;        // seed spacing within a seed row

    // ---- 3. seeds: coarse histogram of I over the window, then ballot refine ----------------
    for (int sd = warp; sd < P.RB * P.G; sd += nwarps) {
        const int band = sd / P.G, g = sd % P.G;
        const int s = g * GW + GW / 2, t = band * BH + BH / 2;  // tile-local output pixel
        const int cu = s - P.xmin, cv = t - P.ymin;             // window centre in the box
        uint32_t* hw = shist + warp * kSeedBins;
        for (int j = lane; j < kSeedBins; j += 32) hw[j] = 0;
        __syncwarp();
        for (int i = 0; i < P.nrows; ++i) {
            const int dy = P.ymin + i;
            const int sp = spans[i];
            const int lo = (int)(int16_t)(sp & 0xffff), hi = sp >> 16;
            const uint16_t* row = ord + (cv + dy) * S + cu;
            for (int dx = lo + lane; dx <= hi; dx += 32) atomicAdd(&hw[row[dx] >> P.hist_shift], 1u);
        }
        __syncwarp();
        uint32_t local = 0;
        for (int j = 0; j < kSeedBins / 32; ++j) local += hw[lane * (kSeedBins / 32) + j];
        uint32_t incl = local;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t tt = __shfl_up_sync(kFull, incl, o);
            if (lane >= o) incl += tt;
        }
        const uint32_t excl = incl - local;
        const bool mine = (int)excl <= target && target < (int)incl;
        const uint32_t who = __ballot_sync(kFull, mine);
        int bin = 0, below = 0;
        if (mine) {
            uint32_t run = excl;
            int j = 0;
            for (; j < kSeedBins / 32 - 1; ++j) {
                const uint32_t c = hw[lane * (kSeedBins / 32) + j];
                if ((int)(run + c) > target) break;
                run += c;
            }
            bin = lane * (kSeedBins / 32) + j;
            below = (int)run;
        }
        const int src_lane = __ffs(who) - 1;
        bin = __shfl_sync(kFull, bin, src_lane);
        below = __shfl_sync(kFull, below, src_lane);
        const int m = ballot_select(om, N, bin << P.hist_shift, below, target, cu - P.cx0, cv - P.cy0, member);
        if (m < 0) set_status(FIM_ERR_INTERNAL);
        if (lane == 0) med[t * T + s] = (uint16_t)max(m, 0);
        __syncwarp();
    }
    __syncthreads();

    // ---- 4. seed rows: horizontal slides, lanes split the kernel rows ----------------------
    for (int job = warp; job < 2 * P.RB * P.G; job += nwarps) {
        const int sd = job >> 1, right = job & 1;
        const int band = sd / P.G, g = sd % P.G;
        int s = g * GW + GW / 2;
        const int t = band * BH + BH / 2;
        const int steps = right ? (GW - GW / 2 - 1) : (GW / 2);
        int cu = s - P.xmin;
        const int cv = t - P.ymin;
        int p = med[t * T + s];
        for (int k = 0; k < steps; ++k) {
            const uint16_t* ctr = ord + cv * S + cu;
            int d = 0;
            for (int i = lane; i < P.nrows; i += 32) {
                const int e = right ? P.hH[i] : P.hL[i] - 1;
                const int l = right ? P.hL[i] : P.hH[i] - 1;
                d += (int)(ctr[e] < p) - (int)(ctr[l] < p);
            }
            d = __reduce_add_sync(kFull, d);
            cu += right ? 1 : -1;
            s += right ? 1 : -1;
            const int m = ballot_select(om, N, p, target + d, target, cu - P.cx0, cv - P.cy0, member);
            if (m < 0) set_status(FIM_ERR_INTERNAL);
            p = max(m, 0);
            if (lane == 0) med[t * T + s] = (uint16_t)p;
        }
    }
    __syncthreads();

    // ---- 5. vertical sweeps: thread per window column, warp-cooperative refinement ----------
    {
        const int groups = T / 32;
        const int cg = warp % groups;
        const int rest = warp / groups;
        const int band = rest % P.RB;
        const int down = rest / P.RB;  // 0: up, 1: down
        const int s = cg * 32 + lane;
        int t = band * BH + BH / 2;
        const int steps = down ? (BH - BH / 2 - 1) : (BH / 2);
        const int cu = s - P.xmin;
        int cv = t - P.ymin;
        int p = med[t * T + s];
        const int ncols = P.ncols;
        for (int k = 0; k < steps; ++k) {
            const uint16_t* ctr = ord + cv * S + cu;
            int d = 0;
            if (down) {
                for (int j = 0; j < ncols; ++j) d += (int)(ctr[P.vB[j]] < p) - (int)(ctr[P.vA[j]] < p);
            } else {
                for (int j = 0; j < ncols; ++j) d += (int)(ctr[P.vA[j] - S] < p) - (int)(ctr[P.vB[j] - S] < p);
            }
            cv += down ? 1 : -1;
            t += down ? 1 : -1;
            const int c = target + d;
            int mine = 0;
            for (int j = 0; j < 32; ++j) {
                const int pj = __shfl_sync(kFull, p, j);
                const int cj = __shfl_sync(kFull, c, j);
                const int m = ballot_select(om, N, pj, cj, target, cu - lane + j - P.cx0, cv - P.cy0, member);
                if (lane == j) mine = m;
            }
            if (mine < 0) set_status(FIM_ERR_INTERNAL);
            p = max(mine, 0);
            med[t * T + s] = (uint16_t)p;
        }
    }
    __syncthreads();

    // ---- 6. output: the input value at Omega[m] ------------------------------------------------
    char* out = static_cast<char*>(P.out);
    for (int idx = tid; idx < T * T; idx += nthreads) {
        const int t = idx / T, s = idx - t * T;
        const int gx = tx0 + s, gy = ty0 + t;
        if (gx >= P.w || gy >= P.h) continue;
        const uint32_t e = om[med[idx]];
        const int u = (int)(int8_t)(e & 0xffu) + P.cx0;
        const int v = (int)(int8_t)(e >> 8) + P.cy0;
        const int sx = clampi(gx0 + u, 0, P.w - 1), sy = clampi(gy0 + v, 0, P.h - 1);
        const V val = reinterpret_cast<const V*>(in + (long long)sy * P.pitch)[sx];
        reinterpret_cast<V*>(out + (long long)gy * P.pitch)[gx] = val;
    }
}

template <int DT, int SHAPE>
fim_status launch_typed(const Plan& p, cudaStream_t stream) {
    auto fn = tile_median_kernel<DT, SHAPE>;
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, p.smem_bytes) != cudaSuccess) {
        cudaGetLastError();
        return FIM_ERR_CUDA;
    }
    const long long tiles = (long long)p.tiles_x * p.tiles_y;
    if (tiles > 0x7fffffffLL) return FIM_ERR_UNSUPPORTED;
    fn<<<(unsigned)tiles, p.threads, p.smem_bytes, stream>>>(p);
    if (cudaGetLastError() != cudaSuccess) return FIM_ERR_CUDA;
    return FIM_OK;
}

}  // namespace

fim_status launch_tile_kernel(const Plan& p, cudaStream_t stream) {
    const bool disk = p.shape == kShapeDisk;
    switch (p.dtype) {
        case FIM_U8: return disk ? launch_typed<FIM_U8, kShapeDisk>(p, stream) : launch_typed<FIM_U8, kShapeSpans>(p, stream);
        case FIM_U16: return disk ? launch_typed<FIM_U16, kShapeDisk>(p, stream) : launch_typed<FIM_U16, kShapeSpans>(p, stream);
        case FIM_F32: return disk ? launch_typed<FIM_F32, kShapeDisk>(p, stream) : launch_typed<FIM_F32, kShapeSpans>(p, stream);
    }
    return FIM_ERR_INVALID_ARG;
}

fim_status read_and_clear_device_status(cudaStream_t stream) {
    int v = 0;
    if (cudaStreamSynchronize(stream) != cudaSuccess) return FIM_ERR_CUDA;
    if (cudaMemcpyFromSymbol(&v, g_status, sizeof(int)) != cudaSuccess) return FIM_ERR_CUDA;
    const int zero = 0;
    if (v != 0 && cudaMemcpyToSymbol(g_status, &zero, sizeof(int)) != cudaSuccess) return FIM_ERR_CUDA;
    return (fim_status)v;
}

}  // namespace fim
