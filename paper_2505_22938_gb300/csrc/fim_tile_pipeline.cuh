#pragma once
// The tile pipeline: one Tx x Ty output tile filtered by one tile group (a CTA, or part of a
// batch CTA) (Sec. 3.3, Sec. 4.2). The single-image and batch kernels include this file.
//
// Phases of one tile, separated by group barriers:
//   1. ordinal transform - the rounded-rectangle footprint (Fig. 10) is read with clamp-to-edge
//                        and key-value sorted by value, giving the omnigram Omega (Sec. 3.3):
//                          8-bit, and 16-bit data in 1024-thread CTAs: counting sort over 256 /
//                                         65536 shared-memory bins, the bucket construction of
//                                         Eq. 5 run by all threads;
//                          float, and 16-bit data in smaller CTAs: LSD radix sort of
//                                         order-preserving keys (Sec. 4.1 float key), 8-bit
//                                         passes (four / two).
//   2. ordinal image   - I(Omega[v]) = v (Eq. 4), exact 16-bit ranks.
//   3. seed solve      - RB*G seed windows, one warp each: coarse histogram of I over the
//                        window, then a ballot scan of Omega to the exact median (Sec. 4.2).
//                        With a learned bracket (an extension), a block-wide MLP proposes a
//                        rank bracket per seed and exact counts at its ends replace the histogram.
//   4. seed rows       - one warp per (seed, direction) slides the window left/right; lanes
//                        split the kernel rows and reduce the count change (Sec. 3.3 step 4).
//   5. vertical sweep  - one thread per (column, band, direction) slides its window up or
//                        down (Fig. 7) and refines it by scanning Omega itself, K 128-bit
//                        groups per step; the last few lanes of a warp hand their long scans to
//                        warp ballots (Sec. 4.1, Eq. 2).
//   6. output          - out = C[m] through the omnigram: the input value at Omega[m].
// Pivots are exact previous medians (Huang's choice, Sec. 3.1): after each solve the count
// below the pivot is exactly the target rank, and a slide only adds the change.
//
// W selects the omnigram encoding: W = 0 packs a location as two int8 coordinates (footprint
// box up to 256 x 256 with one side below 256, Sec. 4.1; -128 marks padding); W = 1 uses two
// int16 coordinates. OG = 1 keeps the omnigram in the CTA's global scratch slice when shared
// memory cannot hold it.
#include <stdint.h>

#include <algorithm>
#include <type_traits>

#include "fim_internal.h"

namespace fim {
namespace {

// First device-side error since the last fim_sync_status(). Each translation unit that includes
// this file has its own word (internal linkage); the host reads and clears all of them.
__device__ int g_status;

constexpr unsigned kFull = 0xffffffffu;

template <int DT>
struct Traits;
template <>
struct Traits<FIM_U8> {
    using T = uint8_t;
    __device__ static uint32_t key(T v) { return v; }
};
template <>
struct Traits<FIM_U16> {
    using T = uint16_t;
    __device__ static uint32_t key(T v) { return v; }
};
template <>
struct Traits<FIM_F32> {
    using T = float;
    // Sign-magnitude to unsigned order (Sec. 4.1): negative values have all bits flipped,
    // non-negative values only the sign bit, so unsigned comparison is IEEE totalOrder.
    __device__ static uint32_t key(T v) {
        const uint32_t b = __float_as_uint(v);
        return b ^ ((uint32_t)((int32_t)b >> 31) | 0x80000000u);
    }
};

// Omnigram entry encodings (locations relative to the footprint box centre cx0, cy0).
template <int W>
struct Loc;
template <>
struct Loc<0> {
    using E = uint16_t;    // entry
    using Pos = uint16_t;  // bounding-box position in the radix lists
    static constexpr int kGroup = 8;  // entries per 128-bit load
    static constexpr E kSentinel = 0x8080;  // (-128, -128): a box side below 256 keeps it out of every window
    __device__ static E pack(int u, int v, int cx0, int cy0) {
        return (E)((uint32_t)(uint8_t)(int8_t)(u - cx0) | ((uint32_t)(uint8_t)(int8_t)(v - cy0) << 8));
    }
    __device__ static int x(uint32_t e) { return (int)(int8_t)(e & 0xffu); }
    __device__ static int y(uint32_t e) { return (int)(int8_t)((e >> 8) & 0xffu); }
};
template <>
struct Loc<1> {
    using E = uint32_t;
    using Pos = uint32_t;
    static constexpr int kGroup = 4;
    static constexpr E kSentinel = 0xC000C000u;  // (-16384, -16384): far outside every window
    __device__ static E pack(int u, int v, int cx0, int cy0) {
        return (E)((uint32_t)(uint16_t)(int16_t)(u - cx0) | ((uint32_t)(uint16_t)(int16_t)(v - cy0) << 16));
    }
    __device__ static int x(uint32_t e) { return (int)(int16_t)(e & 0xffffu); }
    __device__ static int y(uint32_t e) { return (int)(int16_t)(e >> 16); }
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

// This translation unit's device status word, read and cleared by the host.
inline fim_status read_and_clear_unit_status() {
    int v = 0;
    if (cudaMemcpyFromSymbol(&v, g_status, sizeof(int)) != cudaSuccess) return FIM_ERR_CUDA;
    const int zero = 0;
    if (v != 0 && cudaMemcpyToSymbol(g_status, &zero, sizeof(int)) != cudaSuccess) return FIM_ERR_CUDA;
    return (fim_status)v;
}

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return min(max(v, lo), hi); }

// A tile group: the threads that run one tile's pipeline. A CTA holds one group (single-image
// launches) or several equal groups (batches of small configurations), each with its own
// named barrier and its own partition of shared memory (everything after the kernel tables).
struct Grp {
    int tid, lane, warp;  // group-local indices
    int nthreads;         // group size (the plan's CTA size)
    int bar;              // named barrier; 0 is the whole CTA
    int shift;            // byte shift of this group's shared-memory partition
    __device__ __forceinline__ void sync() const {
        if (bar == 0)
            __syncthreads();
        else
            asm volatile("bar.sync %0, %1;" ::"r"(bar), "r"(nthreads) : "memory");
    }
};

// Diagnostics: thread 0 records clock64() at phase boundaries when a buffer is attached. The
// stamps collect in the group's scan scratch (words 48..63, which no phase uses) and go to the
// buffer together at the end of the tile, so that no stamp waits behind the tile's own global
// stores.
__device__ __forceinline__ void stamp(const Plan& P, int tile, int phase, const Grp& G) {
    if (P.phase_clock != nullptr && G.tid == 0 && tile < P.phase_tiles) {
        extern __shared__ __align__(16) unsigned char smem_base[];
        unsigned long long* st = reinterpret_cast<unsigned long long*>(smem_base + G.shift + P.off_misc + 48 * 4);
        st[phase] = clock64();
        if (phase == 7)
            for (int i = 0; i < 8; ++i) P.phase_clock[tile * 8 + i] = st[i];
    }
}

__device__ __forceinline__ int span_lo(int s) { return (int)(int16_t)(s & 0xffff); }
__device__ __forceinline__ int span_hi(int s) { return s >> 16; }

// Region membership of one omnigram entry (Eq. 2); (px, py) is the window centre in the
// entry's coordinate frame.
template <int SHAPE, int W>
struct Member;

template <int W>
struct Member<kShapeDisk, W> {
    int r2;
    __device__ __forceinline__ bool operator()(uint32_t e, int px, int py) const {
        const int dx = Loc<W>::x(e) - px;
        const int dy = Loc<W>::y(e) - py;
        return dx * dx + dy * dy <= r2;   // Eq. 3 on the lattice
    }
};

template <int W>
struct Member<kShapeSpans, W> {
    const int* spans;  // shared memory, per kernel row: lo | hi << 16
    int ymin, nrows;
    __device__ __forceinline__ bool operator()(uint32_t e, int px, int py) const {
        const int i = Loc<W>::y(e) - py - ymin;
        if ((unsigned)i >= (unsigned)nrows) return false;
        const int s = spans[i];
        const int dx = Loc<W>::x(e) - px;
        return dx >= span_lo(s) && dx <= span_hi(s);
    }
};

// Membership of the omnigram entries held in one 32-bit word, for a fixed window: bit k is
// entry k of the word (two 16-bit entries, or one 32-bit entry).
template <int SHAPE, int W>
struct WordTest {
    Member<SHAPE, W> m;
    int px, py;
    __device__ __forceinline__ void init(const Member<SHAPE, W>& mm, int x, int y) {
        m = mm;
        px = x;
        py = y;
    }
    __device__ __forceinline__ uint32_t operator()(uint32_t w) const {
        if constexpr (W == 0)
            return (uint32_t)m(w & 0xffffu, px, py) | ((uint32_t)m(w >> 16, px, py) << 1);
        else
            return (uint32_t)m(w, px, py);
    }
};

// Disk with 8-bit coordinates: (x-px)^2 + (y-py)^2 <= r2 is evaluated as
// x^2 + y^2 - 2(x px + y py) <= r2 - px^2 - py^2 with byte dot products on the packed pair.
template <>
struct WordTest<kShapeDisk, 0> {
    int R;
    int plo, phi;  // (px, py, 0, 0) and (0, 0, px, py) as signed bytes
    __device__ __forceinline__ void init(const Member<kShapeDisk, 0>& mm, int px, int py) {
        R = mm.r2 - px * px - py * py;
        const uint32_t b = (uint32_t)(px & 0xff) | ((uint32_t)(py & 0xff) << 8);
        plo = (int)b;
        phi = (int)(b << 16);
    }
    __device__ __forceinline__ uint32_t operator()(uint32_t w) const {
        const int sq = __dp4a((int)w, (int)w, 0);
        const int sq0 = __dp4a((int)(w & 0xffffu), (int)w, 0);
        const int t0 = sq0 - 2 * __dp4a((int)w, plo, 0);
        const int t1 = (sq - sq0) - 2 * __dp4a((int)w, phi, 0);
        return (uint32_t)(t0 <= R) | ((uint32_t)(t1 <= R) << 1);
    }
};

// Exact selection by ballot scans of the omnigram (Sec. 4.1, Sec. 4.2).
// Given a pivot rank p and c = #{window members with rank < p}, returns the rank m of the
// window element with window-rank `target`. All 32 lanes pass the same arguments and get
// the same result; -1 means the counts were inconsistent (never expected).
template <class E, class M>
__device__ __forceinline__ int ballot_select(const E* __restrict__ om, int N, int p, int c, int target, int px,
                                             int py, const M& member) {
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

// Warp-cooperative exact selection for long walks (seed windows): the same contract as
// ballot_select, but every lane tests two consecutive aligned 128-bit groups of entries per
// step, so a warp covers 64 groups (512 entries of 16 bits) per step. A warp reduction of the
// per-lane member counts says whether the step holds the target; only that last step takes the
// warp prefix sum that finds the lane, and the lane picks the entry. Entries past N up to the
// last group are sentinels, never members; groups outside the omnigram count nothing. The loop is
// bounded by the omnigram length.
template <int SHAPE, int W>
__device__ __forceinline__ int wide_select(const typename Loc<W>::E* __restrict__ om, int N, int p, int c,
                                           int target, int px, int py, const Member<SHAPE, W>& member) {
    constexpr int G = Loc<W>::kGroup;
    constexpr int kShift = G == 8 ? 3 : 2;
    constexpr int kb = G / 4;  // entries per 32-bit word
    constexpr uint32_t kAll = (1u << G) - 1;
    const int lane = threadIdx.x & 31;
    WordTest<SHAPE, W> wt;
    wt.init(member, px, py);
    const uint4* om128 = reinterpret_cast<const uint4*>(om);
    const bool up = c <= target;
    int need = up ? target - c + 1 : c - target;
    const int v0 = up ? p : p - 1;  // first entry to examine
    const int glast = (N - 1) >> kShift;
    const int g0 = v0 >> kShift;    // -1 below entry 0
    const int o0 = v0 & (G - 1);
    const uint32_t first = up ? (kAll << o0) & kAll : kAll >> (G - 1 - o0);
    auto test = [&](int g) -> uint32_t {
        if ((unsigned)g > (unsigned)glast) return 0u;
        const uint4 q = om128[g];
        return wt(q.x) | (wt(q.y) << kb) | (wt(q.z) << (2 * kb)) | (wt(q.w) << (3 * kb));
    };
    for (int it = 0; it * 64 <= glast + 1; ++it) {
        // this lane's two groups, in walking order
        const int ga = up ? g0 + 64 * it + 2 * lane : g0 - 64 * it - 2 * lane;
        const int gb = up ? ga + 1 : ga - 1;
        uint32_t ma = test(ga);
        const uint32_t mb = test(gb);
        if (it == 0 && lane == 0) ma &= first;
        const int cnt = __popc(ma) + __popc(mb);
        const int total = (int)__reduce_add_sync(kFull, (unsigned)cnt);
        if (total >= need) {
            int incl = cnt;
            for (int o = 1; o < 32; o <<= 1) {
                const int t = __shfl_up_sync(kFull, incl, o);
                if (lane >= o) incl += t;
            }
            const uint32_t hit = __ballot_sync(kFull, incl >= need);
            const int j = __ffs(hit) - 1;
            int m = 0;
            if (lane == j) {
                int k = need - (incl - cnt);  // the k-th member of this lane's groups, along the walk
                const int ca = __popc(ma);
                const int g = k <= ca ? ga : gb;
                uint32_t mask = k <= ca ? ma : mb;
                if (k > ca) k -= ca;
                if (up) {
                    for (; k > 1; --k) mask &= mask - 1;
                    m = G * g + __ffs(mask) - 1;
                } else {
                    for (; k > 1; --k) mask ^= 1u << (31 - __clz(mask));
                    m = G * g + 31 - __clz(mask);
                }
            }
            return __shfl_sync(kFull, m, j);
        }
        need -= total;
        if (up ? g0 + 64 * (it + 1) > glast : g0 - 64 * (it + 1) < 0) break;
    }
    return -1;
}

// Members of a window below rank `p` (every lane gets the warp's total). Lane l takes kernel rows
// l, l + 32, ... and reads each row segment of the ordinal image in aligned 8-rank chunks (one
// 128-bit load each), comparing the ranks two per 32-bit word; only a row's first and last chunks
// need a mask. `ctr` is the window centre's ordinal-image position shifted by the kernel's first
// row (ymin) rows, as in window_walk; the image is 16-byte aligned.
__device__ __forceinline__ int window_rows_below(const int* spans, int nrows, const uint16_t* ctr, int SP, int p) {
    const int lane = threadIdx.x & 31;
    const uint32_t up = (uint32_t)p;
    int c = 0;
    for (int i = lane; i < nrows; i += 32) {
        const int sp = spans[i];
        const uint16_t* lo = ctr + i * SP + span_lo(sp);
        const uint16_t* hi = ctr + i * SP + span_hi(sp);
        const uint4* q = reinterpret_cast<const uint4*>((uintptr_t)lo & ~(uintptr_t)15);
        const uint4* qe = reinterpret_cast<const uint4*>((uintptr_t)hi & ~(uintptr_t)15);
        for (; q <= qe; ++q) {
            const uint4 v = *q;
            const uint32_t w[4] = {v.x, v.y, v.z, v.w};
            const uint16_t* e0 = reinterpret_cast<const uint16_t*>(q);
            if (e0 >= lo && e0 + 7 <= hi) {
#pragma unroll
                for (int j = 0; j < 4; ++j) c += (int)((w[j] & 0xffffu) < up) + (int)((w[j] >> 16) < up);
            } else {
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const uint32_t r = (w[j >> 1] >> (16 * (j & 1))) & 0xffffu;
                    c += (int)(e0 + j >= lo && e0 + j <= hi && r < up);
                }
            }
        }
    }
    return (int)__reduce_add_sync(kFull, (unsigned)c);
}

// Per-thread exact selection (vertical sweep): every lane refines its own window. It scans the
// omnigram from its pivot in aligned groups of entries (one 128-bit load), K groups per step
// (the loop's votes and bookkeeping are paid once per K groups: K = 4 where scans are short,
// small kernels; 8 where they are long), counting members, until the group holding the
// target-th member. While at least kHandoff lanes are still
// scanning this is the cheapest schedule; the last few lanes of a warp (long jumps at edges and
// impulses) are finished by warp-cooperative ballot scans instead of keeping 29+ lanes idle.
// Same contract as ballot_select, per lane. All loops are bounded by the omnigram length.
constexpr int kHandoff = 8;
constexpr int kHandoffAfterGroups = 8;

// KS > 0: KS groups per step, fixed at compile time; KS = 0: `groups` per step (at most 8),
// read at run time (smaller code).
template <int SHAPE, int W, int KS>
__device__ __forceinline__ int thread_select(const typename Loc<W>::E* __restrict__ om, int N, int p, int c,
                                             int target, int px, int py, const Member<SHAPE, W>& member,
                                             int groups = KS) {
    constexpr int kUnroll = KS > 0 ? KS : 8;
    const int K = KS > 0 ? KS : groups;
    const int handoff_after = (kHandoffAfterGroups + K - 1) / K;  // steps
    constexpr int G = Loc<W>::kGroup;
    constexpr uint32_t kAll = (1u << G) - 1;
    const int lane = threadIdx.x & 31;
    WordTest<SHAPE, W> wt;
    wt.init(member, px, py);
    const uint4* om128 = reinterpret_cast<const uint4*>(om);
    const bool up = c <= target;
    int need = up ? target - c + 1 : c - target;
    int nextv = up ? p : p - 1;  // next omnigram entry to examine
    const int glast = (N - 1) / G;
    bool done = false;
    int m = -1;
    // Entries past N up to the last group's end are sentinels that are never members, so only
    // the first group needs a mask: the entries on the far side of the pivot.
    const int o0 = nextv & (G - 1);
    uint32_t first = up ? (kAll << o0) & kAll : kAll >> (G - 1 - o0);
    constexpr int kShift = G == 8 ? 3 : 2;
    for (int it = 0; it <= glast + 1; ++it) {
        // the hand-off test costs a vote, so it only starts once the typical scan is over
        if (it >= handoff_after && __popc(__ballot_sync(kFull, !done)) < kHandoff) break;
        if (it < handoff_after && !__any_sync(kFull, !done)) break;
        if (!done) {
            const int g = nextv >> kShift;  // -1 below entry 0
            if ((unsigned)g > (unsigned)glast) {
                done = true;
            } else {
                constexpr int kb = G / 4;  // entries per word
                uint32_t selmask = 0;
                int selg = 0;
                bool found = false;
#pragma unroll
                for (int k = 0; k < kUnroll; ++k) {
                    if (KS == 0 && k >= K) break;  // uniform: every lane has the same K
                    const int gk = up ? g + k : g - k;
                    const bool ok = (unsigned)gk <= (unsigned)glast;
                    const uint4 q = om128[ok ? gk : g];
                    uint32_t mk = wt(q.x) | (wt(q.y) << kb) | (wt(q.z) << (2 * kb)) | (wt(q.w) << (3 * kb));
                    if (!ok) mk = 0;
                    if (k == 0) mk &= first;
                    const int c = __popc(mk);
                    if (!found) {
                        if (c >= need) {
                            found = true;
                            selmask = mk;
                            selg = gk;
                        } else {
                            need -= c;
                        }
                    }
                }
                first = kAll;
                if (found) {
                    uint32_t mask = selmask;
                    if (up) {
                        for (int k = 1; k < need; ++k) mask &= mask - 1;  // drop the lowest need-1
                        m = G * selg + __ffs(mask) - 1;
                    } else {
                        for (int k = 1; k < need; ++k) mask ^= 1u << (31 - __clz(mask));  // drop the highest
                        m = G * selg + 31 - __clz(mask);
                    }
                    done = true;
                } else {
                    nextv = up ? G * (g + K) : G * (g - K + 1) - 1;
                }
            }
        }
    }
    // hand-off: the remaining lanes, one window at a time, by ballot scans
    uint32_t rest = __ballot_sync(kFull, !done);
    while (rest) {
        const int j = __ffs(rest) - 1;
        rest &= rest - 1;
        const int upj = __shfl_sync(kFull, (int)up, j);
        const int nj = __shfl_sync(kFull, nextv, j);
        const int needj = __shfl_sync(kFull, need, j);
        const int pxj = __shfl_sync(kFull, px, j);
        const int pyj = __shfl_sync(kFull, py, j);
        const int pj = upj ? nj : nj + 1;
        const int cj = upj ? target + 1 - needj : target + needj;
        const int mj = ballot_select(om, N, pj, cj, target, pxj, pyj, member);
        if (lane == j) m = mj;
    }
    return m;
}

// Block-wide exclusive scan of 65536 16-bit counters packed two per word (bin 2k in the low
// half of word k). Offsets stay below 2^16 because the footprint holds at most 65535 pixels.
__device__ void scan_bins16(uint32_t* bins, uint32_t* wtot, const Plan& P, const Grp& G) {
    const int lane = G.lane, warp = G.warp;
    const int chunk = 32768 / P.nwarps;  // words per warp, a multiple of 128
    uint4* b4 = reinterpret_cast<uint4*>(bins + warp * chunk);
    uint32_t acc = 0;
    for (int it = 0; it < chunk / 128; ++it) {
        const uint4 q = b4[it * 32 + lane];
        acc += ((q.x + (q.x >> 16)) & 0xffffu) + ((q.y + (q.y >> 16)) & 0xffffu) +
               ((q.z + (q.z >> 16)) & 0xffffu) + ((q.w + (q.w >> 16)) & 0xffffu);
    }
    acc = __reduce_add_sync(kFull, acc);
    if (lane == 0) wtot[warp] = acc;
    G.sync();
    if (warp == 0) {
        const uint32_t x = lane < P.nwarps ? wtot[lane] : 0;
        uint32_t incl = x;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(kFull, incl, o);
            if (lane >= o) incl += t;
        }
        wtot[lane] = incl - x;
    }
    G.sync();
    uint32_t run = wtot[warp];
    for (int it = 0; it < chunk / 128; ++it) {
        uint4 q = b4[it * 32 + lane];
        const uint32_t s = ((q.x + (q.x >> 16)) & 0xffffu) + ((q.y + (q.y >> 16)) & 0xffffu) +
                           ((q.z + (q.z >> 16)) & 0xffffu) + ((q.w + (q.w >> 16)) & 0xffffu);
        uint32_t incl = s;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(kFull, incl, o);
            if (lane >= o) incl += t;
        }
        uint32_t b = run + incl - s;
        uint32_t w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const uint32_t lo = w[k] & 0xffffu, hi = w[k] >> 16;
            w[k] = b | ((b + lo) << 16);
            b += lo + hi;
        }
        b4[it * 32 + lane] = make_uint4(w[0], w[1], w[2], w[3]);
        run += __shfl_sync(kFull, incl, 31);
    }
    G.sync();
}

// Block-wide exclusive scan of 32768 32-bit counters, offset by `base`; returns their total
// (every thread). Each warp owns a contiguous chunk; each lane 4 counters (one 128-bit word) per
// 128-counter slab.
__device__ uint32_t scan_bins32(uint32_t* bins, uint32_t* wtot, uint32_t base, const Plan& P, const Grp& G) {
    const int lane = G.lane, warp = G.warp;
    const int chunk = 32768 / P.nwarps;  // counters per warp, a multiple of 128
    uint4* b4 = reinterpret_cast<uint4*>(bins + warp * chunk);
    uint32_t acc = 0;
    for (int it = 0; it < chunk / 128; ++it) {
        const uint4 q = b4[it * 32 + lane];
        acc += q.x + q.y + q.z + q.w;
    }
    acc = __reduce_add_sync(kFull, acc);
    if (lane == 0) wtot[warp] = acc;
    G.sync();
    if (warp == 0) {
        const uint32_t x = lane < P.nwarps ? wtot[lane] : 0;
        uint32_t incl = x;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(kFull, incl, o);
            if (lane >= o) incl += t;
        }
        wtot[lane] = incl - x;
        if (lane == 31) wtot[32] = incl;
    }
    G.sync();
    uint32_t run = base + wtot[warp];
    const uint32_t total = wtot[32];
    for (int it = 0; it < chunk / 128; ++it) {
        uint4 q = b4[it * 32 + lane];
        const uint32_t sum = q.x + q.y + q.z + q.w;
        uint32_t incl = sum;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(kFull, incl, o);
            if (lane >= o) incl += t;
        }
        uint32_t b = run + incl - sum;
        const uint32_t c0 = q.x, c1 = q.y, c2 = q.z;
        q.x = b;
        q.y = b + c0;
        q.z = q.y + c1;
        q.w = q.z + c2;
        b4[it * 32 + lane] = q;
        run += __shfl_sync(kFull, incl, 31);
    }
    G.sync();
    return total;
}

// The image as the tile pipeline reads it, held in registers.
struct Img {
    const char* in;
    long long pitch;
    int w, h;
    __device__ __forceinline__ explicit Img(const Plan& P)
        : in(static_cast<const char*>(P.in)), pitch(P.pitch), w(P.w), h(P.h) {}
};

template <int DT>
__device__ __forceinline__ typename Traits<DT>::T load_px(const Img& im, int gx, int gy) {
    using V = typename Traits<DT>::T;
    const V* row = reinterpret_cast<const V*>(im.in + (long long)clampi(gy, 0, im.h - 1) * im.pitch);
    return __ldg(row + clampi(gx, 0, im.w - 1));
}

// Where phase 1 reads the footprint from: the box staged in shared memory by the tensor memory
// accelerator (interior tiles), or the image in global memory with clamp-to-edge (every other
// tile). `off` is the staged column of box column 0 (the copy starts on a 16-byte boundary).
// STAGED is fixed per call (the sorts are compiled for both), so the loads of the global-memory
// form stay free of a per-pixel branch.
template <int DT>
struct Footprint {
    using V = typename Traits<DT>::T;
    const unsigned char* stage;  // null: read the image
    int pitch;                   // bytes per staged row
    int off;
    Img im;
    int gx0, gy0;
    template <bool STAGED>
    __device__ __forceinline__ uint32_t key(int u, int v) const {
        if constexpr (STAGED) return Traits<DT>::key(reinterpret_cast<const V*>(stage + v * pitch)[u + off]);
        else return Traits<DT>::key(load_px<DT>(im, gx0 + u, gy0 + v));
    }
};

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// mbarrier of the footprint copies: one arrival (the issuing thread) plus the copy's bytes.
__device__ __forceinline__ void mbar_init(uint64_t* bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Copies the box of `rows` x `cols` elements at image column x0 (a multiple of 16 bytes) and row
// y0 into shared memory at dst, completing on `bar` (issued by one thread).
__device__ __forceinline__ void tma_load_box(const void* tmap, unsigned char* dst, uint64_t* bar, int x0, int y0,
                                             uint32_t bytes) {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
        ::"r"(smem_addr(dst)), "l"(reinterpret_cast<uint64_t>(tmap)), "r"(x0), "r"(y0), "r"(smem_addr(bar))
        : "memory");
}

// Waits for phase `parity` of `bar` to complete; gives up (false) after a bounded number of tries.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
    const uint32_t a = smem_addr(bar);
    for (int i = 0; i < (1 << 22); ++i) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// State of the footprint copies of one CTA across its tiles.
struct TmaState {
    uint32_t parity;  // phase of the next copy's completion
    int off;          // 1 once a copy timed out: global loads from then on
};

// Counting-sort ordinal transform for 8/16-bit data (Sec. 4.1, Eq. 5): histogram of the
// footprint, exclusive prefix, then every pixel takes the next free ordinal of its value.
// Ties get consecutive ordinals in arrival order, which is all the method needs.
template <int DT, int W, bool STAGED>
__device__ void ordinal_transform_count(const Plan& P, const int* frow, uint32_t* bins, uint32_t* misc,
                                        typename Loc<W>::E* om, const Footprint<DT>& fp, const Grp& G) {
    const int tid = G.tid, lane = G.lane, warp = G.warp;
    const int SH = P.SH, nwarps = P.nwarps, cx0 = P.cx0, cy0 = P.cy0;
    constexpr bool k16 = DT == FIM_U16;
    constexpr int kLoads = 8;
    if constexpr (k16) {
        if (P.sort == kSortCount16x2) {
            // Footprints of more than 65535 pixels: the same construction in two rounds over the
            // key range (top bit 0, then 1), each with 32768 32-bit bins in the same 128 KiB; the
            // second round's offsets start after the first round's pixels.
            uint32_t base = 0;
            for (int h = 0; h < 2; ++h) {
                for (int i = tid * 4; i < 32768; i += P.threads * 4)
                    *reinterpret_cast<uint4*>(bins + i) = make_uint4(0, 0, 0, 0);
                G.sync();
                for (int v = warp; v < SH; v += nwarps) {
                    const int fr = frow[v];
                    const int hi = span_hi(fr);
                    for (int u0 = span_lo(fr) + lane; u0 <= hi; u0 += 32 * kLoads) {
                        uint32_t key[kLoads];
#pragma unroll
                        for (int k = 0; k < kLoads; ++k)
                            key[k] = u0 + 32 * k <= hi ? fp.template key<STAGED>(u0 + 32 * k, v) : 0xffffffffu;
#pragma unroll
                        for (int k = 0; k < kLoads; ++k)
                            if ((key[k] >> 15) == (uint32_t)h) atomicAdd(&bins[key[k] & 0x7fffu], 1u);
                    }
                }
                G.sync();
                base += scan_bins32(bins, misc, base, P, G);
                for (int v = warp; v < SH; v += nwarps) {
                    const int fr = frow[v];
                    const int hi = span_hi(fr);
                    for (int u0 = span_lo(fr) + lane; u0 <= hi; u0 += 32 * kLoads) {
                        uint32_t key[kLoads];
#pragma unroll
                        for (int k = 0; k < kLoads; ++k)
                            key[k] = u0 + 32 * k <= hi ? fp.template key<STAGED>(u0 + 32 * k, v) : 0xffffffffu;
#pragma unroll
                        for (int k = 0; k < kLoads; ++k)
                            if ((key[k] >> 15) == (uint32_t)h)
                                om[atomicAdd(&bins[key[k] & 0x7fffu], 1u)] = Loc<W>::pack(u0 + 32 * k, v, cx0, cy0);
                    }
                }
                G.sync();
            }
            return;
        }
    }
    const int nwords = k16 ? 32768 : 256;
    for (int i = tid * 4; i < nwords; i += P.threads * 4)
        *reinterpret_cast<uint4*>(bins + i) = make_uint4(0, 0, 0, 0);
    G.sync();
    // A warp takes one footprint row at a time; each lane loads up to kLoads pixels of it (all in
    // flight at once) before it issues their shared-memory atomics.
    for (int v = warp; v < SH; v += nwarps) {
        const int fr = frow[v];
        const int hi = span_hi(fr);
        for (int u0 = span_lo(fr) + lane; u0 <= hi; u0 += 32 * kLoads) {
            uint32_t key[kLoads];
#pragma unroll
            for (int k = 0; k < kLoads; ++k)
                key[k] = u0 + 32 * k <= hi ? fp.template key<STAGED>(u0 + 32 * k, v) : 0u;
#pragma unroll
            for (int k = 0; k < kLoads; ++k) {
                if (u0 + 32 * k > hi) break;
                if (k16)
                    atomicAdd(&bins[key[k] >> 1], 1u << ((key[k] & 1u) << 4));
                else
                    atomicAdd(&bins[key[k]], 1u);
            }
        }
    }
    G.sync();
    if (k16) {
        scan_bins16(bins, misc, P, G);
    } else {
        if (warp == 0) {
            uint32_t c[8], s = 0;
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                c[k] = bins[lane * 8 + k];
                s += c[k];
            }
            uint32_t incl = s;
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t t = __shfl_up_sync(kFull, incl, o);
                if (lane >= o) incl += t;
            }
            uint32_t b = incl - s;
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                bins[lane * 8 + k] = b;
                b += c[k];
            }
        }
        G.sync();
    }
    for (int v = warp; v < SH; v += nwarps) {
        const int fr = frow[v];
        const int hi = span_hi(fr);
        for (int u0 = span_lo(fr) + lane; u0 <= hi; u0 += 32 * kLoads) {
            uint32_t key[kLoads];
#pragma unroll
            for (int k = 0; k < kLoads; ++k)
                key[k] = u0 + 32 * k <= hi ? fp.template key<STAGED>(u0 + 32 * k, v) : 0u;
#pragma unroll
            for (int k = 0; k < kLoads; ++k) {
                if (u0 + 32 * k > hi) break;
                uint32_t o;
                if (k16) {
                    const uint32_t sh = (key[k] & 1u) << 4;
                    o = (atomicAdd(&bins[key[k] >> 1], 1u << sh) >> sh) & 0xffffu;
                } else {
                    o = atomicAdd(&bins[key[k]], 1u);
                }
                om[o] = Loc<W>::pack(u0 + 32 * k, v, cx0, cy0);
            }
        }
    }
}

// LSD radix ordinal transform over bounding-box positions. Float keys in 1024-thread CTAs (C16):
// a 65536-bin counting pass on the low 16 bits (Eq. 5's construction, like 16-bit data) followed
// by two stable 8-bit passes on the high bytes; otherwise 8-bit passes only, four for 32-bit
// float keys and two for 16-bit data. The first pass may order equal digits arbitrarily
// (shared-memory atomics), since the later passes are stable. In a stable pass each warp owns one
// contiguous segment of the current order, and a pixel's new place is its (digit, warp)-major
// exclusive offset plus its position among equal digits earlier in the segment (warp match).
// Histograms are laid out warp-major with a pad word so that the leaders of one warp never share
// a bank. Where the keys live in global scratch (large footprints), each stable pass first copies
// its digit of every box position into a shared byte array (`dig`, coalesced reads of the keys),
// so that the passes look digits up in shared memory instead of gathering keys from L2 one by one.
// The sorted positions end in list B, which is then rewritten in place as the omnigram.
template <int DT, int W, bool C16, bool STAGED>
__device__ void ordinal_transform_radix(const Plan& P, const int* frow, uint32_t* keys, typename Loc<W>::Pos* bufA,
                                        typename Loc<W>::Pos* bufB, uint32_t* hist, uint32_t* wsum, uint32_t* bins,
                                        uint8_t* dig, const Footprint<DT>& fp, const Grp& G) {
    using Pos = typename Loc<W>::Pos;
    const int tid = G.tid, lane = G.lane, warp = G.warp;
    const int nthreads = P.threads, nwarps = P.nwarps, S = P.S;
    constexpr int HS = kSortBins + 1;
    const int area = S * P.SH;
    uint32_t* hw = hist + warp * HS;
    // Exclusive scan of the per-warp digit counts in (digit, warp) order, in place: each thread
    // takes 8 consecutive counters (256 * nwarps counters over 32 * nwarps threads).
    auto scan_counts = [&]() {
        const int e0 = tid * 8;
        uint32_t c[8];
        uint32_t local = 0;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int e = e0 + j, d = e / nwarps, wq = e - d * nwarps;
            c[j] = hist[wq * HS + d];
            local += c[j];
        }
        uint32_t incl = local;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(kFull, incl, o);
            if (lane >= o) incl += t;
        }
        if (lane == 31) wsum[warp] = incl;
        G.sync();
        if (warp == 0) {
            const uint32_t x = lane < nwarps ? wsum[lane] : 0;
            uint32_t y = x;
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t t = __shfl_up_sync(kFull, y, o);
                if (lane >= o) y += t;
            }
            wsum[lane] = y - x;
        }
        G.sync();
        uint32_t run = incl - local + wsum[warp];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int e = e0 + j, d = e / nwarps, wq = e - d * nwarps;
            hist[wq * HS + d] = run;
            run += c[j];
        }
    };
    // box position i lies in the footprint (Fig. 10)
    auto inside = [&](int i) {
        const int v = (int)__umulhi((unsigned)i, P.div_magic);
        const int fr = frow[v];
        const int u = i - v * S;
        return u >= span_lo(fr) && u <= span_hi(fr);
    };
    // Pass 0, fused with the footprint load: every thread takes box positions tid, tid +
    // nthreads, ... (coalesced rows), four loads in flight, and counts the low digit (8 bits in its
    // warp's histogram, or 16 bits in the block's packed bins); equal digits may then land in any
    // order (returned atomics), since the later passes are stable.
    // Footprints of more than 65535 pixels would overflow the packed 16-bit counters: the 16-bit
    // pass then counts in two rounds over the digit range (top bit 0, then 1), each with 32768
    // 32-bit bins in the same 128 KiB (the first round's histogram fused with the load).
    const bool two = C16 && P.N > 65535;
    if constexpr (C16) {
        for (int i = tid * 4; i < 32768; i += nthreads * 4)
            *reinterpret_cast<uint4*>(bins + i) = make_uint4(0, 0, 0, 0);
        G.sync();
    } else {
        for (int d = lane; d < kSortBins; d += 32) hw[d] = 0;
        __syncwarp();
    }
    for (int i0 = tid; i0 < area; i0 += 4 * nthreads) {
        uint32_t key[4];
        bool in[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int i = i0 + k * nthreads;
            in[k] = i < area && inside(i);
            key[k] = 0;
            if (in[k]) {
                const int v = (int)__umulhi((unsigned)i, P.div_magic);
                key[k] = fp.template key<STAGED>(i - v * S, v);
            }
        }
#pragma unroll
        for (int k = 0; k < 4; ++k)
            if (in[k]) {
                keys[i0 + k * nthreads] = key[k];
                if constexpr (C16) {
                    const uint32_t d = key[k] & 0xffffu;
                    if (!two)
                        atomicAdd(&bins[d >> 1], 1u << ((d & 1u) << 4));
                    else if ((d >> 15) == 0)
                        atomicAdd(&bins[d], 1u);
                } else {
                    atomicAdd(&hw[key[k] & 0xff], 1u);
                }
            }
    }
    G.sync();
    // the first pass's result goes to the list the stable passes start from: with C16 two stable
    // passes follow (B -> A -> B), otherwise an odd number (A -> B -> ... -> B)
    Pos* first = C16 ? bufB : bufA;
    // The keys may live in global scratch: every loop below loads kG of them (all in flight)
    // before it uses the first.
    constexpr int kG = 4;
    if constexpr (C16) {
        if (two) {
            uint32_t base = 0;
            for (int h = 0; h < 2; ++h) {
                if (h == 1) {  // the second round's histogram (the keys, in order, from scratch)
                    for (int i = tid * 4; i < 32768; i += nthreads * 4)
                        *reinterpret_cast<uint4*>(bins + i) = make_uint4(0, 0, 0, 0);
                    G.sync();
                    for (int i0 = tid; i0 < area; i0 += kG * nthreads) {
                        uint32_t key[kG];
                        bool in[kG];
#pragma unroll
                        for (int k = 0; k < kG; ++k) {
                            const int i = i0 + k * nthreads;
                            in[k] = i < area && inside(i);
                            key[k] = in[k] ? keys[i] & 0xffffu : 0u;
                        }
#pragma unroll
                        for (int k = 0; k < kG; ++k)
                            if (in[k] && (key[k] >> 15) == 1u) atomicAdd(&bins[key[k] & 0x7fffu], 1u);
                    }
                    G.sync();
                }
                base += scan_bins32(bins, wsum, base, P, G);
                for (int i0 = tid; i0 < area; i0 += kG * nthreads) {
                    uint32_t key[kG];
                    bool in[kG];
#pragma unroll
                    for (int k = 0; k < kG; ++k) {
                        const int i = i0 + k * nthreads;
                        in[k] = i < area && inside(i);
                        key[k] = in[k] ? keys[i] & 0xffffu : 0u;
                    }
#pragma unroll
                    for (int k = 0; k < kG; ++k)
                        if (in[k] && (key[k] >> 15) == (uint32_t)h)
                            first[atomicAdd(&bins[key[k] & 0x7fffu], 1u)] = (Pos)(i0 + k * nthreads);
                }
                G.sync();
            }
        } else {
            scan_bins16(bins, wsum, P, G);
        }
    } else {
        scan_counts();
        G.sync();
    }
    for (int i0 = tid; i0 < area && !two; i0 += kG * nthreads) {
        uint32_t key[kG];
        bool in[kG];
#pragma unroll
        for (int k = 0; k < kG; ++k) {
            const int i = i0 + k * nthreads;
            in[k] = i < area && inside(i);
            key[k] = in[k] ? keys[i] : 0u;
        }
#pragma unroll
        for (int k = 0; k < kG; ++k)
            if (in[k]) {
                const int i = i0 + k * nthreads;
                if constexpr (C16) {
                    const uint32_t d = key[k] & 0xffffu, sh = (d & 1u) << 4;
                    first[(atomicAdd(&bins[d >> 1], 1u << sh) >> sh) & 0xffffu] = (Pos)i;
                } else {
                    first[atomicAdd(&hw[key[k] & 0xff], 1u)] = (Pos)i;
                }
            }
    }
    G.sync();
    // stable passes over the current order: each warp owns one contiguous segment; a pixel's
    // new place is its (digit, warp)-major exclusive offset plus its position among equal
    // digits earlier in the segment (warp match)
    const Pos* src = first;
    Pos* dst = C16 ? bufA : bufB;
    constexpr int kBits0 = C16 ? 16 : 8;                       // key bits the first pass sorted
    constexpr int kPasses = (DT == FIM_F32 ? 32 - kBits0 : 16 - kBits0) / 8;  // stable 8-bit passes
    static_assert(kPasses % 2 == (C16 ? 0 : 1), "the sorted positions must end in list B");
    const int N = P.N;
    const int seg = ((N + nwarps - 1) / nwarps + 31) & ~31;
    const int s0 = min(N, warp * seg), s1 = min(N, s0 + seg);
    // the stable passes, compiled for digits looked up in `dig` and for digits taken from the keys
    auto stable_passes = [&](auto use_dig) {
        constexpr bool kDig = decltype(use_dig)::value;
        for (int pass = 0; pass < kPasses; ++pass) {
            const int shift = kBits0 + 8 * pass;
            if constexpr (kDig) {
                const int nq = (area + 3) >> 2;  // keys of 4 consecutive box positions per load
                const uint4* k4 = reinterpret_cast<const uint4*>(keys);
                uint32_t* d4 = reinterpret_cast<uint32_t*>(dig);
                for (int j = tid; j < nq; j += nthreads) {
                    const uint4 q = k4[j];
                    d4[j] = ((q.x >> shift) & 0xffu) | (((q.y >> shift) & 0xffu) << 8) |
                            (((q.z >> shift) & 0xffu) << 16) | ((q.w >> shift) << 24);
                }
                G.sync();
            }
            auto digit = [&](int pos) -> int {
                if constexpr (kDig) return dig[pos];
                else return (int)(keys[pos] >> shift) & 0xff;
            };
            for (int d = lane; d < kSortBins; d += 32) hw[d] = 0;
            __syncwarp();
            for (int i0 = s0 + lane; i0 < s1; i0 += 32 * kG) {  // counts do not depend on the order
                int dk[kG];
#pragma unroll
                for (int k = 0; k < kG; ++k) {
                    const int i = i0 + 32 * k;
                    dk[k] = i < s1 ? digit(src[i]) : 0;
                }
#pragma unroll
                for (int k = 0; k < kG; ++k)
                    if (i0 + 32 * k < s1) atomicAdd(&hw[dk[k]], 1u);
            }
            G.sync();
            scan_counts();
            G.sync();
            for (int b0 = s0; b0 < s1; b0 += 32 * kG) {
                int pos[kG], d[kG];
#pragma unroll
                for (int k = 0; k < kG; ++k) {
                    const int i = b0 + 32 * k + lane;
                    pos[k] = i < s1 ? (int)src[i] : -1;
                }
#pragma unroll
                for (int k = 0; k < kG; ++k)
                    d[k] = pos[k] >= 0 ? digit(pos[k]) : kSortBins + lane;
                // batches in segment order, so equal digits keep their order
#pragma unroll
                for (int k = 0; k < kG; ++k) {
                    if (b0 + 32 * k >= s1) break;
                    const bool valid = pos[k] >= 0;
                    const uint32_t peers = __match_any_sync(kFull, d[k]);
                    uint32_t base = 0;
                    if (valid) base = hw[d[k]];
                    __syncwarp();
                    if (valid) {
                        dst[base + __popc(peers & lanemask_lt())] = (Pos)pos[k];
                        if (lane == __ffs(peers) - 1) hw[d[k]] = base + __popc(peers);
                    }
                    __syncwarp();
                }
            }
            G.sync();
            src = dst;
            dst = (dst == bufA) ? bufB : bufA;
        }
    };
    if constexpr (DT == FIM_F32) {  // only float plans place digits (one stable pass otherwise)
        if (dig != nullptr)
            stable_passes(std::true_type{});
        else
            stable_passes(std::false_type{});
    } else {
        stable_passes(std::false_type{});
    }
    // the sorted positions are in B; rewrite them in place as entries
    typename Loc<W>::E* om = reinterpret_cast<typename Loc<W>::E*>(bufB);
    for (int v = tid; v < N; v += nthreads) {
        const int pos = (int)bufB[v];
        const int y = (int)__umulhi((unsigned)pos, P.div_magic);
        om[v] = Loc<W>::pack(pos - y * S, y, P.cx0, P.cy0);
    }
}

// ---- learned rank bracket (seed windows) ---------------------------------------------------

__device__ __forceinline__ float bf16_to_f32(uint16_t b) { return __uint_as_float((uint32_t)b << 16); }

// Features of the seed window centred at box position (cu, cv): the tile's normalised value
// quantiles (already in q[0..31]) and the ranks / N of the 3x3 pixels around the centre
// (the centre's own rank where a neighbour lies outside the footprint).
__device__ __forceinline__ void seed_features(const uint16_t* ord, int SP, const int* frow, int SH, int N, int cu,
                                              int cv, const float* q, float* fa, float* fb) {
    const int lane = threadIdx.x & 31;
    *fa = q[lane];
    float nb = 0.f;
    if (lane < kNeigh) {
        int u = cu + lane % 3 - 1, v = cv + lane / 3 - 1;
        bool in = v >= 0 && v < SH;
        if (in) {
            const int fr = frow[v];
            in = u >= span_lo(fr) && u <= span_hi(fr);
        }
        if (!in) {
            u = cu;
            v = cv;
        }
        nb = (float)ord[v * SP + u] / (float)N;
    }
    *fb = nb;
}

// Visits the ranks of every pixel of a window (row i of the kernel at ctr + (ymin + i) * SP,
// ctr being the window centre's ordinal-image position shifted by ymin rows). Lane l takes
// kernel rows l, l+32, ... and walks each from a lane-dependent column, so the 32 pixels
// visited at once lie far apart (their ranks rarely share a histogram bin). Four ranks are
// loaded before they are handed to `f`, so the loads of a group overlap instead of each
// waiting behind the previous group's shared-memory atomics.
template <class Fn>
__device__ __forceinline__ void window_walk(const int* spans, int nrows, const uint16_t* ctr, int SP, Fn&& f) {
    const int lane = threadIdx.x & 31;
    for (int i = lane; i < nrows; i += 32) {
        const int sp = spans[i];
        const int width = span_hi(sp) - span_lo(sp) + 1;
        const uint16_t* row = ctr + i * SP + span_lo(sp);
        int x = (lane * 37) % width;
        int k = 0;
        for (; k + 4 <= width; k += 4) {
            int x1 = x + 1, x2 = x + 2, x3 = x + 3;
            if (x1 >= width) x1 -= width;
            if (x2 >= width) x2 -= width;
            if (x3 >= width) x3 -= width;
            const int r0 = row[x], r1 = row[x1], r2 = row[x2], r3 = row[x3];
            f(r0);
            f(r1);
            f(r2);
            f(r3);
            x = x3 + 1 == width ? 0 : x3 + 1;
        }
        for (; k < width; ++k) {
            f((int)row[x]);
            x = (x + 1 == width) ? 0 : x + 1;
        }
    }
}

// Target rank of output pixel (gx, gy) under a percentile map (Fig. 14), from the rank image
// the host computed before the launch. Pixels beyond the image (the ragged edge of a tile) take
// the nearest pixel's rank; their results are never stored.
__device__ __forceinline__ int map_rank(const Plan& P, int gx, int gy) {
    return __ldg(P.rank_map + (long long)min(gy, P.h - 1) * P.w + min(gx, P.w - 1));
}

// Seed histogram (kSeedBins bins of one warp): the bin holding window-rank `target` when
// `base` window members lie below bin 0. Returns the bin and, in *below, the members below it.
__device__ __forceinline__ int hist_pick(const uint32_t* hw, int base, int target, int* below) {
    const int lane = threadIdx.x & 31;
    constexpr int per = kSeedBins / 32;
    uint32_t local = 0;
    for (int j = 0; j < per; ++j) local += hw[lane * per + j];
    uint32_t incl = local;
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t tt = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += tt;
    }
    const int excl = base + (int)(incl - local);
    const bool mine = excl <= target && target < base + (int)incl;
    const uint32_t who = __ballot_sync(kFull, mine);
    int bin = 0, run = 0;
    if (mine) {
        run = excl;
        int j = 0;
        for (; j < per - 1; ++j) {
            const int c = (int)hw[lane * per + j];
            if (run + c > target) break;
            run += c;
        }
        bin = lane * per + j;
    }
    const int src = who ? __ffs(who) - 1 : 0;
    *below = __shfl_sync(kFull, run, src);
    return __shfl_sync(kFull, bin, src);
}

template <class T>
__device__ __forceinline__ T* place(unsigned char* smem, unsigned char* gslice, int loc) {
    return reinterpret_cast<T*>(loc >= 0 ? smem + loc : gslice + (-(long long)loc - 1));
}

// Several radii from one transform: keeps, in order, the omnigram entries that lie in a smaller
// disk's footprint (`qfrow`: per box row, its columns lo | hi << 16; rows outside hold an empty
// span), and gives those pixels their new ranks in the ordinal image. The order of the kept
// entries is the sorted order restricted to the smaller footprint, i.e. that footprint's own
// ordinal transform, obtained in one pass with no sort. Each thread takes 4 consecutive entries
// of a 4 * group-size chunk; a block scan of the per-thread counts gives the new places. Every
// write goes to an index no larger than the entry's own, and all reads of a chunk precede its
// first barrier, so the compaction can run in place. Returns the number kept.
template <int W>
__device__ int compact_omnigram(typename Loc<W>::E* om, int N, const int* qfrow, uint16_t* ord, int SP, int cx0,
                                int cy0, uint32_t* wsum, const Grp& G, int nthreads, int nwarps) {
    using E = typename Loc<W>::E;
    const int tid = G.tid, lane = G.lane, warp = G.warp;
    int base = 0;
    for (int c0 = 0; c0 < N; c0 += 4 * nthreads) {
        E e[4];
        bool keep[4];
        int cnt = 0;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int i = c0 + 4 * tid + k;
            keep[k] = false;
            e[k] = 0;
            if (i < N) {
                e[k] = om[i];
                const int u = Loc<W>::x(e[k]) + cx0, v = Loc<W>::y(e[k]) + cy0;
                const int fr = qfrow[v];
                keep[k] = u >= span_lo(fr) && u <= span_hi(fr);
            }
            cnt += keep[k];
        }
        int incl = cnt;
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(kFull, incl, o);
            if (lane >= o) incl += t;
        }
        if (lane == 31) wsum[warp] = (uint32_t)incl;
        G.sync();
        if (warp == 0) {
            const uint32_t x = lane < nwarps ? wsum[lane] : 0u;
            uint32_t y = x;
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t t = __shfl_up_sync(kFull, y, o);
                if (lane >= o) y += t;
            }
            wsum[lane] = y - x;         // exclusive per-warp offsets
            if (lane == 31) wsum[32] = y;  // the chunk's total
        }
        G.sync();
        int idx = base + (int)wsum[warp] + incl - cnt;
#pragma unroll
        for (int k = 0; k < 4; ++k)
            if (keep[k]) {
                om[idx] = e[k];
                ord[(Loc<W>::y(e[k]) + cy0) * SP + Loc<W>::x(e[k]) + cx0] = (uint16_t)idx;
                ++idx;
            }
        base += (int)wsum[32];
        G.sync();  // the offsets are read before the next chunk rewrites them
    }
    const int pad = ((base + Loc<W>::kGroup - 1) & ~(Loc<W>::kGroup - 1)) - base;
    if (tid < pad) om[base + tid] = Loc<W>::kSentinel;
    G.sync();
    return base;
}

// KS: omnigram groups per scan step of the vertical sweep, fixed at compile time (4 or 8; the
// batch class kernels are compiled for both), or 0 to follow the plan's scan_groups at run time.
// XT: 1 compiles the extras — the learned bracket, training-row output, seed statistics and
// several target ranks per launch — and 2 a target rank per output pixel (a percentile map).
// Each lives in kernels of its own: at the 64-register cap of 1024-thread CTAs their code
// changes how the compiler allocates the plain pipeline's registers, and the reverse.
// TMA: how interior footprints are copied into the staging region: 0 not at all; 1 the
// single-image kernels (mbarrier in the scan scratch, tensor map in the kernel parameter);
// 2 the batch kernels (`bar` and `tmap` given: a CTA-wide mbarrier and the job's tensor map in
// the plan array in global memory, since their plans are read from shared memory).
template <int DT, int SHAPE, int W, int OG, int KS = 0, int XT = 0, int TMA = 1>
__device__ __forceinline__ void process_tile(const Plan& P, int tile, unsigned char* gslice, const Grp& G,
                                             TmaState* tma = nullptr, uint64_t* bar = nullptr,
                                             const void* tmap = nullptr) {
    extern __shared__ __align__(16) unsigned char smem_base[];
    unsigned char* const smem = smem_base + G.shift;  // this group's partition (tables excluded)
    using V = typename Traits<DT>::T;
    using E = typename Loc<W>::E;
    const int tid = G.tid;
    const int lane = G.lane;
    const int warp = G.warp;
    const int nthreads = P.threads;
    const int nwarps = P.nwarps;
    const int SP = P.SP, N = P.N, TX = P.Tx, TY = P.Ty;
    const int tx0 = (tile % P.tiles_x) * TX;
    const int ty0 = (tile / P.tiles_x) * TY;
    const int gx0 = tx0 + P.xmin;  // global coordinates of bounding-box pixel (0, 0)
    const int gy0 = ty0 + P.ymin;
    const int cx0 = P.cx0, cy0 = P.cy0, xmin = P.xmin, ymin = P.ymin, hist_shift = P.hist_shift;
    // The ordinal image and the medians hold ranks minus rank_base, clamped to 16 bits: every
    // pivot lies in the tile's feasible median ranks (Fig. 10), which then compare exactly, so
    // footprints beyond 65535 pixels keep a 16-bit ordinal image (rank_base = 0 below that).
    const int rb = P.rank_base;

    const int2* vtab = reinterpret_cast<const int2*>(smem_base + P.off_vtab);
    const int2* htab = reinterpret_cast<const int2*>(smem_base + P.off_htab);
    const int* spans = reinterpret_cast<const int*>(smem_base + P.off_spans);
    const int* frow = reinterpret_cast<const int*>(smem_base + P.off_frow);
    uint32_t* misc = reinterpret_cast<uint32_t*>(smem + P.off_misc);
    // The omnigram's home is fixed per instantiation (OG), so the compiler keeps shared-memory
    // accesses as such; everything else of the solve always lives in shared memory.
    E* om = OG ? reinterpret_cast<E*>(gslice + (-(long long)P.loc_om - 1)) : reinterpret_cast<E*>(smem + P.loc_om);
    uint16_t* ord = reinterpret_cast<uint16_t*>(smem + P.loc_ord);
    uint16_t* med = reinterpret_cast<uint16_t*>(smem + P.loc_med);
    uint32_t* shist = reinterpret_cast<uint32_t*>(smem + P.loc_shist);

    // ---- 1. ordinal transform ------------------------------------------------------------------
    stamp(P, tile, 1, G);
    // The footprint: for an interior tile with a staging region, one thread has the tensor memory
    // accelerator copy the whole box (from the 16-byte boundary at or left of its first column)
    // into shared memory, and every thread waits on the mbarrier (bounded: after a timeout the
    // tile, and the CTA's later tiles, read the image instead).
    Footprint<DT> fp{nullptr, 0, 0, Img(P), gx0, gy0};
    if (TMA != 0 && tma != nullptr && P.use_tma && !tma->off) {
        constexpr int A = 16 / (int)sizeof(V);  // elements per 16 bytes
        const int x0 = gx0 & ~(A - 1);
        if (x0 >= 0 && gy0 >= 0 && x0 + P.stage_bw <= P.w && gy0 + P.SH <= P.h) {
            unsigned char* st = smem + P.loc_stage;
            st += (128u - (smem_addr(st) & 127u)) & 127u;  // the region has 128 bytes of slack
            if constexpr (TMA == 1) {  // the single-image kernel: barrier in the scan scratch
                bar = reinterpret_cast<uint64_t*>(misc + 34);
                tmap = &P.tmap;
            }
            if (tid == 0)
                tma_load_box(tmap, st, bar, x0, gy0, (uint32_t)(P.stage_bw * P.SH * (int)sizeof(V)));
            const bool ok = mbar_wait(bar, tma->parity) || mbar_wait(bar, tma->parity);
            tma->parity ^= 1u;
            if (ok) {
                fp.stage = st;
                fp.pitch = P.stage_bw * (int)sizeof(V);
                fp.off = gx0 - x0;
            } else {
                tma->off = 1;
                set_status(FIM_ERR_TIMEOUT);
            }
        }
    }
    // float data always takes the radix sort; 16-bit data takes it in small CTAs, where the
    // counting sort's 65536 bins would keep other CTAs off the SM
    // the sort, compiled for the staged box and for the image (one branch per tile)
    auto sort = [&](auto staged) {
        constexpr bool ST = decltype(staged)::value;
        if constexpr (DT == FIM_F32) {
            if (P.sort == kSortRadix16)
                ordinal_transform_radix<DT, W, true, ST>(P, frow, place<uint32_t>(smem, gslice, P.loc_keys),
                                                         place<typename Loc<W>::Pos>(smem, gslice, P.loc_a),
                                                         place<typename Loc<W>::Pos>(smem, gslice, P.loc_b),
                                                         reinterpret_cast<uint32_t*>(smem + P.loc_hist), misc,
                                                         reinterpret_cast<uint32_t*>(smem + P.loc_bins),
                                                         P.loc_dig >= 0 ? smem + P.loc_dig : nullptr, fp, G);
            else
                ordinal_transform_radix<DT, W, false, ST>(P, frow, place<uint32_t>(smem, gslice, P.loc_keys),
                                                          place<typename Loc<W>::Pos>(smem, gslice, P.loc_a),
                                                          place<typename Loc<W>::Pos>(smem, gslice, P.loc_b),
                                                          reinterpret_cast<uint32_t*>(smem + P.loc_hist), misc,
                                                          nullptr, P.loc_dig >= 0 ? smem + P.loc_dig : nullptr, fp,
                                                          G);
        } else if (DT == FIM_U16 && P.sort == kSortRadix) {
            ordinal_transform_radix<DT, W, false, ST>(P, frow, place<uint32_t>(smem, gslice, P.loc_keys),
                                                      place<typename Loc<W>::Pos>(smem, gslice, P.loc_a),
                                                      place<typename Loc<W>::Pos>(smem, gslice, P.loc_b),
                                                      reinterpret_cast<uint32_t*>(smem + P.loc_hist), misc, nullptr,
                                                      P.loc_dig >= 0 ? smem + P.loc_dig : nullptr, fp, G);
        } else {
            ordinal_transform_count<DT, W, ST>(P, frow, reinterpret_cast<uint32_t*>(smem + P.loc_bins), misc, om, fp,
                                               G);
        }
    };
    if constexpr (TMA != 0) {
        if (fp.stage != nullptr)
            sort(std::true_type{});
        else
            sort(std::false_type{});
    } else {
        sort(std::false_type{});
    }
    G.sync();

    // ---- 2. ordinal image I (Eq. 4) ------------------------------------------------------------
    stamp(P, tile, 2, G);
    if constexpr (OG) {  // omnigram in global scratch: four entries per thread in flight
        for (int v0 = tid; v0 < N; v0 += 4 * nthreads) {
            uint32_t e[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) e[k] = v0 + k * nthreads < N ? (uint32_t)om[v0 + k * nthreads] : 0u;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int v = v0 + k * nthreads;
                if (v < N)
                    ord[(Loc<W>::y(e[k]) + cy0) * SP + Loc<W>::x(e[k]) + cx0] = (uint16_t)clampi(v - rb, 0, 65535);
            }
        }
    } else {
        for (int v = tid; v < N; v += nthreads) {
            const uint32_t e = om[v];
            ord[(Loc<W>::y(e) + cy0) * SP + Loc<W>::x(e) + cx0] = (uint16_t)clampi(v - rb, 0, 65535);
        }
    }
    {   // pad the last 128-bit group with sentinels no window contains
        const int pad = ((N + Loc<W>::kGroup - 1) & ~(Loc<W>::kGroup - 1)) - N;
        if (tid < pad) om[N + tid] = Loc<W>::kSentinel;
    }
    G.sync();

    Member<SHAPE, W> member;
    if constexpr (SHAPE == kShapeDisk) {
        member.r2 = P.r2;
    } else {
        member.spans = spans;
        member.ymin = P.ymin;
        member.nrows = P.nrows;
    }
    // Extras kernels may take several target ranks (percentiles) of one window size: the
    // ordinal transform and the ordinal image above are built once and serve them all.
    const int nr = XT == 1 ? P.nranks : 1;
    // With a percentile map every output pixel has its own target rank. A slide's pivot is the
    // previous window's result, which has exactly that window's target below it, so the count
    // at the pivot after the slide is the previous target plus the change.
    const bool mapped = XT == 2 && P.rank_map != nullptr;
    int Nq = N;  // omnigram length for this target (several radii: the current disk's footprint)
    for (int q = 0; q < nr; ++q) {
        const int target = q == 0 ? P.rank : P.ranks[q];
        // the kernel of this target: the plan's own, or (several radii) the q-th disk's tables
        const int2* qvtab = vtab;
        const int2* qhtab = htab;
        const int* qspans = spans;
        int qn = P.n, qymin = ymin, qnrows = P.nrows, qncols = P.ncols;
        Member<SHAPE, W> qmember = member;
        if constexpr (XT == 1) {
            if (P.multi) {
                qvtab = reinterpret_cast<const int2*>(smem_base + P.q_vtab[q]);
                qhtab = reinterpret_cast<const int2*>(smem_base + P.q_htab[q]);
                qspans = reinterpret_cast<const int*>(smem_base + P.q_spans[q]);
                qn = P.q_n[q];
                qymin = P.q_ymin[q];
                qnrows = P.q_nrows[q];
                qncols = P.q_ncols[q];
                if constexpr (SHAPE == kShapeDisk) {
                    qmember.r2 = P.q_r2[q];
                } else {
                    qmember.spans = qspans;
                    qmember.ymin = qymin;
                    qmember.nrows = qnrows;
                }
                // targets come largest disk first: narrow the omnigram to this disk's footprint
                if (P.q_N[q] < Nq) {
                    const int kept = compact_omnigram<W>(om, Nq, reinterpret_cast<const int*>(smem_base + P.q_frow[q]),
                                                         ord, SP, cx0, cy0, misc, G, nthreads, nwarps);
                    if (kept != P.q_N[q]) set_status(FIM_ERR_INTERNAL);
                    Nq = P.q_N[q];
                }
            }
        }
        const int qhist_shift = XT == 1 && P.multi ? P.q_hshift[q] : hist_shift;
        const int BH = TY / P.RB;      // band height
        const int GW = TX / P.G;       // seed spacing within a seed row
        // feasible median ranks of any window of this tile (Fig. 10): [lof, hif]
        const int lof = target, hif = Nq - qn + target;

        // ---- 3. seeds: coarse histogram of I over the window, then ballot refine ----------------
        // (or, with a learned bracket, two exact counts at predicted ranks, then ballot refine)
        stamp(P, tile, 3, G);
        const bool learned = XT == 1 && P.model != nullptr;
        const bool sampling = XT == 1 && P.samples != nullptr;
        const bool counting = XT == 1 && P.stats != nullptr;
        float* quant = reinterpret_cast<float*>(misc);  // the sort's scan scratch is free from here on
        if (learned || sampling) {
            if (warp == 0) {  // normalised value quantiles of the footprint: C at N (j + 1/2) / 32
                const int q = min(Nq - 1, (int)(((long long)Nq * (2 * lane + 1)) / (2 * kQuantiles)));
                const uint32_t e = om[q];
                const float v = (float)load_px<DT>(Img(P), gx0 + Loc<W>::x(e) + cx0, gy0 + Loc<W>::y(e) + cy0);
                const float mid = __shfl_sync(kFull, v, kQuantiles / 2);
                const float spread = __shfl_sync(kFull, v, 7 * kQuantiles / 8) - __shfl_sync(kFull, v, kQuantiles / 8);
                const float z = (v - mid) / (spread > 0.f ? spread : 1.f);
                quant[lane] = fminf(fmaxf(z, -8.f), 8.f);
            }
            G.sync();
        }
        const int nseeds = P.RB * P.G;
        static_assert(kHidden <= kSeedBins, "the quantiles' layer-1 pre-activations fit one seed histogram");
        if (learned) {
            // Learned bracket (extension): the layer-1 contribution of the tile's quantiles is
            // computed once, block-wide; then each warp takes one seed at a time and, with no
            // further block barrier, evaluates the bracket MLP for it (lanes hold hidden units
            // lane and lane + 32, activations move by shuffles), counts the window's ranks below
            // the predicted median, and walks Omega 512 entries a step from there to the exact
            // median. It replaces the plain seeds' histogram or long walk.
            const uint16_t* wts =
                P.off_model >= 0 ? reinterpret_cast<const uint16_t*>(smem_base + P.off_model) : P.model;
            float* hbase = reinterpret_cast<float*>(shist);  // layer-1 pre-activation of the quantiles
            for (int j = tid; j < kHidden; j += nthreads) {
                float h = bf16_to_f32(wts[kOffB1 + j]);
                for (int i = 0; i < kQuantiles; ++i) h = fmaf(quant[i], bf16_to_f32(wts[kOffW1 + i * kHidden + j]), h);
                hbase[j] = h;
            }
            G.sync();
            for (int sd = warp; sd < nseeds; sd += nwarps) {
                const int band = sd / P.G, g = sd % P.G;
                const int s = g * GW + GW / 2, t = band * BH + BH / 2;
                const int cu = s - xmin, cv = t - ymin;
                float fa, fb;
                seed_features(ord, SP, frow, P.SH, Nq, cu, cv, quant, &fa, &fb);
                float a0 = hbase[lane], a1 = hbase[lane + 32];
#pragma unroll
                for (int i = 0; i < kNeigh; ++i) {
                    const float x = __shfl_sync(kFull, fb, i);
                    a0 = fmaf(x, bf16_to_f32(wts[kOffW1 + (kQuantiles + i) * kHidden + lane]), a0);
                    a1 = fmaf(x, bf16_to_f32(wts[kOffW1 + (kQuantiles + i) * kHidden + lane + 32]), a1);
                }
                a0 = fmaxf(a0, 0.f);
                a1 = fmaxf(a1, 0.f);
                float b0 = bf16_to_f32(wts[kOffB2 + lane]), b1 = bf16_to_f32(wts[kOffB2 + lane + 32]);
#pragma unroll 8
                for (int k = 0; k < kHidden; ++k) {
                    const float x = __shfl_sync(kFull, k < 32 ? a0 : a1, k & 31);
                    b0 = fmaf(x, bf16_to_f32(wts[kOffW2 + k * kHidden + lane]), b0);
                    b1 = fmaf(x, bf16_to_f32(wts[kOffW2 + k * kHidden + lane + 32]), b1);
                }
                b0 = fmaxf(b0, 0.f);
                b1 = fmaxf(b1, 0.f);
                float o0 = bf16_to_f32(wts[kOffW3 + lane * 2]) * b0 + bf16_to_f32(wts[kOffW3 + (lane + 32) * 2]) * b1;
                float o1 = bf16_to_f32(wts[kOffW3 + lane * 2 + 1]) * b0 + bf16_to_f32(wts[kOffW3 + (lane + 32) * 2 + 1]) * b1;
                for (int o = 16; o > 0; o >>= 1) {
                    o0 += __shfl_xor_sync(kFull, o0, o);
                    o1 += __shfl_xor_sync(kFull, o1, o);
                }
                o0 += bf16_to_f32(wts[kOffB3]);
                o1 += bf16_to_f32(wts[kOffB3 + 1]);
                const float sig = __expf(fminf(fmaxf(o1, -8.f), 2.f)) * P.bracket_z;
                const float span = (float)(hif - lof);
                const int lo = clampi(__float2int_rn(lof + (o0 - sig) * span), 0, Nq - 1);
                const int hi = clampi(__float2int_rn(lof + (o0 + sig) * span), lo, Nq - 1);
                // (pivots stay in the feasible ranks, where the ordinal image's ranks compare exactly)
                const int pivot = clampi(clampi(__float2int_rn(lof + o0 * span), lo, hi), lof, hif);
                // The count at the predicted median is exact, so the walk from it finds the exact
                // median wherever it lies: on a miss it simply walks past the bracket, over the
                // full range if need be. The bracket ends only classify the outcome.
                const int below = window_rows_below(qspans, qnrows, ord + (cv + qymin) * SP + cu, SP, pivot - rb);
                const int m = wide_select<SHAPE, W>(om, Nq, pivot, below, target, cu - cx0, cv - cy0, qmember);
                if (m < 0) set_status(FIM_ERR_INTERNAL);
                if (lane == 0) med[t * TX + s] = (uint16_t)(max(m, 0) - rb);
                if (counting && lane == 0) {
                    const int kind = m < lo ? 2 : (m > hi ? 3 : 1);
                    atomicAdd(P.stats + 0, 1ull);
                    atomicAdd(P.stats + kind, 1ull);
                    atomicAdd(P.stats + 4, (unsigned long long)abs(max(m, 0) - pivot));
                }
            }
        } else {
            for (int sd = warp; sd < nseeds; sd += nwarps) {
                const int band = sd / P.G, g = sd % P.G;
                const int s = g * GW + GW / 2, t = band * BH + BH / 2;  // tile-local output pixel
                const int cu = s - xmin, cv = t - ymin;                 // window centre in the box
                float fa = 0.f, fb = 0.f;
                if (sampling) seed_features(ord, SP, frow, P.SH, Nq, cu, cv, quant, &fa, &fb);
                const int ts = mapped ? map_rank(P, tx0 + s, ty0 + t) : target;
                int pivot = 0, below = 0, m;
                if (P.seed_mode == kSeedHistogram) {
                    // a coarse histogram of the window's ranks (one per concurrently solved seed),
                    // scanned to the bin of the target, then a ballot scan of Omega from that bin
                    uint32_t* hw = shist + (nwarps >= nseeds ? sd : warp) * kSeedBins;
                    for (int j = lane; j < kSeedBins; j += 32) hw[j] = 0;
                    __syncwarp();
                    window_walk(qspans, qnrows, ord + (cv + qymin) * SP + cu, SP,
                                [&](int r) { atomicAdd(&hw[r >> qhist_shift], 1u); });
                    __syncwarp();
                    pivot = hist_pick(hw, 0, ts, &below) << qhist_shift;
                    m = ballot_select(om, Nq, pivot, below, ts, cu - cx0, cv - cy0, qmember);
                } else {
                    if (P.seed_mode == kSeedWalk) {
                        // walk Omega from whichever end is known exactly: nothing lies below
                        // rank 0, and all n members lie below rank N
                        if (2 * ts >= qn) {
                            pivot = Nq;
                            below = qn;
                        }
                    } else {
                        // count the window below the middle of the tile's feasible ranks, walk from there
                        pivot = (lof + hif) >> 1;
                        below = window_rows_below(qspans, qnrows, ord + (cv + qymin) * SP + cu, SP, pivot - rb);
                    }
                    m = wide_select<SHAPE, W>(om, Nq, pivot, below, ts, cu - cx0, cv - cy0, qmember);
                }
                if (m < 0) set_status(FIM_ERR_INTERNAL);
                if (lane == 0) med[t * TX + s] = (uint16_t)(max(m, 0) - rb);
                if (sampling) {  // training row: features and the exact median's place in [lof, hif]
                    unsigned int row = 0;
                    if (lane == 0) row = atomicAdd(P.sample_count, 1u);
                    row = __shfl_sync(kFull, row, 0);
                    if ((int)row < P.sample_cap) {
                        float* dst = P.samples + (size_t)row * (kFeatures + 1);
                        dst[lane] = fa;
                        if (lane < kNeigh) dst[kQuantiles + lane] = fb;
                        if (lane == 0) dst[kFeatures] = hif > lof ? (float)(max(m, 0) - lof) / (float)(hif - lof) : 0.5f;
                    }
                }
                if (counting && lane == 0) {
                    atomicAdd(P.stats + 0, 1ull);
                    atomicAdd(P.stats + 4, (unsigned long long)abs(max(m, 0) - pivot));
                }
                __syncwarp();
            }
        }
        G.sync();

        // ---- 4. seed rows: horizontal slides, lanes split the kernel rows ----------------------
        stamp(P, tile, 4, G);
        for (int job = warp; job < 2 * P.RB * P.G; job += nwarps) {
            const int sd = job >> 1, right = job & 1;
            const int band = sd / P.G, g = sd % P.G;
            int s = g * GW + GW / 2;
            const int t = band * BH + BH / 2;
            const int steps = right ? (GW - GW / 2 - 1) : (GW / 2);
            int cu = s - xmin;
            const int cv = t - ymin;
            int p = med[t * TX + s] + rb;
            constexpr int kRowsPerLane = (kMaxExtent + 31) / 32;
            int eo[kRowsPerLane], lo[kRowsPerLane];  // this lane's rows: entering / leaving offsets
    #pragma unroll
            for (int q = 0; q < kRowsPerLane; ++q) {
                const int i = lane + 32 * q;
                eo[q] = lo[q] = 0;  // rows beyond the kernel compare the centre with itself: no change
                if (i < qnrows) {
                    const int2 o = qhtab[i];
                    eo[q] = right ? o.y : o.x - 1;
                    lo[q] = right ? o.x : o.y - 1;
                }
            }
            for (int k = 0; k < steps; ++k) {
                const uint16_t* ctr = ord + cv * SP + cu;
                const int pr = p - rb;  // the pivot among the ordinal image's ranks
                int d = 0;
    #pragma unroll
                for (int q = 0; q < kRowsPerLane; ++q)
                    if (32 * q < qnrows) d += (int)(ctr[eo[q]] < pr) - (int)(ctr[lo[q]] < pr);
                d = __reduce_add_sync(kFull, d);
                // targets of the pivot's window and of the next one (re-read: no extra live state)
                const int tp = mapped ? map_rank(P, tx0 + s, ty0 + t) : target;
                cu += right ? 1 : -1;
                s += right ? 1 : -1;
                const int tn = mapped ? map_rank(P, tx0 + s, ty0 + t) : target;
                const int m = ballot_select(om, Nq, p, tp + d, tn, cu - cx0, cv - cy0, qmember);
                if (m < 0) set_status(FIM_ERR_INTERNAL);
                p = max(m, 0);
                if (lane == 0) med[t * TX + s] = (uint16_t)(p - rb);
            }
        }
        G.sync();

        // ---- 5. vertical sweeps: thread per window column, per-thread refinement ----------------
        // ---- 6. output, fused: out = C[m], the input value at Omega[m] --------------------------
        // Each sweep thread writes the pixels it solves (the downward threads also the seed row's
        // pixel they start from). The gather of a pixel's value is issued right after its solve
        // and its store waits for the next step, so the L2 latency of the scattered gathers hides
        // behind the next slide instead of queueing at the end of the tile.
        stamp(P, tile, 5, G);
        if (warp < P.vthreads / 32) {
            const int groups = TX / 32;
            const int cg = warp % groups;
            const int rest = warp / groups;
            const int vmix = XT == 1 && P.multi ? P.q_vmix[q] : P.vmix;
            const int band = vmix ? (rest + lane) % P.RB : rest % P.RB;  // per lane with mixing
            const int down = rest / P.RB;  // 0: up, 1: down
            const int s = cg * 32 + lane;
            int t = band * BH + BH / 2;
            const int steps = down ? (BH - BH / 2 - 1) : (BH / 2);
            const int cu = s - xmin;
            int cv = t - ymin;
            int p = med[t * TX + s] + rb;
            const int ncols = qncols;
            const int scan_groups = P.scan_groups;
            const int eoff = down ? 0 : -SP;
            const Img im(P);
            char* const out = static_cast<char*>(q == 0 ? P.out : P.outs[q]);
            const int gx = tx0 + s;
            V pval = V(0);       // value gathered for the last solved pixel, not yet stored
            V* pdst = nullptr;   // where it goes (null: outside the image, or nothing pending)
            auto gather = [&](int m, int tt) {
                const uint32_t e = om[m];
                pval = load_px<DT>(im, gx0 + Loc<W>::x(e) + cx0, gy0 + Loc<W>::y(e) + cy0);
                const int gy = ty0 + tt;
                pdst = (gx < im.w && gy < im.h) ? reinterpret_cast<V*>(out + (long long)gy * im.pitch) + gx : nullptr;
            };
            if (down) gather(p, t);  // the seed row's pixel
            for (int k = 0; k < steps; ++k) {
                const uint16_t* ctr = ord + cv * SP + cu + eoff;
                const int pr = p - rb;  // the pivot among the ordinal image's ranks
                int d = 0;
                // slide unrolled 8 kernel columns deep in the kernels compiled for the 1024-thread
                // tiles (KS = 8), 4 in the others (measured, 4096^2 u16: r = 32-64 +1.2-1.8 % over
                // 4; r = 2-16 -3 to -11 %; KS = 0 kernels serve small CTAs too)
                constexpr int kSlideUnroll = KS == 8 ? 8 : 4;
                if (down) {
    #pragma unroll kSlideUnroll
                    for (int j = 0; j < ncols; ++j) {
                        const int2 o = qvtab[j];
                        d += (int)(ctr[o.y] < pr) - (int)(ctr[o.x] < pr);
                    }
                } else {
    #pragma unroll kSlideUnroll
                    for (int j = 0; j < ncols; ++j) {
                        const int2 o = qvtab[j];
                        d += (int)(ctr[o.x] < pr) - (int)(ctr[o.y] < pr);
                    }
                }
                const int tp = mapped ? map_rank(P, tx0 + s, ty0 + t) : target;
                cv += down ? 1 : -1;
                t += down ? 1 : -1;
                const int tn = mapped ? map_rank(P, tx0 + s, ty0 + t) : target;
                const int mine =
                    thread_select<SHAPE, W, KS>(om, Nq, p, tp + d, tn, cu - cx0, cv - cy0, qmember, scan_groups);
                if (mine < 0) set_status(FIM_ERR_INTERNAL);
                p = max(mine, 0);
                if (pdst) *pdst = pval;  // the previous pixel's value has arrived by now
                gather(p, t);
            }
            if (pdst) *pdst = pval;
        }
        stamp(P, tile, 6, G);  // the first group thread's own sweep is done (output is fused into it)
        G.sync();
        stamp(P, tile, 7, G);
    }
}

__device__ __forceinline__ void load_tables(const Plan& P) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int tid = threadIdx.x, nt = blockDim.x;
    int2* vtab = reinterpret_cast<int2*>(smem + P.off_vtab);
    int2* htab = reinterpret_cast<int2*>(smem + P.off_htab);
    int* spans = reinterpret_cast<int*>(smem + P.off_spans);
    int* frow = reinterpret_cast<int*>(smem + P.off_frow);
    for (int i = tid; i < P.ncols; i += nt) vtab[i] = make_int2(P.vtab[2 * i], P.vtab[2 * i + 1]);
    for (int i = tid; i < P.nrows; i += nt) {
        htab[i] = make_int2(P.htab[2 * i], P.htab[2 * i + 1]);
        spans[i] = P.spans[i];
    }
    for (int i = tid; i < P.SH; i += nt) frow[i] = P.frow[i];
    if (P.xtab != nullptr) {
        int* xt = reinterpret_cast<int*>(smem + P.off_xtab);
        for (int i = tid; i < P.xtab_words; i += nt) xt[i] = P.xtab[i];
    }
    if (P.off_model >= 0 && P.model != nullptr) {  // kMlpParams is even: copy 32-bit pairs
        const uint32_t* src = reinterpret_cast<const uint32_t*>(P.model);
        uint32_t* dst = reinterpret_cast<uint32_t*>(smem + P.off_model);
        for (int i = tid; i < kMlpParams / 2; i += nt) dst[i] = src[i];
    }
}

}  // namespace
}  // namespace fim
