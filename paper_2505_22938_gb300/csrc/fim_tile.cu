// Per-tile median kernel: one CTA filters one Tx x Ty output tile (Sec. 3.3, Sec. 4.2).
//
// Phases, separated by __syncthreads():
//   1. ordinal transform - the rounded-rectangle footprint (Fig. 10) is read with clamp-to-edge
//                        and key-value sorted by value, giving the omnigram Omega (Sec. 3.3):
//                          8/16-bit data: counting sort over 256 / 65536 shared-memory bins, the
//                                         bucket construction of Eq. 5 run by all threads;
//                          float data:    stable LSD radix sort of order-preserving keys
//                                         (Sec. 4.1 float key), four 8-bit passes.
//   2. ordinal image   - I(Omega[v]) = v (Eq. 4), exact 16-bit ranks.
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

// Diagnostics: thread 0 records clock64() at phase boundaries when a buffer is attached.
__device__ __forceinline__ void stamp(const Plan& P, int phase) {
    if (P.phase_clock != nullptr && threadIdx.x == 0 && (int)blockIdx.x < P.phase_tiles)
        P.phase_clock[blockIdx.x * 8 + phase] = clock64();
}

__device__ __forceinline__ int span_lo(int s) { return (int)(int16_t)(s & 0xffff); }
__device__ __forceinline__ int span_hi(int s) { return s >> 16; }

__device__ __forceinline__ uint16_t pack_loc(int u, int v, const Plan& P) {
    return (uint16_t)((uint32_t)(uint8_t)(int8_t)(u - P.cx0) | ((uint32_t)(uint8_t)(int8_t)(v - P.cy0) << 8));
}

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
        return dx >= span_lo(s) && dx <= span_hi(s);
    }
};

// Membership of the two omnigram entries packed in one 32-bit word (entry 2k in the low half,
// entry 2k+1 in the high half). Returns bit 0 / bit 1 for the low / high entry.
// For the disk, (x-px)^2 + (y-py)^2 <= r2 is evaluated as x^2 + y^2 - 2(x px + y py) <= R with
// R = r2 - px^2 - py^2, using byte dot products on the packed int8 coordinates.
template <int SHAPE>
struct Member2;

template <>
struct Member2<kShapeDisk> {
    int R;
    int plo, phi;  // (px, py, 0, 0) and (0, 0, px, py) as signed bytes
    __device__ __forceinline__ void set(int r2, int px, int py) {
        R = r2 - px * px - py * py;
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

template <>
struct Member2<kShapeSpans> {
    Member<kShapeSpans> m;
    int px, py;
    __device__ __forceinline__ uint32_t operator()(uint32_t w) const {
        return (uint32_t)m(w & 0xffffu, px, py) | ((uint32_t)m(w >> 16, px, py) << 1);
    }
};

// Exact selection, 64 omnigram entries per iteration (two per lane from one 32-bit load).
// Same contract as ballot_select below. Entries are taken in rank order: lane l holds ranks
// 2(k+l) and 2(k+l)+1 of the word block starting at word k.
template <class M2>
__device__ __forceinline__ int ballot_select64(const uint16_t* __restrict__ om, int N, int p, int c, int target,
                                               const M2& member2) {
    const int lane = threadIdx.x & 31;
    const uint32_t* om32 = reinterpret_cast<const uint32_t*>(om);
    const int nw = (N + 1) >> 1;
    if (c <= target) {  // the answer is at or above p
        int need = target - c + 1;
        for (int k = p >> 1; k < nw; k += 32) {
            const int kk = k + lane;
            const int e = 2 * kk;
            uint32_t bits = kk < nw ? member2(om32[kk]) : 0u;
            bits &= (uint32_t)(e >= p && e < N) | ((uint32_t)(e + 1 >= p && e + 1 < N) << 1);
            const uint32_t b0 = __ballot_sync(kFull, bits & 1u);
            const uint32_t b1 = __ballot_sync(kFull, bits & 2u);
            const int cnt = __popc(b0) + __popc(b1);
            if (cnt >= need) {
                const uint32_t lt = lanemask_lt();
                const int before = __popc(b0 & lt) + __popc(b1 & lt);
                const int m0 = bits & 1u, m1 = (bits >> 1) & 1u;
                const int sel = (m0 && before + 1 == need) ? 0 : ((m1 && before + m0 + 1 == need) ? 1 : -1);
                const uint32_t hit = __ballot_sync(kFull, sel >= 0);
                const int wl = __ffs(hit) - 1;
                return 2 * (k + wl) + __shfl_sync(kFull, sel, wl);
            }
            need -= cnt;
        }
    } else {  // the answer is below p: walk down, the need-th member met is the answer
        int need = c - target;
        for (int k1 = (p - 1) >> 1; k1 >= 0; k1 -= 32) {
            const int kk = k1 - 31 + lane;
            const int e = 2 * kk;
            uint32_t bits = kk >= 0 ? member2(om32[kk]) : 0u;
            bits &= (uint32_t)(kk >= 0 && e < p) | ((uint32_t)(kk >= 0 && e + 1 < p) << 1);
            const uint32_t b0 = __ballot_sync(kFull, bits & 1u);
            const uint32_t b1 = __ballot_sync(kFull, bits & 2u);
            const int cnt = __popc(b0) + __popc(b1);
            if (cnt >= need) {
                const uint32_t gt = ~lanemask_le();
                const int above = __popc(b0 & gt) + __popc(b1 & gt);
                const int m0 = bits & 1u, m1 = (bits >> 1) & 1u;
                const int sel = (m1 && above + 1 == need) ? 1 : ((m0 && above + m1 + 1 == need) ? 0 : -1);
                const uint32_t hit = __ballot_sync(kFull, sel >= 0);
                const int wl = __ffs(hit) - 1;
                return 2 * (k1 - 31 + wl) + __shfl_sync(kFull, sel, wl);
            }
            need -= cnt;
        }
    }
    return -1;
}

#ifndef FIM_REFINE
#define FIM_REFINE 1
#endif
#ifndef FIM_VREFINE
#define FIM_VREFINE 1
#endif

template <int SHAPE>
__device__ __forceinline__ Member2<SHAPE> make_member2(const Member<SHAPE>& m, int px, int py, int r2) {
    Member2<SHAPE> m2;
    if constexpr (SHAPE == kShapeDisk) {
        m2.set(r2, px, py);
    } else {
        m2.m = m;
        m2.px = px;
        m2.py = py;
    }
    return m2;
}

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

// Per-thread exact selection (vertical sweep): every lane refines its own window. It scans the
// omnigram from its pivot in aligned groups of 8 entries (one 128-bit load), counting members
// with the packed-pair test, until the group holding the target-th member. While at least
// kHandoff lanes are still scanning this is the cheapest schedule; the last few lanes of a warp
// (long jumps at edges and impulses) are finished by warp-cooperative ballot scans instead of
// keeping 29+ lanes idle. Same contract as ballot_select, per lane. All loops are bounded by
// the omnigram length.
constexpr int kHandoff = 4;
constexpr int kHandoffAfter = 16;  // groups of 8 entries

template <int SHAPE>
__device__ __forceinline__ int thread_select(const uint16_t* __restrict__ om, int N, int p, int c, int target,
                                             int px, int py, const Member<SHAPE>& member, int r2) {
    const int lane = threadIdx.x & 31;
    const Member2<SHAPE> member2 = make_member2<SHAPE>(member, px, py, r2);
    const uint4* om128 = reinterpret_cast<const uint4*>(om);
    const bool up = c <= target;
    int need = up ? target - c + 1 : c - target;
    int nextv = up ? p : p - 1;      // next omnigram entry to examine
    const int glast = (N - 1) >> 3;
    bool done = false;
    int m = -1;
    for (int it = 0; it <= glast + 1; ++it) {
        // the hand-off test costs a vote, so it only starts once the typical scan is over
        if (it >= kHandoffAfter && __popc(__ballot_sync(kFull, !done)) < kHandoff) break;
        if (it < kHandoffAfter && !__any_sync(kFull, !done)) break;
        if (!done) {
            const int g = nextv >> 3;
            if (g < 0 || g > glast) {
                done = true;
            } else {
                const uint4 q = om128[g];
                uint32_t mask = member2(q.x) | (member2(q.y) << 2) | (member2(q.z) << 4) | (member2(q.w) << 6);
                mask &= up ? (0xffu << (nextv & 7)) & 0xffu : (0xffu >> (7 - (nextv & 7)));
                if (g == glast) mask &= 0xffu >> (7 - ((N - 1) & 7));
                const int cnt = __popc(mask);
                if (cnt >= need) {
                    if (up) {
                        for (int k = 1; k < need; ++k) mask &= mask - 1;  // drop the lowest need-1
                        m = 8 * g + __ffs(mask) - 1;
                    } else {
                        for (int k = 1; k < need; ++k) mask ^= 1u << (31 - __clz(mask));  // drop the highest
                        m = 8 * g + 31 - __clz(mask);
                    }
                    done = true;
                } else {
                    need -= cnt;
                    nextv = up ? 8 * g + 8 : 8 * g - 1;
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
        const int pj = upj ? nj : nj + 1;
        const int cj = upj ? target + 1 - needj : target + needj;
        const int mj = ballot_select(om, N, pj, cj, target, pxj, py, member);
        if (lane == j) m = mj;
    }
    return m;
}

// Refinement entry point used by every phase: exact rank of the target-th window member.
template <int SHAPE>
__device__ __forceinline__ int refine(const uint16_t* __restrict__ om, int N, int p, int c, int target, int px,
                                      int py, const Member<SHAPE>& member, int r2) {
#if FIM_REFINE == 1
    return ballot_select(om, N, p, c, target, px, py, member);
#else
    return ballot_select64(om, N, p, c, target, make_member2<SHAPE>(member, px, py, r2));
#endif
}

// Block-wide exclusive scan of 65536 16-bit counters packed two per word (bin 2k in the low
// half of word k). Offsets stay below 2^16 because the footprint holds at most 65535 pixels.
__device__ void scan_bins16(uint32_t* bins, const Plan& P) {
    __shared__ uint32_t wtot[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
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
    __syncthreads();
    if (warp == 0) {
        const uint32_t x = lane < P.nwarps ? wtot[lane] : 0;
        uint32_t incl = x;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(kFull, incl, o);
            if (lane >= o) incl += t;
        }
        wtot[lane] = incl - x;
    }
    __syncthreads();
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
}

template <int DT>
__device__ __forceinline__ typename Traits<DT>::T load_px(const char* in, const Plan& P, int gx, int gy) {
    using V = typename Traits<DT>::T;
    const V* row = reinterpret_cast<const V*>(in + (long long)clampi(gy, 0, P.h - 1) * P.pitch);
    return __ldg(row + clampi(gx, 0, P.w - 1));
}

// Counting-sort ordinal transform for 8/16-bit data (Sec. 4.1, Eq. 5): histogram of the
// footprint, exclusive prefix, then every pixel takes the next free ordinal of its value.
// Ties get consecutive ordinals in arrival order, which is all the method needs.
template <int DT>
__device__ void ordinal_transform_count(const Plan& P, const int* frow, uint16_t* om, int gx0, int gy0) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    uint32_t* bins = reinterpret_cast<uint32_t*>(smem + P.off_bins);
    const char* in = static_cast<const char*>(P.in);
    constexpr bool k16 = DT == FIM_U16;
    const int nwords = k16 ? 32768 : 256;
    for (int i = tid * 4; i < nwords; i += P.threads * 4)
        *reinterpret_cast<uint4*>(bins + i) = make_uint4(0, 0, 0, 0);
    __syncthreads();
    for (int v = warp; v < P.SH; v += P.nwarps) {
        const int fr = frow[v];
        for (int u = span_lo(fr) + lane; u <= span_hi(fr); u += 32) {
            const uint32_t key = Traits<DT>::key(load_px<DT>(in, P, gx0 + u, gy0 + v));
            if (k16)
                atomicAdd(&bins[key >> 1], 1u << ((key & 1u) << 4));
            else
                atomicAdd(&bins[key], 1u);
        }
    }
    __syncthreads();
    if (k16) {
        scan_bins16(bins, P);
    } else if (warp == 0) {
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
    __syncthreads();
    for (int v = warp; v < P.SH; v += P.nwarps) {
        const int fr = frow[v];
        for (int u = span_lo(fr) + lane; u <= span_hi(fr); u += 32) {
            const uint32_t key = Traits<DT>::key(load_px<DT>(in, P, gx0 + u, gy0 + v));
            uint32_t o;
            if (k16) {
                const uint32_t sh = (key & 1u) << 4;
                o = (atomicAdd(&bins[key >> 1], 1u << sh) >> sh) & 0xffffu;
            } else {
                o = atomicAdd(&bins[key], 1u);
            }
            om[o] = pack_loc(u, v, P);
        }
    }
}

// Stable LSD radix ordinal transform for 32-bit keys (float data): four 8-bit passes over
// bounding-box positions. Each warp owns one contiguous segment of the current order; a
// pixel's new place is its (digit, warp)-major exclusive offset plus its position among
// equal digits earlier in the segment (warp match). Histograms are laid out warp-major with
// a pad word so that the leaders of one warp never share a bank.
template <int DT>
__device__ void ordinal_transform_radix(const Plan& P, const int* frow, uint16_t* om, int gx0, int gy0) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ uint32_t wsum[32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nthreads = P.threads, nwarps = P.nwarps, S = P.S;
    constexpr int HS = kSortBins + 1;
    uint32_t* keys = reinterpret_cast<uint32_t*>(smem + P.off_keys);
    uint16_t* bufA = reinterpret_cast<uint16_t*>(smem + P.off_a);
    uint16_t* bufB = reinterpret_cast<uint16_t*>(smem + P.off_b);
    uint32_t* hist = reinterpret_cast<uint32_t*>(smem + P.off_hist);
    const char* in = static_cast<const char*>(P.in);
    for (int v = warp; v < P.SH; v += nwarps) {
        const int fr = frow[v];
        for (int u = span_lo(fr) + lane; u <= span_hi(fr); u += 32)
            keys[v * S + u] = Traits<DT>::key(load_px<DT>(in, P, gx0 + u, gy0 + v));
    }
    __syncthreads();
    const int area = S * P.SH;
    const uint16_t* src = nullptr;
    uint16_t* dst = bufA;
    for (int pass = 0; pass < 4; ++pass) {
        const int shift = 8 * pass;
        const int len = pass == 0 ? area : P.N;
        const int seg = ((len + nwarps - 1) / nwarps + 31) & ~31;
        const int s0 = min(len, warp * seg), s1 = min(len, s0 + seg);
        uint32_t* hw = hist + warp * HS;
        for (int d = lane; d < kSortBins; d += 32) hw[d] = 0;
        __syncwarp();
        for (int b = s0; b < s1; b += 32) {
            const int i = b + lane;
            bool valid = i < s1;
            int pos = 0;
            if (valid) {
                if (pass == 0) {
                    const int v = (int)__umulhi((unsigned)i, P.div_magic);
                    const int u = i - v * S;
                    const int fr = frow[v];
                    valid = u >= span_lo(fr) && u <= span_hi(fr);
                    pos = i;
                } else {
                    pos = src[i];
                }
            }
            const int d = valid ? (int)(keys[pos] >> shift) & 0xff : kSortBins + lane;
            const uint32_t peers = __match_any_sync(kFull, d);
            if (valid && lane == __ffs(peers) - 1) hw[d] += __popc(peers);
            __syncwarp();
        }
        __syncthreads();
        {   // exclusive scan in (digit, warp) order: each thread takes 8 consecutive counters
            const int e0 = tid * 8;  // 256 * nwarps counters over 32 * nwarps threads
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
            __syncthreads();
            if (warp == 0) {
                const uint32_t x = lane < nwarps ? wsum[lane] : 0;
                uint32_t y = x;
                for (int o = 1; o < 32; o <<= 1) {
                    const uint32_t t = __shfl_up_sync(kFull, y, o);
                    if (lane >= o) y += t;
                }
                wsum[lane] = y - x;
            }
            __syncthreads();
            uint32_t run = incl - local + wsum[warp];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int e = e0 + j, d = e / nwarps, wq = e - d * nwarps;
                hist[wq * HS + d] = run;
                run += c[j];
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
                    const int fr = frow[v];
                    valid = u >= span_lo(fr) && u <= span_hi(fr);
                    pos = i;
                } else {
                    pos = src[i];
                }
            }
            const int d = valid ? (int)(keys[pos] >> shift) & 0xff : kSortBins + lane;
            const uint32_t peers = __match_any_sync(kFull, d);
            uint32_t base = 0;
            if (valid) base = hw[d];
            __syncwarp();
            if (valid) {
                dst[base + __popc(peers & lanemask_lt())] = (uint16_t)pos;
                if (lane == __ffs(peers) - 1) hw[d] = base + __popc(peers);
            }
            __syncwarp();
        }
        __syncthreads();
        src = dst;
        dst = (dst == bufA) ? bufB : bufA;
    }
    // four passes: the sorted positions are in B; the omnigram goes to A
    for (int v = tid; v < P.N; v += nthreads) {
        const int pos = src[v];
        const int y = (int)__umulhi((unsigned)pos, P.div_magic);
        om[v] = pack_loc(pos - y * S, y, P);
    }
}

template <int DT, int SHAPE>
__global__ void __launch_bounds__(1024, 1) tile_median_kernel(const __grid_constant__ Plan P) {
    using V = typename Traits<DT>::T;
    extern __shared__ __align__(16) unsigned char smem[];

    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int warp = tid >> 5;
    const int nthreads = P.threads;
    const int nwarps = P.nwarps;
    const int SP = P.SP, N = P.N, TX = P.Tx, TY = P.Ty;
    const int tile = blockIdx.x;
    const int tx0 = (tile % P.tiles_x) * TX;
    const int ty0 = (tile / P.tiles_x) * TY;
    const int gx0 = tx0 + P.xmin;  // global coordinates of bounding-box pixel (0, 0)
    const int gy0 = ty0 + P.ymin;

    int2* vtab = reinterpret_cast<int2*>(smem + P.off_vtab);
    int2* htab = reinterpret_cast<int2*>(smem + P.off_htab);
    int* spans = reinterpret_cast<int*>(smem + P.off_spans);
    int* frow = reinterpret_cast<int*>(smem + P.off_frow);
    uint16_t* om = reinterpret_cast<uint16_t*>(smem + P.off_om);
    uint16_t* ord = reinterpret_cast<uint16_t*>(smem + P.off_ord);
    uint16_t* med = reinterpret_cast<uint16_t*>(smem + P.off_med);
    uint32_t* shist = reinterpret_cast<uint32_t*>(smem + P.off_shist);

    stamp(P, 0);
    for (int i = tid; i < P.ncols; i += nthreads) vtab[i] = make_int2(P.vtab[2 * i], P.vtab[2 * i + 1]);
    for (int i = tid; i < P.nrows; i += nthreads) {
        htab[i] = make_int2(P.htab[2 * i], P.htab[2 * i + 1]);
        spans[i] = P.spans[i];
    }
    for (int i = tid; i < P.SH; i += nthreads) frow[i] = P.frow[i];
    __syncthreads();

    // ---- 1. ordinal transform ------------------------------------------------------------------
    stamp(P, 1);
    if constexpr (DT == FIM_F32)
        ordinal_transform_radix<DT>(P, frow, om, gx0, gy0);
    else
        ordinal_transform_count<DT>(P, frow, om, gx0, gy0);
    __syncthreads();

    // ---- 2. ordinal image I (Eq. 4) ------------------------------------------------------------
    stamp(P, 2);
    for (int v = tid; v < N; v += nthreads) {
        const uint32_t e = om[v];
        const int u = (int)(int8_t)(e & 0xffu) + P.cx0;
        const int y = (int)(int8_t)(e >> 8) + P.cy0;
        ord[y * SP + u] = (uint16_t)v;
    }
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
    const int BH = TY / P.RB;      // band height
    const int GW = TX / P.G;       // seed spacing within a seed row

    // ---- 3. seeds: coarse histogram of I over the window, then ballot refine ----------------
    stamp(P, 3);
    for (int sd = warp; sd < P.RB * P.G; sd += nwarps) {
        const int band = sd / P.G, g = sd % P.G;
        const int s = g * GW + GW / 2, t = band * BH + BH / 2;  // tile-local output pixel
        const int cu = s - P.xmin, cv = t - P.ymin;             // window centre in the box
        uint32_t* hw = shist + warp * kSeedBins;
        for (int j = lane; j < kSeedBins; j += 32) hw[j] = 0;
        __syncwarp();
        // Lane l takes kernel rows l, l+32, ... and walks each from a lane-dependent column,
        // so the 32 pixels counted at once lie far apart and rarely share a histogram bin.
        for (int i = lane; i < P.nrows; i += 32) {
            const int sp = spans[i];
            const int width = span_hi(sp) - span_lo(sp) + 1;
            const uint16_t* row = ord + (cv + P.ymin + i) * SP + cu + span_lo(sp);
            int x = (lane * 37) % width;
            for (int k = 0; k < width; ++k) {
                atomicAdd(&hw[row[x] >> P.hist_shift], 1u);
                x = (x + 1 == width) ? 0 : x + 1;
            }
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
        const int m = refine<SHAPE>(om, N, bin << P.hist_shift, below, target, cu - P.cx0, cv - P.cy0, member, P.r2);
        if (m < 0) set_status(FIM_ERR_INTERNAL);
        if (lane == 0) med[t * TX + s] = (uint16_t)max(m, 0);
        __syncwarp();
    }
    __syncthreads();

    // ---- 4. seed rows: horizontal slides, lanes split the kernel rows ----------------------
    stamp(P, 4);
    for (int job = warp; job < 2 * P.RB * P.G; job += nwarps) {
        const int sd = job >> 1, right = job & 1;
        const int band = sd / P.G, g = sd % P.G;
        int s = g * GW + GW / 2;
        const int t = band * BH + BH / 2;
        const int steps = right ? (GW - GW / 2 - 1) : (GW / 2);
        int cu = s - P.xmin;
        const int cv = t - P.ymin;
        int p = med[t * TX + s];
        for (int k = 0; k < steps; ++k) {
            const uint16_t* ctr = ord + cv * SP + cu;
            int d = 0;
            for (int i = lane; i < P.nrows; i += 32) {
                const int2 o = htab[i];
                const int e = right ? o.y : o.x - 1;
                const int l = right ? o.x : o.y - 1;
                d += (int)(ctr[e] < p) - (int)(ctr[l] < p);
            }
            d = __reduce_add_sync(kFull, d);
            cu += right ? 1 : -1;
            s += right ? 1 : -1;
            const int m = refine<SHAPE>(om, N, p, target + d, target, cu - P.cx0, cv - P.cy0, member, P.r2);
            if (m < 0) set_status(FIM_ERR_INTERNAL);
            p = max(m, 0);
            if (lane == 0) med[t * TX + s] = (uint16_t)p;
        }
    }
    __syncthreads();

    // ---- 5. vertical sweeps: thread per window column, warp-cooperative refinement ----------
    stamp(P, 5);
    {
        const int groups = TX / 32;
        const int cg = warp % groups;
        const int rest = warp / groups;
        const int band = rest % P.RB;
        const int down = rest / P.RB;  // 0: up, 1: down
        const int s = cg * 32 + lane;
        int t = band * BH + BH / 2;
        const int steps = down ? (BH - BH / 2 - 1) : (BH / 2);
        const int cu = s - P.xmin;
        int cv = t - P.ymin;
        int p = med[t * TX + s];
        const int ncols = P.ncols;
        const int eoff = down ? 0 : -SP;
        for (int k = 0; k < steps; ++k) {
            const uint16_t* ctr = ord + cv * SP + cu + eoff;
            int d = 0;
            if (down) {
#pragma unroll 4
                for (int j = 0; j < ncols; ++j) {
                    const int2 o = vtab[j];
                    d += (int)(ctr[o.y] < p) - (int)(ctr[o.x] < p);
                }
            } else {
#pragma unroll 4
                for (int j = 0; j < ncols; ++j) {
                    const int2 o = vtab[j];
                    d += (int)(ctr[o.x] < p) - (int)(ctr[o.y] < p);
                }
            }
            cv += down ? 1 : -1;
            t += down ? 1 : -1;
            const int c = target + d;
#if FIM_VREFINE == 0
            int mine = 0;
            for (int j = 0; j < 32; ++j) {
                const int pj = __shfl_sync(kFull, p, j);
                const int cj = __shfl_sync(kFull, c, j);
                const int m = refine<SHAPE>(om, N, pj, cj, target, cu - lane + j - P.cx0, cv - P.cy0, member, P.r2);
                if (lane == j) mine = m;
            }
#else
            const int mine = thread_select<SHAPE>(om, N, p, c, target, cu - P.cx0, cv - P.cy0, member, P.r2);
#endif
            if (mine < 0) set_status(FIM_ERR_INTERNAL);
            p = max(mine, 0);
            med[t * TX + s] = (uint16_t)p;
        }
    }
    __syncthreads();

    // ---- 6. output: the input value at Omega[m] ------------------------------------------------
    stamp(P, 6);
    const char* in = static_cast<const char*>(P.in);
    char* out = static_cast<char*>(P.out);
    for (int idx = tid; idx < TX * TY; idx += nthreads) {
        const int t = idx >> P.txshift, s = idx & (TX - 1);
        const int gx = tx0 + s, gy = ty0 + t;
        if (gx >= P.w || gy >= P.h) continue;
        const uint32_t e = om[med[idx]];
        const int u = (int)(int8_t)(e & 0xffu) + P.cx0;
        const int v = (int)(int8_t)(e >> 8) + P.cy0;
        const V val = load_px<DT>(in, P, gx0 + u, gy0 + v);
        reinterpret_cast<V*>(out + (long long)gy * P.pitch)[gx] = val;
    }
    __syncthreads();
    stamp(P, 7);
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
