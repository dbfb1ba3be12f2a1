// CPU oracle for the exact 2-D rank-order (median / percentile) filter.
//
// TEST INFRASTRUCTURE ONLY. Only tests/, __graft_entry__.smoke() and bench.py's
// cpu_baseline / reference arm may load this library. The CUDA product path shares no
// code with it and never calls it.
//
// What it computes is the plain definition of the filter, written out with no blocking,
// no fusion and no reordering:
//   for each output pixel (x, y):
//     W = { in(clamp(x+dx, 0, w-1), clamp(y+dy, 0, h-1)) : (dx, dy) in K }   (one entry per tap)
//     out(x, y) = the element of 0-based rank k in ascending order of W
// with k = (n-1)/2 for the median (Sec. 3.1: a 7x7 window's median is its 25th smallest
// value, 0-based rank 24),
// K the kernel's offset set (Eq. 1-3: a pixel belongs to the region iff its location
// lies inside the kernel shape), and clamp-to-edge borders (the input tiles of Sec. 3.3
// are padded by the radius; the padding mode is clamp).
// The selection primitive is std::nth_element. Floats are ordered by IEEE 754 totalOrder
// restricted to non-NaN values (-0 < +0), written as a plain comparator; the median is a
// selected input value, so no arithmetic touches the data.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

struct LessU8 {
    bool operator()(uint8_t a, uint8_t b) const { return a < b; }
};
struct LessU16 {
    bool operator()(uint16_t a, uint16_t b) const { return a < b; }
};
struct LessF32 {  // totalOrder on non-NaN floats: numeric order, and -0 before +0
    bool operator()(float a, float b) const {
        if (a < b) return true;
        if (a == b) return std::signbit(a) && !std::signbit(b);
        return false;
    }
};

inline int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

template <typename T, typename Less>
void filter_all(const T* in, size_t in_pitch, T* out, size_t out_pitch, int w, int h,
                const int* dx, const int* dy, int n, int rank, int nthreads) {
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
#pragma omp parallel
    {
        std::vector<T> win((size_t)n);
#pragma omp for schedule(dynamic, 1)
        for (int y = 0; y < h; ++y) {
            for (int x = 0; x < w; ++x) {
                for (int t = 0; t < n; ++t) {
                    int xx = clampi(x + dx[t], 0, w - 1);
                    int yy = clampi(y + dy[t], 0, h - 1);
                    const T* row = (const T*)((const char*)in + (size_t)yy * in_pitch);
                    win[(size_t)t] = row[xx];
                }
                std::nth_element(win.begin(), win.begin() + rank, win.end(), Less());
                T* orow = (T*)((char*)out + (size_t)y * out_pitch);
                orow[x] = win[(size_t)rank];
            }
        }
    }
}

// The same definition with a rank of its own for every output pixel: ranks is w * h ints,
// row-major, each in [0, n) (a spatially varying percentile, Fig. 14).
template <typename T, typename Less>
void filter_ranks(const T* in, size_t in_pitch, T* out, size_t out_pitch, int w, int h,
                  const int* dx, const int* dy, int n, const int* ranks, int nthreads) {
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
#pragma omp parallel
    {
        std::vector<T> win((size_t)n);
#pragma omp for schedule(dynamic, 1)
        for (int y = 0; y < h; ++y) {
            for (int x = 0; x < w; ++x) {
                for (int t = 0; t < n; ++t) {
                    int xx = clampi(x + dx[t], 0, w - 1);
                    int yy = clampi(y + dy[t], 0, h - 1);
                    const T* row = (const T*)((const char*)in + (size_t)yy * in_pitch);
                    win[(size_t)t] = row[xx];
                }
                const int k = ranks[(size_t)y * w + x];
                std::nth_element(win.begin(), win.begin() + k, win.end(), Less());
                T* orow = (T*)((char*)out + (size_t)y * out_pitch);
                orow[x] = win[(size_t)k];
            }
        }
    }
}

template <typename T, typename Less>
void filter_points(const T* in, size_t in_pitch, int w, int h, const int* px, const int* py,
                   long npts, const int* dx, const int* dy, int n, int rank, T* vals, int nthreads) {
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
#pragma omp parallel
    {
        std::vector<T> win((size_t)n);
#pragma omp for schedule(dynamic, 64)
        for (long i = 0; i < npts; ++i) {
            int x = px[i], y = py[i];
            for (int t = 0; t < n; ++t) {
                int xx = clampi(x + dx[t], 0, w - 1);
                int yy = clampi(y + dy[t], 0, h - 1);
                const T* row = (const T*)((const char*)in + (size_t)yy * in_pitch);
                win[(size_t)t] = row[xx];
            }
            std::nth_element(win.begin(), win.begin() + rank, win.end(), Less());
            vals[i] = win[(size_t)rank];
        }
    }
}

}  // namespace

extern "C" {

// dtype: 0 = uint8, 1 = uint16, 2 = float32. Pitches in bytes. Returns 0, or -1 on bad args.
int fim_oracle_filter(int dtype, const void* in, size_t in_pitch, void* out, size_t out_pitch,
                      int w, int h, const int* dx, const int* dy, int n, int rank, int nthreads) {
    if (!in || !out || w <= 0 || h <= 0 || n <= 0 || rank < 0 || rank >= n) return -1;
    switch (dtype) {
        case 0: filter_all<uint8_t, LessU8>((const uint8_t*)in, in_pitch, (uint8_t*)out, out_pitch, w, h, dx, dy, n, rank, nthreads); return 0;
        case 1: filter_all<uint16_t, LessU16>((const uint16_t*)in, in_pitch, (uint16_t*)out, out_pitch, w, h, dx, dy, n, rank, nthreads); return 0;
        case 2: filter_all<float, LessF32>((const float*)in, in_pitch, (float*)out, out_pitch, w, h, dx, dy, n, rank, nthreads); return 0;
    }
    return -1;
}

// Per-pixel ranks (w * h ints, row-major). Returns 0, or -1 on bad args (a rank outside [0, n)).
int fim_oracle_filter_ranks(int dtype, const void* in, size_t in_pitch, void* out, size_t out_pitch,
                            int w, int h, const int* dx, const int* dy, int n, const int* ranks, int nthreads) {
    if (!in || !out || !ranks || w <= 0 || h <= 0 || n <= 0) return -1;
    for (size_t i = 0; i < (size_t)w * h; ++i)
        if (ranks[i] < 0 || ranks[i] >= n) return -1;
    switch (dtype) {
        case 0: filter_ranks<uint8_t, LessU8>((const uint8_t*)in, in_pitch, (uint8_t*)out, out_pitch, w, h, dx, dy, n, ranks, nthreads); return 0;
        case 1: filter_ranks<uint16_t, LessU16>((const uint16_t*)in, in_pitch, (uint16_t*)out, out_pitch, w, h, dx, dy, n, ranks, nthreads); return 0;
        case 2: filter_ranks<float, LessF32>((const float*)in, in_pitch, (float*)out, out_pitch, w, h, dx, dy, n, ranks, nthreads); return 0;
    }
    return -1;
}

// Same definition evaluated at npts chosen pixels (px[i], py[i]); vals[i] receives the result.
int fim_oracle_points(int dtype, const void* in, size_t in_pitch, int w, int h, const int* px,
                      const int* py, long npts, const int* dx, const int* dy, int n, int rank,
                      void* vals, int nthreads) {
    if (!in || !vals || w <= 0 || h <= 0 || n <= 0 || rank < 0 || rank >= n || npts < 0) return -1;
    switch (dtype) {
        case 0: filter_points<uint8_t, LessU8>((const uint8_t*)in, in_pitch, w, h, px, py, npts, dx, dy, n, rank, (uint8_t*)vals, nthreads); return 0;
        case 1: filter_points<uint16_t, LessU16>((const uint16_t*)in, in_pitch, w, h, px, py, npts, dx, dy, n, rank, (uint16_t*)vals, nthreads); return 0;
        case 2: filter_points<float, LessF32>((const float*)in, in_pitch, w, h, px, py, npts, dx, dy, n, rank, (float*)vals, nthreads); return 0;
    }
    return -1;
}

int fim_oracle_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

}  // extern "C"
