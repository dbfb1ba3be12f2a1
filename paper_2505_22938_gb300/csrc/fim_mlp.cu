// Rank-bracket MLP: model object, training and inference kernels, sample collection and the
// learned median filter entry point.
//
// The network maps a seed window's features (the tile's 32 normalised value quantiles and the
// ranks / N of the 3x3 pixels around the window centre) to (mu, s): mu predicts the window's
// median rank as a fraction of the tile's feasible median ranks (Fig. 10), s = log sigma its
// uncertainty. Layers 41 -> 64 (ReLU) -> 64 (ReLU) -> 2 with bf16 weights and fp32 accumulation.
// Training minimises the Gaussian negative log-likelihood 0.5 (y - mu)^2 / sigma^2 + log sigma
// with Adam on fp32 master weights; every forward and backward pass uses the bf16-rounded
// weights (straight-through for the rounding). The filter uses mu +- z sigma as a bracket that
// the exact selection verifies by counting (the seed phase of fim_tile_pipeline.cuh): the network can
// only change how far the omnigram scan walks, never the output.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "fim_internal.h"

using namespace fim;

struct fim_model {
    float* w = nullptr;      // fp32 master parameters
    float* wq = nullptr;     // the same, rounded to bf16 and widened back (GEMM operand)
    uint16_t* wb = nullptr;  // bf16 bits (the filter's copy)
    float* m = nullptr;      // Adam first moment
    float* v = nullptr;      // Adam second moment
    float* g = nullptr;      // gradient
    float bracket_z = 3.0f;
    long long step = 0;
    int device = 0;
};

namespace {

// Round-to-nearest-even of an fp32 value to bf16 (the upper 16 bits), NaN kept quiet.
__host__ __device__ inline uint16_t to_bf16(float f) {
    uint32_t u;
    memcpy(&u, &f, 4);
    if ((u & 0x7fffffffu) > 0x7f800000u) return (uint16_t)((u >> 16) | 0x40u);
    u += 0x7fffu + ((u >> 16) & 1u);
    return (uint16_t)(u >> 16);
}
__host__ __device__ inline float from_bf16(uint16_t b) {
    const uint32_t u = (uint32_t)b << 16;
    float f;
    memcpy(&f, &u, 4);
    return f;
}

// C[i][j] (+)= bias[j] + sum_k A(i, k) B(k, j), optional ReLU; A(i,k) = A[i*sai + k*sak], etc.
// One thread per output element; the shapes here are small (<= 64 wide).
__global__ void gemm_kernel(int M, int Nn, int K, const float* __restrict__ A, long long sai, long long sak,
                            const float* __restrict__ B, long long sbk, long long sbj, float* __restrict__ C,
                            long long sci, long long scj, const float* __restrict__ bias, int relu, int accumulate) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)M * Nn) return;
    const int i = (int)(idx / Nn), j = (int)(idx % Nn);
    float acc = bias ? bias[j] : 0.f;
    for (int k = 0; k < K; ++k) acc = fmaf(A[i * sai + k * sak], B[k * sbk + j * sbj], acc);
    if (relu) acc = fmaxf(acc, 0.f);
    float* c = C + i * sci + j * scj;
    *c = accumulate ? *c + acc : acc;
}

void gemm(cudaStream_t st, int M, int Nn, int K, const float* A, long long sai, long long sak, const float* B,
          long long sbk, long long sbj, float* C, long long sci, long long scj, const float* bias = nullptr,
          int relu = 0, int accumulate = 0) {
    const long long n = (long long)M * Nn;
    gemm_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(M, Nn, K, A, sai, sak, B, sbk, sbj, C, sci, scj, bias,
                                                            relu, accumulate);
}

// Gaussian NLL per row and its gradient with respect to the two outputs (mean over rows).
__global__ void nll_kernel(int rows, const float* __restrict__ O, const float* __restrict__ Y, long long ystride,
                           float* __restrict__ dO, float* __restrict__ loss_sum) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    float l = 0.f;
    if (i < rows) {
        const float mu = O[2 * i], s_raw = O[2 * i + 1];
        const float s = fminf(fmaxf(s_raw, -8.f), 2.f);
        const float inv = expf(-2.f * s);
        const float e = Y[i * ystride] - mu;
        l = 0.5f * e * e * inv + s;
        dO[2 * i] = -e * inv / rows;
        dO[2 * i + 1] = (s_raw > -8.f && s_raw < 2.f) ? (1.f - e * e * inv) / rows : 0.f;
    }
    for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(loss_sum, l);
}

// dZ = dA * [Z > 0]
__global__ void relu_back_kernel(long long n, const float* __restrict__ Z, float* __restrict__ dA) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && Z[i] <= 0.f) dA[i] = 0.f;
}

// column sums of a rows x cols matrix into out (bias gradients)
__global__ void colsum_kernel(int rows, int cols, const float* __restrict__ X, float* __restrict__ out) {
    const int j = blockIdx.x;
    float acc = 0.f;
    for (int i = threadIdx.x; i < rows; i += blockDim.x) acc += X[(long long)i * cols + j];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    __shared__ float part[32];
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.f;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += part[k];
        out[j] = t;
    }
}

__global__ void adam_kernel(int n, float* w, float* wq, uint16_t* wb, float* m, float* v, const float* g, float lr,
                            float b1, float b2, float eps, float c1, float c2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    w[i] = wi;
    const uint16_t b = to_bf16(wi);
    wb[i] = b;
    wq[i] = from_bf16(b);
}

__global__ void quantize_kernel(int n, const float* w, float* wq, uint16_t* wb) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint16_t b = to_bf16(w[i]);
    wb[i] = b;
    wq[i] = from_bf16(b);
}

// Standardised absolute residual |y - mu| / sigma per row (for calibrating the bracket width).
__global__ void zscore_kernel(int rows, const float* __restrict__ O, const float* __restrict__ Y, long long ystride,
                              float* __restrict__ z) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= rows) return;
    const float s = fminf(fmaxf(O[2 * i + 1], -8.f), 2.f);
    z[i] = fabsf(Y[i * ystride] - O[2 * i]) * expf(-s);
}

// Workspace of one forward/backward pass over `rows` rows.
struct Act {
    float *z1, *a1, *z2, *a2, *o, *d_o, *d2, *d1, *loss;
    int rows = 0;
    void release() {
        float* ps[] = {z1, a1, z2, a2, o, d_o, d2, d1, loss};
        for (float* p : ps)
            if (p) cudaFree(p);
    }
    bool alloc(int n) {
        rows = n;
        z1 = a1 = z2 = a2 = o = d_o = d2 = d1 = loss = nullptr;
        const size_t h = (size_t)n * kHidden * 4;
        return cudaMalloc(&z1, h) == cudaSuccess && cudaMalloc(&a1, h) == cudaSuccess &&
               cudaMalloc(&z2, h) == cudaSuccess && cudaMalloc(&a2, h) == cudaSuccess &&
               cudaMalloc(&o, (size_t)n * 8) == cudaSuccess && cudaMalloc(&d_o, (size_t)n * 8) == cudaSuccess &&
               cudaMalloc(&d2, h) == cudaSuccess && cudaMalloc(&d1, h) == cudaSuccess &&
               cudaMalloc(&loss, 4) == cudaSuccess;
    }
};

// Forward pass of `rows` rows of X (row stride xs floats) with the bf16-rounded weights.
void forward(const fim_model* md, cudaStream_t st, const float* X, long long xs, int rows, Act& a) {
    const float* W = md->wq;
    gemm(st, rows, kHidden, kFeatures, X, xs, 1, W + kOffW1, kHidden, 1, a.z1, kHidden, 1, W + kOffB1);
    cudaMemcpyAsync(a.a1, a.z1, (size_t)rows * kHidden * 4, cudaMemcpyDeviceToDevice, st);
    relu_back_kernel<<<(unsigned)(((long long)rows * kHidden + 255) / 256), 256, 0, st>>>((long long)rows * kHidden,
                                                                                          a.z1, a.a1);
    gemm(st, rows, kHidden, kHidden, a.a1, kHidden, 1, W + kOffW2, kHidden, 1, a.z2, kHidden, 1, W + kOffB2);
    cudaMemcpyAsync(a.a2, a.z2, (size_t)rows * kHidden * 4, cudaMemcpyDeviceToDevice, st);
    relu_back_kernel<<<(unsigned)(((long long)rows * kHidden + 255) / 256), 256, 0, st>>>((long long)rows * kHidden,
                                                                                          a.z2, a.a2);
    gemm(st, rows, 2, kHidden, a.a2, kHidden, 1, W + kOffW3, 2, 1, a.o, 2, 1, W + kOffB3);
}

// Mean loss and its gradient (into md->g) over rows of (X, y); y is column kFeatures of X
// when ys == xs and X == Y base, or any strided vector.
void loss_and_grad(fim_model* md, cudaStream_t st, const float* X, long long xs, const float* Y, long long ys,
                   int rows, Act& a) {
    forward(md, st, X, xs, rows, a);
    cudaMemsetAsync(a.loss, 0, 4, st);
    nll_kernel<<<(rows + 255) / 256, 256, 0, st>>>(rows, a.o, Y, ys, a.d_o, a.loss);
    const float* W = md->wq;
    float* g = md->g;
    // layer 3
    gemm(st, kHidden, 2, rows, a.a2, 1, kHidden, a.d_o, 2, 1, g + kOffW3, 2, 1);
    colsum_kernel<<<2, 256, 0, st>>>(rows, 2, a.d_o, g + kOffB3);
    gemm(st, rows, kHidden, 2, a.d_o, 2, 1, W + kOffW3, 1, 2, a.d2, kHidden, 1);
    relu_back_kernel<<<(unsigned)(((long long)rows * kHidden + 255) / 256), 256, 0, st>>>((long long)rows * kHidden,
                                                                                          a.z2, a.d2);
    // layer 2
    gemm(st, kHidden, kHidden, rows, a.a1, 1, kHidden, a.d2, kHidden, 1, g + kOffW2, kHidden, 1);
    colsum_kernel<<<kHidden, 256, 0, st>>>(rows, kHidden, a.d2, g + kOffB2);
    gemm(st, rows, kHidden, kHidden, a.d2, kHidden, 1, W + kOffW2, 1, kHidden, a.d1, kHidden, 1);
    relu_back_kernel<<<(unsigned)(((long long)rows * kHidden + 255) / 256), 256, 0, st>>>((long long)rows * kHidden,
                                                                                          a.z1, a.d1);
    // layer 1
    gemm(st, kFeatures, kHidden, rows, X, 1, xs, a.d1, kHidden, 1, g + kOffW1, kHidden, 1);
    colsum_kernel<<<kHidden, 256, 0, st>>>(rows, kHidden, a.d1, g + kOffB1);
}

fim_status check_cuda() {
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? FIM_OK : FIM_ERR_CUDA;
}

void free_model(fim_model* md) {
    if (!md) return;
    float* fs[] = {md->w, md->wq, md->m, md->v, md->g};
    for (float* p : fs)
        if (p) cudaFree(p);
    if (md->wb) cudaFree(md->wb);
    delete md;
}

fim_status alloc_model(fim_model** out) {
    fim_model* md = new (std::nothrow) fim_model();
    if (!md) return FIM_ERR_OOM;
    cudaGetDevice(&md->device);
    const size_t b = (size_t)kMlpParams * 4;
    if (cudaMalloc(&md->w, b) != cudaSuccess || cudaMalloc(&md->wq, b) != cudaSuccess ||
        cudaMalloc(&md->m, b) != cudaSuccess || cudaMalloc(&md->v, b) != cudaSuccess ||
        cudaMalloc(&md->g, b) != cudaSuccess || cudaMalloc(&md->wb, (size_t)kMlpParams * 2) != cudaSuccess) {
        cudaGetLastError();
        free_model(md);
        return FIM_ERR_OOM;
    }
    cudaMemset(md->m, 0, b);
    cudaMemset(md->v, 0, b);
    cudaMemset(md->g, 0, b);
    *out = md;
    return FIM_OK;
}

fim_status upload_params(fim_model* md, const float* host) {
    if (cudaMemcpy(md->w, host, (size_t)kMlpParams * 4, cudaMemcpyHostToDevice) != cudaSuccess) return FIM_ERR_CUDA;
    quantize_kernel<<<(kMlpParams + 255) / 256, 256>>>(kMlpParams, md->w, md->wq, md->wb);
    if (cudaDeviceSynchronize() != cudaSuccess) return FIM_ERR_CUDA;
    return check_cuda();
}

// run the plain or learned tile kernel with the given hooks
fim_status run_filter(const void* in, void* out, int w, int h, size_t pitch, int dtype, const fim_kernel* k,
                      const fim_model* md, unsigned long long* stats, float* samples, unsigned int* count, int cap,
                      cudaStream_t st) {
    if (!in || !out || !k || w <= 0 || h <= 0) return FIM_ERR_INVALID_ARG;
    if (dtype != FIM_U8 && dtype != FIM_U16 && dtype != FIM_F32) return FIM_ERR_INVALID_ARG;
    const size_t es = dtype == FIM_U8 ? 1 : (dtype == FIM_U16 ? 2 : 4);
    if (pitch < (size_t)w * es || pitch % es != 0) return FIM_ERR_INVALID_ARG;
    const int limit = device_smem_limit();
    if (limit <= 0) return FIM_ERR_CUDA;
    TileShape ts;
    // the bracket's features and labels depend on the tile geometry, so training rows and the
    // learned launches take the large-image shapes whatever the image size
    fim_status s = choose_tile(k, dtype, limit, &ts, 0, 0);
    if (s != FIM_OK) return s;
    Plan* p = new (std::nothrow) Plan;
    if (!p) return FIM_ERR_OOM;
    s = make_plan(k, dtype, (k->n - 1) / 2, w, h, ts, limit, p);
    if (s == FIM_OK) {
        p->in = in;
        p->out = out;
        p->pitch = (long long)pitch;
        p->model = md ? md->wb : nullptr;
        p->bracket_z = md ? md->bracket_z : 0.f;
        s = plan_stage_model(p, limit);
    }
    if (s == FIM_OK) {
        p->stats = stats;
        p->samples = samples;
        p->sample_count = count;
        p->sample_cap = cap;
        get_phase_clock_buffer(&p->phase_clock, &p->phase_tiles);
        s = launch_tile_kernel(*p, st);
    }
    delete p;
    return s;
}

}  // namespace

extern "C" {

fim_status fim_model_create(uint64_t seed, fim_model** out) {
    if (!out) return FIM_ERR_INVALID_ARG;
    *out = nullptr;
    fim_model* md = nullptr;
    fim_status s = alloc_model(&md);
    if (s != FIM_OK) return s;
    // He-uniform initialisation from a splitmix64 stream; biases zero; output layer small
    std::vector<float> h((size_t)kMlpParams, 0.f);
    uint64_t x = seed ? seed : 0x9e3779b97f4a7c15ull;
    auto next = [&]() {
        x += 0x9e3779b97f4a7c15ull;
        uint64_t z = x;
        z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
        z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
        z ^= z >> 31;
        return (double)(z >> 11) / 9007199254740992.0 * 2.0 - 1.0;  // uniform in [-1, 1)
    };
    for (int i = 0; i < kFeatures * kHidden; ++i) h[kOffW1 + i] = (float)(next() * sqrt(6.0 / kFeatures));
    for (int i = 0; i < kHidden * kHidden; ++i) h[kOffW2 + i] = (float)(next() * sqrt(6.0 / kHidden));
    for (int i = 0; i < kHidden * 2; ++i) h[kOffW3 + i] = (float)(next() * 0.01);
    h[kOffB3 + 0] = 0.5f;   // predicted rank starts mid-range
    h[kOffB3 + 1] = -2.0f;  // and sigma = e^-2
    s = upload_params(md, h.data());
    if (s != FIM_OK) {
        free_model(md);
        return s;
    }
    *out = md;
    return FIM_OK;
}

void fim_model_destroy(fim_model* md) {
    cudaDeviceSynchronize();
    free_model(md);
}

int fim_model_param_count(void) { return kMlpParams; }

fim_status fim_model_get_params(const fim_model* md, float* host_fp32, uint16_t* host_bf16) {
    if (!md) return FIM_ERR_INVALID_ARG;
    if (host_fp32 && cudaMemcpy(host_fp32, md->w, (size_t)kMlpParams * 4, cudaMemcpyDeviceToHost) != cudaSuccess)
        return FIM_ERR_CUDA;
    if (host_bf16 && cudaMemcpy(host_bf16, md->wb, (size_t)kMlpParams * 2, cudaMemcpyDeviceToHost) != cudaSuccess)
        return FIM_ERR_CUDA;
    return FIM_OK;
}

fim_status fim_model_set_params(fim_model* md, const float* host_fp32) {
    if (!md || !host_fp32) return FIM_ERR_INVALID_ARG;
    return upload_params(md, host_fp32);
}

float fim_model_bracket_z(const fim_model* md) { return md ? md->bracket_z : 0.f; }

fim_status fim_model_forward(const fim_model* md, const float* x, int rows, int row_stride, float* out, void* stream) {
    if (!md || !x || !out || rows <= 0 || row_stride < kFeatures) return FIM_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    Act a;
    if (!a.alloc(rows)) {
        a.release();
        return FIM_ERR_OOM;
    }
    forward(md, st, x, row_stride, rows, a);
    cudaMemcpyAsync(out, a.o, (size_t)rows * 8, cudaMemcpyDeviceToDevice, st);
    const cudaError_t e = cudaStreamSynchronize(st);
    a.release();
    return e == cudaSuccess ? check_cuda() : FIM_ERR_CUDA;
}

fim_status fim_model_loss_grad(fim_model* md, const float* x, int rows, int row_stride, const float* y,
                               int y_stride, float* grad_out, float* loss_out, void* stream) {
    if (!md || !x || !y || rows <= 0 || row_stride < kFeatures || y_stride < 1) return FIM_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    Act a;
    if (!a.alloc(rows)) {
        a.release();
        return FIM_ERR_OOM;
    }
    loss_and_grad(md, st, x, row_stride, y, y_stride, rows, a);
    float l = 0.f;
    cudaMemcpyAsync(&l, a.loss, 4, cudaMemcpyDeviceToHost, st);
    if (grad_out) cudaMemcpyAsync(grad_out, md->g, (size_t)kMlpParams * 4, cudaMemcpyDeviceToDevice, st);
    const cudaError_t e = cudaStreamSynchronize(st);
    a.release();
    if (e != cudaSuccess) return FIM_ERR_CUDA;
    if (loss_out) *loss_out = l / rows;
    return check_cuda();
}

fim_status fim_model_train(fim_model* md, const float* rows_xy, int rows, int epochs, int batch, float lr,
                           void* stream, float* last_epoch_loss) {
    if (!md || !rows_xy || rows <= 0 || epochs <= 0 || batch <= 0 || !(lr > 0.f)) return FIM_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const int b = std::min(batch, rows);
    Act a;
    if (!a.alloc(b)) {
        a.release();
        return FIM_ERR_OOM;
    }
    const long long stride = kFeatures + 1;
    float* d_epoch = nullptr;
    if (cudaMalloc(&d_epoch, 4) != cudaSuccess) {
        a.release();
        return FIM_ERR_OOM;
    }
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    float ep_loss = 0.f;
    for (int e = 0; e < epochs; ++e) {
        double sum = 0.0;
        int nb = 0;
        for (int r0 = 0; r0 + b <= rows; r0 += b) {
            const float* X = rows_xy + (long long)r0 * stride;
            loss_and_grad(md, st, X, stride, X + kFeatures, stride, b, a);
            ++md->step;
            const float c1 = 1.f - powf(b1, (float)md->step), c2 = 1.f - powf(b2, (float)md->step);
            adam_kernel<<<(kMlpParams + 255) / 256, 256, 0, st>>>(kMlpParams, md->w, md->wq, md->wb, md->m, md->v,
                                                                 md->g, lr, b1, b2, eps, c1, c2);
            float l = 0.f;
            cudaMemcpyAsync(&l, a.loss, 4, cudaMemcpyDeviceToHost, st);
            if (cudaStreamSynchronize(st) != cudaSuccess) {
                a.release();
                cudaFree(d_epoch);
                return FIM_ERR_CUDA;
            }
            sum += l / b;
            ++nb;
        }
        ep_loss = nb ? (float)(sum / nb) : 0.f;
    }
    a.release();
    cudaFree(d_epoch);
    if (last_epoch_loss) *last_epoch_loss = ep_loss;
    return check_cuda();
}

fim_status fim_model_calibrate(fim_model* md, const float* rows_xy, int rows, double coverage, void* stream,
                               float* z_out) {
    if (!md || !rows_xy || rows <= 0 || !(coverage > 0.0 && coverage < 1.0)) return FIM_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    Act a;
    float* dz = nullptr;
    if (!a.alloc(rows) || cudaMalloc(&dz, (size_t)rows * 4) != cudaSuccess) {
        a.release();
        return FIM_ERR_OOM;
    }
    const long long stride = kFeatures + 1;
    forward(md, st, rows_xy, stride, rows, a);
    zscore_kernel<<<(rows + 255) / 256, 256, 0, st>>>(rows, a.o, rows_xy + kFeatures, stride, dz);
    std::vector<float> z((size_t)rows);
    cudaMemcpyAsync(z.data(), dz, (size_t)rows * 4, cudaMemcpyDeviceToHost, st);
    const cudaError_t e = cudaStreamSynchronize(st);
    a.release();
    cudaFree(dz);
    if (e != cudaSuccess) return FIM_ERR_CUDA;
    const size_t q = std::min((size_t)rows - 1, (size_t)(coverage * rows));
    std::nth_element(z.begin(), z.begin() + q, z.end());
    md->bracket_z = std::max(z[q], 1e-3f);
    if (z_out) *z_out = md->bracket_z;
    return FIM_OK;
}

fim_status fim_model_save(const fim_model* md, const char* path) {
    if (!md || !path) return FIM_ERR_INVALID_ARG;
    std::vector<float> w((size_t)kMlpParams), m((size_t)kMlpParams), v((size_t)kMlpParams);
    if (cudaMemcpy(w.data(), md->w, w.size() * 4, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(m.data(), md->m, m.size() * 4, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(v.data(), md->v, v.size() * 4, cudaMemcpyDeviceToHost) != cudaSuccess)
        return FIM_ERR_CUDA;
    FILE* f = fopen(path, "wb");
    if (!f) return FIM_ERR_INVALID_ARG;
    const char magic[8] = {'F', 'I', 'M', 'M', 'L', 'P', '0', '1'};
    const int n = kMlpParams;
    bool ok = fwrite(magic, 1, 8, f) == 8 && fwrite(&n, 4, 1, f) == 1 && fwrite(&md->bracket_z, 4, 1, f) == 1 &&
              fwrite(&md->step, 8, 1, f) == 1 && fwrite(w.data(), 4, w.size(), f) == w.size() &&
              fwrite(m.data(), 4, m.size(), f) == m.size() && fwrite(v.data(), 4, v.size(), f) == v.size();
    ok = (fclose(f) == 0) && ok;
    return ok ? FIM_OK : FIM_ERR_INVALID_ARG;
}

fim_status fim_model_load(const char* path, fim_model** out) {
    if (!path || !out) return FIM_ERR_INVALID_ARG;
    *out = nullptr;
    FILE* f = fopen(path, "rb");
    if (!f) return FIM_ERR_INVALID_ARG;
    char magic[8];
    int n = 0;
    float z = 0.f;
    long long step = 0;
    std::vector<float> w((size_t)kMlpParams), m((size_t)kMlpParams), v((size_t)kMlpParams);
    bool ok = fread(magic, 1, 8, f) == 8 && memcmp(magic, "FIMMLP01", 8) == 0 && fread(&n, 4, 1, f) == 1 &&
              n == kMlpParams && fread(&z, 4, 1, f) == 1 && fread(&step, 8, 1, f) == 1 &&
              fread(w.data(), 4, w.size(), f) == w.size() && fread(m.data(), 4, m.size(), f) == m.size() &&
              fread(v.data(), 4, v.size(), f) == v.size();
    fclose(f);
    if (!ok) return FIM_ERR_INVALID_ARG;
    fim_model* md = nullptr;
    fim_status s = alloc_model(&md);
    if (s != FIM_OK) return s;
    s = upload_params(md, w.data());
    if (s == FIM_OK && (cudaMemcpy(md->m, m.data(), m.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
                        cudaMemcpy(md->v, v.data(), v.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess))
        s = FIM_ERR_CUDA;
    if (s != FIM_OK) {
        free_model(md);
        return s;
    }
    md->bracket_z = z;
    md->step = step;
    *out = md;
    return FIM_OK;
}

fim_status fim_collect_seed_samples(const void* in, void* out, int w, int h, size_t pitch_bytes, fim_dtype dtype,
                                    const fim_kernel* k, float* rows_xy, int capacity, unsigned int* count_dev,
                                    void* stream) {
    if (!rows_xy || capacity <= 0 || !count_dev) return FIM_ERR_INVALID_ARG;
    return run_filter(in, out, w, h, pitch_bytes, dtype, k, nullptr, nullptr, rows_xy, count_dev, capacity,
                      (cudaStream_t)stream);
}

fim_status fim_median_learned(const void* in, void* out, int w, int h, size_t pitch_bytes, fim_dtype dtype,
                              const fim_kernel* k, const fim_model* md, fim_border border, void* stream,
                              unsigned long long* stats_dev) {
    if (border != FIM_BORDER_CLAMP) return FIM_ERR_INVALID_ARG;
    return run_filter(in, out, w, h, pitch_bytes, dtype, k, md, stats_dev, nullptr, nullptr, 0,
                      (cudaStream_t)stream);
}

}  // extern "C"
