// Autotuner: picks the tile configuration (tile width and height, bands, seeds per seed row)
// for a (device, dtype, kernel geometry, image-size class) by timing every valid candidate on the
// caller's data with CUDA events. Results live in a process-wide cache that choose_tile()
// consults first and that can be persisted to a text file named by the FIM_TUNE_CACHE
// environment variable.
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <tuple>

#include "fim_internal.h"

namespace fim {
namespace {

// device name, dtype, kernel hash, CTA size (0: any), image-size class
using Key = std::tuple<std::string, int, uint64_t, int, int>;

std::mutex g_tune_mu;
std::map<Key, TileShape>& tune_map() {
    static std::map<Key, TileShape> m;
    return m;
}
bool g_loaded = false;

std::string device_name() {
    int dev = 0;
    cudaDeviceProp prop;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&prop, dev) != cudaSuccess) return "unknown";
    std::string s(prop.name);
    for (char& c : s)
        if (c == ' ' || c == '\t') c = '_';
    return s;
}

// FNV-1a over the kernel's defining data (shape class, disk bound, row spans).
uint64_t kernel_hash(const fim_kernel* k) {
    uint64_t h = 1469598103934665603ull;
    auto mix = [&](int64_t v) {
        for (int i = 0; i < 8; ++i) {
            h ^= (uint64_t)((v >> (8 * i)) & 0xff);
            h *= 1099511628211ull;
        }
    };
    mix(k->shape);
    mix(k->r2);
    mix(k->ymin);
    for (size_t i = 0; i < k->rlo.size(); ++i) {
        mix(k->rlo[i]);
        mix(k->rhi[i]);
    }
    return h;
}

const char* cache_path() {
    const char* p = getenv("FIM_TUNE_CACHE");
    return (p && *p) ? p : nullptr;
}

void load_locked() {
    if (g_loaded) return;
    g_loaded = true;
    const char* path = cache_path();
    if (!path) return;
    FILE* f = fopen(path, "r");
    if (!f) return;
    char name[256];
    int dtype, cta, sc, tx, ty, rb, g;
    unsigned long long hash;
    while (fscanf(f, "%255s %d %llx %d %d %d %d %d %d", name, &dtype, &hash, &cta, &sc, &tx, &ty, &rb, &g) == 9)
        tune_map()[Key(std::string(name), dtype, (uint64_t)hash, cta, sc)] = TileShape{tx, ty, rb, g};
    fclose(f);
}

void save_locked() {
    const char* path = cache_path();
    if (!path) return;
    std::string tmp = std::string(path) + ".tmp";
    FILE* f = fopen(tmp.c_str(), "w");
    if (!f) return;
    for (const auto& kv : tune_map())
        fprintf(f, "%s %d %llx %d %d %d %d %d %d\n", std::get<0>(kv.first).c_str(), std::get<1>(kv.first),
                (unsigned long long)std::get<2>(kv.first), std::get<3>(kv.first), std::get<4>(kv.first),
                kv.second.Tx, kv.second.Ty, kv.second.RB, kv.second.G);
    fclose(f);
    rename(tmp.c_str(), path);
}

}  // namespace

bool tuned_lookup(const fim_kernel* k, int dtype, TileShape* ts, int size_cls, int cta_threads) {
    std::lock_guard<std::mutex> g(g_tune_mu);
    load_locked();
    auto it = tune_map().find(Key(device_name(), dtype, kernel_hash(k), cta_threads, size_cls));
    if (it == tune_map().end()) return false;
    *ts = it->second;
    return true;
}

void tuned_store(const fim_kernel* k, int dtype, const TileShape& ts, int size_cls, int cta_threads) {
    std::lock_guard<std::mutex> g(g_tune_mu);
    load_locked();
    tune_map()[Key(device_name(), dtype, kernel_hash(k), cta_threads, size_cls)] = ts;
    save_locked();
}

void tuned_clear() {
    std::lock_guard<std::mutex> g(g_tune_mu);
    tune_map().clear();
}

// Candidate tile configurations: tile width 32 or 64 (a warp row of the vertical sweep is 32
// columns), tile height 16..128, 2..16 bands of at least 4 rows, 1..4 seeds per seed row.
void tile_candidates(std::vector<TileShape>* out) {
    static const int txs[] = {64, 32};
    static const int tys[] = {128, 64, 32, 16};
    static const int rbs[] = {2, 4, 8, 16};
    static const int gs[] = {1, 2, 4};
    for (int tx : txs)
        for (int ty : tys)
            for (int rb : rbs)
                for (int g : gs) {
                    if (2 * tx * rb > 1024 || ty % rb != 0 || ty / rb < 4 || tx % g != 0) continue;
                    out->push_back(TileShape{tx, ty, rb, g});
                }
}

}  // namespace fim

using namespace fim;

extern "C" fim_status fim_autotune(const void* in, void* out, int w, int h, size_t pitch_bytes, fim_dtype dtype,
                                   const fim_kernel* k, int cta_threads, void* stream, int* tile_w, int* tile_h) {
    if (cta_threads != 0 && cta_threads != 256 && cta_threads != 512 && cta_threads != 1024) return FIM_ERR_INVALID_ARG;
    if (!in || !out || !k || w <= 0 || h <= 0) return FIM_ERR_INVALID_ARG;
    if (dtype != FIM_U8 && dtype != FIM_U16 && dtype != FIM_F32) return FIM_ERR_INVALID_ARG;
    const int es = dtype == FIM_U8 ? 1 : (dtype == FIM_U16 ? 2 : 4);
    if (pitch_bytes < (size_t)w * es || pitch_bytes % es != 0) return FIM_ERR_INVALID_ARG;
    const int limit = device_smem_limit();
    if (limit <= 0) return FIM_ERR_CUDA;
    cudaStream_t st = (cudaStream_t)stream;
    std::vector<TileShape> cands;
    tile_candidates(&cands);
    Plan* p = new (std::nothrow) Plan;
    if (!p) return FIM_ERR_OOM;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        delete p;
        return FIM_ERR_CUDA;
    }
    float best_ms = 1e30f;
    TileShape best{0, 0, 0, 0};
    fim_status result = FIM_ERR_UNSUPPORTED;
    for (const TileShape& c : cands) {
        if (cta_threads != 0 && 2 * c.Tx * c.RB != cta_threads) continue;
        if (make_plan(k, dtype, (k->n - 1) / 2, w, h, c, limit, p) != FIM_OK) continue;
        p->in = in;
        p->out = out;
        p->pitch = (long long)pitch_bytes;
        if (launch_tile_kernel(*p, st) != FIM_OK) continue;  // warm-up (and workspace growth)
        float ms = 1e30f;
        for (int rep = 0; rep < 2; ++rep) {
            cudaEventRecord(e0, st);
            if (launch_tile_kernel(*p, st) != FIM_OK) break;
            cudaEventRecord(e1, st);
            if (cudaEventSynchronize(e1) != cudaSuccess) break;
            float t = 0.f;
            cudaEventElapsedTime(&t, e0, e1);
            ms = std::min(ms, t);
        }
        if (ms < best_ms) {
            best_ms = ms;
            best = c;
            result = FIM_OK;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    delete p;
    if (cudaGetLastError() != cudaSuccess) return FIM_ERR_CUDA;
    if (result == FIM_OK) {
        tuned_store(k, dtype, best, size_class(w, h), cta_threads);
        if (tile_w) *tile_w = best.Tx;
        if (tile_h) *tile_h = best.Ty;
    }
    return result;
}

extern "C" fim_status fim_autotune_clear(void) {
    tuned_clear();
    return FIM_OK;
}
