// Context internals shared by the C-ABI translation units.
#pragma once

#include <algorithm>
#include <atomic>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>

#include <cuda_runtime.h>

#include "../../include/esp.h"
#include "esp_kernels.h"
#include "pair_builder.h"

namespace esp {

// message of the last failing call in this thread (esp_last_error)
std::string &last_error();

inline esp_status fail(esp_status s, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    last_error() = buf;
    return s;
}

inline esp_status cuda_fail(cudaError_t e, const char *what)
{
    if (e == cudaErrorMemoryAllocation)
        return fail(ESP_ERR_OOM, "%s: %s", what, cudaGetErrorString(e));
    return fail(ESP_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

// Host-side fault injection for the tests of the error paths (no GPU fault
// is involved): the environment variable ESP_FAULT names, comma-separated, the
// operations that fail as if the CUDA call had failed: "alloc" (every device
// allocation of contexts, scratch, batches and surrogates: out of memory),
// "upload" (the environment upload of esp_create), "graph" (instantiating the
// batched driver's CUDA graph).  Read on every use, so a test can set and
// clear it between calls.
inline bool fault(const char *what)
{
    const char *v = std::getenv("ESP_FAULT");
    if (!v || !*v)
        return false;
    const size_t n = std::strlen(what);
    for (const char *p = v; *p;) {
        const char *q = p;
        while (*q && *q != ',')
            ++q;
        if (size_t(q - p) == n && std::strncmp(p, what, n) == 0)
            return true;
        p = *q ? q + 1 : q;
    }
    return false;
}

struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
    void release()
    {
        if (p)
            cudaFree(p);
        p = nullptr;
        bytes = 0;
    }
    cudaError_t ensure(size_t need)
    {
        if (need <= bytes)
            return cudaSuccess;
        if (fault("alloc"))
            return cudaErrorMemoryAllocation;
        release();
        cudaError_t e = cudaMalloc(&p, need);
        if (e != cudaSuccess) {
            p = nullptr;
            return e;
        }
        bytes = need;
        return cudaSuccess;
    }
};

// Restores the caller's current device on scope exit.
struct DeviceGuard {
    int prev = -1;
    bool ok = false;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) == cudaSuccess && cudaSetDevice(dev) == cudaSuccess)
            ok = true;
    }
    ~DeviceGuard()
    {
        if (prev >= 0)
            cudaSetDevice(prev);
    }
};

struct BusyGuard {
    std::atomic<int> &flag;
    bool acquired;
    explicit BusyGuard(std::atomic<int> &f) : flag(f)
    {
        int expect = 0;
        acquired = flag.compare_exchange_strong(expect, 1);
    }
    ~BusyGuard()
    {
        if (acquired)
            flag.store(0);
    }
};

enum class Space { Host, Device, Invalid };

inline Space classify(const void *p, int device)
{
    cudaPointerAttributes at;
    cudaError_t e = cudaPointerGetAttributes(&at, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return Space::Host;
    }
    if (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged)
        return at.device == device ? Space::Device : Space::Invalid;
    return Space::Host;
}

// A set of a context's tiles evaluated together: the whole environment, or a
// subset (the surrogate's near-field tiles).  `tiles` is a device array of
// TileMeta (records stay in the context's rec32 / rec64); the FP32C splits
// are dealt per class group (point charges, L = 0..4; empty groups left out),
// in proportion to each group's estimated FP32 work.
struct TileView {
    const TileMeta *tiles = nullptr;
    int n_tiles = 0;
    int n_groups = 1;
    int grp_tile[kMaxTileGroups + 1] = {0, 0};
    double grp_work[kMaxTileGroups] = {0.0};
    bool point_heavy = false; // >= 90 % of the entries are FP32 point charges
    // FP32 point charges of the view: their records are contiguous in rec32
    // (the builder emits those tiles one after the other)
    int64_t p32_off = 0;
    int n_p32 = 0;
};

// Tile groups of a host tile list (in device order); with fewer than one
// group per class, or tiles not grouped by class, the plain deal.
void set_tile_groups(const std::vector<TileMeta> &T, TileView &v);

} // namespace esp

struct esp_ctx {
    int device = 0;
    int num_sms = 152;
    cudaStream_t stream = nullptr;
    esp_options opt;
    esp::HostEnv env;        // host copy of the tiles (kept for esp_get_info / test hook)
    bool host_copy = true;
    esp::DevBuf tiles, rec32, rec64, boys32, boys64;
    esp::DevBuf in, stage, partial, vout, eout, sortbuf;
    std::atomic<int> busy{0};
    int64_t device_bytes = 0;
    int n_tiles = 0;
    esp::TileView full;      // every tile of the environment, set at creation
    int threads[2] = {128, 128};  // per precision (0 = FP64, 1 = FP32C)
    int ppt[2] = {2, 4};
    bool timing = false;
    bool timed_valid = false;
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr}; // pipeline start, kernel start/end, pipeline end
    uint32_t magic = 0x45535021u;
};

namespace esp {
inline bool valid_ctx(const esp_ctx *c) { return c && c->magic == 0x45535021u; }
// per-split count for n positions in precision prec (0 FP64, 1 FP32C)
int choose_splits(const esp_ctx *c, const TileView &v, int n, int prec);
// Fills the deal of the view's tiles (n_splits and the tile groups) for n
// positions, with at most max_splits partial sums; returns n_splits.  FP32C
// deals each tile group to its own splits, in proportion to the group's work.
int plan_splits(const esp_ctx *c, const TileView &v, int n, int prec, int max_splits, EvalArgs &a);
// Potentials of the view's tiles at n device positions into device V (the
// main pipeline of esp_eval: spatial order for FP32C calls of >= 4,096
// positions, staging, potential kernel, fixed-order reduction), enqueued on
// the context's stream with the context's scratch.  prec: 0 FP64, 1 FP32C.
// The caller holds the context (no other call may run on it meanwhile).
esp_status eval_view(esp_ctx *c, const TileView &v, int prec, const double *d_pos, int64_t n, double *d_V);
} // namespace esp
