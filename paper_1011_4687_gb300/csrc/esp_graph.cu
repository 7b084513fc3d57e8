// A captured few-position evaluation, replayed as one CUDA graph per call.
//
// The paper evaluates one electron position per GPU call, once per Metropolis
// move (Sec. III, Fig. codeStructure: r_new in, U_ES out).  At that size the
// launch overhead matters as much as the sum itself, so this entry point
// captures the few-position pipeline (entries spread over all SMs, then one
// CTA per position for the fixed-order sum) for a fixed device position
// buffer and output once, and each call replays the graph: the caller writes
// the new positions into the same buffer between calls.
#include <cuda_runtime.h>

#include "../../include/esp.h"
#include "esp_ctx.h"

using namespace esp;

struct esp_graph {
    esp_ctx *ctx = nullptr;
    int n = 0;
    DevBuf partial;
    cudaStream_t cap = nullptr;
    cudaGraphExec_t exec = nullptr;
    uint32_t magic = 0x45535047u;
};

namespace {

bool valid_graph(const esp_graph *g) { return g && g->magic == 0x45535047u; }

void release_graph(esp_graph *g)
{
    if (g->exec)
        cudaGraphExecDestroy(g->exec);
    g->exec = nullptr;
    if (g->cap)
        cudaStreamDestroy(g->cap);
    g->cap = nullptr;
    g->partial.release();
}

} // namespace

extern "C" {

esp_status esp_graph_create(esp_ctx *ctx, const double *positions, int64_t n, double *V_out, esp_graph **out)
{
    last_error().clear();
    if (!valid_ctx(ctx) || ctx->device < 0)
        return fail(ESP_ERR_STATE, "invalid or host-only context");
    if (!out || !positions || !V_out || n < 1 || n > ESP_GRAPH_MAX_POSITIONS)
        return fail(ESP_ERR_INVALID, "esp_graph_create takes 1..%d device positions and outputs",
                    ESP_GRAPH_MAX_POSITIONS);
    if (ctx->n_tiles == 0)
        return fail(ESP_ERR_UNSUPPORTED, "empty environment");
    BusyGuard busy(ctx->busy);
    if (!busy.acquired)
        return fail(ESP_ERR_STATE, "context is in use by another thread");
    DeviceGuard dg(ctx->device);
    if (!dg.ok)
        return fail(ESP_ERR_CUDA, "cannot select device %d", ctx->device);
    if (classify(positions, ctx->device) != Space::Device || classify(V_out, ctx->device) != Space::Device)
        return fail(ESP_ERR_INVALID, "esp_graph_create takes device memory of device %d", ctx->device);
    esp_graph *g = new (std::nothrow) esp_graph();
    if (!g)
        return fail(ESP_ERR_OOM, "host allocation of the graph");
    g->ctx = ctx;
    g->n = int(n);
    const int splits = small_n_splits(ctx->n_tiles, ctx->num_sms, int(n));
    SmallArgs sa;
    sa.n_pos = int(n);
    sa.n_tiles = ctx->n_tiles;
    sa.pos_in = positions;
    sa.cx = ctx->opt.qm_center[0];
    sa.cy = ctx->opt.qm_center[1];
    sa.cz = ctx->opt.qm_center[2];
    sa.tiles = ctx->full.tiles;
    sa.rec64 = static_cast<const double *>(ctx->rec64.p);
    sa.rec32 = static_cast<const float *>(ctx->rec32.p);
    sa.boys64 = static_cast<const double *>(ctx->boys64.p);
    sa.quantum = ctx->env.coord_quantum;
    sa.fp32 = ctx->opt.precision == ESP_FP32C && ctx->full.n_p32 > 0;
    sa.p32_off = ctx->full.p32_off;
    sa.n_p32 = ctx->full.n_p32;
    cudaError_t e = g->partial.ensure(size_t(splits) * size_t(n) * sizeof(double));
    if (e == cudaSuccess)
        e = cudaStreamCreateWithFlags(&g->cap, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        release_graph(g);
        delete g;
        return cuda_fail(e, "allocating the graph's scratch");
    }
    sa.partial = static_cast<double *>(g->partial.p);
    e = cudaStreamBeginCapture(g->cap, cudaStreamCaptureModeThreadLocal);
    cudaError_t e1 = e == cudaSuccess ? launch_small_n(sa, splits, V_out, g->cap) : e;
    cudaGraph_t graph = nullptr;
    if (e == cudaSuccess)
        e = cudaStreamEndCapture(g->cap, &graph);
    if (e == cudaSuccess)
        e = e1;
    if (e == cudaSuccess)
        e = fault("graph") ? cudaErrorInvalidValue : cudaGraphInstantiate(&g->exec, graph, 0);
    if (graph)
        cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        release_graph(g);
        delete g;
        return cuda_fail(e, "capturing the few-position graph");
    }
    *out = g;
    return ESP_OK;
}

esp_status esp_graph_launch(esp_graph *g)
{
    last_error().clear();
    if (!valid_graph(g) || !valid_ctx(g->ctx))
        return fail(ESP_ERR_STATE, "invalid graph");
    BusyGuard busy(g->ctx->busy);
    if (!busy.acquired)
        return fail(ESP_ERR_STATE, "context is in use by another thread");
    DeviceGuard dg(g->ctx->device);
    cudaError_t e = cudaGraphLaunch(g->exec, g->ctx->stream);
    return e == cudaSuccess ? ESP_OK : cuda_fail(e, "replaying the few-position graph");
}

void esp_graph_destroy(esp_graph *g)
{
    if (!valid_graph(g))
        return;
    if (valid_ctx(g->ctx)) {
        DeviceGuard dg(g->ctx->device);
        cudaStreamSynchronize(g->ctx->stream);
        release_graph(g);
    }
    g->magic = 0;
    delete g;
}

} // extern "C"
