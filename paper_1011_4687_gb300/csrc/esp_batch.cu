// Batched evaluation of many independent environments in one launch sequence.
//
// The paper evaluates one fragment's field for one electron per call
// (Sec. III); an FMO calculation has many fragments and fragment pairs
// (Eq. FMO), and QMC runs many walkers, so the batch driver evaluates many
// (environment, positions) systems of uneven size together: one staging
// kernel, one persistent potential kernel that takes (system, position block,
// pair split) work items from an atomic counter, largest systems first, and
// one reduction kernel.  The three launches and the upload of the per-call
// table are captured once into a CUDA graph and replayed; sizes and pointers
// travel in the table, so a replay serves any call that fits the capacity.
#include <cmath>
#include <vector>

#include "esp_ctx.h"

using namespace esp;

struct esp_batch {
    std::vector<esp_ctx *> ctxs;
    int device = 0;
    int precision = 1;
    int num_sms = 152;
    int tile_cap = 64;
    cudaStream_t stream = nullptr;      // the caller's stream (may be the legacy default stream)
    cudaStream_t gstream = nullptr;     // the batch's own stream: graphs are captured and replayed here
    cudaEvent_t ev_in = nullptr, ev_out = nullptr; // join points with the caller's stream
    std::atomic<int> busy{0};
    // configuration (autotuned)
    int threads = 128, ppt = 4;
    double split_scale = 1.0;
    // device table and its pinned host image: BatchHeader then SysDesc[n]
    DevBuf table, counter;
    void *host_table = nullptr;
    size_t table_bytes = 0;
    std::vector<DevBuf> scratch;      // per system: staged positions, then partial sums
    std::vector<size_t> scratch_cap;
    cudaGraphExec_t exec = nullptr;
    bool graph_valid = false;
    cudaEvent_t ev_copied = nullptr, ev_start = nullptr, ev_end = nullptr;
    bool copied_pending = false, timed = false;
    uint32_t magic = 0x45535042u;
};

namespace {

bool valid_batch(const esp_batch *b) { return b && b->magic == 0x45535042u; }

int base_splits(const esp_ctx *c)
{
    // work items of about 24 tiles each for every position block
    return std::max(1, (c->n_tiles + 23) / 24);
}

void release_batch(esp_batch *b)
{
    if (b->exec)
        cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
    b->graph_valid = false;
    b->table.release();
    b->counter.release();
    for (DevBuf &d : b->scratch)
        d.release();
    if (b->host_table)
        cudaFreeHost(b->host_table);
    b->host_table = nullptr;
    for (cudaEvent_t *e : {&b->ev_copied, &b->ev_start, &b->ev_end, &b->ev_in, &b->ev_out})
        if (*e) {
            cudaEventDestroy(*e);
            *e = nullptr;
        }
    if (b->gstream)
        cudaStreamDestroy(b->gstream);
    b->gstream = nullptr;
}

esp_status capture_graph(esp_batch *b)
{
    if (b->exec) {
        cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
    }
    b->graph_valid = false;
    cudaStream_t s = b->gstream;
    cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess)
        return cuda_fail(e, "beginning graph capture");
    const BatchHeader *hdr = static_cast<const BatchHeader *>(b->table.p);
    const SysDesc *sys = reinterpret_cast<const SysDesc *>(static_cast<const char *>(b->table.p) + sizeof(BatchHeader));
    cudaError_t e1 = cudaMemcpyAsync(b->table.p, b->host_table, b->table_bytes, cudaMemcpyHostToDevice, s);
    // an external record node: the host can wait on it after each replay
    cudaError_t e2 = e1 == cudaSuccess ? cudaEventRecordWithFlags(b->ev_copied, s, cudaEventRecordExternal) : e1;
    cudaError_t e3 = e2 == cudaSuccess ? cudaMemsetAsync(b->counter.p, 0, sizeof(int), s) : e2;
    const esp_ctx *c0 = b->ctxs[0];
    cudaError_t e4 = e3 == cudaSuccess
                         ? launch_batch(b->precision, hdr, sys, int(b->ctxs.size()), static_cast<int *>(b->counter.p),
                                        1 << 30,
                                        static_cast<const float *>(c0->boys32.p),
                                        static_cast<const double *>(c0->boys64.p), b->tile_cap, b->threads, b->ppt,
                                        b->num_sms, 1 << 30, s)
                         : e3;
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(s, &g);
    if (e4 != cudaSuccess) {
        if (g)
            cudaGraphDestroy(g);
        return cuda_fail(e4, "capturing the batched launch");
    }
    if (e != cudaSuccess)
        return cuda_fail(e, "ending graph capture");
    e = fault("graph") ? cudaErrorInvalidValue : cudaGraphInstantiate(&b->exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess)
        return cuda_fail(e, "instantiating the batched graph");
    b->graph_valid = true;
    return ESP_OK;
}

esp_status batch_eval(esp_batch *b, const double *const *positions, const int64_t *n, double *const *V_out)
{
    const int ns = int(b->ctxs.size());
    if (!positions || !n || !V_out)
        return fail(ESP_ERR_INVALID, "null pointer arrays");
    int64_t total = 0;
    for (int k = 0; k < ns; ++k) {
        if (n[k] < 0 || n[k] > (int64_t(1) << 28))
            return fail(ESP_ERR_INVALID, "system %d: position count out of range", k);
        if (n[k] > 0) {
            if (!positions[k] || !V_out[k])
                return fail(ESP_ERR_INVALID, "system %d: null positions or outputs", k);
            if (classify(positions[k], b->device) != Space::Device || classify(V_out[k], b->device) != Space::Device)
                return fail(ESP_ERR_INVALID, "system %d: batched evaluation takes device memory only", k);
        }
        total += n[k];
    }
    if (total > (int64_t(1) << 30))
        return fail(ESP_ERR_INVALID, "too many positions in one batch");
    // per-system split counts and work items; largest item cost first
    std::vector<int> order(ns), splits(ns), blocks(ns);
    std::vector<double> item_cost(ns);
    const int per_cta = b->threads * b->ppt;
    for (int k = 0; k < ns; ++k) {
        order[size_t(k)] = k;
        const esp_ctx *c = b->ctxs[size_t(k)];
        int sp = int(std::lround(base_splits(c) * b->split_scale));
        splits[size_t(k)] = std::max(1, std::min({sp, 64, std::max(c->n_tiles, 1)}));
        blocks[size_t(k)] = int((n[k] + per_cta - 1) / per_cta);
        item_cost[size_t(k)] = double(c->n_tiles) / splits[size_t(k)];
    }
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return item_cost[size_t(x)] > item_cost[size_t(y)]; });
    // scratch capacity (staged positions + partial sums) per system
    cudaError_t e;
    for (int k = 0; k < ns; ++k) {
        size_t need = size_t(n[k]) * (3 * sizeof(double) + 6 * sizeof(float)) + 256 +
                      size_t(n[k]) * size_t(splits[size_t(k)]) * sizeof(double) + 2 * size_t(n[k]) * sizeof(int);
        if ((e = b->scratch[size_t(k)].ensure(std::max<size_t>(need, 256))) != cudaSuccess)
            return cuda_fail(e, "allocating batched scratch");
    }
    // wait until the previous replay has read the pinned table
    if (b->copied_pending) {
        if ((e = cudaEventSynchronize(b->ev_copied)) != cudaSuccess)
            return cuda_fail(e, "waiting for the previous table upload");
        b->copied_pending = false;
    }
    BatchHeader *hdr = static_cast<BatchHeader *>(b->host_table);
    SysDesc *sys = reinterpret_cast<SysDesc *>(static_cast<char *>(b->host_table) + sizeof(BatchHeader));
    int item = 0, pos = 0;
    for (int r = 0; r < ns; ++r) {
        const int k = order[size_t(r)];
        const esp_ctx *c = b->ctxs[size_t(k)];
        SysDesc &d = sys[r];
        std::memset(&d, 0, sizeof(d));
        d.tiles = static_cast<const TileMeta *>(c->tiles.p);
        d.rec32 = static_cast<const float *>(c->rec32.p);
        d.rec64 = static_cast<const double *>(c->rec64.p);
        d.pos_in = positions[k];
        d.V_out = V_out[k];
        const int nk = int(n[k]);
        char *base = static_cast<char *>(b->scratch[size_t(k)].p);
        d.st.x64 = reinterpret_cast<double *>(base);
        d.st.y64 = d.st.x64 + nk;
        d.st.z64 = d.st.y64 + nk;
        float *f = reinterpret_cast<float *>(d.st.z64 + nk);
        d.st.xh = f;
        d.st.yh = f + nk;
        d.st.zh = f + 2 * nk;
        d.st.xl = f + 3 * nk;
        d.st.yl = f + 4 * nk;
        d.st.zl = f + 5 * nk;
        size_t off = (size_t(nk) * (3 * sizeof(double) + 6 * sizeof(float)) + 255) / 256 * 256;
        d.partial = reinterpret_cast<double *>(base + off);
        // FP32C systems with many positions are staged in spatial order
        d.sorted = (b->precision == 1 && nk >= kSortMinPositions) ? 1 : 0;
        d.slot_of = reinterpret_cast<int *>(d.partial + size_t(nk) * size_t(splits[size_t(k)]));
        d.perm = d.slot_of + nk;
        for (int q = 0; q < 3; ++q)
            d.qm[q] = c->opt.qm_center[q];
        d.quantum = c->env.coord_quantum;
        d.n_tiles = c->n_tiles;
        d.tile_size = c->env.tile_size;
        d.n_pos = nk;
        d.splits = splits[size_t(k)];
        d.blocks = blocks[size_t(k)];
        d.item_begin = item;
        d.pos_begin = pos;
        d.near_r = float(c->opt.near_radius < 0.0 ? kDefaultNearRadius : c->opt.near_radius);
        item += d.blocks * d.splits;
        pos += nk;
    }
    hdr->n_sys = ns;
    hdr->n_items = item;
    hdr->n_pos_total = pos;
    hdr->pad = 0;
    if (!b->graph_valid) {
        esp_status st = capture_graph(b);
        if (st != ESP_OK)
            return st;
    }
    // ordered after earlier work on the caller's stream, and before later work on it
    if ((e = cudaEventRecord(b->ev_in, b->stream)) != cudaSuccess ||
        (e = cudaStreamWaitEvent(b->gstream, b->ev_in, 0)) != cudaSuccess ||
        (e = cudaEventRecord(b->ev_start, b->gstream)) != cudaSuccess ||
        (e = cudaGraphLaunch(b->exec, b->gstream)) != cudaSuccess ||
        (e = cudaEventRecord(b->ev_end, b->gstream)) != cudaSuccess ||
        (e = cudaEventRecord(b->ev_out, b->gstream)) != cudaSuccess ||
        (e = cudaStreamWaitEvent(b->stream, b->ev_out, 0)) != cudaSuccess)
        return cuda_fail(e, "launching the batched graph");
    b->copied_pending = true;
    b->timed = true;
    return ESP_OK;
}

esp_status batch_elapsed(esp_batch *b, double *ms)
{
    if (!b->timed)
        return fail(ESP_ERR_STATE, "no batched evaluation yet");
    cudaError_t e = cudaEventSynchronize(b->ev_end);
    if (e != cudaSuccess)
        return cuda_fail(e, "waiting for the batched evaluation");
    float t = 0.f;
    if ((e = cudaEventElapsedTime(&t, b->ev_start, b->ev_end)) != cudaSuccess)
        return cuda_fail(e, "reading batch timing events");
    *ms = t;
    return ESP_OK;
}

} // namespace

extern "C" {

esp_status esp_batch_create(esp_ctx *const *ctxs, int32_t n_sys, void *cuda_stream, esp_batch **out)
{
    last_error().clear();
    if (!out || !ctxs || n_sys <= 0 || n_sys > 65536)
        return fail(ESP_ERR_INVALID, "bad batch arguments");
    for (int32_t k = 0; k < n_sys; ++k) {
        if (!valid_ctx(ctxs[k]) || ctxs[k]->device < 0)
            return fail(ESP_ERR_STATE, "system %d: invalid or host-only context", k);
        if (ctxs[k]->device != ctxs[0]->device)
            return fail(ESP_ERR_INVALID, "all contexts of a batch must be on one device");
        if (ctxs[k]->opt.precision != ctxs[0]->opt.precision)
            return fail(ESP_ERR_INVALID, "all contexts of a batch must use one precision");
    }
    esp_batch *b = new (std::nothrow) esp_batch();
    if (!b)
        return fail(ESP_ERR_OOM, "host allocation of the batch");
    b->ctxs.assign(ctxs, ctxs + n_sys);
    b->device = ctxs[0]->device;
    b->precision = ctxs[0]->opt.precision == ESP_FP64 ? 0 : 1;
    b->num_sms = ctxs[0]->num_sms;
    b->stream = static_cast<cudaStream_t>(cuda_stream);
    for (esp_ctx *c : b->ctxs)
        b->tile_cap = std::max(b->tile_cap, c->env.tile_size);
    b->threads = b->precision == 1 ? 128 : 128;
    b->ppt = b->precision == 1 ? 4 : 2;
    b->scratch.resize(size_t(n_sys));
    b->scratch_cap.assign(size_t(n_sys), 0);
    DeviceGuard dg(b->device);
    b->table_bytes = sizeof(BatchHeader) + size_t(n_sys) * sizeof(SysDesc);
    cudaError_t e;
    if ((e = b->table.ensure(b->table_bytes)) != cudaSuccess || (e = b->counter.ensure(sizeof(int))) != cudaSuccess ||
        (e = cudaMallocHost(&b->host_table, b->table_bytes)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&b->ev_copied, cudaEventDisableTiming)) != cudaSuccess ||
        (e = cudaEventCreate(&b->ev_start)) != cudaSuccess || (e = cudaEventCreate(&b->ev_end)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming)) != cudaSuccess ||
        (e = cudaStreamCreateWithFlags(&b->gstream, cudaStreamNonBlocking)) != cudaSuccess) {
        release_batch(b);
        delete b;
        return cuda_fail(e, "allocating the batch");
    }
    std::memset(b->host_table, 0, b->table_bytes);
    *out = b;
    return ESP_OK;
}

esp_status esp_batch_eval(esp_batch *b, const double *const *positions, const int64_t *n, double *const *V_out)
{
    last_error().clear();
    if (!valid_batch(b))
        return fail(ESP_ERR_STATE, "invalid batch");
    BusyGuard busy(b->busy);
    if (!busy.acquired)
        return fail(ESP_ERR_STATE, "batch is in use by another thread");
    DeviceGuard dg(b->device);
    if (!dg.ok)
        return fail(ESP_ERR_CUDA, "cannot select device %d", b->device);
    return batch_eval(b, positions, n, V_out);
}

esp_status esp_batch_set_shape(esp_batch *b, int32_t threads, int32_t ppt, double split_scale)
{
    if (!valid_batch(b))
        return fail(ESP_ERR_STATE, "invalid batch");
    if (!batch_shape_supported(b->precision, threads, ppt) || !(split_scale > 0.0) || split_scale > 64.0)
        return fail(ESP_ERR_INVALID, "unsupported batch shape %d x %d (scale %g)", threads, ppt, split_scale);
    BusyGuard busy(b->busy);
    if (!busy.acquired)
        return fail(ESP_ERR_STATE, "batch is in use by another thread");
    if (b->threads != threads || b->ppt != ppt)
        b->graph_valid = false;
    b->threads = threads;
    b->ppt = ppt;
    b->split_scale = split_scale;
    return ESP_OK;
}

esp_status esp_batch_last_ms(esp_batch *b, double *ms)
{
    if (!valid_batch(b) || !ms)
        return fail(ESP_ERR_INVALID, "invalid batch or output");
    DeviceGuard dg(b->device);
    return batch_elapsed(b, ms);
}

esp_status esp_batch_autotune(esp_batch *b, const double *const *positions, const int64_t *n, double *const *V_out,
                              esp_tune_report *rep)
{
    last_error().clear();
    if (!valid_batch(b))
        return fail(ESP_ERR_STATE, "invalid batch");
    BusyGuard busy(b->busy);
    if (!busy.acquired)
        return fail(ESP_ERR_STATE, "batch is in use by another thread");
    DeviceGuard dg(b->device);
    static const int shapes32[][2] = {{128, 4}, {128, 2}, {256, 2}, {64, 4}};
    static const int shapes64[][2] = {{128, 2}, {128, 1}, {256, 1}};
    static const double scales[] = {0.5, 1.0, 2.0};
    const int nshape = b->precision == 1 ? 4 : 3;
    esp_tune_report r;
    std::memset(&r, 0, sizeof(r));
    r.best_ms = 1e300;
    for (int si = 0; si < nshape; ++si) {
        for (double sc : scales) {
            const int t = b->precision == 1 ? shapes32[si][0] : shapes64[si][0];
            const int p = b->precision == 1 ? shapes32[si][1] : shapes64[si][1];
            if (b->threads != t || b->ppt != p)
                b->graph_valid = false;
            b->threads = t;
            b->ppt = p;
            b->split_scale = sc;
            double best = 1e300;
            for (int it = 0; it < 3; ++it) { // one warm-up, two timed
                esp_status st = batch_eval(b, positions, n, V_out);
                double ms = 0.0;
                if (st == ESP_OK)
                    st = batch_elapsed(b, &ms);
                if (st != ESP_OK)
                    return st;
                if (it > 0)
                    best = std::min(best, ms);
            }
            if (r.n_tried < 16) {
                r.tried_threads[r.n_tried] = t;
                r.tried_ppt[r.n_tried] = p;
                r.tried_scale[r.n_tried] = sc;
                r.tried_ms[r.n_tried] = best;
                ++r.n_tried;
            }
            if (best < r.best_ms) {
                r.best_ms = best;
                r.threads_per_block = t;
                r.positions_per_thread = p;
                r.split_scale = sc;
            }
        }
    }
    if (b->threads != r.threads_per_block || b->ppt != r.positions_per_thread)
        b->graph_valid = false;
    b->threads = r.threads_per_block;
    b->ppt = r.positions_per_thread;
    b->split_scale = r.split_scale;
    if (rep)
        *rep = r;
    return ESP_OK;
}

void esp_batch_destroy(esp_batch *b)
{
    if (!valid_batch(b))
        return;
    {
        DeviceGuard dg(b->device);
        if (b->gstream)
            cudaStreamSynchronize(b->gstream);
        release_batch(b);
    }
    b->magic = 0;
    delete b;
}

} // extern "C"
