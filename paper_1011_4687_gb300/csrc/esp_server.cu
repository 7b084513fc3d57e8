// Several clients sharing one GPU context.
//
// The paper runs one MPI process per CPU core and one GPU per process, and
// proposes (Introduction, Discussions) that several processes share one GPU,
// with OpenMP threads on the host.  Here one context serves any number of
// host threads: each client submits its walkers' positions and gets a ticket;
// one worker thread owns the context, takes every request queued when it
// wakes, concatenates their positions into one staging buffer, evaluates them
// in one call (one launch sequence for all clients, so small requests fill
// the GPU together), and scatters the potentials back.  A client that submits
// and then does its own host work before waiting overlaps that work with the
// GPU evaluation.
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/esp.h"
#include "esp_ctx.h"

using namespace esp;

namespace {

struct Request {
    const double *pos;
    int64_t n;
    double *V;
    int64_t ticket;
};

} // namespace

struct esp_server {
    esp_ctx *ctx = nullptr;
    int64_t max_positions = 0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request> queue;
    int64_t next_ticket = 1;
    int64_t done_upto = 0;        // every ticket <= done_upto has completed
    std::vector<int64_t> failed;  // tickets whose batch failed
    esp_status last_status = ESP_OK;
    std::string last_message;
    bool stop = false;
    int64_t batches = 0, served = 0;
    double *h_pos = nullptr, *h_V = nullptr; // pinned staging
    std::thread worker;
    uint32_t magic = 0x45535356u;
};

namespace {

bool valid_server(const esp_server *s) { return s && s->magic == 0x45535356u; }

void serve(esp_server *s)
{
    std::vector<Request> batch;
    for (;;) {
        {
            std::unique_lock<std::mutex> lk(s->mu);
            s->cv_work.wait(lk, [&] { return s->stop || !s->queue.empty(); });
            if (s->queue.empty() && s->stop)
                return;
            batch.clear();
            int64_t total = 0;
            while (!s->queue.empty() && total + s->queue.front().n <= s->max_positions) {
                total += s->queue.front().n;
                batch.push_back(s->queue.front());
                s->queue.pop_front();
            }
        }
        int64_t total = 0;
        for (const Request &r : batch) {
            std::memcpy(s->h_pos + 3 * total, r.pos, size_t(r.n) * 3 * sizeof(double));
            total += r.n;
        }
        esp_status st = esp_eval(s->ctx, s->h_pos, total, s->h_V);
        std::string msg = st == ESP_OK ? std::string() : std::string(esp_last_error());
        if (st == ESP_OK) {
            int64_t o = 0;
            for (const Request &r : batch) {
                std::memcpy(r.V, s->h_V + o, size_t(r.n) * sizeof(double));
                o += r.n;
            }
        }
        {
            std::lock_guard<std::mutex> lk(s->mu);
            for (const Request &r : batch) {
                if (st != ESP_OK)
                    s->failed.push_back(r.ticket);
                s->done_upto = std::max(s->done_upto, r.ticket);
            }
            if (st != ESP_OK) {
                s->last_status = st;
                s->last_message = msg;
            }
            ++s->batches;
            s->served += total;
        }
        s->cv_done.notify_all();
    }
}

} // namespace

extern "C" {

esp_status esp_server_create(esp_ctx *ctx, int64_t max_positions, esp_server **out)
{
    last_error().clear();
    if (!valid_ctx(ctx) || ctx->device < 0)
        return fail(ESP_ERR_STATE, "invalid or host-only context");
    if (!out || max_positions < 1 || max_positions > (int64_t(1) << 28))
        return fail(ESP_ERR_INVALID, "bad server arguments");
    esp_server *s = new (std::nothrow) esp_server();
    if (!s)
        return fail(ESP_ERR_OOM, "host allocation of the server");
    s->ctx = ctx;
    s->max_positions = max_positions;
    DeviceGuard dg(ctx->device);
    cudaError_t e = fault("alloc") ? cudaErrorMemoryAllocation
                                   : cudaMallocHost(&s->h_pos, size_t(max_positions) * 3 * sizeof(double));
    if (e == cudaSuccess)
        e = cudaMallocHost(&s->h_V, size_t(max_positions) * sizeof(double));
    if (e != cudaSuccess) {
        if (s->h_pos)
            cudaFreeHost(s->h_pos);
        delete s;
        return cuda_fail(e, "allocating the server's pinned staging");
    }
    s->worker = std::thread(serve, s);
    *out = s;
    return ESP_OK;
}

esp_status esp_server_submit(esp_server *s, const double *positions, int64_t n, double *V_out, int64_t *ticket)
{
    if (!valid_server(s))
        return fail(ESP_ERR_STATE, "invalid server");
    if (n < 1 || n > s->max_positions || !positions || !V_out || !ticket)
        return fail(ESP_ERR_INVALID, "a request takes 1..%lld host positions", (long long)s->max_positions);
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->stop)
            return fail(ESP_ERR_STATE, "server is stopping");
        *ticket = s->next_ticket++;
        s->queue.push_back(Request{positions, n, V_out, *ticket});
    }
    s->cv_work.notify_one();
    return ESP_OK;
}

esp_status esp_server_wait(esp_server *s, int64_t ticket)
{
    if (!valid_server(s))
        return fail(ESP_ERR_STATE, "invalid server");
    std::unique_lock<std::mutex> lk(s->mu);
    if (ticket < 1 || ticket >= s->next_ticket)
        return fail(ESP_ERR_INVALID, "unknown ticket %lld", (long long)ticket);
    s->cv_done.wait(lk, [&] { return s->done_upto >= ticket; });
    for (int64_t f : s->failed)
        if (f == ticket)
            return fail(s->last_status, "batched evaluation failed: %s", s->last_message.c_str());
    return ESP_OK;
}

esp_status esp_server_stats(esp_server *s, int64_t *batches, int64_t *positions)
{
    if (!valid_server(s))
        return fail(ESP_ERR_STATE, "invalid server");
    std::lock_guard<std::mutex> lk(s->mu);
    if (batches)
        *batches = s->batches;
    if (positions)
        *positions = s->served;
    return ESP_OK;
}

void esp_server_destroy(esp_server *s)
{
    if (!valid_server(s))
        return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    if (s->worker.joinable())
        s->worker.join();
    {
        DeviceGuard dg(s->ctx->device);
        cudaFreeHost(s->h_pos);
        cudaFreeHost(s->h_V);
    }
    s->magic = 0;
    delete s;
}

} // extern "C"
