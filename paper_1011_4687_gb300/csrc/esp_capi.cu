// C ABI of the library (declared in include/esp.h).
//
// Data residency follows the paper (Sec. III): the environment is built and
// uploaded once by esp_create and stays read-only on the device; each
// esp_eval moves only positions in and potentials out.  Device scratch
// (staged positions, per-split partial sums) is owned by the context and
// grows on demand.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>

#include <cuda_runtime.h>

#include "../../include/esp.h"
#include "esp_ctx.h"
#include "esp_eval_core.h"
#include "esp_harmonics.h"

using namespace esp;

std::string &esp::last_error()
{
    static thread_local std::string msg;
    return msg;
}

namespace {

} // namespace

int esp::choose_splits(const esp_ctx *c, const TileView &v, int n, int prec)
{
    if (c->opt.pair_splits > 0)
        return std::max(1, std::min(c->opt.pair_splits, std::max(v.n_tiles, 1)));
    int per_cta = c->threads[prec] * c->ppt[prec];
    int blocks = (n + per_cta - 1) / per_cta;
    // many short CTAs: the round-robin deal of tiles balances, and the last
    // wave leaves little idle time (measured best at ~50 CTAs per SM)
    int target = 48 * c->num_sms;
    int s = (target + blocks - 1) / blocks;
    s = std::min(s, std::max(v.n_tiles, 1));
    s = std::min(s, 64);
    return std::max(s, 1);
}

int esp::plan_splits(const esp_ctx *c, const TileView &v, int n, int prec, int max_splits, EvalArgs &a)
{
    const int total = std::max(1, std::min(choose_splits(c, v, n, prec), max_splits));
    a.n_tiles = v.n_tiles;
    a.tiles = v.tiles;
    a.n_splits = total;
    single_group(a);
    if (prec == 0 || c->opt.pair_splits > 0 || v.n_groups <= 1 || v.n_groups > total)
        return total;
    double work = 0.0;
    for (int g = 0; g < v.n_groups; ++g)
        work += v.grp_work[g];
    int S[kMaxTileGroups], sum = 0;
    for (int g = 0; g < v.n_groups; ++g) {
        const int tiles = v.grp_tile[g + 1] - v.grp_tile[g];
        const int want = int(std::lround(total * v.grp_work[g] / std::max(work, 1e-300)));
        S[g] = std::max(1, std::min(want, tiles));
        sum += S[g];
    }
    while (sum > total) { // give back from the group with the most splits
        int big = 0;
        for (int g = 1; g < v.n_groups; ++g)
            if (S[g] > S[big])
                big = g;
        --S[big];
        --sum;
    }
    a.n_groups = v.n_groups;
    a.grp_split[0] = 0;
    for (int g = 0; g < v.n_groups; ++g) {
        a.grp_tile[g] = v.grp_tile[g];
        a.grp_split[g + 1] = a.grp_split[g] + S[g];
    }
    a.grp_tile[v.n_groups] = v.grp_tile[v.n_groups];
    a.n_splits = sum;
    return sum;
}

void esp::set_tile_groups(const std::vector<TileMeta> &T, TileView &v)
{
    // FP32 operations per evaluation by L (the kernel's algorithmic count) and
    // an FP64 point charge, for the split of the work between groups
    static const double kCost[kMaxL + 1] = {10.0, 26.0, 52.0, 95.0, 170.0};
    const double kPointCost = 12.0, kPoint32Cost = 10.0;
    v.n_tiles = int(T.size());
    int64_t n_small = 0, n_all = 0;
    v.n_p32 = 0;
    v.p32_off = 0;
    bool contiguous = true;
    for (const TileMeta &m : T) {
        n_all += m.n;
        if (m.cls != kClassPoint32)
            continue;
        if (n_small == 0)
            v.p32_off = m.off32;
        else if (int64_t(m.off32) != v.p32_off + n_small * rec32_stride(0))
            contiguous = false;
        n_small += m.n;
    }
    v.point_heavy = n_all > 0 && n_small * 10 >= n_all * 9;
    v.n_p32 = contiguous ? int(n_small) : 0;
    v.n_groups = 1;
    v.grp_tile[0] = 0;
    v.grp_tile[1] = int(T.size());
    v.grp_work[0] = 0.0;
    int n = 0, prev = -1;
    int bounds[kMaxTileGroups + 1];
    double work[kMaxTileGroups] = {0.0};
    for (size_t t = 0; t < T.size(); ++t) {
        const int g = T[t].cls == kClassPoint ? 0 : T[t].cls == kClassPoint32 ? 1 : 2 + (T[t].cls & 7);
        if (g < prev || g > kMaxL + 2)
            return; // not grouped by class: keep the plain deal
        if (g != prev) {
            if (n == kMaxTileGroups)
                return;
            bounds[n++] = int(t);
            prev = g;
        }
        work[n - 1] += T[t].n * (g == 0 ? kPointCost : g == 1 ? kPoint32Cost : kCost[g - 2]);
    }
    if (n == 0)
        return;
    bounds[n] = int(T.size());
    v.n_groups = n;
    for (int g = 0; g <= n; ++g)
        v.grp_tile[g] = bounds[g];
    for (int g = 0; g < n; ++g)
        v.grp_work[g] = work[g];
}

namespace {

esp_status ensure_scratch(esp_ctx *c, int64_t n, int splits, bool host_io, int64_t n_walkers)
{
    cudaError_t e;
    if (host_io && (e = c->in.ensure(size_t(n) * 3 * sizeof(double))) != cudaSuccess)
        return cuda_fail(e, "allocating position staging");
    if ((e = c->stage.ensure(size_t(n) * (3 * sizeof(double) + 6 * sizeof(float)) + 256)) != cudaSuccess)
        return cuda_fail(e, "allocating staged positions");
    if ((e = c->partial.ensure(size_t(n) * splits * sizeof(double))) != cudaSuccess)
        return cuda_fail(e, "allocating partial sums");
    (void)n_walkers;
    return ESP_OK;
}

Staged staged_view(esp_ctx *c, int64_t n)
{
    char *b = static_cast<char *>(c->stage.p);
    Staged st;
    st.x64 = reinterpret_cast<double *>(b);
    st.y64 = st.x64 + n;
    st.z64 = st.y64 + n;
    float *f = reinterpret_cast<float *>(st.z64 + n);
    st.xh = f;
    st.yh = f + n;
    st.zh = f + 2 * n;
    st.xl = f + 3 * n;
    st.yl = f + 4 * n;
    st.zl = f + 5 * n;
    return st;
}

// The device part of an evaluation over the view's tiles, enqueued on the
// context's stream: spatial order (FP32C, >= kSortMinPositions positions),
// staging, potential kernel (or the few-position path), fixed-order reduction
// into dV, and the walker energies into dE when dE is set.  timing: record
// ev[1] / ev[2] around the potential kernel.
esp_status pipeline(esp_ctx *c, const TileView &v, int prec, const double *d_pos, int64_t n, double *dV,
                    int64_t n_walkers, int64_t n_elec, double *dE, bool timing)
{
    // few positions: entries spread over threads instead of positions (up to
    // kSmallN positions for environments of point charges, whose entries the
    // path evaluates in FP32; up to kSmallNDistributions otherwise, since
    // distributions take FP64 there)
    const bool small_n = v.n_tiles > 0 && (n <= kSmallNDistributions || (n <= kSmallN && v.point_heavy));
    EvalArgs a;
    const int splits = small_n ? small_n_splits(v.n_tiles, c->num_sms, int(n)) : plan_splits(c, v, int(n), prec, 1 << 20, a);
    esp_status st = ensure_scratch(c, n, splits, false, n_walkers);
    if (st != ESP_OK)
        return st;
    cudaStream_t s = c->stream;
    cudaError_t e;
    // FP32C with many positions: stage them in spatial order (the kernel's
    // warp-uniform far/near votes then see compact groups of positions)
    const bool sorted = !small_n && prec == 1 && n >= kSortMinPositions;
    if (sorted && (e = c->sortbuf.ensure(sort_scratch_ints(int(n)) * sizeof(int))) != cudaSuccess)
        return cuda_fail(e, "allocating the position order");
    Staged stg = staged_view(c, n);
    int *slot_of = nullptr, *perm = nullptr;
    if (sorted && (e = launch_sort(d_pos, int(n), c->opt.qm_center, static_cast<int *>(c->sortbuf.p), &slot_of, &perm,
                                   s)) != cudaSuccess)
        return cuda_fail(e, "ordering positions");
    // (the few-position kernel reads and recentres the positions itself)
    if (!small_n && (e = launch_stage(d_pos, int(n), c->opt.qm_center, c->env.coord_quantum, stg, s, slot_of)) !=
                        cudaSuccess)
        return cuda_fail(e, "staging positions");
    a.n_pos = int(n);
    a.tile_size = c->env.tile_size;
    a.pos = stg;
    a.tiles = v.tiles;
    a.rec32 = static_cast<const float *>(c->rec32.p);
    a.rec64 = static_cast<const double *>(c->rec64.p);
    a.boys32 = static_cast<const float *>(c->boys32.p);
    a.boys64 = static_cast<const double *>(c->boys64.p);
    a.partial = static_cast<double *>(c->partial.p);
    a.near_r = float(c->opt.near_radius < 0.0 ? kDefaultNearRadius : c->opt.near_radius);
    if (timing && (e = cudaEventRecord(c->ev[1], s)) != cudaSuccess)
        return cuda_fail(e, "recording a timing event");
    if (v.n_tiles == 0) {
        if ((e = cudaMemsetAsync(a.partial, 0, size_t(n) * splits * sizeof(double), s)) != cudaSuccess)
            return cuda_fail(e, "clearing partial sums");
    } else if (small_n) {
        SmallArgs sa;
        sa.n_pos = int(n);
        sa.n_tiles = v.n_tiles;
        sa.pos_in = d_pos;
        sa.cx = c->opt.qm_center[0];
        sa.cy = c->opt.qm_center[1];
        sa.cz = c->opt.qm_center[2];
        sa.tiles = v.tiles;
        sa.rec64 = a.rec64;
        sa.rec32 = a.rec32;
        sa.boys64 = a.boys64;
        sa.quantum = c->env.coord_quantum;
        sa.fp32 = prec == 1 && v.n_p32 > 0;
        sa.p32_off = v.p32_off;
        sa.n_p32 = v.n_p32;
        sa.partial = a.partial;
        if ((e = launch_small_n(sa, splits, dV, s)) != cudaSuccess)
            return cuda_fail(e, "launching the few-position kernels");
    } else if ((e = launch_potential(prec, a, c->threads[prec], c->ppt[prec], s)) != cudaSuccess) {
        return cuda_fail(e, "launching the potential kernel");
    }
    if (timing && (e = cudaEventRecord(c->ev[2], s)) != cudaSuccess)
        return cuda_fail(e, "recording a timing event");
    if ((!small_n || v.n_tiles == 0) && (e = launch_reduce(a.partial, splits, int(n), dV, s, perm)) != cudaSuccess)
        return cuda_fail(e, "launching the partial-sum reduction");
    if (dE && (e = launch_walkers(dV, int(n_walkers), int(n_elec), dE, s)) != cudaSuccess)
        return cuda_fail(e, "launching the walker-energy reduction");
    return ESP_OK;
}

// The evaluation shared by esp_eval and esp_eval_walkers: argument checks,
// host <-> device copies around the pipeline over every tile.
esp_status run_eval(esp_ctx *c, const double *positions, int64_t n, double *V_out, int64_t n_walkers,
                    int64_t n_elec, double *E_out)
{
    if (n < 0 || n > (int64_t(1) << 30))
        return fail(ESP_ERR_INVALID, "position count %lld out of range", (long long)n);
    if (n == 0)
        return ESP_OK;
    if (!positions || (!V_out && !E_out))
        return fail(ESP_ERR_INVALID, "null positions or outputs");
    BusyGuard busy(c->busy);
    if (!busy.acquired)
        return fail(ESP_ERR_STATE, "context is in use by another thread");
    DeviceGuard dg(c->device);
    if (!dg.ok)
        return fail(ESP_ERR_CUDA, "cannot select device %d", c->device);
    Space sp = classify(positions, c->device);
    Space sv = V_out ? classify(V_out, c->device) : sp;
    Space se = E_out ? classify(E_out, c->device) : sp;
    if (sp == Space::Invalid || sv != sp || se != sp)
        return fail(ESP_ERR_INVALID, "positions and outputs must all be host memory or all be device memory of "
                                     "device %d", c->device);
    const bool host_io = sp == Space::Host;
    const int prec = c->opt.precision == ESP_FP64 ? 0 : 1;
    cudaStream_t s = c->stream;
    cudaError_t e;
    if (host_io) {
        if ((e = c->in.ensure(size_t(n) * 3 * sizeof(double))) != cudaSuccess ||
            (e = c->vout.ensure(size_t(n) * sizeof(double))) != cudaSuccess ||
            (n_walkers > 0 && (e = c->eout.ensure(size_t(n_walkers) * sizeof(double))) != cudaSuccess))
            return cuda_fail(e, "allocating host-call staging");
    } else if (!V_out && (e = c->vout.ensure(size_t(n) * sizeof(double))) != cudaSuccess) {
        return cuda_fail(e, "allocating potentials");
    }
    c->timed_valid = false;
    if (c->timing && (e = cudaEventRecord(c->ev[0], s)) != cudaSuccess)
        return cuda_fail(e, "recording a timing event");
    const double *d_pos = positions;
    if (host_io) {
        if ((e = cudaMemcpyAsync(c->in.p, positions, size_t(n) * 3 * sizeof(double), cudaMemcpyHostToDevice, s)) !=
            cudaSuccess)
            return cuda_fail(e, "copying positions to the device");
        d_pos = static_cast<const double *>(c->in.p);
    }
    double *dV = (!host_io && V_out) ? V_out : static_cast<double *>(c->vout.p);
    double *dE = E_out ? (host_io ? static_cast<double *>(c->eout.p) : E_out) : nullptr;
    esp_status st = pipeline(c, c->full, prec, d_pos, n, dV, n_walkers, n_elec, dE, c->timing);
    if (st != ESP_OK)
        return st;
    if (c->timing) {
        if ((e = cudaEventRecord(c->ev[3], s)) != cudaSuccess)
            return cuda_fail(e, "recording a timing event");
        c->timed_valid = true;
    }
    if (host_io) {
        if (V_out && (e = cudaMemcpyAsync(V_out, dV, size_t(n) * sizeof(double), cudaMemcpyDeviceToHost, s)) !=
                         cudaSuccess)
            return cuda_fail(e, "copying potentials to the host");
        if (E_out &&
            (e = cudaMemcpyAsync(E_out, dE, size_t(n_walkers) * sizeof(double), cudaMemcpyDeviceToHost, s)) !=
                cudaSuccess)
            return cuda_fail(e, "copying walker energies to the host");
        if ((e = cudaStreamSynchronize(s)) != cudaSuccess)
            return cuda_fail(e, "evaluation");
    }
    return ESP_OK;
}

} // namespace

esp_status esp::eval_view(esp_ctx *c, const TileView &v, int prec, const double *d_pos, int64_t n, double *d_V)
{
    if (n < 0 || n > (int64_t(1) << 30))
        return fail(ESP_ERR_INVALID, "position count %lld out of range", (long long)n);
    if (n == 0)
        return ESP_OK;
    DeviceGuard dg(c->device);
    if (!dg.ok)
        return fail(ESP_ERR_CUDA, "cannot select device %d", c->device);
    return pipeline(c, v, prec, d_pos, n, d_V, 0, 0, nullptr, false);
}

namespace {

template <typename T>
cudaError_t upload(DevBuf &b, const std::vector<T> &v, int64_t &bytes)
{
    size_t n = v.size() * sizeof(T);
    cudaError_t e = b.ensure(std::max<size_t>(n, 16));
    if (e != cudaSuccess)
        return e;
    bytes += int64_t(b.bytes);
    if (n == 0)
        return cudaSuccess;
    return cudaMemcpy(b.p, v.data(), n, cudaMemcpyHostToDevice);
}

void release_all(esp_ctx *c)
{
    for (cudaEvent_t &ev : c->ev)
        if (ev) {
            cudaEventDestroy(ev);
            ev = nullptr;
        }
    DevBuf *bufs[] = {&c->tiles, &c->rec32, &c->rec64, &c->boys32, &c->boys64,
                      &c->in, &c->stage, &c->partial, &c->vout, &c->eout, &c->sortbuf};
    for (DevBuf *b : bufs)
        b->release();
}

// Host emulation of the FP32C kernel for one position (one split): the same
// per-tile core, the same staging, near test and accumulation.
double host_eval_f32c(const esp_ctx *c, const double *C)
{
    const float *boys32 = boys_table32().data();
    const double *boys64 = boys_table64().data();
    float ch[1][3], cl[1][3];
    double c64[1][3];
    for (int d = 0; d < 3; ++d) {
        c64[0][d] = C[d];
        double h = quantize_hi(C[d], c->env.coord_quantum);
        ch[0][d] = float(h);
        cl[0][d] = float(C[d] - h);
    }
    float S[1] = {0.0f}, Cc[1] = {0.0f};
    double acc64[1] = {0.0};
    const float near_r = float(c->opt.near_radius < 0.0 ? kDefaultNearRadius : c->opt.near_radius);
    for (const TileMeta &m : c->env.tiles) {
        if (m.cls == kClassPoint) {
            tile_points_f64<1>(c->env.rec64.data() + m.off64, m.n, c64, acc64);
            continue;
        }
        if (m.cls == kClassPoint32) {
            const bool none[1] = {false};
            float th0[1][3];
            for (int d = 0; d < 3; ++d)
                th0[0][d] = 0.0f - ch[0][d];
            tile_f32c<0, 1, true, false, false>(c->env.rec32.data() + m.off32, m.n, th0, cl, cl, none, S, Cc, boys32);
            continue;
        }
        bool nearq[1], farq, relq;
        classify_tile(m, ch[0][0], ch[0][1], ch[0][2], near_r, nearq[0], farq, relq);
        const float *r = c->env.rec32.data() + m.off32;
        const float ct[3] = {m.cx, m.cy, m.cz};
        float th[1][3], dq[1][3];
        for (int d = 0; d < 3; ++d) {
            th[0][d] = ct[d] - ch[0][d];
            dq[0][d] = th[0][d] - cl[0][d];
        }
#define ESP_TILE(CLS, LL, SH)                                                                    \
    case CLS:                                                                                    \
        if (relq && !nearq[0])                                                                   \
            tile_f32c<LL, 1, true, SH, false, true>(r, m.n, th, cl, dq, nearq, S, Cc, boys32);   \
        else if (farq)                                                                           \
            tile_f32c<LL, 1, true, SH>(r, m.n, th, cl, dq, nearq, S, Cc, boys32);                \
        else                                                                                     \
            tile_f32c<LL, 1, false, SH>(r, m.n, th, cl, dq, nearq, S, Cc, boys32);               \
        break;
        switch (m.cls) {
            ESP_TILE(0, 0, false)
            ESP_TILE(1, 1, false)
            ESP_TILE(2, 2, false)
            ESP_TILE(3, 3, false)
            ESP_TILE(4, 4, false)
            ESP_TILE(8, 0, true)
            ESP_TILE(9, 1, true)
            ESP_TILE(10, 2, true)
            ESP_TILE(11, 3, true)
            default:
            ESP_TILE(12, 4, true)
        }
#undef ESP_TILE
        if (nearq[0])
            acc64[0] += tile_f64_one_any(m.cls, c->env.rec64.data() + m.off64, m.n, C[0], C[1], C[2], boys64);
    }
    return (double(S[0]) + double(Cc[0])) + acc64[0];
}

double host_eval_f64(const esp_ctx *c, const double *C)
{
    const double *boys = boys_table64().data();
    double s = 0.0, cc = 0.0;
    for (const TileMeta &m : c->env.tiles) {
        const double *r = c->env.rec64.data() + m.off64;
        double v;
        if (is_point_class(m.cls)) {
            double c64[1][3] = {{C[0], C[1], C[2]}}, acc[1] = {0.0};
            tile_points_f64<1>(r, m.n, c64, acc);
            v = acc[0];
        } else {
            v = tile_f64_one_any(m.cls, r, m.n, C[0], C[1], C[2], boys);
        }
        two_sum_acc(s, cc, v);
    }
    return s + cc;
}

} // namespace

extern "C" {

void esp_default_options(esp_options *opt)
{
    if (!opt)
        return;
    std::memset(opt, 0, sizeof(*opt));
    opt->size = int32_t(sizeof(esp_options));
    opt->precision = ESP_FP32C;
    opt->screen_tol = 1e-12;
    opt->cuda_stream = nullptr;
    opt->device = -1;
    opt->near_radius = -1.0;
    opt->point32_max_charge = -1.0;
}

int32_t esp_abi_version(void) { return ESP_ABI_VERSION; }

const char *esp_last_error(void) { return last_error().c_str(); }

const char *esp_status_string(esp_status s)
{
    switch (s) {
    case ESP_OK: return "ok";
    case ESP_ERR_INVALID: return "invalid argument";
    case ESP_ERR_OOM: return "out of memory";
    case ESP_ERR_CUDA: return "CUDA error";
    case ESP_ERR_TIMEOUT: return "device wait timed out";
    case ESP_ERR_STATE: return "context busy or invalid";
    case ESP_ERR_UNSUPPORTED: return "unsupported";
    }
    return "unknown status";
}

esp_status esp_create(const esp_point_charge *charges, int64_t n_charges, const esp_gauss_pair *pairs,
                      const double *weights, int64_t n_pairs, const esp_options *opt_in, esp_ctx **out)
{
    last_error().clear();
    if (!out)
        return fail(ESP_ERR_INVALID, "out is NULL");
    esp_options opt;
    esp_default_options(&opt);
    if (opt_in) {
        if (opt_in->size != int32_t(sizeof(esp_options)))
            return fail(ESP_ERR_INVALID, "esp_options.size is %d, expected %d (call esp_default_options)",
                        opt_in->size, int(sizeof(esp_options)));
        opt = *opt_in;
    }
    if (opt.precision != ESP_FP64 && opt.precision != ESP_FP32C)
        return fail(ESP_ERR_INVALID, "unknown precision %d", opt.precision);
    if (opt.flags & ~ESP_FLAG_HOST_ONLY)
        return fail(ESP_ERR_INVALID, "unknown flags 0x%x", opt.flags);
    if (!(opt.near_radius < 1e6))
        return fail(ESP_ERR_INVALID, "bad near_radius");
    if (!(opt.point32_max_charge < 1e30))
        return fail(ESP_ERR_INVALID, "bad point32_max_charge");
    const int thr_ok[] = {0, 64, 128, 256};
    bool tok = false;
    for (int t : thr_ok)
        tok |= opt.threads_per_block == t;
    if (!tok || opt.positions_per_thread < 0 || opt.positions_per_thread > 4 || opt.pair_splits < 0)
        return fail(ESP_ERR_INVALID, "bad launch-shape options");

    esp_ctx *c = new (std::nothrow) esp_ctx();
    if (!c)
        return fail(ESP_ERR_OOM, "host allocation of the context");
    c->opt = opt;
    std::string err;
    esp_status st = build_environment(charges, n_charges, pairs, weights, n_pairs, opt, c->env, err);
    if (st != ESP_OK) {
        delete c;
        return fail(st, "%s", err.c_str());
    }
    c->n_tiles = int(c->env.tiles.size());
    set_tile_groups(c->env.tiles, c->full);
    if (opt.flags & ESP_FLAG_HOST_ONLY) {
        c->device = -1;
        *out = c;
        return ESP_OK;
    }
    int dev = opt.device;
    if (dev < 0 && cudaGetDevice(&dev) != cudaSuccess) {
        delete c;
        return fail(ESP_ERR_CUDA, "no CUDA device");
    }
    c->device = dev;
    DeviceGuard dg(dev);
    if (!dg.ok) {
        delete c;
        return fail(ESP_ERR_CUDA, "cannot select device %d", dev);
    }
    cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, dev);
    c->stream = static_cast<cudaStream_t>(opt.cuda_stream);
    c->n_tiles = int(c->env.tiles.size());
    if (opt.threads_per_block) {
        c->threads[0] = c->threads[1] = opt.threads_per_block;
    }
    if (opt.positions_per_thread) {
        c->ppt[1] = opt.positions_per_thread;
        c->ppt[0] = std::min(opt.positions_per_thread, 2); // FP64 keeps at most 2 positions per thread
    }
    for (int p = 0; p < 2; ++p) {
        if (!potential_shape_supported(p, c->threads[p], c->ppt[p])) {
            delete c;
            return fail(ESP_ERR_INVALID, "launch shape %d threads x %d positions is not built for %s", c->threads[p],
                        c->ppt[p], p == 0 ? "FP64" : "FP32C");
        }
    }
    cudaError_t e = fault("upload") ? cudaErrorInvalidValue : cudaSuccess;
    int64_t bytes = 0;
    if (e != cudaSuccess || (e = upload(c->tiles, c->env.tiles, bytes)) != cudaSuccess ||
        (e = upload(c->rec32, c->env.rec32, bytes)) != cudaSuccess ||
        (e = upload(c->rec64, c->env.rec64, bytes)) != cudaSuccess ||
        (e = upload(c->boys32, boys_table32(), bytes)) != cudaSuccess ||
        (e = upload(c->boys64, boys_table64(), bytes)) != cudaSuccess) {
        release_all(c);
        delete c;
        return cuda_fail(e, "uploading the environment");
    }
    c->device_bytes = bytes;
    c->full.tiles = static_cast<const TileMeta *>(c->tiles.p);
    // keep a host copy of the records only while it is small (test hook use)
    if (c->env.rec64.size() * sizeof(double) > (size_t(256) << 20)) {
        c->host_copy = false;
        std::vector<float>().swap(c->env.rec32);
        std::vector<double>().swap(c->env.rec64);
    }
    *out = c;
    return ESP_OK;
}

esp_status esp_eval(esp_ctx *ctx, const double *positions, int64_t n, double *V_out)
{
    last_error().clear();
    if (!valid_ctx(ctx) || ctx->device < 0)
        return fail(ESP_ERR_STATE, "invalid or host-only context");
    if (n > 0 && !V_out)
        return fail(ESP_ERR_INVALID, "V_out is NULL");
    return run_eval(ctx, positions, n, V_out, 0, 0, nullptr);
}

esp_status esp_eval_walkers(esp_ctx *ctx, const double *positions, int64_t n_walkers, int64_t n_elec,
                            double *V_out, double *E_out)
{
    last_error().clear();
    if (!valid_ctx(ctx) || ctx->device < 0)
        return fail(ESP_ERR_STATE, "invalid or host-only context");
    if (n_walkers < 0 || n_elec < 0 || n_walkers > (int64_t(1) << 30) || n_elec > (int64_t(1) << 20))
        return fail(ESP_ERR_INVALID, "bad walker counts");
    if (n_walkers * n_elec > (int64_t(1) << 30))
        return fail(ESP_ERR_INVALID, "too many positions");
    if (n_walkers > 0 && !E_out)
        return fail(ESP_ERR_INVALID, "E_out is NULL");
    if (n_walkers > 0 && n_elec == 0) {
        // every walker has zero electrons: its energy is 0
        DeviceGuard dg(ctx->device);
        Space se = classify(E_out, ctx->device);
        if (se == Space::Invalid)
            return fail(ESP_ERR_INVALID, "E_out on another device");
        if (se == Space::Host) {
            std::memset(E_out, 0, size_t(n_walkers) * sizeof(double));
            return ESP_OK;
        }
        cudaError_t e = cudaMemsetAsync(E_out, 0, size_t(n_walkers) * sizeof(double), ctx->stream);
        return e == cudaSuccess ? ESP_OK : cuda_fail(e, "clearing walker energies");
    }
    return run_eval(ctx, positions, n_walkers * n_elec, V_out, n_walkers, n_elec, E_out);
}

esp_status esp_set_precision(esp_ctx *ctx, int32_t precision)
{
    if (!valid_ctx(ctx))
        return fail(ESP_ERR_STATE, "invalid context");
    if (precision != ESP_FP64 && precision != ESP_FP32C)
        return fail(ESP_ERR_INVALID, "unknown precision %d", precision);
    BusyGuard busy(ctx->busy);
    if (!busy.acquired)
        return fail(ESP_ERR_STATE, "context is in use by another thread");
    ctx->opt.precision = precision;
    return ESP_OK;
}

esp_status esp_get_info(const esp_ctx *ctx, esp_info *info)
{
    if (!valid_ctx(ctx) || !info)
        return fail(ESP_ERR_INVALID, "invalid context or info pointer");
    std::memset(info, 0, sizeof(*info));
    info->n_point_charges = ctx->env.n_point_charges;
    info->n_pairs_in = ctx->env.n_pairs_in;
    info->n_distributions = ctx->env.n_distributions;
    info->n_screened = ctx->env.n_screened;
    for (int l = 0; l <= kMaxL; ++l)
        info->n_by_L[l] = ctx->env.n_by_L[l];
    info->n_tiles = ctx->n_tiles;
    info->n_near_tiles = ctx->env.n_near_tiles;
    info->device_bytes = ctx->device_bytes;
    info->precision = ctx->opt.precision;
    info->tile_size = ctx->env.tile_size;
    int p = ctx->opt.precision == ESP_FP64 ? 0 : 1;
    info->threads_per_block = ctx->threads[p];
    info->positions_per_thread = ctx->ppt[p];
    info->pair_splits = ctx->opt.pair_splits;
    info->device = ctx->device;
    return ESP_OK;
}

esp_status esp_set_timing(esp_ctx *ctx, int32_t enable)
{
    if (!valid_ctx(ctx) || ctx->device < 0)
        return fail(ESP_ERR_STATE, "invalid or host-only context");
    BusyGuard busy(ctx->busy);
    if (!busy.acquired)
        return fail(ESP_ERR_STATE, "context is in use by another thread");
    DeviceGuard dg(ctx->device);
    if (enable && !ctx->ev[0]) {
        for (cudaEvent_t &ev : ctx->ev) {
            cudaError_t e = cudaEventCreate(&ev);
            if (e != cudaSuccess)
                return cuda_fail(e, "creating timing events");
        }
    }
    ctx->timing = enable != 0;
    ctx->timed_valid = false;
    return ESP_OK;
}

esp_status esp_last_timing(esp_ctx *ctx, double *potential_ms, double *pipeline_ms)
{
    if (!valid_ctx(ctx) || ctx->device < 0)
        return fail(ESP_ERR_STATE, "invalid or host-only context");
    if (!ctx->timing || !ctx->timed_valid)
        return fail(ESP_ERR_STATE, "no timed evaluation (call esp_set_timing first)");
    DeviceGuard dg(ctx->device);
    cudaError_t e = cudaEventSynchronize(ctx->ev[3]);
    if (e != cudaSuccess)
        return cuda_fail(e, "waiting for the timed evaluation");
    float k = 0.f, t = 0.f;
    if ((e = cudaEventElapsedTime(&k, ctx->ev[1], ctx->ev[2])) != cudaSuccess ||
        (e = cudaEventElapsedTime(&t, ctx->ev[0], ctx->ev[3])) != cudaSuccess)
        return cuda_fail(e, "reading timing events");
    if (potential_ms)
        *potential_ms = k;
    if (pipeline_ms)
        *pipeline_ms = t;
    return ESP_OK;
}

esp_status esp_synchronize(esp_ctx *ctx)
{
    if (!valid_ctx(ctx) || ctx->device < 0)
        return fail(ESP_ERR_STATE, "invalid or host-only context");
    DeviceGuard dg(ctx->device);
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    return e == cudaSuccess ? ESP_OK : cuda_fail(e, "synchronize");
}

void esp_destroy(esp_ctx *ctx)
{
    if (!valid_ctx(ctx))
        return;
    if (ctx->device >= 0) {
        DeviceGuard dg(ctx->device);
        cudaStreamSynchronize(ctx->stream);
        release_all(ctx);
    }
    ctx->magic = 0;
    delete ctx;
}

esp_status esp_debug_boys(int32_t precision, int32_t nmax, double T, double *F_out)
{
    if (!F_out || nmax < 0 || nmax > kMaxL || !(T >= 0.0) || !(T < 1e30))
        return fail(ESP_ERR_INVALID, "bad Boys arguments");
    if (precision == ESP_FP64) {
        const double *tab = boys_table64().data();
        double F[kMaxL + 1];
        switch (nmax) {
        case 0: { double G[1]; boys_eval<0, double>(T, tab, G); F[0] = G[0]; break; }
        case 1: { double G[2]; boys_eval<1, double>(T, tab, G); for (int i = 0; i < 2; ++i) F[i] = G[i]; break; }
        case 2: { double G[3]; boys_eval<2, double>(T, tab, G); for (int i = 0; i < 3; ++i) F[i] = G[i]; break; }
        case 3: { double G[4]; boys_eval<3, double>(T, tab, G); for (int i = 0; i < 4; ++i) F[i] = G[i]; break; }
        default: { double G[5]; boys_eval<4, double>(T, tab, G); for (int i = 0; i < 5; ++i) F[i] = G[i]; break; }
        }
        for (int i = 0; i <= nmax; ++i)
            F_out[i] = F[i];
        return ESP_OK;
    }
    if (precision == ESP_FP32C) {
        const float *tab = boys_table32().data();
        float F[kMaxL + 1];
        float Tf = float(T);
        switch (nmax) {
        case 0: { float G[1]; boys_eval<0, float>(Tf, tab, G); F[0] = G[0]; break; }
        case 1: { float G[2]; boys_eval<1, float>(Tf, tab, G); for (int i = 0; i < 2; ++i) F[i] = G[i]; break; }
        case 2: { float G[3]; boys_eval<2, float>(Tf, tab, G); for (int i = 0; i < 3; ++i) F[i] = G[i]; break; }
        case 3: { float G[4]; boys_eval<3, float>(Tf, tab, G); for (int i = 0; i < 4; ++i) F[i] = G[i]; break; }
        default: { float G[5]; boys_eval<4, float>(Tf, tab, G); for (int i = 0; i < 5; ++i) F[i] = G[i]; break; }
        }
        for (int i = 0; i <= nmax; ++i)
            F_out[i] = F[i];
        return ESP_OK;
    }
    return fail(ESP_ERR_INVALID, "unknown precision");
}

int32_t esp_debug_fault_active(const char *what) { return what && fault(what) ? 1 : 0; }

esp_status esp_debug_solid_harmonics(int32_t L, const double *u, double *out)
{
    if (L < 0 || L > kMaxExpDegree || !u || !out)
        return fail(ESP_ERR_INVALID, "bad solid-harmonic arguments");
    static HarmonicConsts h;
    static bool ready = false;
    if (!ready) {
        harmonic_consts(h);
        ready = true;
    }
    solid_harmonics(u[0], u[1], u[2], L, h.a, h.b, h.sec, h.sub, [&](int k, double v) { out[k] = v; });
    return ESP_OK;
}

esp_status esp_debug_host_eval(const esp_ctx *ctx, const double *positions, int64_t n, double *V_out)
{
    if (!valid_ctx(ctx) || n < 0 || (n > 0 && (!positions || !V_out)))
        return fail(ESP_ERR_INVALID, "bad arguments");
    if (!ctx->host_copy)
        return fail(ESP_ERR_UNSUPPORTED, "host copy of the records was dropped (environment too large)");
    for (int64_t i = 0; i < n; ++i) {
        double C[3];
        for (int d = 0; d < 3; ++d)
            C[d] = positions[3 * i + d] - ctx->opt.qm_center[d];
        V_out[i] = ctx->opt.precision == ESP_FP32C ? host_eval_f32c(ctx, C) : host_eval_f64(ctx, C);
    }
    return ESP_OK;
}

} // extern "C"

// ---------------------------------------------------------------------------
// esp_eval_noalloc: the same pipeline with its scratch in a fixed device array
// instead of context-owned cudaMalloc buffers.
// ---------------------------------------------------------------------------
namespace {

constexpr int64_t kNoallocMaxPositions = ESP_NOALLOC_MAX_POSITIONS;
constexpr int kNoallocMaxSplits = 8;
constexpr size_t kNoallocStageBytes = size_t(kNoallocMaxPositions) * (3 * sizeof(double) + 6 * sizeof(float));
constexpr size_t kNoallocBytes = kNoallocStageBytes + size_t(kNoallocMaxPositions) * kNoallocMaxSplits * sizeof(double);

} // namespace

// Scratch of esp_eval_noalloc: staged positions, then per-split partial sums.
// Host code must not pass this symbol to a kernel; it uses the device address
// obtained by cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

namespace {

// Device address of g_noalloc_scratch on the current device.  Looked up on
// every call (cheap): a cached address would go stale if the device's primary
// context were reset between calls.
esp_status noalloc_scratch(void **out)
{
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
        return cuda_fail(e == cudaSuccess ? cudaErrorInvalidSymbol : e, "locating the no-allocation scratch");
    *out = p;
    return ESP_OK;
}

} // namespace

extern "C" esp_status esp_eval_noalloc(esp_ctx *ctx, const double *positions, int64_t n, double *V_out)
{
    last_error().clear();
    if (!valid_ctx(ctx) || ctx->device < 0)
        return fail(ESP_ERR_STATE, "invalid or host-only context");
    if (n < 0 || n > kNoallocMaxPositions)
        return fail(ESP_ERR_INVALID, "n = %lld outside [0, %lld] for esp_eval_noalloc", (long long)n,
                    (long long)kNoallocMaxPositions);
    if (n == 0)
        return ESP_OK;
    if (!positions || !V_out)
        return fail(ESP_ERR_INVALID, "null positions or V_out");
    BusyGuard busy(ctx->busy);
    if (!busy.acquired)
        return fail(ESP_ERR_STATE, "context is in use by another thread");
    DeviceGuard dg(ctx->device);
    if (!dg.ok)
        return fail(ESP_ERR_CUDA, "cannot select device %d", ctx->device);
    if (classify(positions, ctx->device) != Space::Device || classify(V_out, ctx->device) != Space::Device)
        return fail(ESP_ERR_INVALID, "esp_eval_noalloc takes device memory of device %d only", ctx->device);
    // this call records no timing events: a timing query must not report the
    // kernel times of an earlier esp_eval as this call's
    ctx->timed_valid = false;
    void *base = nullptr;
    esp_status st = noalloc_scratch(&base);
    if (st != ESP_OK)
        return st;
    const int prec = ctx->opt.precision == ESP_FP64 ? 0 : 1;
    EvalArgs a;
    const int splits = plan_splits(ctx, ctx->full, int(n), prec, kNoallocMaxSplits, a);
    char *b = static_cast<char *>(base);
    Staged stg;
    stg.x64 = reinterpret_cast<double *>(b);
    stg.y64 = stg.x64 + n;
    stg.z64 = stg.y64 + n;
    float *f = reinterpret_cast<float *>(stg.z64 + n);
    stg.xh = f;
    stg.yh = f + n;
    stg.zh = f + 2 * n;
    stg.xl = f + 3 * n;
    stg.yl = f + 4 * n;
    stg.zl = f + 5 * n;
    double *partial = reinterpret_cast<double *>(b + kNoallocStageBytes);
    cudaStream_t s = ctx->stream;
    cudaError_t e;
    if ((e = launch_stage(positions, int(n), ctx->opt.qm_center, ctx->env.coord_quantum, stg, s)) != cudaSuccess)
        return cuda_fail(e, "staging positions");
    if (ctx->n_tiles == 0) {
        // nothing writes the partial sums: they must start at zero
        if ((e = cudaMemsetAsync(partial, 0, size_t(n) * splits * sizeof(double), s)) != cudaSuccess)
            return cuda_fail(e, "clearing partial sums");
    } else {
        a.n_pos = int(n);
        a.tile_size = ctx->env.tile_size;
        a.pos = stg;
        a.tiles = static_cast<const TileMeta *>(ctx->tiles.p);
        a.rec32 = static_cast<const float *>(ctx->rec32.p);
        a.rec64 = static_cast<const double *>(ctx->rec64.p);
        a.boys32 = static_cast<const float *>(ctx->boys32.p);
        a.boys64 = static_cast<const double *>(ctx->boys64.p);
        a.partial = partial;
        a.near_r = float(ctx->opt.near_radius < 0.0 ? kDefaultNearRadius : ctx->opt.near_radius);
        if ((e = launch_potential(prec, a, ctx->threads[prec], ctx->ppt[prec], s)) != cudaSuccess)
            return cuda_fail(e, "launching the potential kernel");
    }
    if ((e = launch_reduce(partial, splits, int(n), V_out, s)) != cudaSuccess)
        return cuda_fail(e, "launching the partial-sum reduction");
    return ESP_OK;
}
