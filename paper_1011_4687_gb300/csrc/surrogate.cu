// Learned surrogate of the environment potential over the QM region.
//
//   V_sur(r) = V_near(r) + sum_lm c_lm S_lm(u) + s f_theta(u),  u = (r - centre) / R
//
// V_near : the exact sum (FP32C potential kernel) over the near tiles: every
//          tile whose bounding sphere comes closer to the centre than
//          `far_radius`, or whose Gaussians reach into the QM sphere
//          (p_min (d - R)^2 < 30); near nuclei are therefore always summed
//          exactly;
// c_lm   : FP64 interior expansion of the far tiles' potential, which is
//          harmonic inside the QM sphere (esp_harmonics.h): each coefficient is
//          the projection of the far field on Y_lm over the sphere |u| = 1,
//          computed by Gauss-Legendre x trapezoid quadrature of the far field
//          evaluated there by the exact FP64 kernel (exact up to aliasing from
//          degrees >= L + 25, which fall off as (R / far_radius)^l);
// f_theta: MLP on Fourier features (surrogate_kernels.cu) trained on the
//          normalised residual (V_far - expansion) / s of the far field with
//          the library's own BF16 tensor-core forward/backward kernels and
//          Adam, labels from the exact kernel over the far tiles; inference
//          runs the whole network in one tcgen05 kernel (surrogate_tc.cu).
// Training positions follow the walker law (half) and fill the sphere
// uniformly (half).  A voxel map, built from validation against the exact
// far-tile sum, marks where expansion + network meet the tolerance; positions
// elsewhere, near point charges, or picked by the online probe (every
// probe_stride-th position) are evaluated exactly over all tiles.  A probe
// that misses the tolerance withdraws its voxel, and the positions of the same
// call in withdrawn voxels are evaluated exactly before the call returns.
#include <cmath>
#include <cstdio>
#include <random>
#include <vector>

#include "esp_ctx.h"
#include "esp_harmonics.h"
#include "surrogate_kernels.h"

using namespace esp;
using namespace esp::sur;

namespace {

// flat parameter layout: W1[256x64] b1 W2[256x256] b2 W3 b3 W4 b4 w5[256] b5
struct Layout {
    size_t w[kLayers], b[kLayers], w5, b5, total;
    int in[kLayers];
    Layout()
    {
        size_t o = 0;
        for (int l = 0; l < kLayers; ++l) {
            in[l] = l == 0 ? kFeat : kHidden;
            w[l] = o;
            o += size_t(kHidden) * in[l];
            b[l] = o;
            o += kHidden;
        }
        w5 = o;
        o += kHidden;
        b5 = o;
        o += 1;
        total = o;
    }
};

const Layout &layout()
{
    static Layout L;
    return L;
}

} // namespace

struct esp_surrogate {
    esp_ctx *ctx = nullptr;
    esp_surrogate_cfg cfg;
    double centre[3] = {0, 0, 0};
    double inv_r = 1.0 / 6.0;
    double scale = 1.0;                 // s: residual normalisation
    int degree = 0, ncoef = 0;          // expansion degree L, (L + 1)^2 coefficients
    std::vector<double> coef;           // c_lm (esp_harmonics.h order)
    std::vector<float> freq;            // [kFreq][3]
    std::vector<float> params;          // FP32 master copy (host mirror after training)
    std::vector<unsigned char> trust;   // [dim^3]
    int dim = 0;
    double train_loss = 0.0, valid_max_err = 0.0, trusted_fraction = 0.0;
    double valid_rms_err = 0.0, base_max_err = 0.0, base_rms_err = 0.0; // with the network / expansion alone
    double base_trusted_fraction = 0.0; // the trust map of the expansion alone
    int64_t n_near_entries = 0, n_far_entries = 0;
    int probe_offset = 0;
    // near / far split of the context's tiles
    std::vector<TileMeta> near_tiles, far_tiles;
    TileView near_view, far_view;
    DevBuf d_near_tiles, d_far_tiles;
    // device state
    DevBuf d_params, d_params_bf, d_grad, d_m, d_v, d_coef, d_freq, d_trust;
    DevBuf d_X, d_Z, d_H, d_dZ, d_y, d_dy, d_part, d_t, d_loss;   // per-chunk activations
    DevBuf d_flag, d_pre, d_tot, d_count, d_cpos, d_cidx, d_cV, d_nfail;
    DevBuf d_wpk, d_tcerr, d_ynet;      // packed weights, kernel status, fused-inference outputs
    DevBuf d_gemmerr;                   // status word of the training GEMMs
    bool packed = false;                // d_wpk holds the current BF16 parameters
    int wait_limit = tc_default_wait_limit(); // bounded waits of the network kernel
    int ynet_cap = 0;
    int chunk_cap = 0, fb_cap = 0;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr, ev2 = nullptr;
    double last_mlp_ms = 0.0, last_total_ms = 0.0;
    int64_t last_fallback = 0, probe_fail_total = 0;
    uint32_t magic = 0x45535053u;
};

namespace {

bool valid_sur(const esp_surrogate *s) { return s && s->magic == 0x45535053u; }

esp_status ensure_chunk(esp_surrogate *s, int chunk)
{
    if (chunk <= s->chunk_cap)
        return ESP_OK;
    cudaError_t e;
    const size_t act = size_t(chunk) * kHidden;
    if ((e = s->d_X.ensure(size_t(chunk) * kFeat * 2)) != cudaSuccess ||
        (e = s->d_Z.ensure(act * kLayers * sizeof(float))) != cudaSuccess ||
        (e = s->d_H.ensure(act * kLayers * 2)) != cudaSuccess || (e = s->d_dZ.ensure(act * 2 * 2)) != cudaSuccess ||
        (e = s->d_y.ensure(size_t(chunk) * sizeof(float))) != cudaSuccess ||
        (e = s->d_dy.ensure(size_t(chunk) * sizeof(float))) != cudaSuccess ||
        (e = s->d_t.ensure(size_t(chunk) * sizeof(float))) != cudaSuccess ||
        (e = s->d_loss.ensure(size_t(chunk) * sizeof(float) + 64)) != cudaSuccess ||
        (e = s->d_part.ensure(size_t(16) * kHidden * kHidden * sizeof(float) + 256 * (kHidden + 1) * sizeof(float))) !=
            cudaSuccess ||
        (e = s->d_gemmerr.ensure(16)) != cudaSuccess)
        return cuda_fail(e, "allocating surrogate activations");
    s->chunk_cap = chunk;
    return ESP_OK;
}

// Forward pass of one chunk: features of pos -> y (FP32).  Keeps Z and H.
esp_status forward(esp_surrogate *s, const double *pos, int n, cudaStream_t st)
{
    const Layout &L = layout();
    cudaError_t e;
    __nv_bfloat16 *X = static_cast<__nv_bfloat16 *>(s->d_X.p);
    float *Z = static_cast<float *>(s->d_Z.p);
    __nv_bfloat16 *H = static_cast<__nv_bfloat16 *>(s->d_H.p);
    const float *P = static_cast<const float *>(s->d_params.p);
    const __nv_bfloat16 *Pb = static_cast<const __nv_bfloat16 *>(s->d_params_bf.p);
    if ((e = features(pos, n, static_cast<const float *>(s->d_freq.p), s->centre, s->inv_r, X, st)) != cudaSuccess)
        return cuda_fail(e, "surrogate features");
    const size_t act = size_t(s->chunk_cap) * kHidden;
    for (int l = 0; l < kLayers; ++l) {
        GemmArgs g;
        std::memset(&g, 0, sizeof(g));
        g.M = n;
        g.N = kHidden;
        g.K = L.in[l];
        g.A = l == 0 ? X : H + (l - 1) * act;
        g.lda = L.in[l];
        g.B = Pb + L.w[l]; // W_l [N][K] row-major: op(B)[k][n] = W[n][k]
        g.ldb = L.in[l];
        g.Cf = Z + l * act;
        g.Cb = H + l * act;
        g.ldc = kHidden;
        g.bias = P + L.b[l];
        g.epi = kEpiSiluFwd;
        g.kchunk = g.K;
        if ((e = gemm_tc(false, true, g, 1, static_cast<int *>(s->d_gemmerr.p), s->wait_limit, st)) != cudaSuccess)
            return cuda_fail(e, "surrogate forward GEMM");
    }
    return ESP_OK;
}

esp_status output_layer(esp_surrogate *s, int n, const float *t, cudaStream_t st)
{
    const Layout &L = layout();
    const size_t act = size_t(s->chunk_cap) * kHidden;
    const __nv_bfloat16 *H4 = static_cast<const __nv_bfloat16 *>(s->d_H.p) + (kLayers - 1) * act;
    const float *P = static_cast<const float *>(s->d_params.p);
    cudaError_t e = output(H4, n, P + L.w5, P + L.b5, static_cast<float *>(s->d_y.p), t, static_cast<float *>(s->d_dy.p),
                           t ? static_cast<float *>(s->d_loss.p) : nullptr, st);
    return e == cudaSuccess ? ESP_OK : cuda_fail(e, "surrogate output layer");
}

// Backward pass of one chunk after forward + output_layer with targets: the
// gradient of mean((y - t)^2) into d_grad (flat layout).
esp_status backward(esp_surrogate *s, int n, cudaStream_t st)
{
    const Layout &L = layout();
    cudaError_t e;
    const size_t act = size_t(s->chunk_cap) * kHidden;
    const __nv_bfloat16 *X = static_cast<const __nv_bfloat16 *>(s->d_X.p);
    const float *Z = static_cast<const float *>(s->d_Z.p);
    const __nv_bfloat16 *H = static_cast<const __nv_bfloat16 *>(s->d_H.p);
    __nv_bfloat16 *cur = static_cast<__nv_bfloat16 *>(s->d_dZ.p), *nxt = cur + act;
    const float *P = static_cast<const float *>(s->d_params.p);
    const __nv_bfloat16 *Pb = static_cast<const __nv_bfloat16 *>(s->d_params_bf.p);
    float *G = static_cast<float *>(s->d_grad.p);
    float *part = static_cast<float *>(s->d_part.p);
    const float *dy = static_cast<const float *>(s->d_dy.p);
    const int nparts = std::min(256, std::max(1, n / 64));
    if ((e = out_grad(dy, H + (kLayers - 1) * act, n, part, nparts, G + L.w5, st)) != cudaSuccess)
        return cuda_fail(e, "surrogate output gradient");
    if ((e = out_back(dy, n, P + L.w5, Z + (kLayers - 1) * act, cur, st)) != cudaSuccess)
        return cuda_fail(e, "surrogate output backward");
    for (int l = kLayers - 1; l >= 0; --l) {
        const int kin = L.in[l];
        const __nv_bfloat16 *Hin = l == 0 ? X : H + (l - 1) * act;
        // dW_l [256 x kin] = dZ_l^T [256 x n] . H_{l-1} [n x kin], split over n
        GemmArgs g;
        std::memset(&g, 0, sizeof(g));
        g.M = kHidden;
        g.N = kin;
        g.K = n;
        g.A = cur;
        g.lda = kHidden;
        g.B = Hin;
        g.ldb = kin;
        g.Cf = part;
        g.ldc = kin;
        g.epi = kEpiRaw;
        const int ks = std::min(16, std::max(1, n / 512));
        g.kchunk = ((n + ks - 1) / ks + 31) / 32 * 32;
        const int ksplit = (n + g.kchunk - 1) / g.kchunk;
        if ((e = gemm_tc(true, false, g, ksplit, static_cast<int *>(s->d_gemmerr.p), s->wait_limit, st)) !=
            cudaSuccess)
            return cuda_fail(e, "surrogate weight-gradient GEMM");
        if ((e = sum_parts(part, ksplit, kHidden * kin, G + L.w[l], st)) != cudaSuccess)
            return cuda_fail(e, "surrogate weight-gradient reduction");
        if ((e = colsum(cur, n, part, nparts, G + L.b[l], st)) != cudaSuccess)
            return cuda_fail(e, "surrogate bias gradient");
        if (l > 0) {
            // dZ_{l-1} [n x kin] = (dZ_l [n x 256] . W_l [256 x kin]) * SiLU'(Z_{l-1})
            GemmArgs h;
            std::memset(&h, 0, sizeof(h));
            h.M = n;
            h.N = kin;
            h.K = kHidden;
            h.A = cur;
            h.lda = kHidden;
            h.B = Pb + L.w[l];
            h.ldb = kin;
            h.Cb = nxt;
            h.ldc = kin;
            h.aux = Z + (l - 1) * act;
            h.epi = kEpiGradSilu;
            h.kchunk = kHidden;
            if ((e = gemm_tc(false, false, h, 1, static_cast<int *>(s->d_gemmerr.p), s->wait_limit, st)) !=
                cudaSuccess)
                return cuda_fail(e, "surrogate input-gradient GEMM");
            std::swap(cur, nxt);
        }
    }
    return ESP_OK;
}

// n uniform/walker-law positions inside the sphere (radius R about c)
void sample_positions(std::mt19937_64 &rng, int n, const double *c, double R, double sd, std::vector<double> &out)
{
    std::normal_distribution<double> N01(0.0, 1.0);
    std::uniform_real_distribution<double> U(-1.0, 1.0);
    out.resize(size_t(n) * 3);
    for (int i = 0; i < n; ++i) {
        double x[3];
        for (;;) {
            double r2 = 0.0;
            for (int d = 0; d < 3; ++d) {
                x[d] = (i % 2 == 0) ? sd * N01(rng) : R * U(rng);
                r2 += x[d] * x[d];
            }
            if (r2 < R * R)
                break;
        }
        for (int d = 0; d < 3; ++d)
            out[size_t(i) * 3 + d] = c[d] + x[d];
    }
}

template <typename T>
cudaError_t upload_vec(DevBuf &b, const std::vector<T> &v)
{
    cudaError_t e = b.ensure(std::max<size_t>(v.size() * sizeof(T), 16));
    if (e != cudaSuccess || v.empty())
        return e;
    return cudaMemcpy(b.p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
}

TcLayout tc_layout()
{
    const Layout &L = layout();
    TcLayout t;
    size_t o = 0;
    for (int l = 0; l < kLayers; ++l) {
        t.w[l] = L.w[l];
        t.b[l] = L.b[l];
        t.wpk[l] = o;
        o += size_t(kHidden) * L.in[l];
    }
    t.w5 = L.w5;
    t.b5 = L.b5;
    return t;
}


// Near / far split of the context's tiles.  A tile is far when its bounding
// sphere lies beyond far_radius from the centre and (distributions) every
// Gaussian of it is small inside the QM sphere: p_min (d - R)^2 >=
// far_penetration (30 by default, the FP32 kernel's own threshold for the
// asymptotic, multipole form), d the distance from the centre to the
// bounding sphere's nearest point.
void split_tiles(esp_surrogate *s)
{
    const double R = 1.0 / s->inv_r, Rs = s->cfg.far_radius;
    s->near_tiles.clear();
    s->far_tiles.clear();
    s->n_near_entries = s->n_far_entries = 0;
    for (const TileMeta &m : s->ctx->env.tiles) {
        const double d = std::sqrt(double(m.cx) * m.cx + double(m.cy) * m.cy + double(m.cz) * m.cz) - double(m.rad);
        bool far = d >= Rs;
        if (far && !is_point_class(m.cls))
            far = double(m.pmin) * (d - R) * (d - R) >= s->cfg.far_penetration;
        (far ? s->far_tiles : s->near_tiles).push_back(m);
        (far ? s->n_far_entries : s->n_near_entries) += m.n;
    }
    set_tile_groups(s->near_tiles, s->near_view);
    set_tile_groups(s->far_tiles, s->far_view);
}

esp_status upload_split(esp_surrogate *s)
{
    cudaError_t e;
    if ((e = upload_vec(s->d_near_tiles, s->near_tiles)) != cudaSuccess ||
        (e = upload_vec(s->d_far_tiles, s->far_tiles)) != cudaSuccess)
        return cuda_fail(e, "uploading the near/far tile split");
    s->near_view.tiles = static_cast<const TileMeta *>(s->d_near_tiles.p);
    s->far_view.tiles = static_cast<const TileMeta *>(s->d_far_tiles.p);
    return ESP_OK;
}

// Quadrature nodes on the unit sphere for the projection: Gauss-Legendre in
// cos(theta) (nt nodes) x nf equally spaced phi; weights sum to 4 pi.
void sphere_quadrature(int nt, int nf, std::vector<double> &dirs, std::vector<double> &w)
{
    std::vector<double> x(nt), wx(nt);
    for (int i = 0; i < nt; ++i) {
        double z = std::cos(3.14159265358979323846 * (i + 0.75) / (nt + 0.5));
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = 0.0;
            for (int k = 1; k <= nt; ++k) {
                const double p2 = p1;
                p1 = p0;
                p0 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p2) / k;
            }
            const double dp = nt * (z * p0 - p1) / (z * z - 1.0);
            const double dz = p0 / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-16)
                break;
        }
        double p0 = 1.0, p1 = 0.0;
        for (int k = 1; k <= nt; ++k) {
            const double p2 = p1;
            p1 = p0;
            p0 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p2) / k;
        }
        const double dp = nt * (z * p0 - p1) / (z * z - 1.0);
        x[i] = z;
        wx[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
    dirs.clear();
    w.clear();
    for (int i = 0; i < nt; ++i) {
        const double st = std::sqrt(std::max(0.0, 1.0 - x[i] * x[i]));
        for (int j = 0; j < nf; ++j) {
            const double ph = 2.0 * 3.14159265358979323846 * j / nf;
            dirs.push_back(st * std::cos(ph));
            dirs.push_back(st * std::sin(ph));
            dirs.push_back(x[i]);
            w.push_back(wx[i] * 2.0 * 3.14159265358979323846 / nf);
        }
    }
}

const HarmonicConsts &host_harmonics()
{
    static HarmonicConsts h;
    static bool ready = false;
    if (!ready) {
        harmonic_consts(h);
        ready = true;
    }
    return h;
}

// Far-field potentials of the current call into dV (exact kernel over the far
// tiles; zero when no tile is far).
esp_status far_exact(esp_surrogate *s, const double *pos, int64_t n, double *dV, int prec)
{
    if (s->far_tiles.empty()) {
        cudaError_t e = cudaMemsetAsync(dV, 0, size_t(n) * sizeof(double), s->ctx->stream);
        return e == cudaSuccess ? ESP_OK : cuda_fail(e, "clearing far-field values");
    }
    return eval_view(s->ctx, s->far_view, prec, pos, n, dV);
}

// c_lm = (1 / 4 pi) sum_q w_q V_far(centre + R d_q) Y_lm(d_q).
esp_status project_far_field(esp_surrogate *s)
{
    const int L = s->degree;
    s->ncoef = num_harmonics(L);
    s->coef.assign(size_t(s->ncoef), 0.0);
    if (s->far_tiles.empty())
        return ESP_OK;
    const int nt = L + 13, nf = 2 * L + 25;
    std::vector<double> dirs, w;
    sphere_quadrature(nt, nf, dirs, w);
    const int nq = int(w.size());
    const double R = 1.0 / s->inv_r;
    std::vector<double> qpos(size_t(nq) * 3), Vq(nq);
    for (int q = 0; q < nq; ++q)
        for (int d = 0; d < 3; ++d)
            qpos[size_t(q) * 3 + d] = s->centre[d] + R * dirs[size_t(q) * 3 + d];
    DevBuf dq, dv;
    cudaError_t e;
    if ((e = upload_vec(dq, qpos)) != cudaSuccess || (e = dv.ensure(size_t(nq) * sizeof(double))) != cudaSuccess)
        return cuda_fail(e, "allocating the projection points");
    esp_status r = far_exact(s, static_cast<const double *>(dq.p), nq, static_cast<double *>(dv.p), 0);
    if (r != ESP_OK)
        return r;
    if ((e = cudaMemcpyAsync(Vq.data(), dv.p, size_t(nq) * sizeof(double), cudaMemcpyDeviceToHost, s->ctx->stream)) !=
            cudaSuccess ||
        (e = cudaStreamSynchronize(s->ctx->stream)) != cudaSuccess)
        return cuda_fail(e, "far field at the projection points");
    const HarmonicConsts &h = host_harmonics();
    for (int q = 0; q < nq; ++q) {
        const double f = w[size_t(q)] * Vq[size_t(q)] / (4.0 * 3.14159265358979323846);
        solid_harmonics(dirs[size_t(q) * 3], dirs[size_t(q) * 3 + 1], dirs[size_t(q) * 3 + 2], L, h.a, h.b, h.sec,
                        h.sub, [&](int k, double v) { s->coef[size_t(k)] += f * v; });
    }
    return ESP_OK;
}

// Network outputs y (FP32, normalised residual) at n device positions, by the
// fused tensor-core kernel.  The operand copy of the weights is packed once
// per parameter update (after training or loading), not per call.
esp_status net_forward(esp_surrogate *s, const double *pos, int n, cudaStream_t st)
{
    cudaError_t e;
    if (n > s->ynet_cap) {
        if ((e = s->d_ynet.ensure(size_t(n) * sizeof(float))) != cudaSuccess)
            return cuda_fail(e, "allocating surrogate outputs");
        s->ynet_cap = n;
    }
    const TcLayout lay = tc_layout();
    if (!s->packed) {
        if ((e = s->d_wpk.ensure(tc_packed_elems() * 2)) != cudaSuccess || (e = s->d_tcerr.ensure(16)) != cudaSuccess ||
            (e = tc_pack(static_cast<const __nv_bfloat16 *>(s->d_params_bf.p), lay,
                         static_cast<__nv_bfloat16 *>(s->d_wpk.p), st)) != cudaSuccess)
            return cuda_fail(e, "packing the surrogate weights");
        s->packed = true;
    }
    if ((e = cudaMemsetAsync(s->d_tcerr.p, 0, 4, st)) != cudaSuccess ||
        (e = tc_forward(pos, n, static_cast<const float *>(s->d_freq.p), s->centre, s->inv_r,
                        static_cast<const __nv_bfloat16 *>(s->d_wpk.p), static_cast<const float *>(s->d_params.p), lay,
                        static_cast<float *>(s->d_ynet.p), static_cast<int *>(s->d_tcerr.p), s->wait_limit, st)) !=
        cudaSuccess)
        return cuda_fail(e, "surrogate network (tensor cores)");
    return ESP_OK;
}

// Status word of the fused kernel (read after a synchronisation point).
esp_status net_status(esp_surrogate *s)
{
    if (!s->d_tcerr.p)
        return ESP_OK;
    int err = 0;
    cudaError_t e = cudaMemcpy(&err, s->d_tcerr.p, 4, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess)
        return cuda_fail(e, "reading the surrogate kernel status");
    if (err)
        return fail(ESP_ERR_TIMEOUT, "surrogate network kernel: a bounded wait gave up");
    return ESP_OK;
}

// Status word of the training GEMMs (read after a synchronisation point);
// cleared for the next pass.
esp_status gemm_status(esp_surrogate *s)
{
    if (!s->d_gemmerr.p)
        return ESP_OK;
    int err = 0;
    cudaError_t e = cudaMemcpy(&err, s->d_gemmerr.p, 4, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && err)
        e = cudaMemset(s->d_gemmerr.p, 0, 4);
    if (e != cudaSuccess)
        return cuda_fail(e, "reading the training GEMM status");
    if (err)
        return fail(ESP_ERR_TIMEOUT, "surrogate training GEMM: a bounded wait gave up");
    return ESP_OK;
}

// The far-field approximation (expansion + network) at n device positions:
// V = (accumulate ? V : 0) + expansion + s y.
esp_status far_approx(esp_surrogate *s, const double *pos, int n, double *V, bool accumulate, cudaStream_t st)
{
    esp_status r = net_forward(s, pos, n, st);
    if (r != ESP_OK)
        return r;
    cudaError_t e = expansion(pos, n, s->centre, s->inv_r, static_cast<const double *>(s->d_coef.p), s->degree,
                              static_cast<const float *>(s->d_ynet.p), s->scale, accumulate, V, st);
    return e == cudaSuccess ? ESP_OK : cuda_fail(e, "surrogate expansion");
}

// Surrogate values without fallback: exact near-tile sum + far approximation.
esp_status predict(esp_surrogate *s, const double *pos, int n, double *V, cudaStream_t st)
{
    if (n <= 0)
        return ESP_OK;
    esp_status r;
    if (s->near_tiles.empty()) {
        cudaError_t e = cudaMemsetAsync(V, 0, size_t(n) * sizeof(double), st);
        if (e != cudaSuccess)
            return cuda_fail(e, "clearing surrogate values");
    } else if ((r = eval_view(s->ctx, s->near_view, 1, pos, n, V)) != ESP_OK) {
        return r;
    }
    return far_approx(s, pos, n, V, true, st);
}

void release_sur(esp_surrogate *s)
{
    DevBuf *bufs[] = {&s->d_params, &s->d_params_bf, &s->d_grad, &s->d_m, &s->d_v, &s->d_coef, &s->d_freq,
                      &s->d_trust, &s->d_X, &s->d_Z, &s->d_H, &s->d_dZ, &s->d_y, &s->d_dy, &s->d_part, &s->d_t,
                      &s->d_loss, &s->d_flag, &s->d_pre, &s->d_tot, &s->d_count, &s->d_cpos, &s->d_cidx, &s->d_cV,
                      &s->d_nfail, &s->d_wpk, &s->d_tcerr, &s->d_ynet, &s->d_near_tiles, &s->d_far_tiles,
                      &s->d_gemmerr};
    for (DevBuf *b : bufs)
        b->release();
    for (cudaEvent_t *e : {&s->ev0, &s->ev1, &s->ev2})
        if (*e) {
            cudaEventDestroy(*e);
            *e = nullptr;
        }
}

esp_status init_device(esp_surrogate *s)
{
    const Layout &L = layout();
    cudaError_t e;
    std::vector<__nv_bfloat16> pb(L.total);
    for (size_t i = 0; i < L.total; ++i)
        pb[i] = __float2bfloat16(s->params[i]);
    if ((e = set_harmonic_consts()) != cudaSuccess || (e = upload_vec(s->d_params, s->params)) != cudaSuccess ||
        (e = upload_vec(s->d_params_bf, pb)) != cudaSuccess ||
        (e = s->d_grad.ensure(L.total * sizeof(float))) != cudaSuccess ||
        (e = s->d_m.ensure(L.total * sizeof(float))) != cudaSuccess ||
        (e = s->d_v.ensure(L.total * sizeof(float))) != cudaSuccess ||
        (e = cudaMemset(s->d_m.p, 0, L.total * sizeof(float))) != cudaSuccess ||
        (e = cudaMemset(s->d_v.p, 0, L.total * sizeof(float))) != cudaSuccess ||
        (e = upload_vec(s->d_coef, s->coef)) != cudaSuccess || (e = upload_vec(s->d_freq, s->freq)) != cudaSuccess ||
        (e = upload_vec(s->d_trust, s->trust)) != cudaSuccess)
        return cuda_fail(e, "uploading the surrogate");
    s->packed = false;
    if (!s->ev0 && ((e = cudaEventCreate(&s->ev0)) != cudaSuccess || (e = cudaEventCreate(&s->ev1)) != cudaSuccess ||
                    (e = cudaEventCreate(&s->ev2)) != cudaSuccess))
        return cuda_fail(e, "creating surrogate events");
    return upload_split(s);
}

// Point charges (x, y, z in the caller's frame) within `reach` of the centre,
// read from the device records of the point tiles that come that close.
esp_status nearby_point_charges(esp_surrogate *s, double reach, std::vector<double> &pts)
{
    const esp_ctx *c = s->ctx;
    pts.clear();
    for (const TileMeta &m : c->env.tiles) {
        if (!is_point_class(m.cls))
            continue;
        const double d = std::sqrt(double(m.cx) * m.cx + double(m.cy) * m.cy + double(m.cz) * m.cz) - double(m.rad);
        if (d > reach)
            continue;
        std::vector<double> rec(size_t(m.n) * kPointStride64);
        cudaError_t e = cudaMemcpy(rec.data(), static_cast<const double *>(c->rec64.p) + m.off64,
                                   rec.size() * sizeof(double), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess)
            return cuda_fail(e, "reading point charges");
        for (int j = 0; j < m.n; ++j)
            for (int d2 = 0; d2 < 3; ++d2)
                pts.push_back(rec[size_t(j) * kPointStride64 + d2] + c->opt.qm_center[d2]);
    }
    return ESP_OK;
}

// Voxel trust map from validation errors: a voxel is trusted when it holds at
// least one validation point, every such point met tol/2, and no point charge
// of the environment lies within `exclusion` of the voxel.
esp_status build_trust(esp_surrogate *s, const std::vector<double> &pos, const std::vector<double> &err)
{
    const double vox = s->cfg.voxel, R = 1.0 / s->inv_r;
    s->dim = int(std::ceil(2.0 * R / vox));
    const int dim = s->dim;
    const double h = 0.5 * dim * vox;
    std::vector<float> vmax(size_t(dim) * dim * dim, -1.0f);
    for (size_t i = 0; i < err.size(); ++i) {
        int ix = int(std::floor((pos[3 * i] - s->centre[0] + h) / vox));
        int iy = int(std::floor((pos[3 * i + 1] - s->centre[1] + h) / vox));
        int iz = int(std::floor((pos[3 * i + 2] - s->centre[2] + h) / vox));
        if (ix < 0 || iy < 0 || iz < 0 || ix >= dim || iy >= dim || iz >= dim)
            continue;
        float &v = vmax[(size_t(ix) * dim + iy) * dim + iz];
        v = std::max(v, float(err[i]));
    }
    s->trust.assign(vmax.size(), 0);
    const double excl = s->cfg.nucleus_exclusion + 0.87 * vox; // voxel half-diagonal
    std::vector<double> pts;
    esp_status r = nearby_point_charges(s, h * 1.7321 + excl, pts);
    if (r != ESP_OK)
        return r;
    size_t ntrust = 0, nvis = 0;
    for (int ix = 0; ix < dim; ++ix)
        for (int iy = 0; iy < dim; ++iy)
            for (int iz = 0; iz < dim; ++iz) {
                const size_t k = (size_t(ix) * dim + iy) * dim + iz;
                if (vmax[k] < 0.0f)
                    continue;
                ++nvis;
                if (vmax[k] > 0.5 * s->cfg.tol)
                    continue;
                const double cx = s->centre[0] - h + (ix + 0.5) * vox, cy = s->centre[1] - h + (iy + 0.5) * vox,
                             cz = s->centre[2] - h + (iz + 0.5) * vox;
                bool nearp = false;
                for (size_t p = 0; p + 2 < pts.size() && !nearp; p += 3) {
                    double dx = pts[p] - cx, dy = pts[p + 1] - cy, dz = pts[p + 2] - cz;
                    nearp = dx * dx + dy * dy + dz * dz < excl * excl;
                }
                if (!nearp) {
                    s->trust[k] = 1;
                    ++ntrust;
                }
            }
    s->trusted_fraction = nvis ? double(ntrust) / double(nvis) : 0.0;
    return ESP_OK;
}

// One uniformly placed point in every trust-map voxel whose centre lies inside
// the QM sphere, appended to pos (so that no voxel inside goes untrusted for
// lack of validation points).
void voxel_points(const esp_surrogate *s, std::mt19937_64 &rng, std::vector<double> &pos)
{
    const double vox = s->cfg.voxel, R = 1.0 / s->inv_r;
    const int dim = int(std::ceil(2.0 * R / vox));
    const double h = 0.5 * dim * vox;
    std::uniform_real_distribution<double> U(0.0, 1.0);
    for (int ix = 0; ix < dim; ++ix)
        for (int iy = 0; iy < dim; ++iy)
            for (int iz = 0; iz < dim; ++iz) {
                const double c[3] = {-h + (ix + 0.5) * vox, -h + (iy + 0.5) * vox, -h + (iz + 0.5) * vox};
                if (c[0] * c[0] + c[1] * c[1] + c[2] * c[2] >= R * R)
                    continue;
                for (int d = 0; d < 3; ++d)
                    pos.push_back(s->centre[d] + c[d] + (U(rng) - 0.5) * vox);
            }
}

esp_status download(std::vector<double> &out, const DevBuf &b, size_t n, cudaStream_t st)
{
    out.resize(n);
    cudaError_t e;
    if ((e = cudaMemcpyAsync(out.data(), b.p, n * sizeof(double), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess)
        return cuda_fail(e, "reading surrogate data");
    return ESP_OK;
}

esp_status train(esp_surrogate *s)
{
    const Layout &L = layout();
    esp_ctx *ctx = s->ctx;
    const esp_surrogate_cfg &cfg = s->cfg;
    cudaStream_t st = ctx->stream;
    cudaError_t e;
    esp_status r;
    std::mt19937_64 rng(cfg.seed);
    // frequencies and initial weights
    std::normal_distribution<double> N01(0.0, 1.0);
    s->freq.resize(size_t(kFreq) * 3);
    for (float &f : s->freq)
        f = float(cfg.fourier_sigma * N01(rng));
    s->params.assign(L.total, 0.0f);
    for (int l = 0; l < kLayers; ++l) {
        const double a = std::sqrt(6.0 / L.in[l]);
        std::uniform_real_distribution<double> U(-a, a);
        for (size_t i = 0; i < size_t(kHidden) * L.in[l]; ++i)
            s->params[L.w[l] + i] = float(U(rng));
    }
    {
        std::uniform_real_distribution<double> U(-std::sqrt(3.0 / kHidden), std::sqrt(3.0 / kHidden));
        for (int k = 0; k < kHidden; ++k)
            s->params[L.w5 + k] = float(U(rng));
    }
    // near / far split and the far field's interior expansion
    split_tiles(s);
    s->trust.assign(1, 0);
    s->ncoef = num_harmonics(s->degree);
    s->coef.assign(size_t(s->ncoef), 0.0);
    if ((r = init_device(s)) != ESP_OK || (r = project_far_field(s)) != ESP_OK)
        return r;
    if ((e = upload_vec(s->d_coef, s->coef)) != cudaSuccess)
        return cuda_fail(e, "uploading the expansion");
    // training and validation positions; labels: the exact far-tile sum
    std::vector<double> tpos, vpos;
    sample_positions(rng, cfg.n_train, s->centre, 1.0 / s->inv_r, cfg.position_sd, tpos);
    sample_positions(rng, cfg.n_valid, s->centre, 1.0 / s->inv_r, cfg.position_sd, vpos);
    voxel_points(s, rng, vpos); // every voxel inside the sphere gets validation evidence
    const int n_val = int(vpos.size() / 3);
    DevBuf d_tpos, d_tV, d_tE, d_vpos, d_vV, d_vS;
    if ((e = upload_vec(d_tpos, tpos)) != cudaSuccess || (e = upload_vec(d_vpos, vpos)) != cudaSuccess ||
        (e = d_tV.ensure(size_t(cfg.n_train) * 8)) != cudaSuccess ||
        (e = d_tE.ensure(size_t(cfg.n_train) * 8)) != cudaSuccess ||
        (e = d_vV.ensure(size_t(n_val) * 8)) != cudaSuccess ||
        (e = d_vS.ensure(size_t(n_val) * 8)) != cudaSuccess)
        return cuda_fail(e, "allocating surrogate training data");
    const int lp = cfg.label_precision == ESP_FP64 ? 0 : 1;
    const double *tp = static_cast<const double *>(d_tpos.p), *vp = static_cast<const double *>(d_vpos.p);
    if ((r = far_exact(s, tp, cfg.n_train, static_cast<double *>(d_tV.p), lp)) != ESP_OK ||
        (r = far_exact(s, vp, n_val, static_cast<double *>(d_vV.p), lp)) != ESP_OK)
        return r;
    if ((e = expansion(tp, cfg.n_train, s->centre, s->inv_r, static_cast<const double *>(s->d_coef.p), s->degree,
                       nullptr, 0.0, false, static_cast<double *>(d_tE.p), st)) != cudaSuccess)
        return cuda_fail(e, "expansion at the training positions");
    std::vector<double> tV, tE;
    if ((r = download(tV, d_tV, size_t(cfg.n_train), st)) != ESP_OK ||
        (r = download(tE, d_tE, size_t(cfg.n_train), st)) != ESP_OK)
        return r;
    double ss = 0.0;
    for (int i = 0; i < cfg.n_train; ++i) {
        tV[size_t(i)] -= tE[size_t(i)];
        ss += tV[size_t(i)] * tV[size_t(i)];
    }
    s->scale = std::max(std::sqrt(ss / std::max(cfg.n_train, 1)), 1e-300);
    std::vector<float> tgt(cfg.n_train);
    for (int i = 0; i < cfg.n_train; ++i)
        tgt[size_t(i)] = float(tV[size_t(i)] / s->scale);
    DevBuf d_tgt;
    if ((e = upload_vec(d_tgt, tgt)) != cudaSuccess)
        return cuda_fail(e, "uploading training targets");
    // training: mini-batches over the (already random) training set
    const int B = std::min(cfg.batch, cfg.n_train);
    if ((r = ensure_chunk(s, std::max(B, 1))) != ESP_OK)
        return r;
    if ((e = cudaMemsetAsync(s->d_gemmerr.p, 0, 4, st)) != cudaSuccess)
        return cuda_fail(e, "clearing the training GEMM status");
    int step = 0;
    double last_loss = 0.0;
    std::vector<float> lossh(B);
    const int steps_per_epoch = cfg.n_train / std::max(B, 1);
    for (int ep = 0; ep < cfg.epochs; ++ep) {
        double ep_loss = 0.0;
        for (int bi = 0; bi < steps_per_epoch; ++bi) {
            const int o = bi * B;
            if ((r = forward(s, tp + 3 * size_t(o), B, st)) != ESP_OK ||
                (r = output_layer(s, B, static_cast<const float *>(d_tgt.p) + o, st)) != ESP_OK ||
                (r = backward(s, B, st)) != ESP_OK)
                return r;
            ++step;
            const double lr = cfg.lr * 0.5 * (1.0 + std::cos(3.14159265358979 * double(step) /
                                                             double(std::max(1, cfg.epochs * steps_per_epoch))));
            if ((e = adam(static_cast<float *>(s->d_params.p), static_cast<const float *>(s->d_grad.p),
                          static_cast<float *>(s->d_m.p), static_cast<float *>(s->d_v.p),
                          static_cast<__nv_bfloat16 *>(s->d_params_bf.p), int(L.total), float(lr), 0.9f, 0.999f, step,
                          1e-8f, st)) != cudaSuccess)
                return cuda_fail(e, "surrogate Adam step");
            if (bi == steps_per_epoch - 1) {
                if ((e = cudaMemcpyAsync(lossh.data(), s->d_loss.p, size_t(B) * 4, cudaMemcpyDeviceToHost, st)) !=
                        cudaSuccess ||
                    (e = cudaStreamSynchronize(st)) != cudaSuccess)
                    return cuda_fail(e, "reading the training loss");
                for (float v : lossh)
                    ep_loss += v;
                last_loss = ep_loss / B;
            }
        }
    }
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess)
        return cuda_fail(e, "training the surrogate");
    if ((r = gemm_status(s)) != ESP_OK)
        return r;
    s->train_loss = last_loss;
    s->packed = false; // the parameters changed: repack before the next inference
    if ((e = cudaMemcpy(s->params.data(), s->d_params.p, L.total * 4, cudaMemcpyDeviceToHost)) != cudaSuccess)
        return cuda_fail(e, "reading trained weights");
    // validation of the far approximation against the exact far-tile sum, the
    // expansion alone as the method without the network, and the trust map
    if ((r = far_approx(s, vp, n_val, static_cast<double *>(d_vS.p), false, st)) != ESP_OK)
        return r;
    std::vector<double> vS, vV, vE;
    if ((r = download(vS, d_vS, size_t(n_val), st)) != ESP_OK || (r = net_status(s)) != ESP_OK ||
        (r = download(vV, d_vV, size_t(n_val), st)) != ESP_OK)
        return r;
    if ((e = expansion(vp, n_val, s->centre, s->inv_r, static_cast<const double *>(s->d_coef.p), s->degree,
                       nullptr, 0.0, false, static_cast<double *>(d_vS.p), st)) != cudaSuccess)
        return cuda_fail(e, "expansion at the validation positions");
    if ((r = download(vE, d_vS, size_t(n_val), st)) != ESP_OK)
        return r;
    std::vector<double> err(n_val), berr(n_val);
    double mx = 0.0, sq = 0.0, bmx = 0.0, bsq = 0.0;
    for (int i = 0; i < n_val; ++i) {
        err[size_t(i)] = std::fabs(vS[size_t(i)] - vV[size_t(i)]);
        mx = std::max(mx, err[size_t(i)]);
        sq += err[size_t(i)] * err[size_t(i)];
        berr[size_t(i)] = std::fabs(vE[size_t(i)] - vV[size_t(i)]);
        bmx = std::max(bmx, berr[size_t(i)]);
        bsq += berr[size_t(i)] * berr[size_t(i)];
    }
    s->valid_max_err = mx;
    s->valid_rms_err = std::sqrt(sq / std::max(n_val, 1));
    s->base_max_err = bmx;
    s->base_rms_err = std::sqrt(bsq / std::max(n_val, 1));
    // the trust map the expansion alone would earn (the method without the
    // network), then the surrogate's own
    if ((r = build_trust(s, vpos, berr)) != ESP_OK)
        return r;
    s->base_trusted_fraction = s->trusted_fraction;
    if ((r = build_trust(s, vpos, err)) != ESP_OK)
        return r;
    if ((e = upload_vec(s->d_trust, s->trust)) != cudaSuccess)
        return cuda_fail(e, "uploading the trust map");
    return ESP_OK;
}

esp_status ensure_fallback(esp_surrogate *s, int n)
{
    if (n <= s->fb_cap)
        return ESP_OK;
    cudaError_t e;
    const int nb = (n + 1023) / 1024;
    if ((e = s->d_flag.ensure(size_t(n) * 4)) != cudaSuccess || (e = s->d_pre.ensure(size_t(n) * 4)) != cudaSuccess ||
        (e = s->d_tot.ensure(size_t(nb) * 4 + 4)) != cudaSuccess || (e = s->d_count.ensure(8)) != cudaSuccess ||
        (e = s->d_cpos.ensure(size_t(n) * 24)) != cudaSuccess || (e = s->d_cidx.ensure(size_t(n) * 4)) != cudaSuccess ||
        (e = s->d_cV.ensure(size_t(n) * 8)) != cudaSuccess || (e = s->d_nfail.ensure(8)) != cudaSuccess)
        return cuda_fail(e, "allocating fallback buffers");
    s->fb_cap = n;
    return ESP_OK;
}

// Exact values (all tiles, FP32C) for the positions the trust map or the probe
// selects; probes that miss tol withdraw their voxel (counted in d_nfail).
// Returns the number of positions evaluated exactly.
esp_status fallback_pass(esp_surrogate *s, const double *pos, int n, double *V, int stride, int *count_out)
{
    cudaStream_t st = s->ctx->stream;
    cudaError_t e;
    if ((e = fallback_select(pos, n, s->centre, s->cfg.voxel, s->dim, static_cast<const unsigned char *>(s->d_trust.p),
                             stride, s->probe_offset, static_cast<int *>(s->d_flag.p), static_cast<int *>(s->d_pre.p),
                             static_cast<int *>(s->d_tot.p), static_cast<int *>(s->d_count.p),
                             static_cast<double *>(s->d_cpos.p), static_cast<int *>(s->d_cidx.p), st)) != cudaSuccess)
        return cuda_fail(e, "selecting fallback positions");
    int count = 0;
    if ((e = cudaMemcpyAsync(&count, s->d_count.p, 4, cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess)
        return cuda_fail(e, "reading the fallback count");
    *count_out = count;
    if (count == 0)
        return ESP_OK;
    esp_status r = eval_view(s->ctx, s->ctx->full, 1, static_cast<const double *>(s->d_cpos.p), count,
                             static_cast<double *>(s->d_cV.p));
    if (r != ESP_OK)
        return r;
    if ((e = fallback_scatter(static_cast<const double *>(s->d_cV.p), static_cast<const int *>(s->d_cidx.p),
                              static_cast<const int *>(s->d_count.p), count, V, pos, s->centre, s->cfg.voxel, s->dim,
                              static_cast<unsigned char *>(s->d_trust.p), stride, s->probe_offset, s->cfg.tol,
                              static_cast<int *>(s->d_nfail.p), st)) != cudaSuccess)
        return cuda_fail(e, "merging fallback values");
    return ESP_OK;
}

esp_status sur_eval(esp_surrogate *s, const double *pos, int64_t n64, double *V, esp_surrogate_stats *stats)
{
    esp_ctx *ctx = s->ctx;
    cudaStream_t st = ctx->stream;
    cudaError_t e;
    esp_status r;
    const int n = int(n64);
    if ((e = cudaEventRecord(s->ev0, st)) != cudaSuccess)
        return cuda_fail(e, "recording surrogate events");
    if ((r = predict(s, pos, n, V, st)) != ESP_OK)
        return r;
    if ((e = cudaEventRecord(s->ev1, st)) != cudaSuccess)
        return cuda_fail(e, "recording surrogate events");
    if ((r = ensure_fallback(s, n)) != ESP_OK)
        return r;
    if ((e = cudaMemsetAsync(s->d_nfail.p, 0, 4, st)) != cudaSuccess)
        return cuda_fail(e, "clearing the probe count");
    int count = 0, tc_err = 0, nfail = 0;
    if ((r = fallback_pass(s, pos, n, V, s->cfg.probe_stride, &count)) != ESP_OK)
        return r;
    if ((e = cudaMemcpyAsync(&tc_err, s->d_tcerr.p, 4, cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
        (e = cudaMemcpyAsync(&nfail, s->d_nfail.p, 4, cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess)
        return cuda_fail(e, "reading the probe count");
    if (tc_err)
        return fail(ESP_ERR_TIMEOUT, "surrogate network kernel: a bounded wait gave up");
    if (nfail > 0) {
        // voxels withdrawn by this call's probes: their other positions of this
        // call take the exact value too (no probes in this pass)
        int again = 0;
        if ((r = fallback_pass(s, pos, n, V, 0, &again)) != ESP_OK)
            return r;
        count += again;
    }
    if ((e = cudaEventRecord(s->ev2, st)) != cudaSuccess || (e = cudaEventSynchronize(s->ev2)) != cudaSuccess)
        return cuda_fail(e, "finishing the surrogate evaluation");
    float t1 = 0.f, t2 = 0.f;
    cudaEventElapsedTime(&t1, s->ev0, s->ev1);
    cudaEventElapsedTime(&t2, s->ev0, s->ev2);
    s->last_mlp_ms = t1;
    s->last_total_ms = t2;
    s->last_fallback = count;
    s->probe_fail_total += nfail;
    if (s->cfg.probe_stride > 0)
        s->probe_offset = (s->probe_offset + 1) % s->cfg.probe_stride;
    if (stats) {
        std::memset(stats, 0, sizeof(*stats));
        stats->n_fallback = count;
        stats->n_probe_fail = nfail;
        stats->surrogate_ms = t1;
        stats->total_ms = t2;
        stats->train_loss = s->train_loss;
        stats->valid_max_err = s->valid_max_err;
        stats->trusted_fraction = s->trusted_fraction;
        stats->n_near_entries = s->n_near_entries;
        stats->n_far_entries = s->n_far_entries;
    }
    return ESP_OK;
}

const uint32_t kFileMagic = 0x45535246u, kFileVersion = 2;

uint64_t checksum(const void *p, size_t n, uint64_t h)
{
    const unsigned char *b = static_cast<const unsigned char *>(p);
    for (size_t i = 0; i < n; ++i)
        h = (h ^ b[i]) * 1099511628211ull;
    return h;
}

} // namespace

extern "C" {

void esp_surrogate_default_cfg(esp_surrogate_cfg *cfg)
{
    if (!cfg)
        return;
    std::memset(cfg, 0, sizeof(*cfg));
    cfg->size = int32_t(sizeof(esp_surrogate_cfg));
    cfg->n_train = 1 << 19;
    cfg->n_valid = 1 << 17;
    cfg->epochs = 8;
    cfg->batch = 8192;
    cfg->degree = 12;
    cfg->qm_radius = 6.0;
    cfg->position_sd = 2.0;
    cfg->fourier_sigma = 1.0;
    cfg->lr = 1e-3;
    cfg->tol = 2e-6;
    cfg->voxel = 0.25;
    cfg->nucleus_exclusion = 0.5;
    cfg->probe_stride = 64;
    cfg->label_precision = ESP_FP32C;
    cfg->seed = 1011;
    cfg->far_radius = 10.0;
    cfg->far_penetration = 30.0;
}

esp_status esp_surrogate_train(esp_ctx *ctx, const esp_surrogate_cfg *cfg_in, esp_surrogate **out)
{
    last_error().clear();
    if (!valid_ctx(ctx) || ctx->device < 0)
        return fail(ESP_ERR_STATE, "invalid or host-only context");
    if (!out)
        return fail(ESP_ERR_INVALID, "out is NULL");
    esp_surrogate_cfg cfg;
    esp_surrogate_default_cfg(&cfg);
    if (cfg_in) {
        if (cfg_in->size != int32_t(sizeof(esp_surrogate_cfg)))
            return fail(ESP_ERR_INVALID, "esp_surrogate_cfg.size mismatch (call esp_surrogate_default_cfg)");
        cfg = *cfg_in;
    }
    if (cfg.n_train < 1024 || cfg.n_valid < 64 || cfg.epochs < 0 || cfg.batch < 64 || cfg.degree < 0 ||
        cfg.degree > kMaxExpDegree || !(cfg.qm_radius > 0.0) || !(cfg.voxel > 0.0) || !(cfg.tol > 0.0) ||
        cfg.probe_stride < 0 || cfg.n_train > (1 << 26) || cfg.n_valid > (1 << 24) ||
        (cfg.label_precision != ESP_FP64 && cfg.label_precision != ESP_FP32C) ||
        !(cfg.far_radius >= cfg.qm_radius) || !(cfg.far_radius < 1e6) || !(cfg.far_penetration >= 4.0) ||
        !(cfg.far_penetration < 1e6))
        return fail(ESP_ERR_INVALID, "bad surrogate configuration");
    BusyGuard busy(ctx->busy);
    if (!busy.acquired)
        return fail(ESP_ERR_STATE, "context is in use by another thread");
    esp_surrogate *s = new (std::nothrow) esp_surrogate();
    if (!s)
        return fail(ESP_ERR_OOM, "host allocation of the surrogate");
    s->ctx = ctx;
    s->cfg = cfg;
    for (int d = 0; d < 3; ++d)
        s->centre[d] = ctx->opt.qm_center[d];
    s->inv_r = 1.0 / cfg.qm_radius;
    s->degree = cfg.degree;
    DeviceGuard dg(ctx->device);
    esp_status st = train(s);
    if (st != ESP_OK) {
        release_sur(s);
        delete s;
        return st;
    }
    *out = s;
    return ESP_OK;
}

esp_status esp_surrogate_eval(esp_surrogate *s, const double *positions, int64_t n, double *V_out,
                              esp_surrogate_stats *stats)
{
    last_error().clear();
    if (!valid_sur(s))
        return fail(ESP_ERR_STATE, "invalid surrogate");
    if (n < 0 || n > (int64_t(1) << 28))
        return fail(ESP_ERR_INVALID, "position count out of range");
    if (n == 0)
        return ESP_OK;
    if (!positions || !V_out)
        return fail(ESP_ERR_INVALID, "null positions or outputs");
    DeviceGuard dg(s->ctx->device);
    if (classify(positions, s->ctx->device) != Space::Device || classify(V_out, s->ctx->device) != Space::Device)
        return fail(ESP_ERR_INVALID, "surrogate evaluation takes device memory");
    BusyGuard busy(s->ctx->busy);
    if (!busy.acquired)
        return fail(ESP_ERR_STATE, "context is in use by another thread");
    return sur_eval(s, positions, n, V_out, stats);
}

esp_status esp_surrogate_predict(esp_surrogate *s, const double *positions, int64_t n, double *V_out)
{
    last_error().clear();
    if (!valid_sur(s))
        return fail(ESP_ERR_STATE, "invalid surrogate");
    if (n < 0 || n > (int64_t(1) << 28) || (n > 0 && (!positions || !V_out)))
        return fail(ESP_ERR_INVALID, "bad arguments");
    if (n == 0)
        return ESP_OK;
    DeviceGuard dg(s->ctx->device);
    if (classify(positions, s->ctx->device) != Space::Device || classify(V_out, s->ctx->device) != Space::Device)
        return fail(ESP_ERR_INVALID, "surrogate evaluation takes device memory");
    BusyGuard busy(s->ctx->busy);
    if (!busy.acquired)
        return fail(ESP_ERR_STATE, "context is in use by another thread");
    esp_status r = predict(s, positions, int(n), V_out, s->ctx->stream);
    if (r != ESP_OK)
        return r;
    cudaError_t e = cudaStreamSynchronize(s->ctx->stream);
    return e == cudaSuccess ? net_status(s) : cuda_fail(e, "surrogate prediction");
}

esp_status esp_surrogate_info(const esp_surrogate *s, esp_surrogate_stats *stats)
{
    if (!valid_sur(s) || !stats)
        return fail(ESP_ERR_INVALID, "invalid surrogate or output");
    std::memset(stats, 0, sizeof(*stats));
    stats->n_fallback = s->last_fallback;
    stats->n_probe_fail = s->probe_fail_total;
    stats->surrogate_ms = s->last_mlp_ms;
    stats->total_ms = s->last_total_ms;
    stats->train_loss = s->train_loss;
    stats->valid_max_err = s->valid_max_err;
    stats->trusted_fraction = s->trusted_fraction;
    stats->n_params = int64_t(layout().total);
    stats->n_baseline = s->ncoef;
    stats->valid_rms_err = s->valid_rms_err;
    stats->baseline_max_err = s->base_max_err;
    stats->baseline_rms_err = s->base_rms_err;
    stats->n_near_entries = s->n_near_entries;
    stats->n_far_entries = s->n_far_entries;
    stats->baseline_trusted_fraction = s->base_trusted_fraction;
    return ESP_OK;
}

esp_status esp_surrogate_debug_step(esp_surrogate *s, const double *positions, const float *targets, int32_t n,
                                    float *params_out, float *grad_out, float *y_out)
{
    last_error().clear();
    if (!valid_sur(s) || n <= 0 || n > 65536 || !positions || !targets)
        return fail(ESP_ERR_INVALID, "bad arguments");
    const Layout &L = layout();
    DeviceGuard dg(s->ctx->device);
    cudaStream_t st = s->ctx->stream;
    DevBuf dp, dt;
    cudaError_t e;
    esp_status r;
    if ((e = dp.ensure(size_t(n) * 24)) != cudaSuccess || (e = dt.ensure(size_t(n) * 4)) != cudaSuccess ||
        (e = cudaMemcpy(dp.p, positions, size_t(n) * 24, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(dt.p, targets, size_t(n) * 4, cudaMemcpyHostToDevice)) != cudaSuccess)
        return cuda_fail(e, "staging the debug batch");
    if ((r = ensure_chunk(s, n)) != ESP_OK)
        return r;
    if ((e = cudaMemsetAsync(s->d_gemmerr.p, 0, 4, st)) != cudaSuccess)
        return cuda_fail(e, "clearing the training GEMM status");
    if ((r = forward(s, static_cast<const double *>(dp.p), n, st)) != ESP_OK ||
        (r = output_layer(s, n, static_cast<const float *>(dt.p), st)) != ESP_OK || (r = backward(s, n, st)) != ESP_OK)
        return r;
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess)
        return cuda_fail(e, "debug step");
    if ((r = gemm_status(s)) != ESP_OK)
        return r;
    if (params_out && (e = cudaMemcpy(params_out, s->d_params.p, L.total * 4, cudaMemcpyDeviceToHost)) != cudaSuccess)
        return cuda_fail(e, "reading parameters");
    if (grad_out && (e = cudaMemcpy(grad_out, s->d_grad.p, L.total * 4, cudaMemcpyDeviceToHost)) != cudaSuccess)
        return cuda_fail(e, "reading gradients");
    if (y_out && (e = cudaMemcpy(y_out, s->d_y.p, size_t(n) * 4, cudaMemcpyDeviceToHost)) != cudaSuccess)
        return cuda_fail(e, "reading outputs");
    return ESP_OK;
}

esp_status esp_surrogate_debug_net(esp_surrogate *s, const double *positions, int32_t n, float *y_out)
{
    last_error().clear();
    if (!valid_sur(s) || n <= 0 || n > 65536 || !positions || !y_out)
        return fail(ESP_ERR_INVALID, "bad arguments");
    DeviceGuard dg(s->ctx->device);
    cudaStream_t st = s->ctx->stream;
    DevBuf dp;
    cudaError_t e;
    if ((e = dp.ensure(size_t(n) * 24)) != cudaSuccess ||
        (e = cudaMemcpy(dp.p, positions, size_t(n) * 24, cudaMemcpyHostToDevice)) != cudaSuccess)
        return cuda_fail(e, "staging the debug batch");
    esp_status r = net_forward(s, static_cast<const double *>(dp.p), n, st);
    if (r != ESP_OK)
        return r;
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess)
        return cuda_fail(e, "debug network");
    if ((r = net_status(s)) != ESP_OK)
        return r;
    if ((e = cudaMemcpy(y_out, s->d_ynet.p, size_t(n) * 4, cudaMemcpyDeviceToHost)) != cudaSuccess)
        return cuda_fail(e, "reading outputs");
    return ESP_OK;
}

esp_status esp_surrogate_debug_expansion(esp_surrogate *s, double dc, double *coef_out, int32_t max_coef)
{
    last_error().clear();
    if (!valid_sur(s) || max_coef < 0 || (max_coef > 0 && !coef_out))
        return fail(ESP_ERR_INVALID, "bad arguments");
    if (dc != 0.0) {
        DeviceGuard dg(s->ctx->device);
        s->coef[0] += dc;
        cudaError_t e = cudaMemcpy(s->d_coef.p, s->coef.data(), sizeof(double), cudaMemcpyHostToDevice);
        if (e != cudaSuccess)
            return cuda_fail(e, "updating the expansion");
    }
    for (int k = 0; k < std::min(max_coef, s->ncoef); ++k)
        coef_out[k] = s->coef[size_t(k)];
    return ESP_OK;
}

esp_status esp_surrogate_set_wait_limit(esp_surrogate *s, int32_t limit)
{
    if (!valid_sur(s))
        return fail(ESP_ERR_INVALID, "invalid surrogate");
    s->wait_limit = limit < 0 ? tc_default_wait_limit() : limit;
    return ESP_OK;
}

esp_status esp_surrogate_features(const esp_surrogate *s, float *freq_out, double *centre_inv_r_out)
{
    if (!valid_sur(s) || !freq_out || !centre_inv_r_out)
        return fail(ESP_ERR_INVALID, "bad arguments");
    std::memcpy(freq_out, s->freq.data(), s->freq.size() * 4);
    for (int d = 0; d < 3; ++d)
        centre_inv_r_out[d] = s->centre[d];
    centre_inv_r_out[3] = s->inv_r;
    return ESP_OK;
}

esp_status esp_surrogate_save(const esp_surrogate *s, const char *path)
{
    if (!valid_sur(s) || !path)
        return fail(ESP_ERR_INVALID, "bad arguments");
    FILE *f = std::fopen(path, "wb");
    if (!f)
        return fail(ESP_ERR_INVALID, "cannot open %s", path);
    uint64_t h = 1469598103934665603ull;
    auto put = [&](const void *p, size_t n) {
        h = checksum(p, n, h);
        return std::fwrite(p, 1, n, f) == n;
    };
    int32_t hdr[8] = {int32_t(kFileMagic), int32_t(kFileVersion), s->degree, s->ncoef, s->dim, int32_t(layout().total),
                      kFreq, 0};
    double dd[12] = {s->centre[0], s->centre[1], s->centre[2], s->inv_r, s->scale, s->train_loss, s->valid_max_err,
                     s->trusted_fraction, s->valid_rms_err, s->base_max_err, s->base_rms_err,
                     s->base_trusted_fraction};
    bool ok = put(hdr, sizeof(hdr)) && put(dd, sizeof(dd)) && put(&s->cfg, sizeof(s->cfg)) &&
              put(s->coef.data(), s->coef.size() * 8) && put(s->freq.data(), s->freq.size() * 4) &&
              put(s->params.data(), s->params.size() * 4) && put(s->trust.data(), s->trust.size());
    ok = ok && std::fwrite(&h, 8, 1, f) == 1;
    ok = (std::fclose(f) == 0) && ok;
    return ok ? ESP_OK : fail(ESP_ERR_INVALID, "writing %s failed", path);
}

esp_status esp_surrogate_load(esp_ctx *ctx, const char *path, esp_surrogate **out)
{
    last_error().clear();
    if (!valid_ctx(ctx) || ctx->device < 0 || !path || !out)
        return fail(ESP_ERR_INVALID, "bad arguments");
    FILE *f = std::fopen(path, "rb");
    if (!f)
        return fail(ESP_ERR_INVALID, "cannot open %s", path);
    esp_surrogate *s = new (std::nothrow) esp_surrogate();
    if (!s) {
        std::fclose(f);
        return fail(ESP_ERR_OOM, "host allocation");
    }
    uint64_t h = 1469598103934665603ull;
    auto get = [&](void *p, size_t n) {
        if (std::fread(p, 1, n, f) != n)
            return false;
        h = checksum(p, n, h);
        return true;
    };
    int32_t hdr[8];
    double dd[12];
    bool ok = get(hdr, sizeof(hdr)) && uint32_t(hdr[0]) == kFileMagic && hdr[1] == int32_t(kFileVersion) &&
              hdr[2] >= 0 && hdr[2] <= kMaxExpDegree && hdr[3] == num_harmonics(hdr[2]) && hdr[4] > 0 &&
              hdr[4] < 4096 && hdr[5] == int32_t(layout().total) && hdr[6] == kFreq && get(dd, sizeof(dd)) &&
              get(&s->cfg, sizeof(s->cfg)) && s->cfg.size == int32_t(sizeof(esp_surrogate_cfg));
    if (ok) {
        s->degree = hdr[2];
        s->ncoef = hdr[3];
        s->dim = hdr[4];
        s->coef.resize(size_t(s->ncoef));
        s->freq.resize(size_t(kFreq) * 3);
        s->params.resize(layout().total);
        s->trust.resize(size_t(s->dim) * s->dim * s->dim);
        ok = get(s->coef.data(), s->coef.size() * 8) && get(s->freq.data(), s->freq.size() * 4) &&
             get(s->params.data(), s->params.size() * 4) && get(s->trust.data(), s->trust.size());
        uint64_t stored = 0;
        ok = ok && std::fread(&stored, 8, 1, f) == 1 && stored == h;
    }
    std::fclose(f);
    if (!ok) {
        delete s;
        return fail(ESP_ERR_INVALID, "%s is not a valid surrogate file (header, size or checksum)", path);
    }
    for (int d = 0; d < 3; ++d)
        s->centre[d] = dd[d];
    s->inv_r = dd[3];
    s->scale = dd[4];
    s->train_loss = dd[5];
    s->valid_max_err = dd[6];
    s->trusted_fraction = dd[7];
    s->valid_rms_err = dd[8];
    s->base_max_err = dd[9];
    s->base_rms_err = dd[10];
    s->base_trusted_fraction = dd[11];
    s->ctx = ctx;
    // the near / far split is a function of the context's tiles and the configuration
    split_tiles(s);
    DeviceGuard dg(ctx->device);
    esp_status st = init_device(s);
    if (st != ESP_OK) {
        release_sur(s);
        delete s;
        return st;
    }
    *out = s;
    return ESP_OK;
}

void esp_surrogate_destroy(esp_surrogate *s)
{
    if (!valid_sur(s))
        return;
    {
        DeviceGuard dg(s->ctx->device);
        cudaStreamSynchronize(s->ctx->stream);
        release_sur(s);
    }
    s->magic = 0;
    delete s;
}

} // extern "C"
