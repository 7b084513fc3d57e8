// Host pair builder.
//
// Input: point charges {Z_beta, R_beta} and weighted primitive pairs
// (A, alpha, lmn_a) x (B, beta, lmn_b), w.  Output: tiles of Hermite
// distributions, uploaded once (the paper's read-only, upload-once cell data,
// Sec. III).  Steps:
//   1. validate every input value;
//   2. orient each pair canonically ((A,alpha) <= (B,beta)) and sort, so the
//      component pairs of one shell pair become contiguous;
//   3. fold each shell pair into one distribution: p = alpha+beta,
//      P = (alpha A + beta B)/p, D_tuv = sum_components w E^x_t E^y_u E^z_v with
//      the McMurchie-Davidson coefficients
//        E^{00}_0 = exp(-alpha beta/p X_AB^2),
//        E^{i+1,j}_t = E^{ij}_{t-1}/(2p) + X_PA E^{ij}_t + (t+1) E^{ij}_{t+1},
//        E^{i,j+1}_t = E^{ij}_{t-1}/(2p) + X_PB E^{ij}_t + (t+1) E^{ij}_{t+1};
//   4. screen: drop the distribution when its absolute-charge bound
//        sum_tuv |D_tuv| int |Lambda_tuv| dr = sum |D_tuv| p^{(t+u+v-3)/2} h_t h_u h_v,
//      h_t = int |H_t(y)| e^{-y^2} dy, is below screen_tol;
//   5. scale G_tuv = (2 pi / p) p^{(t+u+v)/2} D_tuv and the far-field moments
//      M_tuv = (pi/p)^{3/2} D_tuv (see esp_internal.h);
//   6. class by L, band by exponent (factors of 4 in p), Morton order of P
//      inside a band, and cut into tiles with a bounding sphere each.
#include "pair_builder.h"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <numeric>
#include <unordered_map>

namespace esp {

namespace {

constexpr double kPi = 3.14159265358979323846;

bool finite3(const double *x) { return std::isfinite(x[0]) && std::isfinite(x[1]) && std::isfinite(x[2]); }

// Gauss-Legendre nodes and weights on [-1, 1] by Newton iteration on P_n.
void gauss_legendre(int n, std::vector<double> &x, std::vector<double> &w)
{
    x.assign(n, 0.0);
    w.assign(n, 0.0);
    for (int i = 0; i < n; ++i) {
        double z = std::cos(kPi * (i + 0.75) / (n + 0.5));
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = 0.0;
            for (int k = 1; k <= n; ++k) {
                double p2 = p1;
                p1 = p0;
                p0 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p2) / k;
            }
            double dp = n * (z * p0 - p1) / (z * z - 1.0);
            double dz = p0 / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-16)
                break;
        }
        double p0 = 1.0, p1 = 0.0;
        for (int k = 1; k <= n; ++k) {
            double p2 = p1;
            p1 = p0;
            p0 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p2) / k;
        }
        double dp = n * (z * p0 - p1) / (z * z - 1.0);
        x[i] = z;
        w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

// F_n(T) = int_0^1 t^{2n} exp(-T t^2) dt by composite Gauss-Legendre quadrature.
void boys_by_quadrature(double T, int nmax, double *F)
{
    static std::vector<double> gx, gw;
    static std::once_flag once;
    std::call_once(once, [] { gauss_legendre(24, gx, gw); });
    const int panels = 24;
    for (int n = 0; n <= nmax; ++n)
        F[n] = 0.0;
    for (int pnl = 0; pnl < panels; ++pnl) {
        double a = double(pnl) / panels, b = double(pnl + 1) / panels;
        double h = 0.5 * (b - a), c = 0.5 * (a + b);
        for (size_t k = 0; k < gx.size(); ++k) {
            double t = c + h * gx[k];
            double g = gw[k] * h * std::exp(-T * t * t);
            double t2 = t * t, tp = 1.0;
            for (int n = 0; n <= nmax; ++n) {
                F[n] += g * tp;
                tp *= t2;
            }
        }
    }
}

template <typename R>
std::vector<R> make_boys_table(int rows, int row_len, int nmax, int exp_col, int lo_col)
{
    std::vector<R> tab(size_t(rows) * row_len, R(0));
    std::vector<double> F(nmax + 1);
    for (int i = 0; i < rows; ++i) {
        double T = i * 0.125;
        boys_by_quadrature(T, nmax, F.data());
        for (int n = 0; n <= nmax; ++n)
            tab[size_t(i) * row_len + n] = R(F[n]);
        tab[size_t(i) * row_len + exp_col] = R(std::exp(-T));
        if (lo_col > 0) {
            for (int n = 0; n <= kMaxL; ++n)
                tab[size_t(i) * row_len + lo_col + n] = R(F[n] - double(R(F[n])));
            tab[size_t(i) * row_len + lo_col + kMaxL + 1] = R(std::exp(-T) - double(R(std::exp(-T))));
        }
    }
    return tab;
}

// h_t = int |H_t(y)| exp(-y^2) dy for physicists' Hermite polynomials, t <= 4.
const double *hermite_abs_moments()
{
    static double h[kMaxL + 1];
    static std::once_flag once;
    std::call_once(once, [] {
        const int n = 400000;
        const double a = -12.0, b = 12.0, dx = (b - a) / n;
        for (int t = 0; t <= kMaxL; ++t)
            h[t] = 0.0;
        for (int i = 0; i <= n; ++i) {
            double y = a + i * dx;
            double wgt = (i == 0 || i == n) ? 1.0 : (i % 2 ? 4.0 : 2.0);
            double Hm = 1.0, H = 2.0 * y;
            double e = std::exp(-y * y);
            h[0] += wgt * e;
            h[1] += wgt * std::fabs(H) * e;
            for (int t = 2; t <= kMaxL; ++t) {
                double Hn = 2.0 * y * H - 2.0 * (t - 1) * Hm;
                Hm = H;
                H = Hn;
                h[t] += wgt * std::fabs(H) * e;
            }
        }
        for (int t = 0; t <= kMaxL; ++t)
            h[t] *= dx / 3.0;
    });
    return h;
}

struct Oriented {
    double A[3], alpha, B[3], beta;
    int la[3], lb[3];
    double w;
};

bool key_less(const Oriented &x, const Oriented &y)
{
    for (int d = 0; d < 3; ++d)
        if (x.A[d] != y.A[d])
            return x.A[d] < y.A[d];
    if (x.alpha != y.alpha)
        return x.alpha < y.alpha;
    for (int d = 0; d < 3; ++d)
        if (x.B[d] != y.B[d])
            return x.B[d] < y.B[d];
    return x.beta < y.beta;
}

bool same_key(const Oriented &x, const Oriented &y)
{
    return !key_less(x, y) && !key_less(y, x);
}

// E^{ij}_t for one direction, i <= imax, j <= jmax (both <= 4).
struct ETable {
    double e[kMaxL + 1][kMaxL + 1][2 * kMaxL + 2];
};

void fill_E(ETable &E, int imax, int jmax, double XAB, double XPA, double XPB, double p, double mu)
{
    std::memset(&E, 0, sizeof(E));
    E.e[0][0][0] = std::exp(-mu * XAB * XAB);
    double o2p = 0.5 / p;
    for (int i = 0; i <= imax; ++i) {
        if (i > 0) {
            for (int t = 0; t <= i; ++t) {
                double v = XPA * E.e[i - 1][0][t] + (t + 1) * E.e[i - 1][0][t + 1];
                if (t > 0)
                    v += o2p * E.e[i - 1][0][t - 1];
                E.e[i][0][t] = v;
            }
        }
        for (int j = 1; j <= jmax; ++j) {
            for (int t = 0; t <= i + j; ++t) {
                double v = XPB * E.e[i][j - 1][t] + (t + 1) * E.e[i][j - 1][t + 1];
                if (t > 0)
                    v += o2p * E.e[i][j - 1][t - 1];
                E.e[i][j][t] = v;
            }
        }
    }
}

struct Dist {
    double P[3];
    double p;
    int L;
    bool onsite;   // A == B: centred exactly on P = A
    bool shortr;   // monopole moved into the point charge at P
    double G[35];
    double M[35];
    double qabs;
    uint64_t key;
};

uint64_t spread10(uint32_t v)
{
    uint64_t x = v & 0x3ff;
    x = (x | (x << 16)) & 0x030000FFull;
    x = (x | (x << 8)) & 0x0300F00Full;
    x = (x | (x << 4)) & 0x030C30C3ull;
    x = (x | (x << 2)) & 0x09249249ull;
    return x;
}

uint64_t morton(const double *P, const double *lo, double inv)
{
    uint32_t q[3];
    for (int d = 0; d < 3; ++d) {
        double f = (P[d] - lo[d]) * inv;
        f = std::min(std::max(f, 0.0), 1023.0);
        q[d] = uint32_t(f);
    }
    return spread10(q[0]) | (spread10(q[1]) << 1) | (spread10(q[2]) << 2);
}

void bounding_sphere(const double *xyz, size_t stride, int n, TileMeta &m)
{
    double c[3] = {0, 0, 0};
    for (int k = 0; k < n; ++k)
        for (int d = 0; d < 3; ++d)
            c[d] += xyz[k * stride + d];
    for (int d = 0; d < 3; ++d)
        c[d] /= std::max(n, 1);
    double r2 = 0.0;
    for (int k = 0; k < n; ++k) {
        double s = 0.0;
        for (int d = 0; d < 3; ++d) {
            double e = xyz[k * stride + d] - c[d];
            s += e * e;
        }
        r2 = std::max(r2, s);
    }
    m.cx = float(c[0]);
    m.cy = float(c[1]);
    m.cz = float(c[2]);
    // float rounding of the centre is covered by a small margin
    m.rad = float(std::sqrt(r2) * (1.0 + 1e-6) + 1e-5);
}

} // namespace

const std::vector<float> &boys_table32()
{
    static std::vector<float> t;
    static std::once_flag once;
    std::call_once(once, [] {
        t = make_boys_table<float>(kBoys32Rows, kBoys32Row, kMaxL + kBoys32Terms - 1,
                                   BoysConst<float>::kExpCol, kBoys32LoCol);
    });
    return t;
}

const std::vector<double> &boys_table64()
{
    static std::vector<double> t;
    static std::once_flag once;
    std::call_once(once, [] {
        t = make_boys_table<double>(kBoys64Rows, kBoys64Row, kMaxL + kBoys64Terms - 1,
                                    BoysConst<double>::kExpCol, 0);
    });
    return t;
}

esp_status build_environment(const esp_point_charge *charges, int64_t n_charges,
                             const esp_gauss_pair *pairs, const double *weights, int64_t n_pairs,
                             const esp_options &opt, HostEnv &out, std::string &err)
{
    if (n_charges < 0 || n_pairs < 0) {
        err = "negative count";
        return ESP_ERR_INVALID;
    }
    if ((n_charges > 0 && !charges) || (n_pairs > 0 && (!pairs || !weights))) {
        err = "null input array with a positive count";
        return ESP_ERR_INVALID;
    }
    if (n_charges > (int64_t(1) << 28) || n_pairs > (int64_t(1) << 30)) {
        err = "input too large";
        return ESP_ERR_INVALID;
    }
    const double *qc = opt.qm_center;
    if (!finite3(qc) || !(opt.screen_tol >= 0.0) || !std::isfinite(opt.screen_tol)) {
        err = "bad options (qm_center or screen_tol)";
        return ESP_ERR_INVALID;
    }
    int tile = opt.tile_size == 0 ? 64 : opt.tile_size;
    if (tile != 32 && tile != 64 && tile != 128 && tile != 256) {
        err = "tile_size must be 32, 64, 128 or 256";
        return ESP_ERR_INVALID;
    }
    for (int64_t i = 0; i < n_charges; ++i) {
        if (!finite3(charges[i].xyz) || !std::isfinite(charges[i].Z)) {
            err = "non-finite point charge " + std::to_string(i);
            return ESP_ERR_INVALID;
        }
    }
    std::vector<Oriented> ps;
    ps.reserve(size_t(n_pairs));
    for (int64_t i = 0; i < n_pairs; ++i) {
        const esp_gauss_pair &g = pairs[i];
        int la = 0, lb = 0;
        bool ok = finite3(g.A) && finite3(g.B) && std::isfinite(g.alpha) && std::isfinite(g.beta) &&
                  g.alpha > 0.0 && g.beta > 0.0 && std::isfinite(weights[i]);
        for (int d = 0; d < 3; ++d) {
            ok = ok && g.lmn_a[d] >= 0 && g.lmn_b[d] >= 0 && g.lmn_a[d] <= kMaxL && g.lmn_b[d] <= kMaxL;
            la += g.lmn_a[d];
            lb += g.lmn_b[d];
        }
        if (!ok || la + lb > kMaxL) {
            err = "invalid Gaussian pair " + std::to_string(i) +
                  " (non-finite value, exponent <= 0, or la+lb > 4)";
            return ESP_ERR_INVALID;
        }
        if (weights[i] == 0.0)
            continue;
        Oriented o;
        // canonical orientation: (A, alpha) <= (B, beta) lexicographically
        int cmp = 0;
        for (int d = 0; d < 3 && cmp == 0; ++d)
            if (g.A[d] != g.B[d])
                cmp = g.B[d] < g.A[d] ? 1 : -1;
        bool swap = cmp != 0 ? cmp > 0 : g.beta < g.alpha;
        const double *A = swap ? g.B : g.A, *B = swap ? g.A : g.B;
        const int32_t *lA = swap ? g.lmn_b : g.lmn_a, *lB = swap ? g.lmn_a : g.lmn_b;
        for (int d = 0; d < 3; ++d) {
            o.A[d] = A[d] - qc[d];
            o.B[d] = B[d] - qc[d];
            o.la[d] = lA[d];
            o.lb[d] = lB[d];
        }
        o.alpha = swap ? g.beta : g.alpha;
        o.beta = swap ? g.alpha : g.beta;
        o.w = weights[i];
        ps.push_back(o);
    }
    std::stable_sort(ps.begin(), ps.end(), key_less);

    const double *habs = hermite_abs_moments();
    std::vector<Dist> dist;
    dist.reserve(ps.size() / 3 + 16);
    int64_t screened = 0;
    ETable Ex, Ey, Ez;
    for (size_t g0 = 0; g0 < ps.size();) {
        size_t g1 = g0 + 1;
        while (g1 < ps.size() && same_key(ps[g0], ps[g1]))
            ++g1;
        const Oriented &o = ps[g0];
        double p = o.alpha + o.beta, mu = o.alpha * o.beta / p;
        double P[3], PA[3], PB[3], AB[3];
        int imax[3] = {0, 0, 0}, jmax[3] = {0, 0, 0}, L = 0;
        for (int d = 0; d < 3; ++d) {
            P[d] = (o.alpha * o.A[d] + o.beta * o.B[d]) / p;
            PA[d] = P[d] - o.A[d];
            PB[d] = P[d] - o.B[d];
            AB[d] = o.A[d] - o.B[d];
        }
        for (size_t k = g0; k < g1; ++k) {
            int l = 0;
            for (int d = 0; d < 3; ++d) {
                imax[d] = std::max(imax[d], ps[k].la[d]);
                jmax[d] = std::max(jmax[d], ps[k].lb[d]);
                l += ps[k].la[d] + ps[k].lb[d];
            }
            L = std::max(L, l);
        }
        fill_E(Ex, imax[0], jmax[0], AB[0], PA[0], PB[0], p, mu);
        fill_E(Ey, imax[1], jmax[1], AB[1], PA[1], PB[1], p, mu);
        fill_E(Ez, imax[2], jmax[2], AB[2], PA[2], PB[2], p, mu);
        double D[35];
        std::fill(D, D + 35, 0.0);
        for (size_t k = g0; k < g1; ++k) {
            const Oriented &c = ps[k];
            for (int t = 0; t <= c.la[0] + c.lb[0]; ++t)
                for (int u = 0; u <= c.la[1] + c.lb[1]; ++u)
                    for (int v = 0; v <= c.la[2] + c.lb[2]; ++v)
                        D[hidx(t, u, v)] += c.w * Ex.e[c.la[0]][c.lb[0]][t] * Ey.e[c.la[1]][c.lb[1]][u] *
                                            Ez.e[c.la[2]][c.lb[2]][v];
        }
        Dist ds;
        double qabs = 0.0;
        for (int N = 0; N <= L; ++N)
            for (int t = N; t >= 0; --t)
                for (int u = N - t; u >= 0; --u) {
                    int v = N - t - u, h = hidx(t, u, v);
                    qabs += std::fabs(D[h]) * std::pow(p, 0.5 * (N - 3)) * habs[t] * habs[u] * habs[v];
                    ds.G[h] = 2.0 * kPi / p * std::pow(p, 0.5 * N) * D[h];
                    ds.M[h] = std::pow(kPi / p, 1.5) * D[h];
                }
        g0 = g1;
        if (qabs < opt.screen_tol || qabs == 0.0) {
            ++screened;
            continue;
        }
        for (int d = 0; d < 3; ++d)
            ds.P[d] = P[d];
        ds.onsite = o.A[0] == o.B[0] && o.A[1] == o.B[1] && o.A[2] == o.B[2];
        if (ds.onsite)
            for (int d = 0; d < 3; ++d)
                ds.P[d] = o.A[d];
        ds.shortr = false;
        ds.p = p;
        ds.L = L;
        ds.qabs = qabs;
        dist.push_back(ds);
    }

    // Point charges (recentred).  On-site distributions (A == B) that sit on a
    // point charge, or that share their centre with at least 8 others, hand
    // their monopole Q_d = M_000 to a point charge at that centre; they keep
    // only the short-range remainder V_d - Q_d/|P - C|.  The many on-site
    // distributions of one atom otherwise share one rounded FP32 value of
    // 1/|P - C| and their errors add up coherently.
    struct PointQ {
        double x[3];
        double Z;
    };
    std::vector<PointQ> pts;
    pts.reserve(size_t(n_charges) + 16);
    for (int64_t i = 0; i < n_charges; ++i) {
        PointQ q;
        for (int d = 0; d < 3; ++d)
            q.x[d] = charges[i].xyz[d] - qc[d];
        q.Z = charges[i].Z;
        pts.push_back(q);
    }
    {
        auto ckey = [](const double *x) {
            uint64_t k = 1469598103934665603ull;
            for (int d = 0; d < 3; ++d) {
                uint64_t b;
                std::memcpy(&b, &x[d], 8);
                k = (k ^ b) * 1099511628211ull;
            }
            return k;
        };
        std::unordered_map<uint64_t, int64_t> at_point;
        for (size_t i = 0; i < pts.size(); ++i)
            at_point.emplace(ckey(pts[i].x), int64_t(i));
        std::unordered_map<uint64_t, std::vector<size_t>> groups;
        for (size_t k = 0; k < dist.size(); ++k)
            if (dist[k].onsite)
                groups[ckey(dist[k].P)].push_back(k);
        const double c0 = 0.88622692545275801365; // sqrt(pi)/2
        for (auto &g : groups) {
            const Dist &d0 = dist[g.second[0]];
            auto it = at_point.find(g.first);
            bool on_point = it != at_point.end() && pts[size_t(it->second)].x[0] == d0.P[0] &&
                            pts[size_t(it->second)].x[1] == d0.P[1] && pts[size_t(it->second)].x[2] == d0.P[2];
            if (!on_point && g.second.size() < 8)
                continue;
            double Q = 0.0;
            for (size_t k : g.second) {
                Q += dist[k].G[0] * c0 / std::sqrt(dist[k].p);
                dist[k].shortr = true;
            }
            if (on_point) {
                pts[size_t(it->second)].Z += Q;
            } else {
                PointQ q;
                for (int d = 0; d < 3; ++d)
                    q.x[d] = d0.P[d];
                q.Z = Q;
                pts.push_back(q);
            }
        }
    }

    // order: class L, exponent band (factor 4), Morton code of P
    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
    for (const Dist &d : dist)
        for (int k = 0; k < 3; ++k) {
            lo[k] = std::min(lo[k], d.P[k]);
            hi[k] = std::max(hi[k], d.P[k]);
        }
    for (int64_t i = 0; i < n_charges; ++i)
        for (int k = 0; k < 3; ++k) {
            lo[k] = std::min(lo[k], charges[i].xyz[k] - qc[k]);
            hi[k] = std::max(hi[k], charges[i].xyz[k] - qc[k]);
        }
    double ext = 1e-9;
    for (int k = 0; k < 3; ++k)
        ext = std::max(ext, hi[k] - lo[k]);
    double inv = 1023.0 / ext;
    for (Dist &d : dist) {
        int band = int(std::floor(std::log(d.p) / std::log(4.0))) + 64;
        band = std::min(std::max(band, 0), 127);
        d.key = (uint64_t(d.L) << 41) | (uint64_t(d.shortr) << 40) | (uint64_t(band) << 32) | morton(d.P, lo, inv);
    }
    std::stable_sort(dist.begin(), dist.end(), [](const Dist &a, const Dist &b) { return a.key < b.key; });

    out = HostEnv();
    out.tile_size = tile;
    // Coordinate grid: offsets P - C stay below 4 max|P| for positions inside the
    // environment's extent, so 2^24 q >= 4 max|P| keeps P_hi - C_hi exact.
    {
        double m = 1.0;
        for (int k = 0; k < 3; ++k)
            m = std::max(m, std::max(std::fabs(lo[k]), std::fabs(hi[k])));
        out.coord_quantum = std::ldexp(1.0, int(std::ceil(std::log2(4.0 * m))) - 24);
    }
    out.n_pairs_in = n_pairs;
    out.n_distributions = int64_t(dist.size());
    out.n_screened = screened;

    // point-charge tiles (FP64 records [x, y, z, Z]), Morton order
    const int64_t n_pts = int64_t(pts.size());
    std::vector<int64_t> pidx{};
    pidx.resize(size_t(n_pts));
    std::iota(pidx.begin(), pidx.end(), 0);
    std::vector<uint64_t> pkey{};
    pkey.resize(size_t(n_pts));
    for (int64_t i = 0; i < n_pts; ++i)
        pkey[size_t(i)] = morton(pts[size_t(i)].x, lo, inv);
    std::stable_sort(pidx.begin(), pidx.end(), [&](int64_t a, int64_t b) { return pkey[size_t(a)] < pkey[size_t(b)]; });
    int64_t kept_charges = 0;
    for (int64_t i = 0; i < n_pts; ++i)
        kept_charges += pts[size_t(i)].Z != 0.0;
    out.n_point_charges = kept_charges;

    // FP64 point tiles (|Z| above the FP32 threshold: nuclei, merged
    // monopoles), then FP32 point tiles (small charges such as the paper's
    // density cells), each in Morton order
    const double q32 = opt.point32_max_charge < 0.0 ? kDefaultPoint32Max : opt.point32_max_charge;
    size_t off64 = 0, off32 = 0;
    std::vector<double> pbuf;
    for (int pass = 0; pass < 2; ++pass) {
        const bool small = pass == 1;
        for (int64_t s = 0; s < n_pts;) {
            TileMeta m;
            std::memset(&m, 0, sizeof(m));
            m.cls = small ? kClassPoint32 : kClassPoint;
            m.off64 = int32_t(off64);
            m.off32 = int32_t(off32);
            pbuf.clear();
            double qsum = 0.0;
            while (s < n_pts && m.n < tile) {
                const PointQ &c = pts[size_t(pidx[size_t(s)])];
                ++s;
                if (c.Z == 0.0 || (std::fabs(c.Z) <= q32) != small)
                    continue;
                for (int d = 0; d < 3; ++d)
                    pbuf.push_back(c.x[d]);
                pbuf.push_back(c.Z);
                qsum += std::fabs(c.Z);
                ++m.n;
                if (small) {
                    // FP32 record in the L = 0 layout: centre hi / lo, M_000 = Z + lo word
                    const size_t b32 = out.rec32.size();
                    out.rec32.resize(b32 + rec32_stride(0), 0.0f);
                    for (int d = 0; d < 3; ++d) {
                        const double h = quantize_hi(c.x[d], out.coord_quantum);
                        out.rec32[b32 + d] = float(h);
                        out.rec32[b32 + rec32_lo(0) + d] = float(c.x[d] - h);
                    }
                    out.rec32[b32 + rec32_m(0)] = float(c.Z);
                    out.rec32[b32 + rec32_lo(0) + 3] = float(c.Z - double(float(c.Z)));
                }
            }
            if (m.n == 0)
                continue;
            bounding_sphere(pbuf.data(), kPointStride64, m.n, m);
            m.qabs = float(qsum);
            out.rec64.insert(out.rec64.end(), pbuf.begin(), pbuf.end());
            off64 += pbuf.size();
            off32 = out.rec32.size();
            out.tiles.push_back(m);
        }
    }

    // distribution tiles: never span a class or an exponent band
    std::vector<double> cbuf;
    for (size_t s = 0; s < dist.size();) {
        size_t e = s + 1;
        uint64_t grp = dist[s].key >> 32;
        while (e < dist.size() && e - s < size_t(tile) && (dist[e].key >> 32) == grp)
            ++e;
        const int L = dist[s].L;
        const bool shortr = dist[s].shortr;
        const int nh = num_hermite(L);
        const int st32 = rec32_stride(L), st64 = rec64_stride(L);
        TileMeta m;
        std::memset(&m, 0, sizeof(m));
        m.cls = L | (shortr ? kClassShortBit : 0);
        m.n = int32_t(e - s);
        m.off32 = int32_t(off32);
        m.off64 = int32_t(off64);
        double pmin = 1e300, qsum = 0.0, vmax = 0.0;
        cbuf.clear();
        for (size_t k = s; k < e; ++k) {
            const Dist &d = dist[k];
            for (int c = 0; c < 3; ++c)
                cbuf.push_back(d.P[c]);
            pmin = std::min(pmin, d.p);
            qsum += d.qabs;
            if (!shortr)
                vmax = std::max(vmax, std::fabs(d.M[0]) * 2.0 * std::sqrt(d.p / kPi));
            out.n_by_L[L] += 1;
            size_t b32 = out.rec32.size();
            out.rec32.resize(b32 + st32, 0.0f);
            for (int c = 0; c < 3; ++c)
                out.rec32[b32 + c] = float(quantize_hi(d.P[c], out.coord_quantum));
            const double psv = L == 0 ? d.p : std::sqrt(d.p);
            out.rec32[b32 + 3] = float(psv);
            out.rec32[b32 + rec32_pslo(L)] = float(psv - double(float(psv)));
            for (int c = 0; c < 3; ++c)
                out.rec32[b32 + rec32_lo(L) + c] = float(d.P[c] - quantize_hi(d.P[c], out.coord_quantum));
            out.rec32[b32 + rec32_lo(L) + 3] = shortr ? 0.0f : float(d.M[0] - double(float(d.M[0])));
            out.rec32[b32 + rec32_g0lo(L)] = float(d.G[0] - double(float(d.G[0])));
            for (int h = 0; h < nh; ++h) {
                out.rec32[b32 + rec32_m(L) + h] = (shortr && h == 0) ? 0.0f : float(d.M[h]);
                out.rec32[b32 + rec32_g(L) + h] = float(d.G[h]);
            }
            size_t b64 = out.rec64.size();
            out.rec64.resize(b64 + st64, 0.0);
            out.rec64[b64 + 0] = d.P[0];
            out.rec64[b64 + 1] = d.P[1];
            out.rec64[b64 + 2] = d.P[2];
            out.rec64[b64 + 3] = std::sqrt(d.p);
            for (int h = 0; h < nh; ++h)
                out.rec64[b64 + 4 + h] = d.G[h];
        }
        off32 = out.rec32.size();
        off64 = out.rec64.size();
        bounding_sphere(cbuf.data(), 3, m.n, m);
        // The tile's reference point T on the coordinate grid (the moved
        // centre stays inside the sphere grown by 2q), and the records' hi
        // words stored as Px_hi - T_x: exact, since both lie on the grid and
        // the difference needs fewer than 24 bits of q.
        {
            const double q = out.coord_quantum;
            const double T[3] = {quantize_hi(m.cx, q), quantize_hi(m.cy, q), quantize_hi(m.cz, q)};
            m.cx = float(T[0]);
            m.cy = float(T[1]);
            m.cz = float(T[2]);
            m.rad = float(double(m.rad) + 2.0 * q);
            for (int k = 0; k < m.n; ++k)
                for (int c = 0; c < 3; ++c) {
                    float &h = out.rec32[size_t(m.off32) + size_t(k) * st32 + c];
                    h = float(double(h) - T[c]);
                }
        }
        m.pmin = float(pmin);
        m.qabs = float(qsum);
        m.vmax = float(vmax);
        out.n_near_tiles += vmax >= kNearVmax;
        out.tiles.push_back(m);
        s = e;
    }
    if (off32 > size_t(INT32_MAX) || off64 > size_t(INT32_MAX)) {
        err = "environment too large for 32-bit record offsets";
        return ESP_ERR_INVALID;
    }
    return ESP_OK;
}

} // namespace esp
