// Internal definitions shared by the pair builder (host) and the kernels.
//
// A Hermite distribution is the Gaussian product chi_a chi_b of one shell pair
// written in McMurchie-Davidson form (Helgaker, Joergensen & Olsen, Sec. 9.5):
//   chi_a chi_b = sum_{t+u+v<=L} D_tuv  d^t/dPx^t d^u/dPy^u d^v/dPz^v exp(-p|r-P|^2)
// and its potential at C is (2 pi / p) sum D_tuv R_tuv(p, P - C) with
//   R^n_000 = (-2p)^n F_n(p|P-C|^2),
//   R^n_{t+1,u,v} = t R^{n+1}_{t-1,u,v} + X_PC R^{n+1}_{t,u,v}  (same in u, v).
// Substituting R^n_tuv = p^{n+(t+u+v)/2} S^n_tuv removes p from the recursion:
//   S^n_000 = (-2)^n F_n(T),  S^n_{t+1,u,v} = t S^{n+1}_{t-1,u,v} + x S^{n+1}_{t,u,v},
// with scaled coordinates x = sqrt(p) (P - C) and T = |x|^2.  The builder
// therefore stores G_tuv = (2 pi / p) p^{(t+u+v)/2} D_tuv, and a distribution's
// potential is sum_tuv G_tuv S^0_tuv.  This is the generalisation of one cell
// term rho(r_m)/|r_new - r_m| of Eq. ElectrostaticField: an s distribution
// with p -> infinity gives G_000 F_0 -> q / |P - C|.
#pragma once

#include <cstring>

#include <math.h>
#include <stdint.h>

#if defined(__CUDACC__)
#define ESP_HD __host__ __device__ __forceinline__
#else
#define ESP_HD inline
#endif

namespace esp {

constexpr int kMaxL = 4;
constexpr int kClassPoint = 5;          // tile class of point charges summed in FP64
// Tile class of small point charges (|Z| <= point32_max_charge, the paper's
// density cells) summed in compensated FP32: FP32 records in the L = 0 layout
// (centre hi/lo, M_000 = Z with its low word) evaluated by the far form, and
// FP64 records in the point layout [x, y, z, Z] for the FP64 paths.
constexpr int kClassPoint32 = 6;
constexpr double kDefaultPoint32Max = 0.25;
ESP_HD constexpr bool is_point_class(int cls) { return cls == kClassPoint || cls == kClassPoint32; }
// FP32 record stride of a tile class (point charges use the L = 0 layout)
ESP_HD constexpr int rec32_stride_cls(int cls);
// FP64 re-evaluation radius of the FP32C kernel when the caller leaves it unset.
// It applies only to tiles holding a distribution whose potential can exceed
// kNearVmax (|Q| 2 sqrt(p/pi) bounds the potential of a charge Q spread with
// exponent p); nuclei and on-site monopoles are FP64 point charges already.
constexpr double kDefaultNearRadius = 1.5;
constexpr float kNearVmax = 2.0f;
// Tile class bit: the distributions are centred on a point charge whose FP64
// charge already includes their monopoles, so the tile holds only the
// short-range remainder V_d - Q_d/|P - C| (Q_d = (pi/p)^{3/2} D_000).
constexpr int kClassShortBit = 8;
ESP_HD constexpr int num_hermite(int L) { return (L + 1) * (L + 2) * (L + 3) / 6; }

// FP32 record (floats), L = total angular momentum, n = num_hermite(L):
//   [0..3]          Px_hi - T_x, Py_hi - T_y, Pz_hi - T_z, p (L = 0) or sqrt(p) (L > 0)
//                   (hi words relative to the tile's reference point T =
//                   (cx, cy, cz) of its TileMeta; both on the coordinate grid,
//                   so the difference is exact; FP32 point charges store
//                   absolute hi words)
//   [4..7]          Px_lo, Py_lo, Pz_lo, M_0 lo word
//   [8, 8+n)        M_tuv = (pi/p)^{3/2} D_tuv   (far-field multipole moments)
//   [8+n]           G_0 lo word
//   [9+n]           lo word of p (L = 0) or sqrt(p) (L > 0)
//   [10+n, 10+2n)   G_tuv                        (general form, see above)
// padded to a multiple of 4 floats.
ESP_HD constexpr int rec32_lo(int) { return 4; }
ESP_HD constexpr int rec32_m(int) { return 8; }
ESP_HD constexpr int rec32_g0lo(int L) { return 8 + (L + 1) * (L + 2) * (L + 3) / 6; }
ESP_HD constexpr int rec32_pslo(int L) { return 9 + (L + 1) * (L + 2) * (L + 3) / 6; }
ESP_HD constexpr int rec32_g(int L) { return 10 + (L + 1) * (L + 2) * (L + 3) / 6; }
ESP_HD constexpr int rec32_stride(int L) { return ((10 + 2 * ((L + 1) * (L + 2) * (L + 3) / 6) + 3) / 4) * 4; }
constexpr int kRec32MaxStride = 80;
ESP_HD constexpr int rec32_stride_cls(int cls) { return cls == kClassPoint32 ? rec32_stride(0) : rec32_stride(cls & 7); }
// FP64 record stride (doubles): [Px, Py, Pz, sqrt(p), G_0 .. G_{n-1}], padded to 2.
ESP_HD constexpr int rec64_stride(int L) { return ((4 + (L == 0 ? 1 : L == 1 ? 4 : L == 2 ? 10 : L == 3 ? 20 : 35) + 1) / 2) * 2; }
constexpr int kPointStride64 = 4;        // [x, y, z, Z]

// Boys tables: rows at T_i = i / 8 (exact in binary), each row F_0 .. F_{nmax}
// followed by exp(-T_i).
constexpr float kBoysStep = 0.125f;
constexpr float kBoysInvStep = 8.0f;
constexpr int kBoys32Terms = 6;          // Taylor terms (k = 0..5) of the FP32 table
constexpr float kBoys32Tmax = 30.0f;     // asymptotic form at and above this T
constexpr int kBoys32Rows = 241;         // T_i up to 30
// F_0..F_9, exp(-T_i), pad, lo words of F_0..F_4 and exp, pad x3.  The odd row
// stride spreads the rows of a warp's gathers (one row per lane, rows a few
// apart) over distinct shared-memory banks.
constexpr int kBoys32Row = 21;
constexpr int kBoys32LoCol = 12;         // low words: F_n at kBoys32LoCol + n (n <= 4), exp at + 5
constexpr int kBoys64Terms = 9;          // Taylor terms (k = 0..8) of the FP64 table
constexpr double kBoys64Tmax = 45.0;
constexpr int kBoys64Rows = 361;         // T_i up to 45
constexpr int kBoys64Row = 16;           // F_0..F_12, exp(-T_i), pad x2

struct TileMeta {
    int32_t cls;      // 0..4 = L of every distribution in the tile, 5 = point charges
    int32_t n;        // entries in the tile
    int32_t off32;    // float offset of the first FP32 record (distributions only)
    int32_t off64;    // double offset of the first FP64 record
    float cx, cy, cz; // bounding-sphere centre (recentred coordinates); for distribution
                      // tiles rounded onto the coordinate grid: the FP32 records' reference point
    float rad;        // bounding-sphere radius (about that centre)
    float pmin;       // smallest exponent p in the tile (0 for point tiles)
    float qabs;       // sum of absolute charge bounds of the tile's entries
    float vmax;       // largest |Q_d| 2 sqrt(p_d/pi) of an unmerged distribution (0 if none)
    float pad1;
};
static_assert(sizeof(TileMeta) == 48, "TileMeta layout");

// Canonical order of Hermite indices: by N = t+u+v, then t descending, then u descending.
ESP_HD constexpr int hidx(int t, int u, int v)
{
    int N = t + u + v;
    int base = N * (N + 1) * (N + 2) / 6;
    int off = 0;
    for (int tt = N; tt > t; --tt)
        off += N - tt + 1;
    return base + off + (N - t - u);
}

// ---------------------------------------------------------------------------
// Boys function from a Taylor table + downward recursion (T < Tmax) or the
// asymptotic series with upward recursion (T >= Tmax).  Templated on the real
// type so the FP32 and FP64 kernels (and host test hooks) share one definition.
//   F_n(T_i + d) = sum_k F_{n+k}(T_i) (-d)^k / k!            (Taylor in T)
//   F_n = (2 T F_{n+1} + e^{-T}) / (2n+1)                    (downward)
//   F_0 ~ sqrt(pi) / (2 sqrt(T)),  F_{n+1} ~ (2n+1)/(2T) F_n  (asymptotic)
// ---------------------------------------------------------------------------
template <typename R> struct BoysConst;
template <> struct BoysConst<float> {
    static constexpr int kTerms = kBoys32Terms;
    static constexpr int kRow = kBoys32Row;
    static constexpr int kExpCol = 10;
    ESP_HD static float tmax() { return kBoys32Tmax; }
};
template <> struct BoysConst<double> {
    static constexpr int kTerms = kBoys64Terms;
    static constexpr int kRow = kBoys64Row;
    static constexpr int kExpCol = 13;
    ESP_HD static double tmax() { return kBoys64Tmax; }
};

ESP_HD float esp_fma(float a, float b, float c) { return fmaf(a, b, c); }
ESP_HD double esp_fma(double a, double b, double c) { return fma(a, b, c); }

// ---------------------------------------------------------------------------
// Two FP32 lanes (two positions) per value.  On sm_100 and later every
// operation is one packed instruction (FADD2 / FMUL2 / FFMA2) that does both
// lanes, which halves the FP32 instructions the potential kernel issues; each
// lane rounds exactly as the scalar operation would.  Host code (test hooks)
// computes the lanes one after the other.
// ---------------------------------------------------------------------------
struct f2 {
    float x, y;
    ESP_HD f2() = default;
    ESP_HD constexpr f2(float a, float b) : x(a), y(b) {}
    ESP_HD constexpr explicit f2(float a) : x(a), y(a) {}
};
#if defined(__CUDA_ARCH__)
ESP_HD float2 f2_v(f2 a) { return make_float2(a.x, a.y); }
ESP_HD f2 v_f2(float2 a) { return f2(a.x, a.y); }
ESP_HD f2 operator+(f2 a, f2 b) { return v_f2(__fadd2_rn(f2_v(a), f2_v(b))); }
ESP_HD f2 operator-(f2 a, f2 b) { return v_f2(__fadd2_rn(f2_v(a), make_float2(-b.x, -b.y))); }
ESP_HD f2 operator*(f2 a, f2 b) { return v_f2(__fmul2_rn(f2_v(a), f2_v(b))); }
ESP_HD f2 esp_fma(f2 a, f2 b, f2 c) { return v_f2(__ffma2_rn(f2_v(a), f2_v(b), f2_v(c))); }
#else
ESP_HD f2 operator+(f2 a, f2 b) { return f2(a.x + b.x, a.y + b.y); }
ESP_HD f2 operator-(f2 a, f2 b) { return f2(a.x - b.x, a.y - b.y); }
ESP_HD f2 operator*(f2 a, f2 b) { return f2(a.x * b.x, a.y * b.y); }
ESP_HD f2 esp_fma(f2 a, f2 b, f2 c) { return f2(fmaf(a.x, b.x, c.x), fmaf(a.y, b.y, c.y)); }
#endif
ESP_HD f2 operator-(f2 a) { return f2(-a.x, -a.y); }
ESP_HD f2 &operator+=(f2 &a, f2 b) { return a = a + b; }
ESP_HD f2 esp_fma(float a, f2 b, f2 c) { return esp_fma(f2(a), b, c); }
ESP_HD f2 operator*(float a, f2 b) { return f2(a) * b; }

// Scalar type of a lane: float for f2.
template <typename R> struct lane_of { using type = R; };
template <> struct lane_of<f2> { using type = float; };

// y / 2 for a normal positive y by decrementing its exponent: an integer
// instruction, so it leaves the FP32 pipe to the arithmetic (exact; the
// reciprocal square roots below are normal for every finite offset)
ESP_HD float half_normal(float y)
{
#if defined(__CUDA_ARCH__)
    return __int_as_float(__float_as_int(y) - (1 << 23));
#else
    uint32_t b;
    std::memcpy(&b, &y, 4);
    b -= 1u << 23;
    std::memcpy(&y, &b, 4);
    return y;
#endif
}

ESP_HD float esp_rsqrt(float x)
{
#if defined(__CUDA_ARCH__)
    float y = rsqrtf(x);
#else
    float y = 1.0f / sqrtf(x);
#endif
    // one Newton step makes the error symmetric about zero (no bias across
    // terms): y + (1 - x y^2) y / 2
    float h = x * y;
    float e = fmaf(-h, y, 1.0f);
    return fmaf(e, half_normal(y), y);
}
ESP_HD f2 esp_rsqrt(f2 x)
{
#if defined(__CUDA_ARCH__)
    f2 y(rsqrtf(x.x), rsqrtf(x.y));
#else
    f2 y(1.0f / sqrtf(x.x), 1.0f / sqrtf(x.y));
#endif
    // the scalar version's Newton step, both lanes per instruction
    f2 h = x * y;
    f2 e = esp_fma(-h, y, f2(1.0f));
    return esp_fma(e, f2(half_normal(y.x), half_normal(y.y)), y);
}
ESP_HD double esp_rsqrt(double x)
{
#if defined(__CUDA_ARCH__)
    return rsqrt(x);
#else
    return 1.0 / sqrt(x);
#endif
}


// x * k with the constant k carried as hi + lo words, rounded once:
// fma(x, hi, x * lo).  Adding x * lo after rounding x * hi would be lost to
// that rounding and leave the one-signed error of k in every term (a bias).
template <typename R>
ESP_HD R mul_const(R x, double k)
{
    using S = typename lane_of<R>::type;
    const S hi = S(k);
    const S lo = S(k - double(hi));
    if (lo == S(0)) // k exact in R (folded at compile time for constant k)
        return x * R(hi);
    return esp_fma(x, R(hi), x * R(lo));
}

template <int L, typename R>
ESP_HD void boys_eval(R T, const R *__restrict__ tab, R (&F)[L + 1])
{
    using C = BoysConst<R>;
    if (T >= C::tmax()) {
        R rs = esp_rsqrt(T);
        F[0] = mul_const(rs, 0.88622692545275801365); // sqrt(pi)/2 / sqrt(T)
        R h = R(0.5) * rs * rs;                         // 1/(2T)
#pragma unroll
        for (int n = 1; n <= L; ++n)
            F[n] = F[n - 1] * (R(2 * n - 1) * h);
    } else {
        int i = (int)(T * R(8) + R(0.5));
        R d = T - R(i) * R(0.125);             // exact: T and T_i are within 1/16
        const R *row = tab + i * C::kRow;
        R md = -d;
        R f = row[L + C::kTerms - 1];
#pragma unroll
        for (int k = C::kTerms - 2; k >= 1; --k)
            f = f * (md * R(1.0 / (k + 1))) + row[L + k];
        f = f * md; // sum_{k>=1} F_{L+k}(T_i) (-d)^k / k!
        if constexpr (sizeof(R) == 4)
            F[L] = row[L] + (row[kBoys32LoCol + L] + f); // leading value carries a low word
        else
            F[L] = row[L] + f;
        if constexpr (L > 0) {
            // exp(-T) = exp(-T_i) * exp(-d), exp(-d) - 1 by its Taylor series (|d| <= 1/16)
            R q = R(1);
#pragma unroll
            for (int k = C::kTerms; k >= 2; --k)
                q = q * (md * R(1.0 / k)) + R(1);
            q = q * md;
            R e;
            if constexpr (sizeof(R) == 4)
                e = row[C::kExpCol] + esp_fma(row[C::kExpCol], q, row[kBoys32LoCol + 5]);
            else
                e = row[C::kExpCol] + row[C::kExpCol] * q;
            R T2 = T + T;
#pragma unroll
            for (int n = L - 1; n >= 0; --n)
                F[n] = mul_const(T2 * F[n + 1] + e, 1.0 / (2 * n + 1));
        }
    }
}

// Both lanes of a pair: the asymptotic form when both lanes are at or above
// Tmax, the table when both are below, else each lane by the scalar code.
template <int L>
ESP_HD void boys_eval(f2 T, const float *__restrict__ tab, f2 (&F)[L + 1])
{
    using C = BoysConst<float>;
    const bool a0 = T.x >= C::tmax(), a1 = T.y >= C::tmax();
    if (a0 && a1) {
        f2 rs = esp_rsqrt(T);
        F[0] = mul_const(rs, 0.88622692545275801365);
        f2 h = f2(0.5f) * rs * rs;
#pragma unroll
        for (int n = 1; n <= L; ++n)
            F[n] = F[n - 1] * (f2(float(2 * n - 1)) * h);
    } else if (!a0 && !a1) {
        const int i0 = (int)(T.x * 8.0f + 0.5f), i1 = (int)(T.y * 8.0f + 0.5f);
        const f2 d = T - f2(float(i0) * 0.125f, float(i1) * 0.125f); // exact: |T - T_i| <= 1/16
        const float *r0 = tab + i0 * C::kRow, *r1 = tab + i1 * C::kRow;
        const f2 md = -d;
        f2 f(r0[L + C::kTerms - 1], r1[L + C::kTerms - 1]);
#pragma unroll
        for (int k = C::kTerms - 2; k >= 1; --k)
            f = esp_fma(f, md * f2(float(1.0 / (k + 1))), f2(r0[L + k], r1[L + k]));
        f = f * md;
        F[L] = f2(r0[L], r1[L]) + (f2(r0[kBoys32LoCol + L], r1[kBoys32LoCol + L]) + f);
        if constexpr (L > 0) {
            f2 q(1.0f);
#pragma unroll
            for (int k = C::kTerms; k >= 2; --k)
                q = esp_fma(q, md * f2(float(1.0 / k)), f2(1.0f));
            q = q * md;
            const f2 ex(r0[C::kExpCol], r1[C::kExpCol]);
            const f2 e = ex + esp_fma(ex, q, f2(r0[kBoys32LoCol + 5], r1[kBoys32LoCol + 5]));
            const f2 T2 = T + T;
#pragma unroll
            for (int n = L - 1; n >= 0; --n)
                F[n] = mul_const(esp_fma(T2, F[n + 1], e), 1.0 / (2 * n + 1));
        }
    } else {
        float G0[L + 1], G1[L + 1];
        boys_eval<L, float>(T.x, tab, G0);
        boys_eval<L, float>(T.y, tab, G1);
#pragma unroll
        for (int n = 0; n <= L; ++n)
            F[n] = f2(G0[n], G1[n]);
    }
}

ESP_HD float esp_erfc(float x) { return erfcf(x); }
ESP_HD double esp_erfc(double x) { return erfc(x); }

// F_0(T) - sqrt(pi)/(2 sqrt(T)) = -sqrt(pi)/2 erfc(sqrt(T))/sqrt(T): the part of
// F_0 left after the monopole moved to a point charge, formed without
// cancellation; zero to working precision at and above Tmax.
template <typename R>
ESP_HD R boys_f0_short(R T)
{
    if (T >= BoysConst<R>::tmax())
        return R(0);
    R rs = esp_rsqrt(T);
    return -mul_const(esp_erfc(T * rs) * rs, 0.88622692545275801365);
}

ESP_HD f2 boys_f0_short(f2 T) { return f2(boys_f0_short<float>(T.x), boys_f0_short<float>(T.y)); }

// Far-field Boys values in units of sqrt(pi)/2 and for unit exponent:
// Fh_0 = 1/sqrt(r2), Fh_n = Fh_{n-1} (2n-1) / (2 r2).  With these, the
// recursion below evaluated at the unscaled offset P - C gives the Cartesian
// derivatives of 1/|P - C| (the exact potential of a Hermite Gaussian once
// exp(-p|P-C|^2) is negligible), and the multipole moments M_tuv complete it.
// Returned pre-multiplied by the recursion's level factor (-2)^n, i.e.
// F[n] = (-2)^n Fh_n = F[n-1] (-(2n-1)) / r2: the same values as scaling
// afterwards (powers of two are exact), with fewer multiplications.
template <int L, typename R>
ESP_HD void boys_far(R r2, R (&F)[L + 1])
{
    R rs = esp_rsqrt(r2);
    F[0] = rs;
    R h = rs * rs;
#pragma unroll
    for (int n = 1; n <= L; ++n)
        F[n] = F[n - 1] * (R(-(2 * n - 1)) * h);
}

// ---------------------------------------------------------------------------
// sum_tuv G_tuv S^0_tuv for one distribution of total angular momentum L at
// scaled offset (x, y, z) = sqrt(p) (P - C), given F_0..F_L(T).
// ---------------------------------------------------------------------------
// g0lo is the low word of G_0: the leading product is rounded once with it.
// With ACC, the terms are added into acc0 (one fewer operation per term than
// forming the sum and adding it); without, acc0 is ignored.  PRE: F[n] carries
// the level factor (-2)^n already (boys_far).
template <int L, typename R, typename G_t = R, bool ACC = false, bool PRE = false>
ESP_HD R hermite_contract(const R (&F)[L + 1], R x, R y, R z, const G_t *__restrict__ G, G_t g0lo = G_t(0),
                          R acc0 = R(0))
{
    if constexpr (L == 0) {
        if constexpr (ACC)
            return esp_fma(G[0], F[0], esp_fma(g0lo, F[0], acc0));
        else
            return esp_fma(G[0], F[0], g0lo * F[0]);
    } else {
    // S[n][h] for levels n = 0..L; level n needs N <= L - n
    R S[L + 1][35];
#pragma unroll
    for (int n = L; n >= 0; --n) {
        R s0 = F[n];
        if constexpr (!PRE) {
#pragma unroll
            for (int k = 0; k < n; ++k)
                s0 = -R(2) * s0;
        }
        S[n][0] = s0;
#pragma unroll
        for (int N = 1; N <= L - n; ++N) {
#pragma unroll
            for (int t = N; t >= 0; --t) {
#pragma unroll
                for (int u = N - t; u >= 0; --u) {
                    const int v = N - t - u;
                    R val;
                    if (t > 0) {
                        val = x * S[n + 1][hidx(t - 1, u, v)];
                        if (t > 1)
                            val = esp_fma(R(t - 1), S[n + 1][hidx(t - 2, u, v)], val);
                    } else if (u > 0) {
                        val = y * S[n + 1][hidx(t, u - 1, v)];
                        if (u > 1)
                            val = esp_fma(R(u - 1), S[n + 1][hidx(t, u - 2, v)], val);
                    } else {
                        val = z * S[n + 1][hidx(t, u, v - 1)];
                        if (v > 1)
                            val = esp_fma(R(v - 1), S[n + 1][hidx(t, u, v - 2)], val);
                    }
                    S[n][hidx(t, u, v)] = val;
                }
            }
        }
    }
    R acc;
    if constexpr (ACC)
        acc = esp_fma(G[0], S[0][0], esp_fma(g0lo, S[0][0], acc0));
    else
        acc = esp_fma(G[0], S[0][0], g0lo * S[0][0]);
#pragma unroll
    for (int h = 1; h < num_hermite(L); ++h)
        acc = esp_fma(G[h], S[0][h], acc);
    return acc;
    }
}

} // namespace esp
