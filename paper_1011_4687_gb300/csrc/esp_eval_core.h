// Per-tile evaluation cores shared by the CUDA kernels and the host test hook.
//
// One definition serves both, so the host emulation of a kernel performs the
// same operations in the same order (the device may fuse a*b+c into one FMA
// where the host rounds twice; the statistics of the errors are the same).
#pragma once

#include "esp_internal.h"

namespace esp {

#ifndef ESP_SUM_BLOCK
#define ESP_SUM_BLOCK 4
#endif
// distributions summed in plain FP32 before a TwoSum into the running pair
constexpr int kSumBlock = ESP_SUM_BLOCK;

#ifndef ESP_REL_RATIO
#define ESP_REL_RATIO 2
#endif
// far tiles at least this many of their radii away take the one-addition
// offset (see tile_f32c)
constexpr float kRelRatio = ESP_REL_RATIO;

// error-free S + x = s + e (Knuth TwoSum); e is added into the compensation C
ESP_HD void two_sum_acc(float &S, float &C, float x)
{
    float s = S + x;
    float bp = s - S;
    float e = (S - (s - bp)) + (x - bp);
    S = s;
    C += e;
}

ESP_HD void two_sum_acc(double &S, double &C, double x)
{
    double s = S + x;
    double bp = s - S;
    double e = (S - (s - bp)) + (x - bp);
    S = s;
    C += e;
}

// One distribution (FP64 record [Px, Py, Pz, sqrt(p), G...]) at one position.
// SHORT: the monopole Q/|P - C| (Q = G_000 sqrt(pi)/(2 sqrt(p))) is left out
// because the point charge at P carries it.
template <int L, bool SHORT = false>
ESP_HD double dist_f64(const double *__restrict__ r, double cx, double cy, double cz,
                       const double *__restrict__ boys64)
{
    double dx = r[0] - cx, dy = r[1] - cy, dz = r[2] - cz;
    double sp = r[3];
    double F[L + 1];
    double v;
    if constexpr (L == 0) {
        double T = (sp * sp) * (dx * dx + dy * dy + dz * dz);
        boys_eval<L, double>(T, boys64, F);
        v = r[4] * F[0];
    } else {
        double x = sp * dx, y = sp * dy, z = sp * dz;
        double T = x * x + y * y + z * z;
        boys_eval<L, double>(T, boys64, F);
        v = hermite_contract<L, double>(F, x, y, z, r + 4);
    }
    if constexpr (SHORT)
        v -= r[4] * 0.88622692545275801365 / sp * esp_rsqrt(dx * dx + dy * dy + dz * dz);
    return v;
}

// A whole tile of one class at one position in FP64.
template <int L, bool SHORT>
ESP_HD double tile_f64_one(const double *__restrict__ rec, int n, double cx, double cy, double cz,
                           const double *__restrict__ boys64)
{
    constexpr int st = rec64_stride(L);
    double acc = 0.0;
    for (int j = 0; j < n; ++j)
        acc += dist_f64<L, SHORT>(rec + j * st, cx, cy, cz, boys64);
    return acc;
}

// cls: tile class (L, possibly with kClassShortBit)
ESP_HD double tile_f64_one_any(int cls, const double *rec, int n, double cx, double cy, double cz,
                               const double *boys64)
{
    switch (cls) {
    case 0: return tile_f64_one<0, false>(rec, n, cx, cy, cz, boys64);
    case 1: return tile_f64_one<1, false>(rec, n, cx, cy, cz, boys64);
    case 2: return tile_f64_one<2, false>(rec, n, cx, cy, cz, boys64);
    case 3: return tile_f64_one<3, false>(rec, n, cx, cy, cz, boys64);
    case 4: return tile_f64_one<4, false>(rec, n, cx, cy, cz, boys64);
    case 8: return tile_f64_one<0, true>(rec, n, cx, cy, cz, boys64);
    case 9: return tile_f64_one<1, true>(rec, n, cx, cy, cz, boys64);
    case 10: return tile_f64_one<2, true>(rec, n, cx, cy, cz, boys64);
    case 11: return tile_f64_one<3, true>(rec, n, cx, cy, cz, boys64);
    default: return tile_f64_one<4, true>(rec, n, cx, cy, cz, boys64);
    }
}

// Point charges [x, y, z, Z] at PPT positions in FP64.
template <int PPT>
ESP_HD void tile_points_f64(const double *__restrict__ pts, int n, const double (&c64)[PPT][3], double (&acc)[PPT])
{
    for (int j = 0; j < n; ++j) {
        const double *a = pts + 4 * j;
#pragma unroll
        for (int q = 0; q < PPT; ++q) {
            double dx = a[0] - c64[q][0], dy = a[1] - c64[q][1], dz = a[2] - c64[q][2];
            acc[q] += a[3] * esp_rsqrt(dx * dx + dy * dy + dz * dz);
        }
    }
}

// ---------------------------------------------------------------------------
// FP32-compensated tiles of class L at PPT positions (record layout in
// esp_internal.h).  The centre carries a low word, and the offset is formed as
//   offset = (P_hi - C_hi) + (P_lo - C_lo),
// so that the fixed rounding of stored coordinates does not add up coherently
// over the electrons of a walker; the leading coefficient carries a low word
// for the same reason.  Distribution records store their hi words relative
// to the tile's grid point T (stored = P_hi - T, exact: both on the grid), and
// the caller passes th = T - C_hi per position (exact), so the offset is
//   offset = (stored + th) + (P_lo - C_lo),
// the same value as above.  REL (far tiles at least kRelRatio radii away):
//   offset = (stored + P_lo) + dq,   dq = th - C_lo per tile and position,
// one addition per coordinate and term instead of three.  The record's part is
// rounded once, the same way for every position (a fixed shift of at most
// 2^-24 |P - T| <= 2^-24 radius), which is why REL is kept to tiles where
// that shift is a small fraction of the distance.
// Terms are summed in FP32 over blocks of kSumBlock (4) distributions and
// each block sum is added into a per-position (S, C) pair by TwoSum.
// Positions flagged near add nothing here (the caller evaluates the tile for
// them in FP64).
//
// FAR:   every position of the warp is in the asymptotic regime
//        (p_min * dist^2 >= Tmax): v = sum_tuv M_tuv d^{tuv}(1/|P - C|).
// !FAR:  general form sum_tuv G_tuv S^0_tuv with the Boys function from the
//        Taylor table or the asymptotic series per evaluation.
// SHORT: the monopole sits in the point charge at P (M_000 is stored as 0 for
//        the far form; the general form uses F_0 - F_0^asymptotic).
// ---------------------------------------------------------------------------
// SEL: some position may be flagged near (its terms are selected away); a
// caller that knows none is can drop the select.
template <int L, int PPT, bool FAR, bool SHORT, bool SEL = true, bool REL = false>
ESP_HD void tile_f32c(const float *__restrict__ s_rec, int n, const float (&th)[PPT][3], const float (&cl)[PPT][3],
                      const float (&dq)[PPT][3], const bool (&nearq)[PPT], float (&S)[PPT], float (&Cc)[PPT],
                      const float *__restrict__ s_boys)
{
    constexpr int st = rec32_stride(L);
    constexpr int nh = num_hermite(L);
    constexpr int lo = rec32_lo(L);
    constexpr int co = FAR ? rec32_m(L) : rec32_g(L);
    constexpr int c0lo = FAR ? rec32_lo(L) + 3 : rec32_g0lo(L);
    // one distribution j at the PPT positions, added into blk
    auto one = [&](int j, float (&blk)[PPT]) {
        const float *r = s_rec + j * st;
        const float4 r0 = reinterpret_cast<const float4 *>(r)[0];
        const float4 r1 = reinterpret_cast<const float4 *>(r)[1];
        const float ps = r0.w;
        const float plx = r1.x, ply = r1.y, plz = r1.z;
        // (REL: the record's offset from T, rounded once)
        float px = r0.x, py = r0.y, pz = r0.z;
        if constexpr (REL) {
            px += plx;
            py += ply;
            pz += plz;
        }
        const float k0lo = FAR ? r1.w : r[c0lo];
        float K[nh];
        if constexpr (FAR) {
            // the moments start 16-byte aligned: whole float4 loads
#pragma unroll
            for (int h = 0; h + 3 < nh; h += 4) {
                const float4 k4 = reinterpret_cast<const float4 *>(r + co)[h / 4];
                K[h] = k4.x;
                K[h + 1] = k4.y;
                K[h + 2] = k4.z;
                K[h + 3] = k4.w;
            }
#pragma unroll
            for (int h = nh - nh % 4; h < nh; ++h)
                K[h] = r[co + h];
        } else {
#pragma unroll
            for (int h = 0; h < nh; ++h)
                K[h] = r[co + h];
        }
#pragma unroll
        for (int q = 0; q < PPT; ++q) {
            float dx, dy, dz;
            if constexpr (REL) {
                dx = px + dq[q][0];
                dy = py + dq[q][1];
                dz = pz + dq[q][2];
            } else {
                dx = (px + th[q][0]) + (plx - cl[q][0]);
                dy = (py + th[q][1]) + (ply - cl[q][1]);
                dz = (pz + th[q][2]) + (plz - cl[q][2]);
            }
            float v;
            float F[L + 1];
            if constexpr (FAR) {
                boys_far<L, float>(dx * dx + dy * dy + dz * dz, F);
                v = hermite_contract<L, float, float, false, true>(F, dx, dy, dz, K, k0lo);
            } else if constexpr (L == 0) {
                const float r2 = dx * dx + dy * dy + dz * dz;
                float T = esp_fma(ps, r2, r[rec32_pslo(L)] * r2);
                if constexpr (SHORT)
                    F[0] = boys_f0_short<float>(T);
                else
                    boys_eval<L, float>(T, s_boys, F);
                v = hermite_contract<L, float>(F, dx, dy, dz, K, k0lo);
            } else {
                const float pslo = r[rec32_pslo(L)];
                float x = esp_fma(ps, dx, pslo * dx), y = esp_fma(ps, dy, pslo * dy), z = esp_fma(ps, dz, pslo * dz);
                float T = x * x + y * y + z * z;
                boys_eval<L, float>(T, s_boys, F);
                if constexpr (SHORT)
                    F[0] = boys_f0_short<float>(T);
                v = hermite_contract<L, float>(F, x, y, z, K, k0lo);
            }
            if constexpr (SEL)
                blk[q] += nearq[q] ? 0.0f : v;
            else
                blk[q] += v;
        }
    };
    for (int j0 = 0; j0 < n; j0 += kSumBlock) {
        float blk[PPT];
#pragma unroll
        for (int q = 0; q < PPT; ++q)
            blk[q] = 0.0f;
        // (unrolling the block measured slower: more live registers at the
        // 128-register cap of 4 positions per thread)
        const int j1 = (j0 + kSumBlock < n) ? j0 + kSumBlock : n;
        for (int j = j0; j < j1; ++j)
            one(j, blk);
#pragma unroll
        for (int q = 0; q < PPT; ++q)
            two_sum_acc(S[q], Cc[q], blk[q]);
    }
}

// Paired form of tile_f32c for the kernel: NP pairs of positions, each pair
// held as two FP32 lanes (f2) so that every FP32 operation of the two
// positions is one packed instruction.  Lane by lane it performs the
// operations of tile_f32c in the same order; positions flagged near take a
// zero weight (wq = 0) instead of a select.
ESP_HD void two_sum_acc(f2 &S, f2 &C, f2 x)
{
    f2 s = S + x;
    f2 bp = s - S;
    f2 e = (S - (s - bp)) + (x - bp);
    S = s;
    C += e;
}

template <int L, int NP, bool FAR, bool SHORT, bool SEL, bool REL = false>
ESP_HD void tile_f32c2(const float *__restrict__ s_rec, int n, const f2 (&th)[NP][3], const f2 (&cl)[NP][3],
                       const f2 (&dq)[NP][3], const f2 (&wq)[NP], f2 (&S)[NP], f2 (&Cc)[NP],
                       const float *__restrict__ s_boys)
{
    constexpr int st = rec32_stride(L);
    constexpr int nh = num_hermite(L);
    constexpr int co = FAR ? rec32_m(L) : rec32_g(L);
    constexpr int c0lo = FAR ? rec32_lo(L) + 3 : rec32_g0lo(L);
    auto one = [&](int j, f2 (&blk)[NP]) {
        const float *r = s_rec + j * st;
        const float4 r0 = reinterpret_cast<const float4 *>(r)[0];
        const float4 r1 = reinterpret_cast<const float4 *>(r)[1];
        const f2 plx(r1.x), ply(r1.y), plz(r1.z);
        // (REL: the record's offset from T, rounded once)
        float hx = r0.x, hy = r0.y, hz = r0.z;
        if constexpr (REL) {
            hx += r1.x;
            hy += r1.y;
            hz += r1.z;
        }
        const f2 px(hx), py(hy), pz(hz);
        const float ps = r0.w;
        const float k0lo = FAR ? r1.w : r[c0lo];
        float K[nh];
        if constexpr (FAR) {
#pragma unroll
            for (int h = 0; h + 3 < nh; h += 4) {
                const float4 k4 = reinterpret_cast<const float4 *>(r + co)[h / 4];
                K[h] = k4.x;
                K[h + 1] = k4.y;
                K[h + 2] = k4.z;
                K[h + 3] = k4.w;
            }
#pragma unroll
            for (int h = nh - nh % 4; h < nh; ++h)
                K[h] = r[co + h];
        } else {
#pragma unroll
            for (int h = 0; h < nh; ++h)
                K[h] = r[co + h];
        }
#pragma unroll
        for (int q = 0; q < NP; ++q) {
            f2 dx, dy, dz;
            if constexpr (REL) {
                dx = px + dq[q][0];
                dy = py + dq[q][1];
                dz = pz + dq[q][2];
            } else {
                dx = (px + th[q][0]) + (plx - cl[q][0]);
                dy = (py + th[q][1]) + (ply - cl[q][1]);
                dz = (pz + th[q][2]) + (plz - cl[q][2]);
            }
            f2 v;
            f2 F[L + 1];
            if constexpr (FAR && !SEL) {
                // the common case: the terms go straight into the block sum
                const f2 r2 = esp_fma(dx, dx, esp_fma(dy, dy, dz * dz));
                boys_far<L, f2>(r2, F);
                blk[q] = hermite_contract<L, f2, float, true, true>(F, dx, dy, dz, K, k0lo, blk[q]);
                continue;
            } else if constexpr (FAR) {
                const f2 r2 = esp_fma(dx, dx, esp_fma(dy, dy, dz * dz));
                boys_far<L, f2>(r2, F);
                v = hermite_contract<L, f2, float, false, true>(F, dx, dy, dz, K, k0lo);
            } else if constexpr (L == 0) {
                const f2 r2 = esp_fma(dx, dx, esp_fma(dy, dy, dz * dz));
                const f2 T = esp_fma(f2(ps), r2, f2(r[rec32_pslo(L)]) * r2);
                if constexpr (SHORT)
                    F[0] = boys_f0_short(T);
                else
                    boys_eval<L>(T, s_boys, F);
                v = hermite_contract<L, f2, float>(F, dx, dy, dz, K, k0lo);
            } else {
                const f2 sp(ps), pslo(r[rec32_pslo(L)]);
                const f2 x = esp_fma(sp, dx, pslo * dx), y = esp_fma(sp, dy, pslo * dy),
                         z = esp_fma(sp, dz, pslo * dz);
                const f2 T = esp_fma(x, x, esp_fma(y, y, z * z));
                boys_eval<L>(T, s_boys, F);
                if constexpr (SHORT)
                    F[0] = boys_f0_short(T);
                v = hermite_contract<L, f2, float>(F, x, y, z, K, k0lo);
            }
            if constexpr (SEL)
                blk[q] = esp_fma(v, wq[q], blk[q]);
            else
                blk[q] += v;
        }
    };
    for (int j0 = 0; j0 < n; j0 += kSumBlock) {
        f2 blk[NP];
#pragma unroll
        for (int q = 0; q < NP; ++q)
            blk[q] = f2(0.0f);
        const int j1 = (j0 + kSumBlock < n) ? j0 + kSumBlock : n;
        for (int j = j0; j < j1; ++j)
            one(j, blk);
#pragma unroll
        for (int q = 0; q < NP; ++q)
            two_sum_acc(S[q], Cc[q], blk[q]);
    }
}

// Per-position classification of a tile: near (FP64 instead; only with a
// positive near_r and for tiles whose distributions can produce potentials
// above kNearVmax), far (the asymptotic form is exact to FP32 for every
// distribution of the tile) and rel (far, and at least kRelRatio radii from
// the tile's sphere: the one-addition offset of tile_f32c applies).
ESP_HD void classify_tile(const TileMeta &m, float cx, float cy, float cz, float near_r, bool &nearq, bool &farq,
                          bool &relq)
{
    float ex = cx - m.cx, ey = cy - m.cy, ez = cz - m.cz;
    float d = sqrtf(ex * ex + ey * ey + ez * ez) - m.rad;
    nearq = near_r > 0.0f && m.vmax >= kNearVmax && d < near_r;
    farq = nearq || (d > 0.0f && m.pmin * d * d >= kBoys32Tmax);
    relq = nearq || (farq && d >= kRelRatio * m.rad);
}

} // namespace esp
