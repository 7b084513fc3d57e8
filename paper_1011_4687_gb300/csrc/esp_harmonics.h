// Real regular solid harmonics: the basis of the interior expansion of the
// far environment's potential over the QM sphere.
//
// Every charge farther from the QM centre than the sphere's radius R makes a
// potential that is harmonic inside the sphere, so there it equals its
// interior multipole expansion (the addition theorem of 1/|r - r'|):
//   V_far(r) = sum_{l, m} c_lm S_lm(u),  u = (r - centre) / R,
//   S_lm(u) = |u|^l Y_lm(u / |u|),
// with Y_lm the real spherical harmonics fully normalised over the unit sphere
// to 4 pi (int Y_lm Y_l'm' dOmega = 4 pi delta delta), and
//   c_lm = (1 / 4 pi) int_{|u| = 1} V_far Y_lm dOmega.
//
// S_lm is evaluated as Re / Im of the complex solid harmonic
// A_l^m = |u|^l Pbar_l^m(cos theta) e^{i m phi} (Pbar fully normalised, no
// Condon-Shortley phase) by the standard recursions, all polynomial in x, y, z:
//   A_0^0 = 1,  A_1^1 = sqrt(3) (x + i y),
//   A_m^m = sqrt((2m + 1) / (2m)) (x + i y) A_{m-1}^{m-1}            (m >= 2),
//   A_{m+1}^m = sqrt(2m + 3) z A_m^m,
//   A_l^m = a_lm z A_{l-1}^m - b_lm |u|^2 A_{l-2}^m                  (l >= m + 2),
//   a_lm = sqrt((2l - 1)(2l + 1) / ((l - m)(l + m))),
//   b_lm = sqrt((2l + 1)(l + m - 1)(l - m - 1) / ((l - m)(l + m)(2l - 3))).
// Coefficient order: for l = 0..L, (l, 0), then (l, m, cos), (l, m, sin) for
// m = 1..l: index l^2 for m = 0, l^2 + 2m - 1 (cos) and l^2 + 2m (sin).
#pragma once

#include <math.h>

#if defined(__CUDACC__)
#define ESP_HH __host__ __device__ __forceinline__
#else
#define ESP_HH inline
#endif

namespace esp {

constexpr int kMaxExpDegree = 40;
ESP_HH constexpr int num_harmonics(int L) { return (L + 1) * (L + 1); }

// Recursion constants for degree <= L, laid out [m][l] (stride kMaxExpDegree + 1):
// rc[0][m][l] = a_lm, rc[1][m][l] = b_lm (zero where unused); sec[m] = the
// sectoral factor of A_m^m, sub[m] = sqrt(2m + 3).
struct HarmonicConsts {
    double a[kMaxExpDegree + 1][kMaxExpDegree + 1];
    double b[kMaxExpDegree + 1][kMaxExpDegree + 1];
    double sec[kMaxExpDegree + 1];
    double sub[kMaxExpDegree + 1];
};

inline void harmonic_consts(HarmonicConsts &h)
{
    for (int m = 0; m <= kMaxExpDegree; ++m) {
        h.sec[m] = m == 0 ? 1.0 : (m == 1 ? sqrt(3.0) : sqrt((2.0 * m + 1.0) / (2.0 * m)));
        h.sub[m] = sqrt(2.0 * m + 3.0);
        for (int l = 0; l <= kMaxExpDegree; ++l) {
            h.a[m][l] = 0.0;
            h.b[m][l] = 0.0;
            if (l >= m + 2) {
                const double lm = double(l - m), lp = double(l + m);
                h.a[m][l] = sqrt((2.0 * l - 1.0) * (2.0 * l + 1.0) / (lm * lp));
                h.b[m][l] = sqrt((2.0 * l + 1.0) * (lp - 1.0) * (lm - 1.0) / (lm * lp * (2.0 * l - 3.0)));
            }
        }
    }
}

// Calls f(k, value) for every S_k(u), k < num_harmonics(L), m-major (all l of
// one m before the next m).  a, b, sec, sub: the HarmonicConsts arrays (any
// memory space the caller can read).
template <typename F>
ESP_HH void solid_harmonics(double x, double y, double z, int L, const double (*a)[kMaxExpDegree + 1],
                            const double (*b)[kMaxExpDegree + 1], const double *sec, const double *sub, F &&f)
{
    const double r2 = x * x + y * y + z * z;
    double sr = 1.0, si = 0.0; // A_m^m
    for (int m = 0; m <= L; ++m) {
        if (m > 0) {
            const double nr = sec[m] * (x * sr - y * si), ni = sec[m] * (x * si + y * sr);
            sr = nr;
            si = ni;
        }
        // l = m
        if (m == 0) {
            f(0, sr);
        } else {
            f(m * m + 2 * m - 1, sr);
            f(m * m + 2 * m, si);
        }
        if (m + 1 > L)
            break;
        double pr = sr, pi = si;                              // A_{l-2}^m
        double qr = sub[m] * z * sr, qi = sub[m] * z * si;    // A_{l-1}^m = A_{m+1}^m
        {
            const int l = m + 1;
            if (m == 0) {
                f(l * l, qr);
            } else {
                f(l * l + 2 * m - 1, qr);
                f(l * l + 2 * m, qi);
            }
        }
        for (int l = m + 2; l <= L; ++l) {
            const double al = a[m][l] * z, bl = b[m][l] * r2;
            const double nr = al * qr - bl * pr, ni = al * qi - bl * pi;
            pr = qr;
            pi = qi;
            qr = nr;
            qi = ni;
            if (m == 0) {
                f(l * l, qr);
            } else {
                f(l * l + 2 * m - 1, qr);
                f(l * l + 2 * m, qi);
            }
        }
    }
}

} // namespace esp
