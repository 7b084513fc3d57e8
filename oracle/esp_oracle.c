/*
 * Plain FP64 CPU oracle for the environment electrostatic potential.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load this file's library.  It shares no
 * code, header, table or constant with the CUDA library.
 *
 * What it computes (the plain definition, term by term, in input order):
 *
 *   V(C) = sum_beta Z_beta / |C - R_beta|
 *        + sum_ab w_ab * int chi_a(r) chi_b(r) / |r - C| dr
 *
 * with chi(r) = (x-Ax)^i (y-Ay)^j (z-Az)^k exp(-alpha |r-A|^2), an
 * unnormalised Cartesian primitive.  The first sum is the nuclear term of the
 * paper's Eq. ElectrostaticField (Sec. II.B); the second is its cell sum with
 * each discretised cell rho(r_m) generalised to a weighted Gaussian product
 * (a cell is the exponent -> infinity limit).  The paper's U_ES equals -V for
 * an electron.
 *
 * Each Gaussian-pair integral is an Obara-Saika nuclear-attraction integral
 * (Obara & Saika, J. Chem. Phys. 84, 3963 (1986)): the vertical recurrence
 * builds (a|0)^(m) from (0|0)^(m) = (2 pi / p) K_AB F_m(p |P-C|^2), and the
 * horizontal recurrence (a|b+1_i) = (a+1_i|b) + (A_i - B_i)(a|b) moves angular
 * momentum onto b.  This is a different algorithm from the McMurchie-Davidson
 * Hermite path used on the GPU.
 *
 * The Boys function F_m(T) = int_0^1 t^{2m} exp(-T t^2) dt is evaluated as
 *   T <  30: the positive-term series
 *            F_m(T) = e^{-T} sum_k (2T)^k / ((2m+1)(2m+3)...(2m+2k+1))
 *            at the highest order, then downward recursion
 *            F_n = (2T F_{n+1} + e^{-T}) / (2n+1);
 *   T >= 30: F_0 = (1/2) sqrt(pi/T) erf(sqrt(T)) from the C library, then
 *            upward recursion F_{n+1} = ((2n+1) F_n - e^{-T}) / (2T).
 * Sums over terms use Neumaier's compensated summation in a fixed order.
 */
#include <math.h>
#include <stdint.h>
#include <stddef.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_PI 3.14159265358979323846
#define OR_LPRIM 4            /* largest angular momentum per primitive */
#define OR_LTOT (2 * OR_LPRIM) /* largest la + lb */
#define OR_D (OR_LTOT + 1)

int oracle_boys(int nmax, double T, double *F)
{
    if (nmax < 0 || nmax > 64 || !(T >= 0.0) || !F)
        return -1;
    double e = exp(-T);
    if (T < 30.0) {
        double term = 1.0 / (2.0 * nmax + 1.0);
        double sum = term;
        for (int k = 1; k < 2000; ++k) {
            term *= 2.0 * T / (2.0 * nmax + 2.0 * k + 1.0);
            sum += term;
            if (term < 1e-18 * sum)
                break;
        }
        F[nmax] = e * sum;
        for (int n = nmax - 1; n >= 0; --n)
            F[n] = (2.0 * T * F[n + 1] + e) / (2.0 * n + 1.0);
    } else {
        F[0] = 0.5 * sqrt(OR_PI / T) * erf(sqrt(T));
        for (int n = 0; n < nmax; ++n)
            F[n + 1] = ((2.0 * n + 1.0) * F[n] - e) / (2.0 * T);
    }
    return 0;
}

/* Vertical recurrence table: vrr[m][i][j][k] = (a|0)^(m), a = (i,j,k). */
typedef struct {
    double v[OR_D][OR_D][OR_D][OR_D];
} or_vrr;

static double or_hrr(const or_vrr *t, int ai, int aj, int ak, int bi, int bj, int bk, const double AB[3])
{
    if (bi > 0)
        return or_hrr(t, ai + 1, aj, ak, bi - 1, bj, bk, AB) + AB[0] * or_hrr(t, ai, aj, ak, bi - 1, bj, bk, AB);
    if (bj > 0)
        return or_hrr(t, ai, aj + 1, ak, bi, bj - 1, bk, AB) + AB[1] * or_hrr(t, ai, aj, ak, bi, bj - 1, bk, AB);
    if (bk > 0)
        return or_hrr(t, ai, aj, ak + 1, bi, bj, bk - 1, AB) + AB[2] * or_hrr(t, ai, aj, ak, bi, bj, bk - 1, AB);
    return t->v[0][ai][aj][ak];
}

/* int chi_a chi_b / |r - C| dr for one primitive pair (Obara-Saika). */
double oracle_pair_potential(const double A[3], double alpha, const int32_t la[3],
                             const double B[3], double beta, const int32_t lb[3], const double C[3])
{
    int L = la[0] + la[1] + la[2] + lb[0] + lb[1] + lb[2];
    if (L > OR_LTOT)
        return NAN;
    double p = alpha + beta;
    double P[3], PA[3], PC[3], AB[3];
    double ab2 = 0.0, pc2 = 0.0;
    for (int d = 0; d < 3; ++d) {
        P[d] = (alpha * A[d] + beta * B[d]) / p;
        PA[d] = P[d] - A[d];
        PC[d] = P[d] - C[d];
        AB[d] = A[d] - B[d];
        ab2 += AB[d] * AB[d];
        pc2 += PC[d] * PC[d];
    }
    double K = exp(-alpha * beta / p * ab2);
    double F[OR_D + 1];
    oracle_boys(L, p * pc2, F);

    static __thread or_vrr t; /* per-thread scratch, fully written before read */
    double pref = 2.0 * OR_PI / p * K;
    for (int m = 0; m <= L; ++m)
        t.v[m][0][0][0] = pref * F[m];
    double o2p = 0.5 / p;
    for (int l = 1; l <= L; ++l) {
        for (int i = l; i >= 0; --i) {
            for (int j = l - i; j >= 0; --j) {
                int k = l - i - j;
                int a[3] = {i, j, k};
                int d = (i > 0) ? 0 : ((j > 0) ? 1 : 2);
                int am[3] = {i, j, k};
                am[d] -= 1;                 /* a - 1_d */
                int nd = am[d];             /* N_d(a - 1_d) */
                for (int m = 0; m <= L - l; ++m) {
                    double val = PA[d] * t.v[m][am[0]][am[1]][am[2]]
                               - PC[d] * t.v[m + 1][am[0]][am[1]][am[2]];
                    if (nd > 0) {
                        int a2[3] = {am[0], am[1], am[2]};
                        a2[d] -= 1;
                        val += nd * o2p * (t.v[m][a2[0]][a2[1]][a2[2]] - t.v[m + 1][a2[0]][a2[1]][a2[2]]);
                    }
                    t.v[m][a[0]][a[1]][a[2]] = val;
                }
            }
        }
    }
    return or_hrr(&t, la[0], la[1], la[2], lb[0], lb[1], lb[2], AB);
}

typedef struct {
    double s, c;
} or_acc;

static inline void or_add(or_acc *a, double x)
{
    double t = a->s + x;
    if (fabs(a->s) >= fabs(x))
        a->c += (a->s - t) + x;
    else
        a->c += (x - t) + a->s;
    a->s = t;
}

/*
 * V[n_pos]: potential at each position.  Arrays are row-major:
 *   nuc_xyz [n_nuc][3], nuc_Z [n_nuc];
 *   A [n_pairs][3], alpha [n_pairs], la [n_pairs][3] (same for B, beta, lb), w [n_pairs];
 *   pos [n_pos][3].
 * n_threads <= 0 uses the OpenMP default.  Returns 0, or -1 on a bad argument.
 */
int oracle_potential(const double *nuc_xyz, const double *nuc_Z, int64_t n_nuc,
                     const double *A, const double *alpha, const int32_t *la,
                     const double *B, const double *beta, const int32_t *lb,
                     const double *w, int64_t n_pairs,
                     const double *pos, int64_t n_pos, double *V, int n_threads)
{
    if (n_nuc < 0 || n_pairs < 0 || n_pos < 0 || (n_pos > 0 && (!pos || !V)))
        return -1;
    for (int64_t q = 0; q < n_pairs; ++q) {
        int L = la[3 * q] + la[3 * q + 1] + la[3 * q + 2] + lb[3 * q] + lb[3 * q + 1] + lb[3 * q + 2];
        if (L > OR_LTOT || la[3 * q] < 0 || la[3 * q + 1] < 0 || la[3 * q + 2] < 0 ||
            lb[3 * q] < 0 || lb[3 * q + 1] < 0 || lb[3 * q + 2] < 0 || !(alpha[q] > 0.0) || !(beta[q] > 0.0))
            return -1;
    }
#ifdef _OPENMP
    if (n_threads > 0)
        omp_set_num_threads(n_threads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int64_t i = 0; i < n_pos; ++i) {
        const double *C = pos + 3 * i;
        or_acc acc = {0.0, 0.0};
        for (int64_t b = 0; b < n_nuc; ++b) {
            double dx = C[0] - nuc_xyz[3 * b], dy = C[1] - nuc_xyz[3 * b + 1], dz = C[2] - nuc_xyz[3 * b + 2];
            or_add(&acc, nuc_Z[b] / sqrt(dx * dx + dy * dy + dz * dz));
        }
        for (int64_t q = 0; q < n_pairs; ++q)
            or_add(&acc, w[q] * oracle_pair_potential(A + 3 * q, alpha[q], la + 3 * q,
                                                      B + 3 * q, beta[q], lb + 3 * q, C));
        V[i] = acc.s + acc.c;
    }
    return 0;
}

/*
 * K[n_pos]: condition of the sum at each position, sum of the absolute values
 * of its terms: sum_beta |Z_beta / |C - R_beta|| + sum_ab |w_ab (a|1/r_C|b)|.
 * Same layout and return value as oracle_potential.
 */
int oracle_abs_terms(const double *nuc_xyz, const double *nuc_Z, int64_t n_nuc,
                     const double *A, const double *alpha, const int32_t *la,
                     const double *B, const double *beta, const int32_t *lb,
                     const double *w, int64_t n_pairs,
                     const double *pos, int64_t n_pos, double *K, int n_threads)
{
    if (n_nuc < 0 || n_pairs < 0 || n_pos < 0 || (n_pos > 0 && (!pos || !K)))
        return -1;
#ifdef _OPENMP
    if (n_threads > 0)
        omp_set_num_threads(n_threads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int64_t i = 0; i < n_pos; ++i) {
        const double *C = pos + 3 * i;
        double acc = 0.0;
        for (int64_t b = 0; b < n_nuc; ++b) {
            double dx = C[0] - nuc_xyz[3 * b], dy = C[1] - nuc_xyz[3 * b + 1], dz = C[2] - nuc_xyz[3 * b + 2];
            acc += fabs(nuc_Z[b] / sqrt(dx * dx + dy * dy + dz * dz));
        }
        for (int64_t q = 0; q < n_pairs; ++q)
            acc += fabs(w[q] * oracle_pair_potential(A + 3 * q, alpha[q], la + 3 * q, B + 3 * q, beta[q], lb + 3 * q, C));
        K[i] = acc;
    }
    return 0;
}

/* E[w] = -sum_e V[w*n_elec + e]: the walker's environment energy sum_e U_ES(r_e). */
int oracle_walker_energies(const double *V, int64_t n_walkers, int64_t n_elec, double *E)
{
    if (n_walkers < 0 || n_elec < 0 || (n_walkers > 0 && (!V || !E)))
        return -1;
    for (int64_t w = 0; w < n_walkers; ++w) {
        or_acc acc = {0.0, 0.0};
        for (int64_t e = 0; e < n_elec; ++e)
            or_add(&acc, -V[w * n_elec + e]);
        E[w] = acc.s + acc.c;
    }
    return 0;
}

int oracle_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
