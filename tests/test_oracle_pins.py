"""Pins of the FP64 oracle against facts fixed by mathematics, not by the oracle.

Each test targets a plausible mistake in the oracle:
  * Boys function vs mpmath's 1F1 and SciPy's incomplete gamma (branch at T=30,
    recursions, prefactor);
  * s-Gaussian charge vs its closed form q erf(sqrt(alpha) r)/r, its r->0 limit
    and the point-charge limit of the paper's cell sum (Eq. ElectrostaticField);
  * p/d pairs vs brute-force 3-D quadrature of the charge density (catches a
    wrong sign, index or dropped term in the Obara-Saika recurrences);
  * p/d pairs vs an independent McMurchie-Davidson implementation;
  * far-field multipole expansion, Gauss's law and the mean-value property;
  * rotation (with the density rotated tensorially), translation, A<->B swap.
"""
import math

import numpy as np
import pytest

import oracle
from tests.md_reference import boys_scipy, md_pair_potential
from workloads import PairList, small_environment, tiny_pd_environment
from workloads.generate import CART


# ----------------------------------------------------------------------------
# helpers (independent of the oracle)
# ----------------------------------------------------------------------------
def density(pairs: PairList, pts: np.ndarray) -> np.ndarray:
    """rho(r) = sum w chi_a chi_b at points [M,3]."""
    rho = np.zeros(pts.shape[0])
    for q in range(len(pairs)):
        ua = pts - pairs.A[q]
        ub = pts - pairs.B[q]
        fa = np.prod(ua ** pairs.la[q], axis=1) * np.exp(-pairs.alpha[q] * np.einsum("ij,ij->i", ua, ua))
        fb = np.prod(ub ** pairs.lb[q], axis=1) * np.exp(-pairs.beta[q] * np.einsum("ij,ij->i", ub, ub))
        rho += pairs.w[q] * fa * fb
    return rho


def quadrature_potential(pairs: PairList, C: np.ndarray, nseg=10, nr=32, nth=48, nph=96) -> float:
    """int rho(r)/|r-C| dr = int_0^inf s ds int rho(C + s n) dOmega (spherical grid at C)."""
    p_min = float(np.min(pairs.alpha + pairs.beta))
    P = (pairs.alpha[:, None] * pairs.A + pairs.beta[:, None] * pairs.B) / (pairs.alpha + pairs.beta)[:, None]
    smax = float(np.max(np.linalg.norm(P - C, axis=1))) + 12.0 / math.sqrt(p_min)
    xg, wg = np.polynomial.legendre.leggauss(nr)
    edges = np.linspace(0.0, smax, nseg + 1)
    s = np.concatenate([0.5 * (b - a) * xg + 0.5 * (a + b) for a, b in zip(edges[:-1], edges[1:])])
    ws = np.concatenate([0.5 * (b - a) * wg for a, b in zip(edges[:-1], edges[1:])])
    ct, wt = np.polynomial.legendre.leggauss(nth)
    ph = np.arange(nph) * (2.0 * math.pi / nph)
    st = np.sqrt(1.0 - ct * ct)
    dirs = np.stack([np.outer(st, np.cos(ph)), np.outer(st, np.sin(ph)),
                     np.outer(ct, np.ones(nph))], -1).reshape(-1, 3)
    wdir = np.outer(wt, np.full(nph, 2.0 * math.pi / nph)).reshape(-1)
    total = 0.0
    for k in range(s.size):
        rho = density(pairs, C + s[k] * dirs)
        total += ws[k] * s[k] * float(np.dot(wdir, rho))
    return total


def gh_moments(pairs: PairList, order: int = 2):
    """Charge, dipole and second moments of sum w chi_a chi_b by separable
    Gauss-Hermite quadrature (exact for these polynomial degrees)."""
    y, wy = np.polynomial.hermite.hermgauss(12)
    Q = 0.0
    mu = np.zeros(3)
    M2 = np.zeros((3, 3))
    for q in range(len(pairs)):
        a, b = pairs.alpha[q], pairs.beta[q]
        p = a + b
        A, B = pairs.A[q], pairs.B[q]
        P = (a * A + b * B) / p
        K = math.exp(-a * b / p * float(np.dot(A - B, A - B)))
        # 1-D moments m[d][k] = int x^k (x-A)^i (x-B)^j exp(-p (x-P)^2) dx
        m = np.zeros((3, 3))
        for d in range(3):
            x = P[d] + y / math.sqrt(p)
            f = (x - A[d]) ** pairs.la[q, d] * (x - B[d]) ** pairs.lb[q, d]
            for k in range(3):
                m[d, k] = float(np.dot(wy, f * x ** k)) / math.sqrt(p)
        w = pairs.w[q] * K
        Q += w * m[0, 0] * m[1, 0] * m[2, 0]
        for d in range(3):
            e = [0, 0, 0]
            e[d] = 1
            mu[d] += w * m[0, e[0]] * m[1, e[1]] * m[2, e[2]]
            for d2 in range(3):
                e2 = [0, 0, 0]
                e2[d] += 1
                e2[d2] += 1
                M2[d, d2] += w * m[0, e2[0]] * m[1, e2[1]] * m[2, e2[2]]
    return Q, mu, M2


def rotation_matrix(rng) -> np.ndarray:
    q, r = np.linalg.qr(rng.normal(size=(3, 3)))
    q = q * np.sign(np.diag(r))
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    return q


def rotate_monomial(lmn, Rm):
    """(R^T u)^lmn expanded as {monomial in u: coefficient}."""
    poly = {(0, 0, 0): 1.0}
    for d in range(3):
        for _ in range(int(lmn[d])):
            new = {}
            for mono, c in poly.items():
                for e in range(3):
                    m2 = list(mono)
                    m2[e] += 1
                    new[tuple(m2)] = new.get(tuple(m2), 0.0) + c * Rm[e, d]
            poly = new
    return poly


def rotate_pairs(pairs: PairList, Rm) -> PairList:
    rows = []
    for q in range(len(pairs)):
        pa = rotate_monomial(pairs.la[q], Rm)
        pb = rotate_monomial(pairs.lb[q], Rm)
        for ma, ca in pa.items():
            for mb, cb in pb.items():
                rows.append((Rm @ pairs.A[q], pairs.alpha[q], ma, Rm @ pairs.B[q], pairs.beta[q], mb,
                             pairs.w[q] * ca * cb))
    return PairList(np.array([r[0] for r in rows]), np.array([r[1] for r in rows]),
                    np.array([r[2] for r in rows], np.int32), np.array([r[3] for r in rows]),
                    np.array([r[4] for r in rows]), np.array([r[5] for r in rows], np.int32),
                    np.array([r[6] for r in rows]))


def single(A, a, la, B, b, lb, w=1.0) -> PairList:
    return PairList(np.array([A], float), np.array([a], float), np.array([la], np.int32),
                    np.array([B], float), np.array([b], float), np.array([lb], np.int32),
                    np.array([w], float))


# ----------------------------------------------------------------------------
# Boys function
# ----------------------------------------------------------------------------
T_GRID = np.concatenate([[0.0, 1e-12, 1e-8, 1e-4], np.geomspace(1e-3, 1e3, 61),
                         [29.0, 29.999, 30.0, 30.001, 31.0, 45.0, 60.0]])


def test_boys_at_zero():
    for n in range(9):
        F = oracle.boys(n, 0.0)
        assert F[n] == pytest.approx(1.0 / (2 * n + 1), rel=1e-15)


def test_boys_vs_mpmath():
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 40
    for T in T_GRID:
        F = oracle.boys(8, float(T))
        for n in range(9):
            ref = mpmath.hyp1f1(n + 0.5, n + 1.5, -mpmath.mpf(float(T))) / (2 * n + 1)
            assert abs(F[n] - float(ref)) <= 2e-14 * float(ref), (n, T)


def test_boys_vs_incomplete_gamma():
    for T in T_GRID[T_GRID > 1e-6]:
        F = oracle.boys(6, float(T))
        for n in range(7):
            ref = boys_scipy(n, float(T))
            assert abs(F[n] - ref) <= 1e-12 * ref, (n, T)


def test_boys_rejects_bad_input():
    with pytest.raises(ValueError):
        oracle.boys(2, -1.0)
    with pytest.raises(ValueError):
        oracle.boys(2, float("nan"))


# ----------------------------------------------------------------------------
# closed forms: s-Gaussian charge and the point-cell limit
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_s_gaussian_closed_form(seed):
    rng = np.random.default_rng(seed)
    for _ in range(50):
        alpha = math.exp(rng.uniform(math.log(0.05), math.log(5e3)))
        q = rng.normal()
        A = rng.normal(size=3) * 5
        r = math.exp(rng.uniform(math.log(1e-3), math.log(30.0)))
        d = rng.normal(size=3)
        C = A + r * d / np.linalg.norm(d)
        w = q * (alpha / math.pi) ** 1.5
        v = w * oracle.pair_potential(A, alpha / 2, [0, 0, 0], A, alpha / 2, [0, 0, 0], C)
        ref = q * math.erf(math.sqrt(alpha) * r) / r
        assert v == pytest.approx(ref, rel=1e-13, abs=1e-300)


def test_s_gaussian_at_center():
    for alpha in [0.1, 1.0, 37.0, 5000.0]:
        A = np.array([0.3, -1.0, 2.0])
        v = (alpha / math.pi) ** 1.5 * oracle.pair_potential(A, alpha / 2, [0, 0, 0], A, alpha / 2,
                                                            [0, 0, 0], A)
        assert v == pytest.approx(2.0 * math.sqrt(alpha / math.pi), rel=1e-14)


def test_point_cell_limit():
    """A very tight s-Gaussian of charge q is the paper's point cell: q/|r - r_m|."""
    alpha = 1e9
    for r in [0.5, 2.0, 17.0]:
        C = np.array([r, 0.0, 0.0])
        v = -0.7 * (alpha / math.pi) ** 1.5 * oracle.pair_potential(np.zeros(3), alpha / 2, [0, 0, 0],
                                                                    np.zeros(3), alpha / 2, [0, 0, 0], C)
        assert v == pytest.approx(-0.7 / r, rel=1e-14)


def test_nuclear_sum_and_superposition():
    wl = small_environment(n_nuclei=20, n_charges=30, n_walkers=2, n_elec=4)
    V = oracle.potential(wl.nuclei_xyz, wl.nuclei_Z, wl.pairs, wl.positions)
    for i, C in enumerate(wl.positions):
        ref = sum(Z / np.linalg.norm(C - R) for R, Z in zip(wl.nuclei_xyz, wl.nuclei_Z))
        r = np.linalg.norm(C - wl.meta["s_centers"], axis=1)
        ref += sum(wl.meta["s_q"][k] * math.erf(math.sqrt(wl.meta["s_alpha"][k]) * r[k]) / r[k]
                   for k in range(r.size))
        assert V[i] == pytest.approx(ref, rel=1e-12, abs=1e-12)


# ----------------------------------------------------------------------------
# p/d pairs: brute-force quadrature and McMurchie-Davidson
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("la,lb", [((1, 0, 0), (0, 0, 0)), ((0, 1, 0), (0, 0, 1)),
                                   ((2, 0, 0), (0, 0, 0)), ((1, 1, 0), (0, 1, 0)),
                                   ((0, 1, 1), (1, 0, 1)), ((0, 0, 2), (2, 0, 0))])
def test_pd_pair_vs_quadrature(la, lb):
    rng = np.random.default_rng(hash((la, lb)) % 2 ** 32)
    A = rng.normal(size=3) * 0.8
    B = A + rng.normal(size=3) * 0.6
    a, b = rng.uniform(0.6, 1.6), rng.uniform(0.6, 1.6)
    pl = single(A, a, la, B, b, lb)
    for C in [A + np.array([1.3, -0.4, 0.9]), B + np.array([-0.2, 0.1, 0.35])]:
        v = oracle.pair_potential(A, a, la, B, b, lb, C)
        ref = quadrature_potential(pl, C)
        assert abs(v - ref) <= 1e-8 * max(abs(ref), 1e-3), (v, ref)


def test_pd_pairs_vs_mcmurchie_davidson():
    rng = np.random.default_rng(7)
    comps = [c for l in range(3) for c in CART[l]]
    for _ in range(300):
        la = comps[rng.integers(len(comps))]
        lb = comps[rng.integers(len(comps))]
        A = rng.normal(size=3) * 2
        B = A + rng.normal(size=3) * rng.choice([0.0, 0.5, 2.0])
        a = math.exp(rng.uniform(math.log(0.1), math.log(50.0)))
        b = math.exp(rng.uniform(math.log(0.1), math.log(50.0)))
        C = rng.normal(size=3) * rng.choice([0.5, 3.0, 12.0])
        v = oracle.pair_potential(A, a, la, B, b, lb, C)
        ref = md_pair_potential(A, a, la, B, b, lb, C)
        scale = abs(oracle.pair_potential(A, a, [0, 0, 0], B, b, [0, 0, 0], C)) + abs(ref)
        assert abs(v - ref) <= 1e-11 * scale + 1e-300, (la, lb, a, b, v, ref)


def test_swap_symmetry():
    rng = np.random.default_rng(11)
    comps = [c for l in range(3) for c in CART[l]]
    for _ in range(100):
        la, lb = comps[rng.integers(len(comps))], comps[rng.integers(len(comps))]
        A, B, C = rng.normal(size=(3, 3)) * 2
        a, b = rng.uniform(0.2, 8.0, size=2)
        v1 = oracle.pair_potential(A, a, la, B, b, lb, C)
        v2 = oracle.pair_potential(B, b, lb, A, a, la, C)
        assert v1 == pytest.approx(v2, rel=1e-12, abs=1e-14)


# ----------------------------------------------------------------------------
# field-level laws
# ----------------------------------------------------------------------------
def test_far_field_multipoles():
    wl = tiny_pd_environment(3, n_pairs=5, n_nuclei=0, exp_range=(0.5, 3.0), spread=0.8)
    Q, mu, M2 = gh_moments(wl.pairs)
    rng = np.random.default_rng(3)
    for _ in range(5):
        d = rng.normal(size=3)
        n = d / np.linalg.norm(d)
        R = 400.0
        V = oracle.potential(np.zeros((0, 3)), np.zeros(0), wl.pairs, (R * n)[None])[0]
        quad = 0.5 * (3.0 * n @ M2 @ n - np.trace(M2))
        ref = Q / R + (mu @ n) / R ** 2 + quad / R ** 3
        assert V == pytest.approx(ref, rel=1e-7, abs=1e-12)


def _sphere_grid(nth=24, nph=48):
    ct, wt = np.polynomial.legendre.leggauss(nth)
    ph = (np.arange(nph) + 0.5) * (2 * math.pi / nph)
    st = np.sqrt(1 - ct * ct)
    n = np.stack([np.outer(st, np.cos(ph)), np.outer(st, np.sin(ph)), np.outer(ct, np.ones(nph))], -1)
    w = np.outer(wt, np.full(nph, 2 * math.pi / nph))
    return n.reshape(-1, 3), w.reshape(-1)


def test_gauss_law_flux():
    wl = tiny_pd_environment(5, n_pairs=6, n_nuclei=3, exp_range=(0.8, 3.0), spread=0.7)
    wl.nuclei_xyz[:] = np.clip(wl.nuclei_xyz, -2, 2)
    Q, _, _ = gh_moments(wl.pairs)
    Qtot = Q + wl.nuclei_Z.sum()
    n, w = _sphere_grid()
    Rs, h = 14.0, 1e-3
    flux = 0.0
    pts = []
    for sgn in (+1, -1):
        pts.append((Rs + sgn * h) * n)
    Vp = oracle.potential(wl.nuclei_xyz, wl.nuclei_Z, wl.pairs, pts[0])
    Vm = oracle.potential(wl.nuclei_xyz, wl.nuclei_Z, wl.pairs, pts[1])
    dVdr = (Vp - Vm) / (2 * h)
    flux = -float(np.dot(w, dVdr)) * Rs * Rs
    assert flux == pytest.approx(4 * math.pi * Qtot, rel=1e-7)


def test_mean_value_property_in_charge_free_ball():
    wl = tiny_pd_environment(9, n_pairs=6, n_nuclei=4, exp_range=(1.0, 3.0), spread=0.7)
    X = np.array([9.0, -8.0, 7.5])
    n, w = _sphere_grid()
    V0 = oracle.potential(wl.nuclei_xyz, wl.nuclei_Z, wl.pairs, X[None])[0]
    Vs = oracle.potential(wl.nuclei_xyz, wl.nuclei_Z, wl.pairs, X + 1.2 * n)
    assert float(np.dot(w, Vs)) / (4 * math.pi) == pytest.approx(V0, rel=1e-11)


# ----------------------------------------------------------------------------
# invariances
# ----------------------------------------------------------------------------
def test_rotation_invariance_pd():
    rng = np.random.default_rng(21)
    wl = tiny_pd_environment(21, n_pairs=8, n_nuclei=3, n_pos=6)
    Rm = rotation_matrix(rng)
    V = oracle.potential(wl.nuclei_xyz, wl.nuclei_Z, wl.pairs, wl.positions)
    rp = rotate_pairs(wl.pairs, Rm)
    Vr = oracle.potential(wl.nuclei_xyz @ Rm.T, wl.nuclei_Z, rp, wl.positions @ Rm.T)
    assert np.allclose(Vr, V, rtol=1e-11, atol=1e-12)


def test_translation_invariance_and_linearity():
    wl = tiny_pd_environment(23, n_pairs=8, n_nuclei=3, n_pos=6)
    t = np.array([3.7, -12.1, 0.4])
    V = oracle.potential(wl.nuclei_xyz, wl.nuclei_Z, wl.pairs, wl.positions)
    p2 = wl.pairs.copy()
    p2.A += t
    p2.B += t
    Vt = oracle.potential(wl.nuclei_xyz + t, wl.nuclei_Z, p2, wl.positions + t)
    assert np.allclose(Vt, V, rtol=1e-11, atol=1e-12)
    half = wl.pairs.copy()
    half.w *= 0.5
    Vh = oracle.potential(np.zeros((0, 3)), np.zeros(0), half, wl.positions)
    Ve = oracle.potential(np.zeros((0, 3)), np.zeros(0), wl.pairs, wl.positions)
    assert np.allclose(2 * Vh, Ve, rtol=1e-13, atol=1e-14)


def test_walker_energies_definition():
    V = np.arange(12, dtype=float) * 0.25 - 1.0
    E = oracle.walker_energies(V, 3, 4)
    assert np.array_equal(E, -V.reshape(3, 4).sum(1))


def test_rejects_bad_pairs():
    pl = single([0, 0, 0], -1.0, [0, 0, 0], [0, 0, 0], 1.0, [0, 0, 0])
    with pytest.raises(ValueError):
        oracle.potential(np.zeros((0, 3)), np.zeros(0), pl, np.zeros((1, 3)))


# ----------------------------------------------------------------------------
# oracle.abs_terms: kappa = sum of |terms|, the condition of the sum.  It
# widens the FP32C per-point bound on the synthetic p/d environments, so it is
# pinned here by facts that do not come from its own formula.
# ----------------------------------------------------------------------------
def _no_pairs():
    return PairList.empty()


def test_abs_terms_nuclei_only_closed_form():
    """Point charges alone: kappa = sum_beta |Z_beta| / |C - R_beta| (signs mixed)."""
    rng = np.random.default_rng(41)
    R = rng.uniform(-9, 9, size=(37, 3))
    Z = rng.choice([-3.0, -1.0, 1.0, 6.0, 8.0], size=37)
    C = rng.normal(size=(11, 3))
    K = oracle.abs_terms(R, Z, _no_pairs(), C)
    for i in range(C.shape[0]):
        ref = math.fsum(abs(z) / math.sqrt(float(np.sum((C[i] - r) ** 2))) for r, z in zip(R, Z))
        assert K[i] == pytest.approx(ref, rel=1e-14)


@pytest.mark.parametrize("q", [-1.3, 0.4])
def test_abs_terms_single_s_charge(q):
    """One s-Gaussian charge: kappa = |q erf(sqrt(alpha) r) / r|, for either sign of q."""
    rng = np.random.default_rng(43)
    for alpha in [0.1, 2.0, 75.0]:
        A = rng.normal(size=3)
        for r in [0.01, 0.8, 6.0]:
            d = rng.normal(size=3)
            C = (A + r * d / np.linalg.norm(d))[None, :]
            pl = single(A, alpha / 2, [0, 0, 0], A, alpha / 2, [0, 0, 0], q * (alpha / math.pi) ** 1.5)
            K = oracle.abs_terms(np.zeros((0, 3)), np.zeros(0), pl, C)
            assert K[0] == pytest.approx(abs(q * math.erf(math.sqrt(alpha) * r) / r), rel=1e-13)


def test_abs_terms_single_pd_pair_vs_quadrature():
    """One p/d pair (a term whose sign depends on the position): kappa = |quadrature potential|."""
    pl = single([0.2, -0.1, 0.3], 0.8, [1, 0, 0], [-0.3, 0.2, 0.0], 1.1, [0, 1, 1], w=-1.7)
    for C in ([1.1, 0.4, -0.2], [-0.6, 0.9, 0.5]):
        C = np.array(C)
        ref = quadrature_potential(pl, C)
        K = oracle.abs_terms(np.zeros((0, 3)), np.zeros(0), pl, C[None, :])
        assert K[0] == pytest.approx(abs(ref), rel=1e-8)


def test_abs_terms_split_by_sign():
    """Nuclei and s-charges have a position-independent sign (that of Z or q), so
    kappa = sum over the positive sources - sum over the negative ones, each an
    s-Gaussian closed form or a Coulomb term; and kappa >= |V|, with equality
    when every source has one sign."""
    wl = small_environment(n_nuclei=25, n_charges=60, n_walkers=2, n_elec=5)
    K = oracle.abs_terms(wl.nuclei_xyz, wl.nuclei_Z, wl.pairs, wl.positions)
    V = oracle.potential(wl.nuclei_xyz, wl.nuclei_Z, wl.pairs, wl.positions)
    q, a, S = wl.meta["s_q"], wl.meta["s_alpha"], wl.meta["s_centers"]
    for i, C in enumerate(wl.positions):
        terms = [z / np.linalg.norm(C - R) for R, z in zip(wl.nuclei_xyz, wl.nuclei_Z)]
        r = np.linalg.norm(C - S, axis=1)
        terms += [q[k] * math.erf(math.sqrt(a[k]) * r[k]) / r[k] for k in range(r.size)]
        pos = math.fsum(t for t in terms if t > 0)
        neg = math.fsum(t for t in terms if t < 0)
        assert K[i] == pytest.approx(pos - neg, rel=1e-12)
        assert K[i] >= abs(V[i]) * (1 - 1e-14)
    # one sign only: kappa = V
    Zp = np.abs(wl.nuclei_Z)
    Kp = oracle.abs_terms(wl.nuclei_xyz, Zp, _no_pairs(), wl.positions)
    Vp = oracle.potential(wl.nuclei_xyz, Zp, _no_pairs(), wl.positions)
    assert np.allclose(Kp, Vp, rtol=1e-14, atol=0)


def test_abs_terms_bounds_and_scaling_pd():
    """Random p/d environments: kappa >= |V| (triangle inequality), kappa >= the
    kappa of any subset of the sources, and kappa(c w, c Z) = |c| kappa(w, Z)."""
    wl = tiny_pd_environment(913, n_pairs=40, n_nuclei=6, n_pos=9, exp_range=(0.2, 20.0), spread=2.0,
                             pos_radius=2.5)
    K = oracle.abs_terms(wl.nuclei_xyz, wl.nuclei_Z, wl.pairs, wl.positions)
    V = oracle.potential(wl.nuclei_xyz, wl.nuclei_Z, wl.pairs, wl.positions)
    assert np.all(K >= np.abs(V) * (1 - 1e-14))
    half = wl.pairs.subset(np.arange(len(wl.pairs) // 2))
    Kh = oracle.abs_terms(wl.nuclei_xyz[:3], wl.nuclei_Z[:3], half, wl.positions)
    assert np.all(K >= Kh * (1 - 1e-14))
    # the sum of the single-pair values is kappa of the pairs
    Kpairs = oracle.abs_terms(np.zeros((0, 3)), np.zeros(0), wl.pairs, wl.positions)
    for i in range(3):
        C = wl.positions[i]
        ref = math.fsum(abs(wl.pairs.w[q] * oracle.pair_potential(wl.pairs.A[q], wl.pairs.alpha[q], wl.pairs.la[q],
                                                                  wl.pairs.B[q], wl.pairs.beta[q], wl.pairs.lb[q], C))
                        for q in range(len(wl.pairs)))
        assert Kpairs[i] == pytest.approx(ref, rel=1e-13)
    for c in (-2.5, 0.5):
        scaled = wl.pairs.copy()
        scaled.w = scaled.w * c
        Ks = oracle.abs_terms(wl.nuclei_xyz, wl.nuclei_Z * c, scaled, wl.positions)
        assert np.allclose(Ks, abs(c) * K, rtol=1e-13, atol=0)


def test_walker_energies_compensated_vs_exact_sum():
    """E_w = -sum_e V: against math.fsum (the correctly rounded sum, Shewchuk's
    algorithm), on sums whose plain left-to-right evaluation loses every digit."""
    V = np.array([1e16, 1.0, -1e16, 3.0, 2.0 ** -30, -2.0 ** -30, 0.5, 1e-3])
    E = oracle.walker_energies(V, 2, 4)
    assert E[0] == -math.fsum(V[:4]) == -4.0
    assert E[1] == pytest.approx(-math.fsum(V[4:]), rel=1e-16)
    rng = np.random.default_rng(47)
    W = rng.normal(size=(50, 64)) * 10.0 ** rng.integers(-3, 4, size=(50, 64))
    E = oracle.walker_energies(W.reshape(-1), 50, 64)
    for w in range(50):
        assert E[w] == pytest.approx(-math.fsum(W[w]), rel=1e-15, abs=1e-300)
