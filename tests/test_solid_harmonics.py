"""The real regular solid harmonics of the surrogate's far-field expansion
(esp_harmonics.h, run on the host through esp_debug_solid_harmonics), pinned
by facts of the mathematics: closed forms of the first degrees, homogeneity,
orthonormality over the unit sphere (Gauss-Legendre x trapezoid quadrature),
harmonicity (finite-difference Laplacian) and the addition theorem of
1/|r - r'|, which is what makes the expansion exact for far charges."""
import math

import numpy as np
import pytest

from paper_1011_4687_gb300 import build_lib, esp


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build_lib.build()
    esp.load()


def S(L, u):
    return esp.debug_solid_harmonics(L, u)


def test_low_degrees_closed_form():
    rng = np.random.default_rng(1)
    for _ in range(20):
        x, y, z = rng.normal(size=3)
        r2 = x * x + y * y + z * z
        s = S(2, [x, y, z])
        ref = [1.0,
               math.sqrt(3) * z, math.sqrt(3) * x, math.sqrt(3) * y,
               math.sqrt(5) * 0.5 * (3 * z * z - r2),
               math.sqrt(15) * x * z, math.sqrt(15) * y * z,
               math.sqrt(15) * 0.5 * (x * x - y * y), math.sqrt(15) * x * y]
        assert np.allclose(s, ref, rtol=1e-13, atol=1e-13)


def test_homogeneity():
    rng = np.random.default_rng(2)
    L = 30
    deg = np.concatenate([[l] * (2 * l + 1) for l in range(L + 1)])
    for _ in range(10):
        u = rng.normal(size=3)
        lam = rng.uniform(0.3, 1.7)
        assert np.allclose(S(L, lam * u), lam ** deg * S(L, u), rtol=1e-11, atol=1e-300)


def _sphere_grid(nt, nf):
    ct, wt = np.polynomial.legendre.leggauss(nt)
    ph = np.arange(nf) * (2 * math.pi / nf)
    st = np.sqrt(1 - ct * ct)
    d = np.stack([np.outer(st, np.cos(ph)), np.outer(st, np.sin(ph)), np.outer(ct, np.ones(nf))], -1).reshape(-1, 3)
    w = np.outer(wt, np.full(nf, 2 * math.pi / nf)).reshape(-1)
    return d, w


def test_orthonormal_over_the_sphere():
    L = 16
    d, w = _sphere_grid(L + 2, 2 * L + 3)
    Y = np.array([S(L, p) for p in d])          # [points, (L+1)^2]
    G = (Y * w[:, None]).T @ Y / (4 * math.pi)
    assert np.abs(G - np.eye(G.shape[0])).max() <= 1e-12


def test_harmonic():
    rng = np.random.default_rng(3)
    L, h = 12, 3e-4
    for _ in range(5):
        u = rng.normal(size=3) * 0.5
        lap = -6 * S(L, u)
        for k in range(3):
            e = np.zeros(3)
            e[k] = h
            lap += S(L, u + e) + S(L, u - e)
        lap /= h * h
        assert np.abs(lap).max() <= 1e-4 * max(1.0, np.abs(S(L, u)).max())  # O(h^2) stencil error


def test_addition_theorem():
    """1/|u - P| = sum_l sum_m S_lm(u) S_lm(P) / ((2l + 1) |P|^(2l+1)) for |u| < |P|."""
    rng = np.random.default_rng(4)
    L = 40
    deg = np.concatenate([[l] * (2 * l + 1) for l in range(L + 1)])
    for _ in range(20):
        P = rng.normal(size=3)
        P *= rng.uniform(2.0, 5.0) / np.linalg.norm(P)
        u = rng.normal(size=3)
        u *= rng.uniform(0.0, 1.0) / np.linalg.norm(u)
        rp = np.linalg.norm(P)
        series = np.sum(S(L, u) * S(L, P) / ((2 * deg + 1) * rp ** (2 * deg + 1)))
        assert series == pytest.approx(1.0 / np.linalg.norm(u - P), rel=1e-11)


def test_rejects_bad_degree():
    with pytest.raises(esp.EspError):
        S(41, [0.1, 0.2, 0.3])
