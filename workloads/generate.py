"""Seeded generators for the environment workloads.

Every array is float64 (int32 for Cartesian exponents).  A Gaussian
primitive is unnormalised and Cartesian,
    chi(r) = (x-Ax)^i (y-Ay)^j (z-Az)^k exp(-alpha |r-A|^2),
and a *pair* is one product chi_a chi_b with a density weight w.  The weight
carries everything the caller folds in: contraction and normalisation
constants, the density-matrix element, the factor 2 for a != b, and the sign
of the charge (-1 for electrons).  The environment potential is then
    V(C) = sum_beta Z_beta / |C - R_beta| + sum_ab w_ab * int chi_a chi_b / |r - C| dr,
the potential of the paper's Eq. ElectrostaticField with the sign flipped
(U_ES = -V for an electron), generalised from point cells to Gaussian
pairs.  Nothing here evaluates that potential.

The density normalisation and the input-side screening of config "realistic"
need overlaps and absolute charges of Gaussian products; those are written
out below from the Gaussian product theorem and 1-D Gaussian moments, which
is workload construction, not the potential method.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Dict, List, Optional

import numpy as np

QM_RADIUS = 6.0          # bohr, radius of the QM sphere about the origin
POSITION_SD = 2.0        # bohr, sd of the Gaussian walker-electron law
BASE_SEED = 1011


def seed_for_config(i: int) -> int:
    """Seed of configuration i (1-based): 1011*100 + i."""
    return BASE_SEED * 100 + int(i)


# Cartesian components of a shell, in a fixed order.
CART = {
    0: [(0, 0, 0)],
    1: [(1, 0, 0), (0, 1, 0), (0, 0, 1)],
    2: [(2, 0, 0), (0, 2, 0), (0, 0, 2), (1, 1, 0), (1, 0, 1), (0, 1, 1)],
}


@dataclasses.dataclass
class PairList:
    """Structure-of-arrays list of weighted Gaussian primitive pairs."""
    A: np.ndarray       # [n,3] f64
    alpha: np.ndarray   # [n]   f64
    la: np.ndarray      # [n,3] int32
    B: np.ndarray       # [n,3] f64
    beta: np.ndarray    # [n]   f64
    lb: np.ndarray      # [n,3] int32
    w: np.ndarray       # [n]   f64

    def __len__(self) -> int:
        return int(self.alpha.shape[0])

    @staticmethod
    def empty() -> "PairList":
        z3 = np.zeros((0, 3))
        zi = np.zeros((0, 3), np.int32)
        z = np.zeros(0)
        return PairList(z3, z, zi, z3.copy(), z.copy(), zi.copy(), z.copy())

    def subset(self, idx) -> "PairList":
        return PairList(self.A[idx], self.alpha[idx], self.la[idx], self.B[idx],
                        self.beta[idx], self.lb[idx], self.w[idx])

    @staticmethod
    def concat(lists: List["PairList"]) -> "PairList":
        if not lists:
            return PairList.empty()
        return PairList(*[np.concatenate([getattr(p, f.name) for p in lists])
                          for f in dataclasses.fields(PairList)])

    def copy(self) -> "PairList":
        return PairList(*[getattr(self, f.name).copy() for f in dataclasses.fields(PairList)])

    def validate(self) -> None:
        n = len(self)
        for f in dataclasses.fields(PairList):
            a = getattr(self, f.name)
            assert a.shape[0] == n, f.name
        assert self.la.dtype == np.int32 and self.lb.dtype == np.int32


@dataclasses.dataclass
class Workload:
    name: str
    nuclei_xyz: np.ndarray     # [K,3]
    nuclei_Z: np.ndarray       # [K]
    pairs: PairList
    positions: np.ndarray      # [N,3], walker-major
    n_walkers: int
    n_elec: int
    qm_center: np.ndarray      # [3]
    meta: Dict

    @property
    def n_positions(self) -> int:
        return int(self.positions.shape[0])


# ----------------------------------------------------------------------------
# positions
# ----------------------------------------------------------------------------
def qm_positions(rng: np.random.Generator, n: int, sd: float = POSITION_SD,
                 radius: float = QM_RADIUS, center=(0.0, 0.0, 0.0)) -> np.ndarray:
    """n positions ~ N(center, sd^2 I) rejection-sampled to |r - center| < radius."""
    out = np.empty((0, 3))
    while out.shape[0] < n:
        m = int((n - out.shape[0]) * 1.1) + 16
        x = rng.normal(0.0, sd, size=(m, 3))
        x = x[np.einsum("ij,ij->i", x, x) < radius * radius]
        out = np.concatenate([out, x])
    return out[:n] + np.asarray(center, dtype=np.float64)


def _uniform_outside_sphere(rng, n, half_box, radius):
    out = np.empty((0, 3))
    while out.shape[0] < n:
        m = 2 * (n - out.shape[0]) + 16
        x = rng.uniform(-half_box, half_box, size=(m, 3))
        x = x[np.einsum("ij,ij->i", x, x) >= radius * radius]
        out = np.concatenate([out, x])
    return out[:n]


# ----------------------------------------------------------------------------
# config "small": point nuclei + s-type Gaussian charges
# ----------------------------------------------------------------------------
def s_charge_pairs(centers: np.ndarray, alpha: np.ndarray, q: np.ndarray) -> PairList:
    """A normalised s-Gaussian charge q (alpha/pi)^{3/2} exp(-alpha r^2) as one pair.

    The pair is (A, alpha/2, s) x (A, alpha/2, s) with weight q (alpha/pi)^{3/2}:
    the product of the two primitives is exp(-alpha |r-A|^2)."""
    n = centers.shape[0]
    z = np.zeros((n, 3), np.int32)
    return PairList(centers.copy(), alpha / 2.0, z, centers.copy(), alpha / 2.0, z.copy(),
                    q * (alpha / math.pi) ** 1.5)


def small_environment(seed: int = seed_for_config(1), n_nuclei: int = 200,
                      n_charges: int = 2000, n_walkers: int = 100, n_elec: int = 100,
                      half_box: float = 10.0) -> Workload:
    """200 nuclei (Z in {1,6,7,8}) and 2,000 s-Gaussian charges, uniform in a 20 bohr
    cube outside the 6 bohr QM sphere; exponents log-uniform in [0.1, 50] bohr^-2;
    charges ~ N(-1, 0.3); positions = walkers x electrons inside the QM sphere."""
    rng = np.random.default_rng(seed)
    R = _uniform_outside_sphere(rng, n_nuclei, half_box, QM_RADIUS)
    Z = rng.choice(np.array([1.0, 6.0, 7.0, 8.0]), size=n_nuclei)
    Cg = _uniform_outside_sphere(rng, n_charges, half_box, QM_RADIUS)
    alpha = np.exp(rng.uniform(math.log(0.1), math.log(50.0), size=n_charges))
    q = rng.normal(-1.0, 0.3, size=n_charges)
    pairs = s_charge_pairs(Cg, alpha, q)
    pos = qm_positions(rng, n_walkers * n_elec)
    return Workload("small: 200 nuclei + 2000 s-Gaussian charges", R, Z, pairs, pos,
                    n_walkers, n_elec, np.zeros(3),
                    dict(seed=seed, n_charges=n_charges, s_alpha=alpha, s_q=q, s_centers=Cg))


def point_cells_environment(seed: int, n_cells: int = 268782, n_nuclei: int = 36,
                            n_positions: int = 1) -> Workload:
    """The paper's literal workload shape: M point cells rho(r_m) plus K nuclei,
    evaluated at a handful of positions.  Cells are point charges of value -rho."""
    rng = np.random.default_rng(seed)
    R = _uniform_outside_sphere(rng, n_nuclei, 10.0, QM_RADIUS)
    Z = rng.choice(np.array([1.0, 6.0, 7.0, 8.0]), size=n_nuclei)
    cells = _uniform_outside_sphere(rng, n_cells, 10.0, QM_RADIUS)
    rho = np.abs(rng.normal(0.0, 1.0, size=n_cells))
    rho *= Z.sum() / rho.sum()
    xyz = np.concatenate([R, cells])
    q = np.concatenate([Z, -rho])
    pos = qm_positions(rng, n_positions)
    return Workload("point cells", xyz, q, PairList.empty(), pos, 1, n_positions,
                    np.zeros(3), dict(seed=seed, n_cells=n_cells))


# ----------------------------------------------------------------------------
# tiny p/d environment for unit tests
# ----------------------------------------------------------------------------
def tiny_pd_environment(seed: int, n_pairs: int = 6, n_nuclei: int = 3, n_pos: int = 5,
                        lmax: int = 2, spread: float = 1.5, exp_range=(0.3, 3.0),
                        pos_radius: float = 3.0, same_center_frac: float = 0.3) -> Workload:
    """A few random Cartesian pairs with angular momentum up to lmax per primitive."""
    rng = np.random.default_rng(seed)
    comps = [c for l in range(lmax + 1) for c in CART[l]]
    A = rng.normal(0.0, spread, size=(n_pairs, 3))
    B = A + rng.normal(0.0, spread * 0.7, size=(n_pairs, 3))
    same = rng.uniform(size=n_pairs) < same_center_frac
    B[same] = A[same]
    lo, hi = exp_range
    alpha = np.exp(rng.uniform(math.log(lo), math.log(hi), size=n_pairs))
    beta = np.exp(rng.uniform(math.log(lo), math.log(hi), size=n_pairs))
    la = np.array([comps[k] for k in rng.integers(0, len(comps), size=n_pairs)], np.int32)
    lb = np.array([comps[k] for k in rng.integers(0, len(comps), size=n_pairs)], np.int32)
    w = rng.normal(0.0, 1.0, size=n_pairs)
    pairs = PairList(A, alpha, la.reshape(-1, 3), B, beta, lb.reshape(-1, 3), w)
    R = rng.normal(0.0, 4.0, size=(n_nuclei, 3))
    Z = rng.choice(np.array([1.0, 6.0, 7.0, 8.0]), size=n_nuclei)
    pos = rng.uniform(-pos_radius, pos_radius, size=(n_pos, 3))
    return Workload("tiny p/d", R, Z, pairs, pos, 1, n_pos, np.zeros(3), dict(seed=seed))


# ----------------------------------------------------------------------------
# Gaussian-product helpers used only to normalise and screen generated inputs
# ----------------------------------------------------------------------------
def _moments(p: np.ndarray, absolute: bool) -> List[np.ndarray]:
    """[int u^k exp(-p u^2) du for k = 0..4] (|u|^k if absolute)."""
    sq = np.sqrt(math.pi / p)
    ip = 1.0 / p
    m = [sq, ip * 0.5, sq * 0.5 * ip, ip * ip * 0.5, sq * 0.75 * ip * ip]
    if not absolute:
        z = np.zeros_like(p)
        m[1] = z
        m[3] = z
    # int |u| e^{-p u^2} du = 1/p ; int |u|^3 e^{-p u^2} du = 1/p^2
    else:
        m[1] = ip
        m[3] = ip * ip
    return m


_COMB = np.array([[math.comb(n, k) for k in range(5)] for n in range(5)], np.float64)


def _poly_moment_1d(i, j, PA, PB, mom):
    """int (u+PA)^i (u+PB)^j exp(-p u^2) du for integer arrays i, j <= 2, where
    mom[k] is the k-th (possibly absolute) Gaussian moment."""
    # coefficients of u^0, u^1, u^2 in (u+PA)^i and (u+PB)^j
    ca = [np.where(i == 0, 1.0, np.where(i == 1, PA, PA * PA)),
          np.where(i == 0, 0.0, np.where(i == 1, 1.0, 2.0 * PA)),
          np.where(i == 2, 1.0, 0.0)]
    cb = [np.where(j == 0, 1.0, np.where(j == 1, PB, PB * PB)),
          np.where(j == 0, 0.0, np.where(j == 1, 1.0, 2.0 * PB)),
          np.where(j == 2, 1.0, 0.0)]
    out = np.zeros_like(PA)
    for k1 in range(3):
        for k2 in range(3):
            out += ca[k1] * cb[k2] * mom[k1 + k2]
    return out


def product_overlap(A, alpha, la, B, beta, lb, absolute=False, pad=0.0):
    """int chi_a chi_b dr (or int |chi_a chi_b| dr) for arrays of primitive pairs.

    With absolute=True and pad=1, |PA| and |PB| are replaced by 1+|PA| and
    1+|PB|, which bounds every component pair of shells with these l values."""
    p = alpha + beta
    P = (alpha[:, None] * A + beta[:, None] * B) / p[:, None]
    AB2 = np.einsum("ij,ij->i", A - B, A - B)
    out = np.exp(-alpha * beta / p * AB2)
    mom = _moments(p, absolute)
    for d in range(3):
        PA = P[:, d] - A[:, d]
        PB = P[:, d] - B[:, d]
        if absolute:
            PA = np.abs(PA) + pad
            PB = np.abs(PB) + pad
        out = out * _poly_moment_1d(la[:, d], lb[:, d], PA, PB, mom)
    return out


def primitive_norm(alpha, lmn):
    """Normalisation constant of an unnormalised Cartesian primitive."""
    lmn = np.asarray(lmn)
    dfact = np.array([1.0, 1.0, 3.0, 15.0, 105.0])
    l = lmn.sum(axis=-1)
    den = dfact[lmn[..., 0]] * dfact[lmn[..., 1]] * dfact[lmn[..., 2]]
    return np.sqrt((2.0 * alpha / math.pi) ** 1.5 * (4.0 * alpha) ** l / den)


# ----------------------------------------------------------------------------
# config "realistic": cc-pVDZ-shaped primitives and a local PSD density
# ----------------------------------------------------------------------------
def _atom_shells(rng, Z):
    """Primitive shells (l, exponent) of one atom; cc-pVDZ *shape* only."""
    jit = lambda n: np.exp(rng.normal(0.0, 0.08, size=n))
    if Z == 1:
        s = np.geomspace(0.1, 50.0, 4) * jit(4)
        p = np.array([1.0]) * jit(1)
        d = np.zeros(0)
    else:
        s = np.geomspace(0.1, 5000.0, 9) * jit(9)
        p = np.geomspace(0.1, 30.0, 4) * jit(4)
        d = np.array([math.sqrt(0.3 * 1.5)]) * jit(1)
    return [(0, e) for e in s] + [(1, e) for e in p] + [(2, e) for e in d]


def realistic_environment(seed: int = seed_for_config(2), n_atoms: int = 2000,
                          n_walkers: int = 4096, n_elec: int = 32, spacing: float = 2.8,
                          n_side: Optional[int] = None, jitter: float = 0.15,
                          support_radius: float = 3.4, neighbour_amp: float = 0.35,
                          screen_tol: float = 1e-12, with_positions: bool = True) -> Workload:
    """Atoms on a jittered lattice outside the QM sphere, each with a cc-pVDZ-shaped
    primitive set (H: 4s 1p; C/N/O: 9s 4p 1d, Cartesian d), and a density
    D = B B^T with B local: each column belongs to one atom and is supported on
    the primitives of that atom and of its neighbours within `support_radius`.
    D is scaled so sum_ab D_ab S_ab equals sum Z (neutral environment).  Pairs
    whose absolute charge |w| int|chi_a chi_b| is below `screen_tol` are dropped.
    """
    from scipy.spatial import cKDTree
    import scipy.sparse as sp

    rng = np.random.default_rng(seed)
    if n_side is None:
        n_side = int(math.ceil((n_atoms * 1.15) ** (1.0 / 3.0))) + 1
        while True:
            g = (np.arange(n_side) - (n_side - 1) / 2.0) * spacing
            sites = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
            sites = sites[np.einsum("ij,ij->i", sites, sites) >= QM_RADIUS ** 2]
            if sites.shape[0] >= n_atoms:
                break
            n_side += 1
    else:
        g = (np.arange(n_side) - (n_side - 1) / 2.0) * spacing
        sites = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
        sites = sites[np.einsum("ij,ij->i", sites, sites) >= QM_RADIUS ** 2]
    pick = np.sort(rng.choice(sites.shape[0], size=n_atoms, replace=False))
    R = sites[pick] + rng.normal(0.0, jitter, size=(n_atoms, 3))
    Z = rng.choice(np.array([1, 6, 7, 8]), size=n_atoms)

    # shells and basis functions
    sh_atom, sh_l, sh_exp = [], [], []
    for a in range(n_atoms):
        for (l, e) in _atom_shells(rng, Z[a]):
            sh_atom.append(a)
            sh_l.append(l)
            sh_exp.append(e)
    sh_atom = np.array(sh_atom)
    sh_l = np.array(sh_l)
    sh_exp = np.array(sh_exp)
    sh_nbf = np.array([len(CART[l]) for l in sh_l])
    sh_bf0 = np.concatenate([[0], np.cumsum(sh_nbf)[:-1]])
    n_bf = int(sh_nbf.sum())
    bf_shell = np.repeat(np.arange(sh_l.size), sh_nbf)
    bf_lmn = np.concatenate([np.array(CART[l], np.int32) for l in sh_l])
    bf_atom = sh_atom[bf_shell]
    bf_norm = primitive_norm(sh_exp[bf_shell], bf_lmn)
    atom_bf0 = np.searchsorted(bf_atom, np.arange(n_atoms))
    atom_nbf = np.bincount(bf_atom, minlength=n_atoms)
    atom_sh0 = np.searchsorted(sh_atom, np.arange(n_atoms))
    atom_nsh = np.bincount(sh_atom, minlength=n_atoms)

    # B: columns per atom (ceil(Z/2) of them), local support
    tree = cKDTree(R)
    neigh = tree.query_ball_point(R, r=support_radius)
    rows, cols, vals = [], [], []
    col = 0
    for k in range(n_atoms):
        ncol = (int(Z[k]) + 1) // 2
        for _ in range(ncol):
            for m in neigh[k]:
                r0, nb = atom_bf0[m], atom_nbf[m]
                amp = 1.0 if m == k else neighbour_amp
                rr = np.arange(r0, r0 + nb)
                rows.append(rr)
                cols.append(np.full(nb, col))
                vals.append(bf_norm[rr] * amp * rng.normal(0.0, 1.0, size=nb))
            col += 1
    Bm = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                       shape=(n_bf, col))
    Daa = np.asarray(Bm.multiply(Bm).sum(axis=1)).ravel()

    # candidate atom pairs: D is nonzero only within 2*support_radius
    ap = np.array(sorted(tree.query_pairs(r=2.0 * support_radius + 1e-9)), dtype=np.int64).reshape(-1, 2)
    ap = np.concatenate([np.stack([np.arange(n_atoms), np.arange(n_atoms)], 1), ap])

    est_scale = float(Z.sum()) / float(np.sum(Daa / bf_norm ** 2))
    sh_dmax = np.sqrt(np.maximum.reduceat(Daa, sh_bf0))
    safety = 2.0 * est_scale * 10.0

    def _expand(cnt):
        tot = int(cnt.sum())
        pid = np.repeat(np.arange(cnt.size), cnt)
        local = np.arange(tot) - np.repeat(np.cumsum(cnt) - cnt, cnt)
        return pid, local

    def _chunk(c0):
        """Surviving component pairs of atom pairs [c0, c0 + ap_chunk)."""
        X, Y = ap[c0:c0 + ap_chunk, 0], ap[c0:c0 + ap_chunk, 1]
        nX, nY = atom_nsh[X], atom_nsh[Y]
        pid, local = _expand(nX * nY)
        sa = atom_sh0[X][pid] + local // nY[pid]
        sb = atom_sh0[Y][pid] + local % nY[pid]
        keep = ~((X[pid] == Y[pid]) & (sa > sb))
        sa, sb = sa[keep], sb[keep]
        # exp(-mu R^2) < 1e-26 cannot survive any bound below
        dAB = R[sh_atom[sa]] - R[sh_atom[sb]]
        mu = sh_exp[sa] * sh_exp[sb] / (sh_exp[sa] + sh_exp[sb])
        keep = mu * np.einsum("ij,ij->i", dAB, dAB) < 60.0
        sa, sb = sa[keep], sb[keep]
        if sa.size == 0:
            return None
        # shell-level screen: |D_ab| <= sqrt(D_aa D_bb) times a padded absolute-moment
        # bound that dominates every component pair of the two shells
        lA = np.repeat(sh_l[sa][:, None], 3, 1).astype(np.int32)
        lB = np.repeat(sh_l[sb][:, None], 3, 1).astype(np.int32)
        qb = product_overlap(R[sh_atom[sa]], sh_exp[sa], lA, R[sh_atom[sb]], sh_exp[sb], lB,
                             absolute=True, pad=1.0)
        keep = qb * sh_dmax[sa] * sh_dmax[sb] * safety >= screen_tol
        sa, sb = sa[keep], sb[keep]
        if sa.size == 0:
            return None
        # component pairs of each surviving shell pair
        na, nb_ = sh_nbf[sa], sh_nbf[sb]
        spid, local = _expand(na * nb_)
        a_bf = sh_bf0[sa][spid] + local // nb_[spid]
        b_bf = sh_bf0[sb][spid] + local % nb_[spid]
        keep = ~((sa[spid] == sb[spid]) & (a_bf > b_bf))
        a_bf, b_bf = a_bf[keep], b_bf[keep]
        ea, eb = sh_exp[bf_shell[a_bf]], sh_exp[bf_shell[b_bf]]
        qabs = product_overlap(R[bf_atom[a_bf]], ea, bf_lmn[a_bf], R[bf_atom[b_bf]], eb, bf_lmn[b_bf],
                               absolute=True)
        keep = np.sqrt(Daa[a_bf] * Daa[b_bf]) * qabs * safety >= screen_tol
        a_bf, b_bf = a_bf[keep], b_bf[keep]
        if a_bf.size == 0:
            return None
        D = np.asarray(Bm[a_bf].multiply(Bm[b_bf]).sum(axis=1)).ravel()
        ea, eb = sh_exp[bf_shell[a_bf]], sh_exp[bf_shell[b_bf]]
        S = product_overlap(R[bf_atom[a_bf]], ea, bf_lmn[a_bf], R[bf_atom[b_bf]], eb, bf_lmn[b_bf])
        return a_bf, b_bf, D, S, qabs[keep]

    # Streamed in chunks of atom pairs (large numpy temporaries are slow); the
    # chunks run on threads (numpy and scipy.sparse release the GIL in their
    # array loops) and are joined in chunk order, so the result does not depend
    # on the thread count.
    import concurrent.futures as cf
    import os
    ap_chunk = 1500
    starts = range(0, ap.shape[0], ap_chunk)
    n_thr = max(1, min(16, os.cpu_count() or 1, len(starts)))
    if n_thr > 1:
        with cf.ThreadPoolExecutor(max_workers=n_thr) as ex:
            parts = [r for r in ex.map(_chunk, starts) if r is not None]
    else:
        parts = [r for r in map(_chunk, starts) if r is not None]
    a_keep, b_keep, d_keep, s_keep, q_keep = (list(x) for x in zip(*parts))
    a = np.concatenate(a_keep)
    b = np.concatenate(b_keep)
    Dab = np.concatenate(d_keep)
    Sab = np.concatenate(s_keep)
    qabs = np.concatenate(q_keep)
    mult = np.where(a == b, 1.0, 2.0)
    n_e = float(Z.sum())
    scale = n_e / float(np.sum(mult * Dab * Sab))
    w = -mult * Dab * scale
    sel = np.nonzero(qabs * np.abs(w) >= screen_tol)[0]
    a, b, w, Sab = a[sel], b[sel], w[sel], Sab[sel]
    pairs = PairList(R[bf_atom[a]], sh_exp[bf_shell[a]], bf_lmn[a].astype(np.int32),
                     R[bf_atom[b]], sh_exp[bf_shell[b]], bf_lmn[b].astype(np.int32), w)
    spk = bf_shell[a].astype(np.int64) * sh_l.size + bf_shell[b]
    n_dist = int(np.count_nonzero(np.diff(spk)) + 1) if spk.size else 0  # shell pairs are contiguous
    lsum = bf_lmn[a].sum(1) + bf_lmn[b].sum(1)
    pos = qm_positions(rng, n_walkers * n_elec) if with_positions else np.zeros((0, 3))
    meta = dict(seed=seed, n_atoms=n_atoms, n_bf=n_bf, n_columns=col, support_radius=support_radius,
                n_shell_pairs=n_dist, n_component_pairs=len(pairs), n_electrons=n_e,
                electron_charge=float(np.sum(w * Sab)),
                component_L_hist=np.bincount(lsum, minlength=5).tolist())
    return Workload("realistic: %d atoms, cc-pVDZ-shaped primitives, local PSD density" % n_atoms,
                    R, Z.astype(np.float64), pairs, pos, n_walkers, n_elec, np.zeros(3), meta)


def batched_specs(seed: int = seed_for_config(3), n_sys: int = 64,
                  pair_range=(1e4, 1e6), pos_range=(1e3, 2e5), n_elec: int = 32,
                  distributions_per_atom: Optional[float] = None,
                  max_atoms: Optional[int] = None) -> List[dict]:
    """Per-system generator arguments of batched_environments (no environment
    is built): distribution-count targets log-uniform in pair_range, position
    counts log-uniform in pos_range rounded to whole walkers of n_elec
    electrons, atom counts from the measured distributions-per-atom ratio of
    the realistic generator."""
    rng = np.random.default_rng(seed)
    tgt = np.exp(rng.uniform(math.log(pair_range[0]), math.log(pair_range[1]), size=n_sys))
    npos = np.exp(rng.uniform(math.log(pos_range[0]), math.log(pos_range[1]), size=n_sys))
    nw = np.maximum(1, np.round(npos / n_elec)).astype(int)
    if distributions_per_atom is None:
        probe = realistic_environment(seed=seed + 7, n_atoms=200, with_positions=False)
        distributions_per_atom = probe.meta["n_shell_pairs"] / 200.0
    specs = []
    for s in range(n_sys):
        na = max(8, int(round(tgt[s] / distributions_per_atom)))
        if max_atoms is not None:
            na = min(na, max_atoms)
        specs.append({"seed": seed * 1000 + s, "n_atoms": na, "n_walkers": int(nw[s]), "n_elec": n_elec,
                      "target_distributions": float(tgt[s])})
    return specs


def batched_system(spec: dict) -> Workload:
    """One system of batched_specs (a realistic environment with its walkers)."""
    wl = realistic_environment(seed=spec["seed"], n_atoms=spec["n_atoms"], n_walkers=spec["n_walkers"],
                               n_elec=spec["n_elec"])
    wl.meta["target_distributions"] = spec["target_distributions"]
    return wl


def batched_environments(seed: int = seed_for_config(3), n_sys: int = 64,
                         pair_range=(1e4, 1e6), pos_range=(1e3, 2e5), n_elec: int = 32,
                         distributions_per_atom: Optional[float] = None,
                         max_atoms: Optional[int] = None) -> List[Workload]:
    """n_sys independent environments of uneven size (see batched_specs); each
    system is a realistic environment."""
    return [batched_system(sp) for sp in batched_specs(seed, n_sys, pair_range, pos_range, n_elec,
                                                        distributions_per_atom, max_atoms)]
