"""Seeded synthetic UCCSD problems (inputs only; no arithmetic of the method).

The paper's workloads are molecules whose orbitals, integrals and MP2 start
amplitudes come from PySCF (Methods section). None of that data is available
here, so this module draws problems with the same *shape*: a real symmetric
one-electron matrix h, an 8-fold-symmetric two-electron tensor g in chemist
notation (pq|rs), the spin-conserving singles and doubles of Eq. 2 enumerated
over spin-orbitals, and one angle theta per factor of Eq. 3.

Conventions shared by every consumer of these inputs:

* spin-orbital index p = 2*spatial + spin (spin 0 = alpha, 1 = beta), so the
  Jordan-Wigner qubit of spin-orbital p is bit p of the determinant key (one
  64-bit word up to 64 spin-orbitals, two words up to 128);
* the reference determinant occupies spatial orbitals 0..n_alpha-1 (alpha) and
  0..n_beta-1 (beta);
* an excitation row (i, j, a, b) stands for tau = a+_a a+_b a_j a_i (a single
  is (i, -1, a, -1), tau = a+_a a_i); row 0 of the list is applied first, i.e.
  it is the rightmost factor U_1 of Eq. 3;
* doubles are ordered by |theta| descending (the Methods section orders them by
  the magnitude of their initial amplitude, largest applied first) and the
  singles follow, applied last; an optional M_D keeps only the M_D doubles of
  largest |theta| (Methods section's ansatz truncation).

This module is imported by the tests, the oracle's callers and the benchmark;
it holds no part of the apply, energy or gradient arithmetic.
"""
from __future__ import annotations

import dataclasses
import itertools
import math
from typing import Optional

import numpy as np

__all__ = [
    "Problem",
    "make_integrals",
    "enumerate_excitations",
    "order_and_truncate",
    "make_problem",
    "config_problem",
    "batch_job_problem",
    "hilbert_size",
    "CONFIGS",
]


@dataclasses.dataclass
class Problem:
    """One synthetic UCCSD problem.

    h      : (n_spatial, n_spatial) float64, symmetric.
    g      : (n_spatial,)*4 float64, chemist (pq|rs), 8-fold symmetric.
    exc    : (K, 4) int32 spin-orbital rows (i, j, a, b) in application order.
    theta  : (K,) float64 angles, same order as exc.
    """

    n_spatial: int
    n_alpha: int
    n_beta: int
    h: np.ndarray
    g: np.ndarray
    exc: np.ndarray
    theta: np.ndarray
    eps: float = 0.0
    e_nuc: float = 0.0
    name: str = ""
    n_max: int = 0   # Methods-section cut: above n_max determinants keep n_cut (0 = off)
    n_cut: int = 0

    @property
    def n_so(self) -> int:
        return 2 * self.n_spatial

    @property
    def n_elec(self) -> int:
        return self.n_alpha + self.n_beta

    @property
    def n_exc(self) -> int:
        return int(self.exc.shape[0])

    @property
    def hf_key(self) -> int:
        key = 0
        for s in range(self.n_alpha):
            key |= 1 << (2 * s)
        for s in range(self.n_beta):
            key |= 1 << (2 * s + 1)
        return key

    def prefix(self, n_factors: int) -> "Problem":
        """The same problem restricted to the first n_factors factors."""
        return dataclasses.replace(
            self, exc=self.exc[:n_factors].copy(), theta=self.theta[:n_factors].copy(),
            name=f"{self.name}[:{n_factors}]")

    def with_theta(self, theta: np.ndarray) -> "Problem":
        theta = np.ascontiguousarray(theta, dtype=np.float64)
        assert theta.shape == self.theta.shape
        return dataclasses.replace(self, theta=theta.copy())


def make_integrals(rng: np.random.Generator, n_spatial: int):
    """Synthetic integrals with the symmetry of real molecular integrals.

    h: diagonal linspace(-2, +1) Ha ascending (an orbital-energy-like spread),
    off-diagonal N(0, 0.1), symmetric.  g_pqrs = sum_{l<4} L^l_pq L^l_rs with
    L^l = (X + X^T)/2, X ~ N(0, 0.2^2): symmetric in p<->q, r<->s and
    (pq)<->(rs), i.e. 8-fold symmetric, and positive semidefinite as a matrix
    over orbital pairs, as a Coulomb kernel is.
    """
    n = n_spatial
    h = np.zeros((n, n))
    h[np.diag_indices(n)] = np.linspace(-2.0, 1.0, n)
    iu = np.triu_indices(n, 1)
    off = rng.normal(0.0, 0.1, size=len(iu[0]))
    h[iu] = off
    h[(iu[1], iu[0])] = off
    g = np.zeros((n, n, n, n))
    for _ in range(4):
        x = rng.normal(0.0, 0.2, size=(n, n))
        L = 0.5 * (x + x.T)
        g += np.einsum("pq,rs->pqrs", L, L)
    return h, g


def _occupied(n_spatial: int, n_alpha: int, n_beta: int):
    occ = [2 * s for s in range(n_alpha)] + [2 * s + 1 for s in range(n_beta)]
    vir = [p for p in range(2 * n_spatial) if p not in set(occ)]
    return sorted(occ), sorted(vir)


def enumerate_excitations(n_spatial: int, n_alpha: int, n_beta: int):
    """Spin-conserving UCCSD excitations of Eq. 2 in canonical order.

    Singles (i, -1, a, -1) with spin(i) == spin(a), then doubles (i, j, a, b)
    with i < j occupied, a < b virtual and {spin i, spin j} == {spin a, spin b},
    each block lexicographic in its spin-orbital indices.
    """
    occ, vir = _occupied(n_spatial, n_alpha, n_beta)
    singles = [(i, -1, a, -1) for i in occ for a in vir if (i & 1) == (a & 1)]
    doubles = []
    for i, j in itertools.combinations(occ, 2):
        for a, b in itertools.combinations(vir, 2):
            if sorted((i & 1, j & 1)) == sorted((a & 1, b & 1)):
                doubles.append((i, j, a, b))
    s = np.array(singles, dtype=np.int32).reshape(-1, 4)
    d = np.array(doubles, dtype=np.int32).reshape(-1, 4)
    return s, d


def order_and_truncate(singles, doubles, th_s, th_d, m_doubles: Optional[int] = None):
    """Factor order of the Methods section: doubles by |theta| descending
    (stable on canonical index, largest first = rightmost in Eq. 3), optionally
    cut to the M_D largest, then all singles in canonical order."""
    order = np.argsort(-np.abs(th_d), kind="stable")
    if m_doubles is not None:
        order = order[:m_doubles]
    exc = np.concatenate([doubles[order], singles], axis=0).astype(np.int32)
    theta = np.concatenate([th_d[order], th_s]).astype(np.float64)
    return np.ascontiguousarray(exc), np.ascontiguousarray(theta)


def make_problem(seed: int, n_spatial: int, n_alpha: int, n_beta: int, sigma_theta: float,
                 eps: float = 0.0, m_doubles: Optional[int] = None, name: str = "") -> Problem:
    """Draw one problem: integrals first, then theta in canonical order
    (singles, then doubles), then order and truncate the factor list."""
    if not (0 < n_alpha <= n_spatial and 0 < n_beta <= n_spatial):
        raise ValueError("electron counts out of range")
    if 2 * n_spatial > 128:
        raise ValueError("at most 128 spin-orbitals (two-word determinant keys)")
    rng = np.random.default_rng(seed)
    h, g = make_integrals(rng, n_spatial)
    s, d = enumerate_excitations(n_spatial, n_alpha, n_beta)
    th_s = rng.normal(0.0, sigma_theta, size=len(s))
    th_d = rng.normal(0.0, sigma_theta, size=len(d))
    exc, theta = order_and_truncate(s, d, th_s, th_d, m_doubles)
    return Problem(n_spatial, n_alpha, n_beta, h, g, exc, theta, eps=eps,
                   name=name or f"seed{seed}_{2 * n_spatial}so_{n_alpha + n_beta}e")


# The five workload shapes: seed, spatial orbitals, alpha/beta electrons,
# theta spread, pruning threshold and the number of doubles kept.
CONFIGS = {
    1: dict(seed=1001, n_spatial=6, n_alpha=2, n_beta=2, sigma_theta=0.05, eps=0.0, m_doubles=None),
    2: dict(seed=1002, n_spatial=12, n_alpha=4, n_beta=4, sigma_theta=0.02, eps=0.0, m_doubles=None),
    3: dict(seed=1003, n_spatial=20, n_alpha=6, n_beta=6, sigma_theta=0.01, eps=1e-8, m_doubles=None,
            n_max=10_000_000, n_cut=6_250_000),
    4: dict(seed=1004, n_spatial=32, n_alpha=8, n_beta=8, sigma_theta=0.005, eps=1e-6, m_doubles=29616,
            n_max=10_000_000, n_cut=6_250_000),
}
CONFIG_NAMES = {
    1: "12so_4e_uccsd",
    2: "24so_8e_uccsd",
    3: "40so_12e_uccsd_eps1e-8_cut1e7",
    4: "64so_16e_uccsd30k_eps1e-6_cut1e7",
}


def config_problem(cfg: int) -> Problem:
    """The workload shapes.  The 40- and 64-spin-orbital ones also carry the
    Methods section's wavefunction cut (N_MAX = 1e7 determinants, N_CUT =
    6.25e6, the paper's 8,000 : 5,000 ratio): with eps alone the 64-so map
    passes 1e9 determinants by factor 3,000 of 30,000, and the 40-so map 5.9e7
    by factor 400 of 9,954."""
    c = CONFIGS[cfg]
    p = make_problem(c["seed"], c["n_spatial"], c["n_alpha"], c["n_beta"], c["sigma_theta"],
                     eps=c["eps"], m_doubles=c["m_doubles"], name=CONFIG_NAMES[cfg])
    p.n_max = c.get("n_max", 0)
    p.n_cut = c.get("n_cut", 0)
    return p


def batch_job_shape(j: int):
    """Shape of job j of the 256-job batch: 16-36 spin-orbitals, 4-12 electrons."""
    n_spatial = 8 + (j % 11)
    n_elec = 4 + 2 * ((j // 11) % 5)
    n_elec = min(n_elec, 2 * n_spatial - 4)
    return n_spatial, n_elec // 2, n_elec // 2


def batch_job_problem(j: int, sigma_theta: float = 0.02, eps: float = 1e-8) -> Problem:
    n_spatial, na, nb = batch_job_shape(j)
    return make_problem(5000 + j, n_spatial, na, nb, sigma_theta, eps=eps,
                        name=f"job{j}_{2 * n_spatial}so_{na + nb}e")


def hilbert_size(n_spatial: int, n_alpha: int, n_beta: int) -> int:
    """Number of determinants with fixed alpha and beta electron counts."""
    return math.comb(n_spatial, n_alpha) * math.comb(n_spatial, n_beta)


def fig3_problem(m_doubles: int = 5000) -> Problem:
    """The shape of the paper's NH3/cc-pCVDZ study of the cut (Results,
    discussion of Fig. 3): 32 spatial orbitals (64 spin-orbitals, the highest
    virtual removed), 10 electrons, the m_doubles largest doubles plus all
    singles, and the optimisation-time cut N_MAX = 8,000 / N_CUT = 5,000.
    Synthetic integrals and angles; no eps (the cut alone bounds the map)."""
    p = make_problem(3200, 32, 5, 5, 0.02, eps=0.0, m_doubles=m_doubles, name=f"64so_10e_md{m_doubles}_cut8000")
    p.n_max, p.n_cut = 8000, 5000
    return p
