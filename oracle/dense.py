"""Dense state-vector brute force (test infrastructure only; n_so <= 16).

An implementation of the same physics that shares nothing with the sparse
oracle: every operator is a Jordan-Wigner map on the full 2^n state vector,
each UCC factor is the matrix exponential exp(theta (tau - tau^+)) evaluated
by its Taylor series to machine precision (Eqs. 3-5, no 2x2 closed form), and
the energy is contracted from one- and two-particle reduced density matrices
with the antisymmetrised spin-orbital integrals (no Slater-Condon rules).

Conventions: basis index x is the determinant bit string (bit p = spin-orbital
p = 2*spatial + spin); a_p|x> = (-1)^popcount(x below p) |x - p>.
"""
from __future__ import annotations

import numpy as np

MAX_QUBITS = 16


class Dense:
    def __init__(self, prob):
        n = prob.n_so
        if n > MAX_QUBITS:
            raise ValueError("dense brute force is limited to 16 spin-orbitals")
        self.prob = prob
        self.n = n
        self.dim = 1 << n
        idx = np.arange(self.dim, dtype=np.int64)
        self._idx = idx
        # Jordan-Wigner sign and occupation of every basis state for every mode.
        self._occ = [((idx >> p) & 1).astype(bool) for p in range(n)]
        below = [np.bitwise_count(idx & ((1 << p) - 1)) for p in range(n)]
        self._sign = [np.where(b % 2 == 1, -1.0, 1.0) for b in below]
        self._build_integrals()

    # --- second quantisation -------------------------------------------------
    def ann(self, p, v):
        """a_p v"""
        out = np.zeros_like(v)
        m = self._occ[p]
        src = self._idx[m]
        out[src ^ (1 << p)] = self._sign[p][m] * v[m]
        return out

    def cre(self, p, v):
        """a+_p v"""
        out = np.zeros_like(v)
        m = ~self._occ[p]
        src = self._idx[m]
        out[src | (1 << p)] = self._sign[p][m] * v[m]
        return out

    def tau(self, row, v):
        i, j, a, b = (int(x) for x in row)
        w = self.ann(i, v)
        if j >= 0:
            w = self.ann(j, w)
            w = self.cre(b, w)
        return self.cre(a, w)

    def tau_dagger(self, row, v):
        i, j, a, b = (int(x) for x in row)
        w = self.ann(a, v)
        if j >= 0:
            w = self.ann(b, w)
            w = self.cre(j, w)
        return self.cre(i, w)

    # --- Eq. 3 by matrix exponentials ----------------------------------------
    def expm_factor(self, row, theta, v):
        """exp(theta (tau - tau^+)) v by its Taylor series."""
        out = v.copy()
        term = v.copy()
        for m in range(1, 80):
            term = (theta / m) * (self.tau(row, term) - self.tau_dagger(row, term))
            out = out + term
            if np.max(np.abs(term)) < 1e-22:
                break
        return out

    def reference(self):
        v = np.zeros(self.dim)
        v[self.prob.hf_key] = 1.0
        return v

    def state(self, theta=None, n_factors=None):
        th = self.prob.theta if theta is None else theta
        nf = len(th) if n_factors is None else n_factors
        v = self.reference()
        for k in range(nf):
            v = self.expm_factor(self.prob.exc[k], th[k], v)
        return v

    # --- Hamiltonian from reduced density matrices ---------------------------
    def _build_integrals(self):
        p = self.prob
        n = self.n
        sp = np.arange(n) // 2
        spin = np.arange(n) % 2
        same = (spin[:, None] == spin[None, :])
        self.h_so = np.where(same, p.h[sp[:, None], sp[None, :]], 0.0)
        # <pq|rs> = (pr|qs) delta(spin p, spin r) delta(spin q, spin s)
        g = p.g[np.ix_(sp, sp, sp, sp)].transpose(0, 2, 1, 3)  # [p,q,r,s] = (p r | q s)
        mask = same[:, None, :, None] & same[None, :, None, :]  # spin p == spin r, spin q == spin s
        phys = np.where(mask, g, 0.0)
        self.anti = phys - phys.transpose(0, 1, 3, 2)

    def transition(self, bra, ket):
        """<bra|H|ket> = sum h_pq <a_p bra|a_q ket> + 1/4 sum <pq||rs> <a_q a_p bra|a_s a_r ket>."""
        n = self.n
        A_bra = np.stack([self.ann(p, bra) for p in range(n)])
        A_ket = np.stack([self.ann(p, ket) for p in range(n)])
        d1 = A_bra @ A_ket.T  # d1[p, q] = <bra| a+_p a_q |ket>
        W_bra = np.stack([self.ann(q, A_bra[p]) for p in range(n) for q in range(n)])
        W_ket = np.stack([self.ann(s, A_ket[r]) for r in range(n) for s in range(n)])
        d2 = (W_bra @ W_ket.T).reshape(n, n, n, n)  # d2[p,q,r,s] = <bra| a+_p a+_q a_s a_r |ket>
        return float(np.sum(self.h_so * d1) + 0.25 * np.sum(self.anti * d2))

    def energy(self, v):
        return self.transition(v, v) / float(v @ v)

    def hmat(self, I, J):
        """<J|H|I> between two determinants."""
        bra = np.zeros(self.dim)
        ket = np.zeros(self.dim)
        bra[int(J)] = 1.0
        ket[int(I)] = 1.0
        return self.transition(bra, ket)
