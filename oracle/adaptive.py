"""Adaptive choice of the integration domain (Section 6, "Adaptive approach for the choice of the
integration domain [-b,b]"), in numpy on the FP64 oracle's moments.

TEST INFRASTRUCTURE ONLY, like the rest of this package: only the tests may import it.

The method as the paper states it, with the readings this build takes where it is silent:
 1. Each primitive pair j = (j1, j2) of a basis pair (mu, nu) carries the Gaussian factor
    sigma_j(x_l) = exp(-p_j (x_l - P_{j,l})^2) of the Gaussian product rule; its numerical support
    in dimension l is where sigma_j > tau_adaptive, |x_l - P_{j,l}| < sqrt(ln(1/tau) / p_j).
 2. The basis pair's support is the smallest cube [c - b, c + b]^3, centred at the centre c of the
    atoms' extent (the default box's centre), that holds the supports of all its primitive pairs
    in all three dimensions: b_{mu nu} = max_{j, l} (|P_{j,l} - c_l| + sqrt(ln(1/tau) / p_j)).
    (Reading: the paper's boxes are [-b, b] about the molecule; the polynomial prefactors are
    ignored, as in the paper's criterion.)
 3. The supports are clustered into N_partitions boxes [c - b_s, c + b_s]^3 (reading: the pairs
    sorted by b, cut into N_partitions groups of about equal count, each cut moved past a run of
    equal b so that equal supports - the Cartesian components of one shell pair - stay together;
    empty groups dropped; b_s the largest b of its group).
 4. A pair's moment matrices are integrated over its partition's box, with the Chebyshev
    polynomials mapped to that box (eq. defV on [c - b_s, c + b_s]).
 5. Between partitions s and s' the kernel exp(-s_p^2 (x - y)^2), x in box s, y in box s', is
    interpolated on the two boxes' Chebyshev grids (Definition 1 with the two intervals):
       A^(p)_{ss'}(a, b) = c_a c_b / n^2 sum_{k, k'} exp(-s_p^2 (b_s u_k - b_s' u_k')^2) T_a(u_k) T_b(u_k'),
    so that A_{s's} = A_{ss'}^T and A_{ss} is Definition 1's matrix on box s.
 6. B(mu nu, ka la) = (w/sqrt(pi)) sum_p w_p sum_{j, j'} c_j c_j' prod_d (S^s_d(j) A^(p)_{ss',d} S^{s'}_d(j')^T),
    s and s' the partitions of (mu, nu) and (ka, la): Algorithm 1 with the partition boxes.
One Chebyshev order n serves every partition (reading; the paper allows N_s per partition).
With one partition whose half-width is the default box's, this is the single-box oracle.
"""
from __future__ import annotations

import math
from typing import List, Sequence, Tuple

import numpy as np

import oracle


def atom_centre(mol) -> np.ndarray:
    """Centre of the atoms' extent (the default box's centre)."""
    C = np.array([s.center for s in mol.shells], dtype=np.float64)
    return 0.5 * (C.min(axis=0) + C.max(axis=0))


def _unique_pairs(nbf: int) -> List[Tuple[int, int]]:
    return [(mu, nu) for mu in range(nbf) for nu in range(mu, nbf)]


def pair_support(o, mu: int, nu: int, centre: np.ndarray, tau: float) -> float:
    """Step 2: half-width b_{mu nu} of the smallest centred cube holding every primitive pair's
    support (sigma_j > tau) in every dimension."""
    A, _, ea, _ = o.basis_function(mu)
    B, _, eb, _ = o.basis_function(nu)
    r = math.log(1.0 / tau)
    b = 0.0
    for a in ea:
        for e in eb:
            p = a + e
            P = (a * A + e * B) / p
            half = math.sqrt(r / p)
            b = max(b, float(np.max(np.abs(P - centre))) + half)
    return b


def partitions(mol, tau: float, npart: int):
    """Steps 2-3: (partition index of every unique pair in row-major upper-triangle order, the
    partitions' half-widths b_s ascending, the common centre c)."""
    centre = atom_centre(mol)
    o = oracle.Oracle.from_molecule(mol, n=1, P=1)
    pairs = _unique_pairs(o.nbf)
    b = np.array([pair_support(o, mu, nu, centre, tau) for mu, nu in pairs])
    order = np.argsort(b, kind="stable")
    N = len(pairs)
    cuts = [0]
    for k in range(1, npart):
        c = max(cuts[-1], (k * N) // npart)
        while 0 < c < N and b[order[c]] == b[order[c - 1]]:
            c += 1
        cuts.append(c)
    cuts.append(N)
    part = np.zeros(N, dtype=np.int64)
    bs = []
    for k in range(npart):
        g = order[cuts[k]:cuts[k + 1]]
        if len(g) == 0:
            continue
        part[g] = len(bs)
        bs.append(float(b[g].max()))
    return part, np.array(bs), centre


def cheb_cross(s_p: float, bx: float, by: float, n: int) -> np.ndarray:
    """Step 5: coefficients of exp(-s_p^2 (x - y)^2) with x = c + bx u, y = c + by v on the
    first-kind Chebyshev grids of the two intervals (a literal double sum)."""
    k = np.arange(1, n + 1)
    u = np.cos((2 * k - 1) * np.pi / (2 * n))
    T = np.array([np.cos(a * np.arccos(u)) for a in range(n)])  # T[a, k] = T_a(u_k)
    F = np.exp(-(s_p ** 2) * (bx * u[:, None] - by * u[None, :]) ** 2)
    cw = np.where(np.arange(n) == 0, 1.0, 2.0)
    A = np.zeros((n, n))
    for a in range(n):
        for bb in range(n):
            A[a, bb] = cw[a] * cw[bb] / n ** 2 * np.sum(F * np.outer(T[a], T[bb]))
    return A


class Adaptive:
    """The adaptive-box TA of one molecule at (omega, n, P, tau_adaptive, N_partitions)."""

    def __init__(self, mol, omega: float, n: int, P: int, tau: float, npart: int):
        self.mol, self.omega, self.n, self.P = mol, float(omega), int(n), int(P)
        self.part, self.bs, self.centre = partitions(mol, tau, npart)
        self.npart = len(self.bs)
        # one oracle context per partition box (moments of eq. defV over that box)
        self.ctx = []
        for s in range(self.npart):
            lo, hi = self.centre - self.bs[s], self.centre + self.bs[s]
            self.ctx.append(oracle.Oracle.from_molecule(mol, omega=omega, n=n, P=P, box_lo=lo, box_hi=hi))
        self.nbf = self.ctx[0].nbf
        self.s, self.w = self.ctx[0].nodes()
        self.index = {pq: i for i, pq in enumerate(_unique_pairs(self.nbf))}
        self.coefs = [self.ctx[0].basis_function(mu)[3] for mu in range(self.nbf)]
        self._A = {}
        self._S = {}

    def cheb(self, s: int, t: int, p: int) -> np.ndarray:
        key = (s, t, p)
        if key not in self._A:
            self._A[key] = cheb_cross(self.s[p], self.bs[s], self.bs[t], self.n)
        return self._A[key]

    def moments(self, mu: int, nu: int):
        """(partition, [S_x, S_y, S_z], c_j) of the unique pair (mu, nu)."""
        key = (min(mu, nu), max(mu, nu))
        if key not in self._S:
            s = int(self.part[self.index[key]])
            S = [self.ctx[s].moments(key[0], key[1], d) for d in range(3)]
            c = np.outer(self.coefs[key[0]], self.coefs[key[1]]).ravel()
            self._S[key] = (s, S, c)
        return self._S[key]

    def entry(self, mu: int, nu: int, ka: int, la: int) -> float:
        """Step 6 (Algorithm 1 with the partition boxes), node sum by math.fsum."""
        s, S1, c1 = self.moments(mu, nu)
        t, S2, c2 = self.moments(ka, la)
        terms = []
        for p in range(self.P):
            G = np.ones((len(c1), len(c2)))
            for d in range(3):
                G = G * (S1[d] @ self.cheb(s, t, p) @ S2[d].T)
            terms.append(self.w[p] * float(c1 @ G @ c2))
        return self.omega / math.sqrt(math.pi) * math.fsum(terms)

    def assemble_B(self) -> np.ndarray:
        nb = self.nbf
        pairs = _unique_pairs(nb)
        Bu = np.zeros((len(pairs), len(pairs)))
        for i, (mu, nu) in enumerate(pairs):
            for j in range(i, len(pairs)):
                ka, la = pairs[j]
                Bu[i, j] = Bu[j, i] = self.entry(mu, nu, ka, la)
        idx = np.zeros((nb, nb), dtype=np.int64)
        for i, (mu, nu) in enumerate(pairs):
            idx[mu, nu] = idx[nu, mu] = i
        flat = idx.ravel()
        return Bu[np.ix_(flat, flat)]
