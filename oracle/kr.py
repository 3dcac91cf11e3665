"""Khatri-Rao low-rank compression of the factored form (Section 6, "Compression by using
low-rank methods": eq. SVD, then eq. approxepsilon), in numpy on the FP64 oracle's factors.

TEST INFRASTRUCTURE ONLY, like the rest of this package: only the tests may import it.

With one Chebyshev order n for every node, the moment matrix W~^(d) of a dimension d (the rows of
all primitive pairs of all unique pairs, n columns) is the same for every node.  Its truncated SVD
W~^(d) ~ U^(d) V^(d)T (U: the first R_d left singular vectors times the singular values, V: the
first R_d right singular vectors, n x R_d) and the mixed-product property of the Khatri-Rao and
Kronecker products give

    B_u ~ (omega / sqrt(pi)) U~ [sum_p w_p (x)_d V^(d)T A_d^(p) V^(d)] U~^T,

U~ (unique pairs x R_1 R_2 R_3) being the c_j-weighted sum over a pair's rows j of the row-wise
Kronecker products U^(1)(j, :) (x) U^(2)(j, :) (x) U^(3)(j, :).  (The paper prints the middle
factor as V A V^T with V^T of size R x n; with V of size n x R the contraction is V^T A V.)
R_d = n reproduces the uncompressed factored form.
"""
from __future__ import annotations

from typing import Sequence

import numpy as np


def moment_rows(o):
    """(S[d] (rows x n) for d = 0, 1, 2; c_j per row; unique-pair index per row), rows ordered by
    unique pair (mu <= nu) then j = j1 * I_nu + j2 (eq. approx4 for c_j)."""
    nbf = o.nbf
    coefs = [o.basis_function(mu)[3] for mu in range(nbf)]
    S = [[], [], []]
    cj, pair = [], []
    r = 0
    for mu in range(nbf):
        for nu in range(mu, nbf):
            cc = np.outer(coefs[mu], coefs[nu]).ravel()
            for d in range(3):
                S[d].append(o.moments(mu, nu, d))
            cj.append(cc)
            pair.append(np.full(cc.size, r))
            r += 1
    return [np.vstack(s) for s in S], np.concatenate(cj), np.concatenate(pair)


def truncated_factors(S: np.ndarray, rank: int):
    """eq. SVD: W~ ~ U V^T with U = u[:, :R] sigma[:R] (rows x R) and V = v[:, :R] (n x R)."""
    u, sv, vt = np.linalg.svd(S, full_matrices=False)
    return u[:, :rank] * sv[:rank], vt[:rank].T, sv


def ranks_for_eps(o, eps: float):
    """eq. approxepsilon's truncation, read as: keep in dimension d the singular values of W~^(d)
    that are at least eps times the largest (eps = 0 keeps all n)."""
    S, _, _ = moment_rows(o)
    out = []
    for d in range(3):
        sv = np.linalg.svd(S[d], compute_uv=False)
        out.append(o.n if eps == 0 else max(1, int(np.count_nonzero(sv >= eps * sv[0]))))
    return out


def compressed_Bu(o, ranks: Sequence[int]):
    """B_u (unique pairs x unique pairs) by eq. approxepsilon with ranks (R_1, R_2, R_3); also
    returns the three singular value vectors."""
    if getattr(o, "tau_screening", 0.0):
        raise ValueError("the compressed form here takes every primitive pair (no screening)")
    S, cj, pair = moment_rows(o)
    U, V, sig = [], [], []
    for d in range(3):
        u, v, sv = truncated_factors(S[d], int(ranks[d]))
        U.append(u)
        V.append(v)
        sig.append(sv)
    npair = o.nbf * (o.nbf + 1) // 2
    rowkron = np.einsum("j,ja,jb,jc->jabc", cj, U[0], U[1], U[2]).reshape(cj.size, -1)
    Ut = np.zeros((npair, rowkron.shape[1]))
    np.add.at(Ut, pair, rowkron)
    _, w = o.nodes()
    KR = np.zeros((Ut.shape[1], Ut.shape[1]))
    for p in range(o.P):
        C = [V[d].T @ o.cheb(d, p) @ V[d] for d in range(3)]
        KR += w[p] * np.kron(C[0], np.kron(C[1], C[2]))
    return o.omega / np.sqrt(np.pi) * Ut @ KR @ Ut.T, sig


def expand(o, Bu: np.ndarray) -> np.ndarray:
    """Full B (N_b^2 x N_b^2, row mu N_b + nu) from B_u over unique pairs."""
    nbf = o.nbf
    idx = np.zeros((nbf, nbf), dtype=np.int64)
    r = 0
    for mu in range(nbf):
        for nu in range(mu, nbf):
            idx[mu, nu] = idx[nu, mu] = r
            r += 1
    flat = idx.ravel()
    return Bu[np.ix_(flat, flat)]


def compressed_B(o, ranks: Sequence[int]) -> np.ndarray:
    return expand(o, compressed_Bu(o, ranks)[0])
