"""Long-range exchange matrix (appendix "The Hartree-Fock exchange", eq. exchange) in numpy on the
FP64 oracle.

TEST INFRASTRUCTURE ONLY, like the rest of this package: only the tests may import it.

K^lr(mu, nu) = 2 sum_j sum_{lambda, kappa} q_{j lambda} q_{j kappa} B^lr(mu, lambda, kappa, nu) for
orbital coefficients q (N_orb x N_b); lambda and kappa run over the N_b basis functions (the
printed range N_b^2 is garbled).  With B^lr(mu lambda, kappa nu) = (omega / sqrt(pi))
M(mu lambda, :) K M(kappa nu, :)^T (eq. tensors, K = sum_p w_p (x)_d A_d^(p)) and the pair
symmetry of M, the factored representation of the appendix is
K^lr = 2 sum_j X_j (omega / sqrt(pi)) K X_j^T with X_j(mu, :) = sum_lambda q_{j lambda} M(mu lambda, :).
"""
from __future__ import annotations

import numpy as np


def exchange_direct(o, Q: np.ndarray, threads=None) -> np.ndarray:
    """eq. exchange from the full B^lr (Algorithm 1 entries); Q: N_orb x N_b."""
    nb = o.nbf
    B4 = o.assemble_B(threads=threads).reshape(nb, nb, nb, nb)  # [mu, lambda, kappa, nu]
    D = Q.T @ Q  # D(lambda, kappa) = sum_j q_{j lambda} q_{j kappa}
    return 2.0 * np.einsum("mlkn,lk->mn", B4, D)


def exchange_factored(o, Q: np.ndarray, threads=None) -> np.ndarray:
    """The appendix's factored representation through M (eq. tensors) and the node sum K."""
    nb, n = o.nbf, o.n
    M3 = o.factor_M(threads=threads).reshape(nb, nb, n ** 3)  # [mu, lambda, m]
    _, w = o.nodes()
    K = sum(w[p] * np.kron(o.cheb(0, p), np.kron(o.cheb(1, p), o.cheb(2, p))) for p in range(o.P))
    K *= o.omega / np.sqrt(np.pi)
    out = np.zeros((nb, nb))
    for q in np.atleast_2d(Q):
        X = np.einsum("l,mlc->mc", q, M3)
        out += 2.0 * X @ K @ X.T
    return out
