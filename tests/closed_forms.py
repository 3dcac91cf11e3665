"""Textbook closed forms used to pin the oracle (test-only; independent of ``oracle/``).

* erf-attenuated Coulomb integral of four unnormalised s-type Gaussians (range-separated
  Boys function): for exponents a, b, c, d at A, B, C, D, with p = a+b, q = c+d,
  rho = pq/(p+q), P, Q the Gaussian-product centres (Proposition 1) and
  T = rho w^2/(rho + w^2) |P-Q|^2,
      (ab|erf(w r)/r|cd) = 2 pi^{5/2} / (p q sqrt(p+q)) sqrt(w^2/(w^2+rho)) K_AB K_CD F0(T),
  F0(T) = sqrt(pi/T) erf(sqrt(T)) / 2.
* Cartesian powers by differentiation with respect to the centre:
  (x-A)   g = (1/2a) d/dA g,
  (x-A)^2 g = (d^2/dA^2 g + 2a g) / (4a^2).
* Normalisation of a Cartesian primitive on R^3 and of a contraction (unit self-overlap).
"""
from __future__ import annotations

import itertools
import math

import mpmath as mp
import numpy as np


def dfact(k: int) -> int:
    r = 1
    while k > 1:
        r *= k
        k -= 2
    return r


def cart_components(l: int):
    out = []
    for lx in range(l, -1, -1):
        for ly in range(l - lx, -1, -1):
            out.append((lx, ly, l - lx - ly))
    return out


def prim_norm(a: float, pw) -> float:
    L = sum(pw)
    return (2 * a / math.pi) ** 0.75 * (4 * a) ** (L / 2) / math.sqrt(dfact(2 * pw[0] - 1) * dfact(2 * pw[1] - 1) * dfact(2 * pw[2] - 1))


def contracted_coefs(exps, coefs, pw):
    """Coefficients (incl. primitive normalisation) of a unit-norm contracted component."""
    c = np.array([coefs[k] * prim_norm(exps[k], pw) for k in range(len(exps))])
    S = 0.0
    for k, q in itertools.product(range(len(exps)), repeat=2):
        pq = exps[k] + exps[q]
        ov = 1.0
        for d in range(3):
            ov *= dfact(2 * pw[d] - 1) / (2 * pq) ** pw[d] * math.sqrt(math.pi / pq)
        S += c[k] * c[q] * ov
    return c / math.sqrt(S)


def ss_erf(a, A, b, B, c, C, d, D, omega):
    """(ab|erf(omega r)/r|cd) for unnormalised s primitives, mpmath precision."""
    a, b, c, d, om = (mp.mpf(v) for v in (a, b, c, d, omega))
    A = [mp.mpf(v) for v in A]
    B = [mp.mpf(v) for v in B]
    C = [mp.mpf(v) for v in C]
    D = [mp.mpf(v) for v in D]
    p, q = a + b, c + d
    rho = p * q / (p + q)
    P = [(a * A[i] + b * B[i]) / p for i in range(3)]
    Q = [(c * C[i] + d * D[i]) / q for i in range(3)]
    kab = mp.e ** (-a * b / p * sum((A[i] - B[i]) ** 2 for i in range(3)))
    kcd = mp.e ** (-c * d / q * sum((C[i] - D[i]) ** 2 for i in range(3)))
    T = rho * om ** 2 / (rho + om ** 2) * sum((P[i] - Q[i]) ** 2 for i in range(3))
    F0 = mp.mpf(1) if T == 0 else mp.sqrt(mp.pi / T) / 2 * mp.erf(mp.sqrt(T))
    return 2 * mp.pi ** mp.mpf(2.5) / (p * q * mp.sqrt(p + q)) * mp.sqrt(om ** 2 / (om ** 2 + rho)) * kab * kcd * F0


def cart_erf(exps4, centers4, pows4, omega, dps=30):
    """(g1 g2|erf|g3 g4) for unnormalised Cartesian primitives by differentiating ss_erf
    with respect to the centre coordinates (mpmath numerical derivatives)."""
    with mp.workdps(dps):
        vars_, orders = [], []
        for f in range(4):
            for d in range(3):
                k = pows4[f][d]
                if k:
                    vars_.append((f, d))
                    orders.append(k)

        def base(*xs):
            cs = [list(map(mp.mpf, centers4[f])) for f in range(4)]
            for (f, d), x in zip(vars_, xs):
                cs[f][d] = x
            return ss_erf(exps4[0], cs[0], exps4[1], cs[1], exps4[2], cs[2], exps4[3], cs[3], omega)

        if not vars_:
            return float(base())
        x0 = [mp.mpf(centers4[f][d]) for (f, d) in vars_]
        # Expand each power-2 factor (d^2 + 2a)/(4a^2) into derivative-order terms.
        total = mp.mpf(0)
        choices = []
        for (f, d), k in zip(vars_, orders):
            a = mp.mpf(exps4[f])
            if k == 1:
                choices.append([(1, 1 / (2 * a))])
            elif k == 2:
                choices.append([(2, 1 / (4 * a * a)), (0, 2 * a / (4 * a * a))])
            else:
                raise ValueError("powers up to 2 only")
        for combo in itertools.product(*choices):
            ords = tuple(o for o, _ in combo)
            coef = mp.mpf(1)
            for _, cf in combo:
                coef *= cf
            if all(o == 0 for o in ords):
                val = base(*x0)
            else:
                val = mp.diff(base, tuple(x0), ords)
            total += coef * val
        return float(total)


def contracted_entry(bf4, omega):
    """B(mu,nu,ka,la) for contracted, normalised Cartesian functions given as
    (center, pow, exps, raw coefs) tuples, from the closed forms above."""
    cs = [contracted_coefs(e, c, pw) for (_, pw, e, c) in bf4]
    total = 0.0
    for ks in itertools.product(*[range(len(b[2])) for b in bf4]):
        coef = 1.0
        for f in range(4):
            coef *= cs[f][ks[f]]
        total += coef * cart_erf([bf4[f][2][ks[f]] for f in range(4)], [bf4[f][0] for f in range(4)],
                                 [bf4[f][1] for f in range(4)], omega)
    return total
