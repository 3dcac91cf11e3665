"""Planted mistakes: each mutation of a copy of the oracle's C source must fail the pins.

The copy is compiled into a temporary directory and loaded beside the real oracle; the
committed oracle source is never touched.  This shows that the pins in
``test_oracle_pins.py`` would catch a dropped term, a wrong sign, a wrong index or a wrong
constant anywhere along the oracle's chain (normalisation, box, nodes, Chebyshev
coefficients, moments, Algorithm 1, factored form).
"""
import math
import os
import subprocess

import numpy as np
import pytest
from scipy import special

import oracle
from tests import closed_forms as cf

SRC_DIR = os.path.dirname(oracle.__file__)

MUTATIONS = {
    "drop_contraction_norm": ("for (int k = 0; k < K; ++k) f->coefs[k] /= sqrt(S);", ""),
    "chebyshev_recurrence_sign": ("T[m] = 2.0 * u * T[m - 1] - T[m - 2];", "T[m] = 2.0 * u * T[m - 1] + T[m - 2];"),
    "wrong_pair_index": ("const double* Wkl = moments_cached(c, ka, la, d);",
                         "const double* Wkl = moments_cached(c, mu, nu, d);"),
    "prefactor": ("return c->omega / sqrt(M_PI) * (s + comp);", "return 2.0 * c->omega / sqrt(M_PI) * (s + comp);"),
    "node_map": ("c->s[p] = 0.5 * omega * (1.0 + z[p]);", "c->s[p] = omega * (1.0 + z[p]);"),
    "cheb_weight": ("((a == 0 || b == 0) ? 2.0 : 4.0)", "((a == 0 || b == 0) ? 2.0 : 2.0)"),
    "box_centre": ("c->cen[d] = 0.5 * (c->lo[d] + c->hi[d]);", "c->cen[d] = 0.5 * c->hi[d];"),
    "dropped_panel": ("for (int q = 0; q < npan; ++q) {", "for (int q = 0; q < npan - 1; ++q) {"),
    "power_on_wrong_centre": ("pow(x - Ad, i) * pow(x - Bd, k)", "pow(x - Ad, i) * pow(x - Ad, k)"),
    "transposed_cheb": ("t += Wmn[(size_t)j * n + a] * A[a * n + b];", "t += Wmn[(size_t)j * n + a] * A[b * n + a + (a == 0 && b == 1)];"),
    "hadamard_skip_dim": ("for (int t = 0; t < I1 * I2; ++t) F[t] *= G[t];",
                          "if (d != 2) for (int t = 0; t < I1 * I2; ++t) F[t] *= G[t];"),
}


def build_mutant(tmp_path, name):
    old, new = MUTATIONS[name]
    src = open(os.path.join(SRC_DIR, "lrtei_oracle.c")).read()
    assert src.count(old) == 1, f"mutation anchor for {name} not unique/present"
    d = tmp_path / name
    d.mkdir()
    (d / "lrtei_oracle.c").write_text(src.replace(old, new))
    (d / "lrtei_oracle.h").write_text(open(os.path.join(SRC_DIR, "lrtei_oracle.h")).read())
    so = d / "lib.so"
    subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off", "-o", str(so),
                    str(d / "lrtei_oracle.c"), "-lm"], check=True)
    return oracle.load_library(str(so))


_REF = {}


def _ref(key, fn):
    if key not in _REF:
        _REF[key] = fn()
    return _REF[key]


def pins_pass(lib) -> bool:
    """A compact battery of the pins (closed forms, brute force, node and Chebyshev identities);
    stops at the first pin that fails."""
    # quadrature nodes reproduce erf(omega r)/r
    centers = np.array([[0.0, 0.0, 0.0], [1.1, 0.4, -0.7]])
    o = oracle.Oracle(centers, np.array([0, 0], np.int32), np.array([2, 1], np.int32), np.array([0.8, 2.0, 1.5]),
                      np.array([0.7, 0.3, 1.0]), 0.3, 32, 24, lib=lib)
    s, w = o.nodes()
    r = np.linspace(0.01, 15, 50)
    approx = 0.3 / math.sqrt(math.pi) * (w[None, :] * np.exp(-np.outer(r * r, s * s))).sum(1)
    if not np.max(np.abs(approx / (special.erf(0.3 * r) / r) - 1)) < 1e-12:
        return False
    # contracted s closed form
    raw = [((0.8, 2.0), (0.7, 0.3)), ((1.5,), (1.0,))]
    bf = [(centers[i], (0, 0, 0), raw[i][0], raw[i][1]) for i in range(2)]
    for q in [(0, 0, 0, 0), (0, 1, 0, 1), (0, 0, 1, 1), (1, 0, 1, 1)]:
        ref = _ref(("s",) + q, lambda: cf.contracted_entry([bf[i] for i in q], 0.3))
        if not abs(o.entry(*q) - ref) <= 1e-11 * abs(ref):
            return False
    # p/d closed form
    c2 = ((0.0, 0.0, 0.0), (0.9, -0.3, 0.5))
    o2 = oracle.Oracle(np.array(c2), np.array([1, 2], np.int32), np.array([1, 1], np.int32), np.array([1.2, 0.9]),
                       np.array([1.0, 1.0]), 0.25, 40, 24, lib=lib)
    comps = [(0, pw) for pw in cf.cart_components(1)] + [(1, pw) for pw in cf.cart_components(2)]
    bfs = [(c2[sh], pw, ((1.2, 0.9)[sh],), (1.0,)) for sh, pw in comps]
    for q in [(0, 3, 1, 8), (3, 6, 8, 2), (0, 0, 4, 5)]:
        ref = _ref(("pd",) + q, lambda: cf.contracted_entry([bfs[i] for i in q], 0.25))
        if not abs(o2.entry(*q) - ref) <= 1e-9 * max(abs(ref), 1e-3):
            return False
    # box-truncated brute force (a box that cuts the Gaussians)
    box = ((-1.2, -1.0, -1.1), (1.0, 1.3, 0.9))
    c3 = ((0.2, -0.1, 0.3), (-0.4, 0.5, -0.2))
    o3 = oracle.Oracle(np.array(c3), np.array([0, 0], np.int32), np.array([1, 1], np.int32), np.array([0.6, 0.9]),
                       np.array([1.0, 1.0]), 0.7, 24, 32, box_lo=box[0], box_hi=box[1], lib=lib)
    ref = _ref("brute", lambda: _brute(box, c3))
    return bool(abs(o3.entry(0, 1, 0, 1) - ref) <= 1e-6 * abs(ref))


def _brute(box, c3):
    z, wq = np.polynomial.legendre.leggauss(12)
    lo, hi = np.array(box[0]), np.array(box[1])
    X = [0.5 * (hi[d] - lo[d]) * z + 0.5 * (hi[d] + lo[d]) for d in range(3)]
    W = [0.5 * (hi[d] - lo[d]) * wq for d in range(3)]
    gx = np.stack(np.meshgrid(*X, indexing="ij"), -1).reshape(-1, 3)
    wx = np.einsum("i,j,k->ijk", *W).reshape(-1)
    g = [(2 * e / math.pi) ** 0.75 * np.exp(-e * ((gx - np.array(c3[i])) ** 2).sum(1)) for i, e in enumerate((0.6, 0.9))]
    rr = np.sqrt(((gx[:, None, :] - gx[None, :, :]) ** 2).sum(-1))
    K = np.where(rr > 0, special.erf(0.7 * rr) / np.where(rr > 0, rr, 1), 2 * 0.7 / math.sqrt(math.pi))
    return (wx * g[0] * g[1]) @ K @ (wx * g[0] * g[1])


def test_pristine_oracle_passes_battery():
    assert pins_pass(oracle._load())


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(tmp_path, name):
    lib = build_mutant(tmp_path, name)
    assert not pins_pass(lib), f"mutation {name} slipped through the pins"
