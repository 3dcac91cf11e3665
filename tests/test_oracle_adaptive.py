"""Pins of the adaptive-box oracle (oracle/adaptive.py; Section 6, adaptive choice of the
integration domain) against what the paper and the mathematics fix (no GPU).

- The cross-interval Chebyshev coefficients reproduce the kernel on the two boxes' grids (the
  interpolation property of Definition 1), are transposed by swapping the boxes, and on one box
  equal the C oracle's Definition 1 coefficients.
- Every pair's support lies in its partition's cube; partitions are ascending; equal supports
  (the components of one shell pair) share a partition.
- One partition: Algorithm 1 with the partition box equals the C oracle's Algorithm 1 with that
  box as an explicit box (two independent implementations).
- The paper's Table 3 trend on a synthetic molecule with diffuse functions: against the erf-Boys
  closed form, a fixed box that cuts the diffuse functions (b = 10) stalls at its truncation error,
  a generous one (b = 20) needs more nodes, and the adaptive boxes reach the accuracy of the
  best fixed box (b = 15) at the same n.
"""
import itertools
import math

import numpy as np
import pytest

import oracle
from oracle import adaptive as ad
from paper_2210_13069_gb300 import synth
from tests import closed_forms as cf


def mol_diffuse():
    return synth.random_molecule(3003, natoms=4, cube=12.0, shells_per_atom=(("s", 2),), nprim=1,
                                 alpha_range=(0.08, 20.0), omega=0.3, n=32, P=24)


@pytest.mark.parametrize("bx,by", [(3.0, 3.0), (2.5, 9.0), (12.0, 4.0)])
def test_cross_coefficients_interpolate_on_both_grids(bx, by):
    n, s = 14, 0.37
    A = ad.cheb_cross(s, bx, by, n)
    k = np.arange(1, n + 1)
    u = np.cos((2 * k - 1) * np.pi / (2 * n))
    T = np.array([np.cos(a * np.arccos(u)) for a in range(n)])
    interp = T.T @ A @ T  # sum_ab A(a, b) T_a(u_k) T_b(u_k')
    exact = np.exp(-s * s * (bx * u[:, None] - by * u[None, :]) ** 2)
    assert np.max(np.abs(interp - exact)) <= 1e-14
    assert np.max(np.abs(ad.cheb_cross(s, by, bx, n) - A.T)) <= 1e-15 * np.abs(A).max()


def test_cross_coefficients_on_one_box_equal_definition_1():
    m = synth.random_molecule(3004, natoms=2, cube=3.0, shells_per_atom=(("s", 1),), nprim=1, omega=0.6, n=12, P=6)
    c = ad.atom_centre(m)
    b = 7.5
    o = oracle.Oracle.from_molecule(m, box_lo=c - b, box_hi=c + b)
    s, _ = o.nodes()
    for p in range(m.P):
        A = ad.cheb_cross(s[p], b, b, m.n)
        ref = o.cheb(0, p)
        assert np.max(np.abs(A - ref)) <= 1e-14 * np.abs(ref).max()


def test_partitions_hold_every_support():
    m = synth.random_molecule(3005, natoms=3, cube=6.0, nprim=2, alpha_range=(0.05, 500.0), omega=0.4, n=8, P=8)
    part, bs, c = ad.partitions(m, 1e-20, 4)
    o = oracle.Oracle.from_molecule(m, n=1, P=1)
    pairs = [(mu, nu) for mu in range(o.nbf) for nu in range(mu, o.nbf)]
    b = np.array([ad.pair_support(o, mu, nu, c, 1e-20) for mu, nu in pairs])
    assert np.all(np.diff(bs) > 0)
    assert np.all(b <= bs[part] * (1 + 1e-15))
    for s in range(len(bs)):  # no smaller box would do for the group
        assert b[part == s].max() == bs[s]
    for v in np.unique(b):  # equal supports share a partition
        assert len(np.unique(part[b == v])) == 1
    # a pair's support: the Gaussian factor of each primitive pair is tau at the edge it reaches
    mu, nu = pairs[int(np.argmax(b))]
    A, _, ea, _ = o.basis_function(mu)
    B, _, eb, _ = o.basis_function(nu)
    hits = [max(abs((a * A + e * B) / (a + e) - c)) + math.sqrt(math.log(1e20) / (a + e)) for a in ea for e in eb]
    assert math.isclose(max(hits), b.max(), rel_tol=1e-15)


def test_one_partition_is_algorithm_1_on_that_box():
    m = synth.random_molecule(3006, natoms=2, cube=3.0, shells_per_atom=(("s", 1), ("p", 1)), nprim=2,
                              alpha_range=(0.3, 20.0), omega=0.5, n=10, P=8)
    a = ad.Adaptive(m, m.omega, m.n, m.P, 1e-20, 1)
    c, b = a.centre, a.bs[0]
    o = oracle.Oracle.from_molecule(m, box_lo=c - b, box_hi=c + b)
    rng = np.random.default_rng(4)
    idx = rng.integers(0, m.nbf, size=(40, 4))
    got = np.array([a.entry(*q) for q in idx])
    ref = o.entries(idx.astype(np.int32))
    assert np.max(np.abs(got - ref)) <= 1e-13 * np.abs(ref).max()


def test_table_3_trend_against_the_closed_form():
    m = mol_diffuse()
    rng = np.random.default_rng(0)
    idx = rng.integers(0, m.nbf, size=(60, 4))
    bf = [(s.center, (0, 0, 0), s.exps, s.coefs) for s in m.shells]
    ref = np.array([cf.contracted_entry([bf[i] for i in q], m.omega) for q in idx])
    a = ad.Adaptive(m, m.omega, m.n, m.P, 1e-20, 3)
    e_ad = np.linalg.norm(np.array([a.entry(*q) for q in idx]) - ref) / np.linalg.norm(ref)
    errs = {}
    for b in (20.0, 15.0, 10.0):
        o = oracle.Oracle.from_molecule(m, box_lo=a.centre - b, box_hi=a.centre + b)
        errs[b] = np.linalg.norm(o.entries(idx.astype(np.int32)) - ref) / np.linalg.norm(ref)
    print(f"adaptive (boxes {np.round(a.bs, 1)}): {e_ad:.1e}; fixed b=20 {errs[20.0]:.1e}, b=15 {errs[15.0]:.1e}, "
          f"b=10 {errs[10.0]:.1e}")
    assert errs[10.0] > 100 * e_ad          # the cut box stalls
    assert errs[20.0] > 10 * e_ad           # the generous box needs more nodes
    assert e_ad <= 3 * errs[15.0]            # as good as the best fixed box
