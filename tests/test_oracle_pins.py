"""Pins of the FP64 oracle against what the paper and the mathematics fix (no GPU).

Each test checks the oracle against something other than itself: a library routine, a
textbook closed form, brute-force quadrature, or an invariant of the method.  The
planted-mistake test at the end shows that typical slips in the oracle's arithmetic
(a dropped term, a wrong sign or index) fail these pins.
"""
import itertools
import math

import numpy as np
import pytest
from scipy import integrate, special

import oracle
from paper_2210_13069_gb300 import synth
from tests import closed_forms as cf

pytestmark = pytest.mark.filterwarnings("ignore::scipy.integrate.IntegrationWarning")


def small_mol(ls=(0, 0), nprim=(1, 1), exps=(0.8, 1.5), coefs=(1.0, 1.0),
              centers=((0.0, 0.0, 0.0), (1.1, 0.4, -0.7)), omega=0.3, n=32, P=24, box=None, tau=0.0):
    c = np.array(centers, dtype=np.float64)
    kw = {"tau_screening": tau}
    if box is not None:
        kw.update(box_lo=box[0], box_hi=box[1])
    return oracle.Oracle(c, np.array(ls, np.int32), np.array(nprim, np.int32), np.array(exps, np.float64),
                         np.array(coefs, np.float64), omega, n, P, **kw)


# --------------------------------------------------------------- Proposition 3 ----

@pytest.mark.parametrize("N", [1, 2, 5, 16, 20, 32, 48, 64])
def test_gauss_legendre_matches_numpy(N):
    z, w = oracle.gauss_legendre(N)
    zr, wr = np.polynomial.legendre.leggauss(N)
    assert np.max(np.abs(z - zr)) < 2e-15
    # numpy's own weights lose digits for large N (1e-12 at N = 48); the mpmath pin below is tight
    assert np.max(np.abs(w - wr) / wr) < 5e-12
    assert abs(w.sum() - 2.0) < 1e-14


@pytest.mark.parametrize("N", [7, 20, 48])
def test_gauss_legendre_matches_mpmath(N):
    """40-digit roots of P_N (mpmath findroot from numpy's nodes) and w = 2/((1-x^2) P_N'(x)^2)."""
    import mpmath as mp
    z, w = oracle.gauss_legendre(N)
    zr, _ = np.polynomial.legendre.leggauss(N)
    with mp.workdps(40):
        for i in range(N):
            x = mp.findroot(lambda t: mp.legendre(N, t), mp.mpf(zr[i]))
            dp = mp.diff(lambda t: mp.legendre(N, t), x)
            wx = 2 / ((1 - x * x) * dp * dp)
            assert abs(z[i] - float(x)) < 2e-16
            # 1 ulp of a node next to +-1 is ~1e-13 relative in (1 - x^2): that bounds the weight
            tol = 2e-14 + 4e-16 / (1 - abs(float(x)))
            assert abs(w[i] - float(wx)) < tol * float(wx)


@pytest.mark.parametrize("omega,P", [(0.5, 20), (0.4, 32), (1.0, 40)])
def test_quadrature_reproduces_erf_kernel(omega, P):
    """eq. kernel/TEI2: (omega/sqrt(pi)) sum_p w_p exp(-s_p^2 r^2) -> erf(omega r)/r."""
    o = small_mol(omega=omega, P=P, n=4)
    s, w = o.nodes()
    assert np.all(s > 0) and np.all(s < omega)
    r = np.linspace(1e-3, 6.0 / omega, 300)
    approx = omega / math.sqrt(math.pi) * (w[None, :] * np.exp(-np.outer(r * r, s * s))).sum(1)
    exact = special.erf(omega * r) / r
    assert np.max(np.abs(approx - exact) / exact) < 1e-12
    # r -> 0 limit: 2 omega / sqrt(pi)
    assert abs(omega / math.sqrt(math.pi) * w.sum() - 2 * omega / math.sqrt(math.pi)) < 1e-14


# --------------------------------------------------------- Definition 1 / chebcheb ----

def cheb_T(n, u):
    th = np.arccos(np.clip(u, -1, 1))
    return np.cos(np.outer(np.arange(n), th))  # n x len(u)


@pytest.mark.parametrize("n", [8, 16, 24])
def test_cheb_interpolant_reproduces_kernel_on_grid(n):
    o = small_mol(n=n, P=12, omega=0.5)
    lo, hi = o.box()
    b = 0.5 * (hi - lo)
    s, _ = o.nodes()
    uk = np.cos((2 * np.arange(1, n + 1) - 1) * np.pi / (2 * n))
    Tk = cheb_T(n, uk)
    for p in (0, 5, 11):
        for d in range(3):
            A = o.cheb(d, p)
            f = np.exp(-(s[p] * b[d]) ** 2 * (uk[:, None] - uk[None, :]) ** 2)
            rec = Tk.T @ A @ Tk
            assert np.max(np.abs(rec - f)) < 1e-13
            # f(u,v) = f(-u,-v) = f(v,u): odd total degree vanishes, matrix symmetric
            odd = (np.add.outer(np.arange(n), np.arange(n)) % 2) == 1
            assert np.max(np.abs(A[odd])) < 1e-14 * np.abs(A).max()
            assert np.max(np.abs(A - A.T)) < 1e-14 * np.abs(A).max()


def test_cheb_interpolant_converges_off_grid():
    rng = np.random.default_rng(0)
    u, v = rng.uniform(-1, 1, 200), rng.uniform(-1, 1, 200)
    errs = []
    for n in (8, 16, 32):
        o = small_mol(n=n, P=8, omega=0.3)
        lo, hi = o.box()
        b = 0.5 * (hi[0] - lo[0])
        s, _ = o.nodes()
        A = o.cheb(0, 7)
        approx = np.einsum("ai,ab,bi->i", cheb_T(n, u), A, cheb_T(n, v))
        exact = np.exp(-(s[7] * b) ** 2 * (u - v) ** 2)
        errs.append(np.max(np.abs(approx - exact)))
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 1e-12


# ------------------------------------------------------------------ eq. defV ----

def quad_moment(o, mu, nu, d, j1, j2):
    c1, p1, e1, _ = o.basis_function(mu)
    c2, p2, e2, _ = o.basis_function(nu)
    lo, hi = o.box()
    cen, half = 0.5 * (lo[d] + hi[d]), 0.5 * (hi[d] - lo[d])
    a, b = e1[j1], e2[j2]
    A, B = c1[d], c2[d]
    p = a + b
    P = (a * A + b * B) / p
    out = []
    for m in range(o.n):
        f = lambda x: (x - A) ** p1[d] * (x - B) ** p2[d] * math.exp(-a * (x - A) ** 2 - b * (x - B) ** 2) * \
            math.cos(m * math.acos(max(-1.0, min(1.0, (x - cen) / half))))
        pts = [x for x in (P - 3 / math.sqrt(p), P, P + 3 / math.sqrt(p)) if lo[d] < x < hi[d]]
        val, _ = integrate.quad(f, lo[d], hi[d], points=pts or None, limit=400, epsabs=0, epsrel=1e-13)
        out.append(val)
    return np.array(out)


def test_moments_match_scipy_quad():
    """Moments of p/d pairs, including Gaussians cut by a small box, against QUADPACK."""
    centers = ((0.0, 0.2, -0.3), (1.3, -0.5, 0.9), (0.4, 0.4, 0.4))
    o = small_mol(ls=(1, 2, 0), nprim=(2, 1, 2), exps=(0.9, 0.15, 2.5, 40.0, 0.3), coefs=(0.6, 0.4, 1.0, 0.5, 0.5),
                  centers=centers, n=12, P=4, box=((-2.0, -2.5, -1.5), (2.5, 2.0, 2.0)))
    rng = np.random.default_rng(1)
    for _ in range(8):
        mu, nu = rng.integers(0, o.nbf, 2)
        d = int(rng.integers(0, 3))
        W = o.moments(int(mu), int(nu), d)
        k2 = len(o.basis_function(int(nu))[2])
        for j in range(W.shape[0]):
            ref = quad_moment(o, int(mu), int(nu), d, j // k2, j % k2)
            scale = np.max(np.abs(ref))
            assert np.max(np.abs(W[j] - ref)) <= 1e-12 * scale + 1e-300


@pytest.mark.parametrize("half", [2.5, 25.0])
def test_moments_match_scipy_quad_high_order(half):
    """The same at the highest orders the library takes (n = 64, T_63 oscillating across the box),
    in a small box that cuts diffuse functions and in a large one, with exponents from 0.05 to 800."""
    centers = ((0.0, 0.3, -0.2), (0.8, -0.6, 0.5))
    box = ((-half, -half, -half), (half, half, half))
    o = small_mol(ls=(2, 1), nprim=(2, 2), exps=(800.0, 0.05, 3.0, 0.3), coefs=(0.5, 0.5, 0.7, 0.3),
                  centers=centers, n=64, P=2, box=box)
    rng = np.random.default_rng(7)
    checked = 0
    for _ in range(3):
        mu, nu = (int(x) for x in rng.integers(0, o.nbf, 2))
        d = int(rng.integers(0, 3))
        W = o.moments(mu, nu, d)
        k2 = len(o.basis_function(nu)[2])
        for j in range(W.shape[0]):
            ref = quad_moment(o, mu, nu, d, j // k2, j % k2)
            scale = np.max(np.abs(ref))
            assert np.max(np.abs(W[j] - ref)) <= 1e-12 * scale, (mu, nu, d, j)
            checked += 1
    assert checked >= 6


def test_moments_closed_form_inside_box():
    """A Gaussian pair deep inside the box: int e^{-p(x-P)^2} K_AB T_m((x-c)/b) for m = 0, 1, 2
    equals K_AB sqrt(pi/p) (1, (P-c)/b, 2((P-c)^2 + 1/(2p))/b^2 - 1)."""
    o = small_mol(exps=(3.0, 5.0), n=4, P=2)
    lo, hi = o.box()
    for d in range(3):
        W = o.moments(0, 1, d)[0]
        c1, _, e1, _ = o.basis_function(0)
        c2, _, e2, _ = o.basis_function(1)
        a, b = e1[0], e2[0]
        p = a + b
        P = (a * c1[d] + b * c2[d]) / p
        K = math.exp(-a * b / p * (c1[d] - c2[d]) ** 2)
        cen, half = 0.5 * (lo[d] + hi[d]), 0.5 * (hi[d] - lo[d])
        m0 = K * math.sqrt(math.pi / p)
        assert abs(W[0] - m0) < 1e-14 * m0
        assert abs(W[1] - m0 * (P - cen) / half) < 1e-14 * m0
        assert abs(W[2] - m0 * (2 * ((P - cen) ** 2 + 1 / (2 * p)) / half ** 2 - 1)) < 1e-14 * m0


# ------------------------------------------------ Theorem 1 / Algorithm 1 ----

def test_entries_match_closed_form_contracted_s():
    """Contracted s functions, generous box, high (n, P): Algorithm 1 -> erf-Boys closed form."""
    centers = ((0.0, 0.0, 0.0), (1.1, 0.4, -0.7), (-0.6, 0.9, 0.5))
    o = small_mol(ls=(0, 0, 0), nprim=(2, 1, 2), exps=(0.8, 2.0, 1.5, 1.1, 3.0), coefs=(0.7, 0.3, 1.0, 0.5, 0.5),
                  centers=centers, omega=0.3, n=32, P=24)
    raw = [((0.8, 2.0), (0.7, 0.3)), ((1.5,), (1.0,)), ((1.1, 3.0), (0.5, 0.5))]
    bf = [(centers[i], (0, 0, 0), raw[i][0], raw[i][1]) for i in range(3)]
    for q in itertools.product(range(3), repeat=4):
        ref = cf.contracted_entry([bf[i] for i in q], 0.3)
        assert abs(o.entry(*q) - ref) <= 1e-12 * abs(ref)


def test_entries_match_closed_form_p_and_d():
    """p and d functions via derivatives of the s closed form with respect to the centres."""
    centers = ((0.0, 0.0, 0.0), (0.9, -0.3, 0.5))
    exps = (1.2, 0.9)
    o = small_mol(ls=(1, 2), nprim=(1, 1), exps=exps, coefs=(1.0, 1.0), centers=centers, omega=0.25, n=40, P=24)
    comps = [(0, pw) for pw in cf.cart_components(1)] + [(1, pw) for pw in cf.cart_components(2)]
    bf = [(centers[s], pw, (exps[s],), (1.0,)) for s, pw in comps]
    rng = np.random.default_rng(3)
    quads = []
    while len(quads) < 10:  # total Cartesian power <= 4 keeps mpmath's derivative stencils small
        q = tuple(int(v) for v in rng.integers(0, len(bf), 4))
        if sum(sum(bf[i][1]) for i in q) <= 4:
            quads.append(q)
    quads += [(0, 3, 1, 8), (3, 6, 8, 2), (4, 0, 8, 0), (3, 3, 1, 1)]
    for q in quads:
        ref = cf.contracted_entry([bf[i] for i in q], 0.25)
        got = o.entry(*q)
        assert abs(got - ref) <= 1e-9 * max(abs(ref), 1e-3), (q, got, ref)


def test_brute_force_box_truncated_6d():
    """A box that cuts the Gaussians: Algorithm 1 equals the box-truncated 6D integral of the
    exact erf kernel, done by a 16^6-point tensor Gauss-Legendre rule (eq. compact)."""
    centers = ((0.2, -0.1, 0.3), (-0.4, 0.5, -0.2))
    box = ((-1.2, -1.0, -1.1), (1.0, 1.3, 0.9))
    exps = (0.6, 0.9)
    o = small_mol(exps=exps, centers=centers, omega=0.7, n=24, P=32, box=box)
    z, w = np.polynomial.legendre.leggauss(16)
    lo, hi = np.array(box[0]), np.array(box[1])
    X = [0.5 * (hi[d] - lo[d]) * z + 0.5 * (hi[d] + lo[d]) for d in range(3)]
    W = [0.5 * (hi[d] - lo[d]) * w for d in range(3)]
    gx = np.stack(np.meshgrid(*X, indexing="ij"), -1).reshape(-1, 3)
    wx = np.einsum("i,j,k->ijk", *W).reshape(-1)
    N = [(2 * e / math.pi) ** 0.75 for e in exps]
    g = [N[i] * np.exp(-exps[i] * ((gx - np.array(centers[i])) ** 2).sum(1)) for i in range(2)]
    r = np.sqrt(((gx[:, None, :] - gx[None, :, :]) ** 2).sum(-1))
    with np.errstate(invalid="ignore", divide="ignore"):
        K = np.where(r > 0, special.erf(0.7 * r) / np.where(r > 0, r, 1), 2 * 0.7 / math.sqrt(math.pi))
    for q in [(0, 0, 0, 0), (0, 1, 0, 1), (0, 0, 1, 1), (1, 1, 0, 1)]:
        f = wx * g[q[0]] * g[q[1]]
        h = wx * g[q[2]] * g[q[3]]
        ref = f @ K @ h
        assert abs(o.entry(*q) - ref) <= 2e-9 * abs(ref), q


# ----------------------------------------------------------------- invariants ----

@pytest.fixture(scope="module")
def small_B():
    m = synth.workload_small_s()
    o = oracle.Oracle.from_molecule(m)
    return m, o, o.assemble_B()


def test_eightfold_symmetry(small_B):
    m, o, B = small_B
    nb = o.nbf
    T = B.reshape(nb, nb, nb, nb)
    scale = np.abs(B).max()
    for perm in [(1, 0, 2, 3), (0, 1, 3, 2), (2, 3, 0, 1), (3, 2, 1, 0)]:
        assert np.max(np.abs(T - T.transpose(perm))) < 1e-14 * scale


def test_positive_semidefinite(small_B):
    """w_p > 0 and every A^(p) congruent to a Gaussian Gram matrix make B PSD."""
    _, _, B = small_B
    ev = np.linalg.eigvalsh(B)
    assert ev.min() >= -1e-13 * ev.max()


def test_hadamard_form_equals_factored_form(small_B):
    """Theorem 1: Algorithm 1 (Hadamard form) == (omega/sqrt(pi)) sum_p w_p M (A(x)A(x)A) M^T."""
    m, o, B = small_B
    M = o.factor_M()
    s, w = o.nodes()
    Bf = np.zeros_like(B)
    for p in range(o.P):
        K = np.kron(np.kron(o.cheb(0, p), o.cheb(1, p)), o.cheb(2, p))
        Bf += w[p] * (M @ K @ M.T)
    Bf *= o.omega / math.sqrt(math.pi)
    assert np.linalg.norm(Bf - B) <= 1e-13 * np.linalg.norm(B)


def test_jbuild_factored_equals_dense(small_B):
    m, o, B = small_B
    D = synth.random_densities(7, o.nbf, 3)
    J = o.jbuild_factored(D)
    Jd = np.einsum("ij,rj->ri", B, D.reshape(3, -1)).reshape(D.shape)
    assert np.linalg.norm(J - Jd) <= 1e-13 * np.linalg.norm(Jd)
    assert np.max(np.abs(J - J.transpose(0, 2, 1))) <= 1e-14 * np.abs(J).max()


def test_omega_to_zero_limit():
    """B/omega -> (2/sqrt(pi)) O_{mu nu} O_{ka la}, O the overlap (closed form for s functions)."""
    centers = ((0.0, 0.0, 0.0), (1.0, -0.5, 0.3))
    exps = (0.9, 1.7)
    o = small_mol(exps=exps, centers=centers, omega=1e-6, n=8, P=4)
    N = [(2 * e / math.pi) ** 0.75 for e in exps]

    def ov(i, j):
        a, b = exps[i], exps[j]
        r2 = sum((centers[i][d] - centers[j][d]) ** 2 for d in range(3))
        return N[i] * N[j] * (math.pi / (a + b)) ** 1.5 * math.exp(-a * b / (a + b) * r2)

    for q in itertools.product(range(2), repeat=4):
        ref = 2 / math.sqrt(math.pi) * ov(q[0], q[1]) * ov(q[2], q[3])
        assert abs(o.entry(*q) / 1e-6 - ref) <= 1e-10 * ref


def test_axis_permutation():
    """Swapping x and y of every centre (and of the Cartesian powers) in a cube box permutes B."""
    centers = np.array([[0.0, 0.1, 0.2], [0.8, -0.4, 0.3]])
    args = dict(ls=(1, 0), nprim=(1, 2), exps=(0.7, 1.1, 0.4), coefs=(1.0, 0.6, 0.4), omega=0.4, n=16, P=12)
    box = ((-6.0, -6.0, -6.0), (6.0, 6.0, 6.0))
    o1 = small_mol(centers=centers, box=box, **args)
    o2 = small_mol(centers=centers[:, [1, 0, 2]], box=box, **args)
    perm = [1, 0, 2, 3]  # p_x <-> p_y, s unchanged
    for q in itertools.product(range(4), repeat=4):
        a = o1.entry(*q)
        b = o2.entry(*[perm[i] for i in q])
        assert abs(a - b) <= 1e-14 * max(abs(a), 1e-300) + 1e-18


# ------------------------------------------------- screening (Section 6, compression) ----

def _screened(a, A, b, B, tau):
    """The screening criterion of Section 6 for one primitive pair, written out here:
    exp(-a b / (a + b) |A - B|^2) <= tau."""
    d2 = sum((A[l] - B[l]) ** 2 for l in range(3))
    return tau > 0 and math.exp(-(a * b / (a + b)) * d2) <= tau


def test_screening_discards_exactly_the_far_pair():
    """Two one-primitive s functions 4 bohr apart, exponents 2 and 3: overlap factor
    exp(-1.2 * 16) = 4.6e-9.  Above that tau, screening removes the pair's only term: every entry
    with (0,1) or (1,0) in either slot is exactly 0 and every other entry is unchanged bit for
    bit; below it, or with tau = 0, nothing changes."""
    kw = dict(ls=(0, 0), nprim=(1, 1), exps=(2.0, 3.0), coefs=(1.0, 1.0),
              centers=((0.0, 0.0, 0.0), (4.0, 0.0, 0.0)), omega=0.4, n=16, P=16)
    B0 = small_mol(**kw).assemble_B(threads=1)
    cross = [1, 2]  # rows / columns mu * 2 + nu of the pairs (0, 1) and (1, 0)
    keep = [0, 3]
    assert np.all(B0[np.ix_(cross, cross)] != 0.0)
    for tau, discard in ((1e-8, True), (1e-9, False), (0.0, False)):
        B = small_mol(tau=tau, **kw).assemble_B(threads=1)
        assert np.array_equal(B[np.ix_(keep, keep)], B0[np.ix_(keep, keep)])
        if discard:
            assert np.all(B[cross, :] == 0.0) and np.all(B[:, cross] == 0.0)
        else:
            assert np.array_equal(B, B0)


def test_screening_contracted_matches_closed_form_over_kept_pairs():
    """Contracted s functions with a spread of exponents, tau = 1e-3: some primitive pairs of
    distinct centres are discarded.  Every entry equals the erf-Boys closed form summed over the
    kept primitive pairs only (the criterion evaluated here, independently of the oracle)."""
    centers = ((0.0, 0.0, 0.0), (1.6, 0.4, -0.7), (-0.6, 1.2, 0.5))
    raw = [((0.8, 6.0), (0.7, 0.3)), ((1.5, 9.0), (1.0, 0.4)), ((1.1, 3.0), (0.5, 0.5))]
    tau, omega = 1e-3, 0.3
    o = small_mol(ls=(0, 0, 0), nprim=(2, 2, 2), exps=tuple(e for r in raw for e in r[0]),
                  coefs=tuple(c for r in raw for c in r[1]), centers=centers, omega=omega, n=32, P=24, tau=tau)
    bf = [(centers[i], (0, 0, 0), raw[i][0], raw[i][1]) for i in range(3)]
    flags = [_screened(a, centers[i], b, centers[j], tau) for i in range(3) for j in range(3)
             for a in raw[i][0] for b in raw[j][0]]
    assert any(flags) and not all(flags)

    def screened_entry(bf4):
        cs = [cf.contracted_coefs(e, c, pw) for (_, pw, e, c) in bf4]
        total = 0.0
        for ks in itertools.product(*[range(len(b[2])) for b in bf4]):
            ex = [bf4[f][2][ks[f]] for f in range(4)]
            if _screened(ex[0], bf4[0][0], ex[1], bf4[1][0], tau) or _screened(ex[2], bf4[2][0], ex[3], bf4[3][0], tau):
                continue
            coef = 1.0
            for f in range(4):
                coef *= cs[f][ks[f]]
            total += coef * cf.cart_erf(ex, [bf4[f][0] for f in range(4)], [bf4[f][1] for f in range(4)], omega)
        return total

    for q in itertools.product(range(3), repeat=4):
        ref = screened_entry([bf[i] for i in q])
        assert abs(o.entry(*q) - ref) <= 1e-12 * abs(ref), q


# ------------------------------------- Khatri-Rao low-rank compression (Section 6) ----

def _kr_mol():
    m = synth.random_molecule(4101, natoms=2, cube=3.0, nprim=2, alpha_range=(0.2, 20.0), omega=0.4, n=8, P=8)
    return oracle.Oracle.from_molecule(m)


def test_khatri_rao_full_rank_is_the_factored_form():
    """With R_d = n the compressed form (eq. approxepsilon) is the factored form: it reproduces
    Algorithm 1's B (the oracle's assemble_B) to rounding."""
    from oracle import kr
    o = _kr_mol()
    B = o.assemble_B(threads=1)
    Bk = kr.compressed_B(o, (o.n, o.n, o.n))
    assert np.linalg.norm(Bk - B) <= 1e-12 * np.linalg.norm(B)


@pytest.mark.parametrize("ranks", [(6, 6, 6), (5, 7, 4), (3, 3, 3)])
def test_khatri_rao_truncation_is_a_projection_of_the_factored_form(ranks):
    """Truncated ranks: U^(d) = W~^(d) V^(d), so the compressed F_u is F_u (x)_d V^(d) V^(d)T and
    B_KR = (omega / sqrt(pi)) F Pi K Pi F^T with Pi = (x)_d V V^T and K = sum_p w_p (x)_d A_d^(p).
    Checked against that product built from the C oracle's F_u (factor_M) and its factors, a route
    that shares nothing with the compressed one but the SVD; the error shrinks as the ranks grow."""
    from oracle import kr
    o = _kr_mol()
    n = o.n
    S, _, _ = kr.moment_rows(o)
    V = [kr.truncated_factors(S[d], ranks[d])[1] for d in range(3)]
    Pi = np.kron(V[0] @ V[0].T, np.kron(V[1] @ V[1].T, V[2] @ V[2].T))
    _, w = o.nodes()
    K = sum(w[p] * np.kron(o.cheb(0, p), np.kron(o.cheb(1, p), o.cheb(2, p))) for p in range(o.P))
    M = o.factor_M(threads=1)  # rows mu N_b + nu, n^3 columns
    ref = o.omega / np.sqrt(np.pi) * M @ Pi @ K @ Pi @ M.T
    Bk = kr.compressed_B(o, ranks)
    assert np.linalg.norm(Bk - ref) <= 1e-12 * np.linalg.norm(ref)
    B = o.assemble_B(threads=1)
    e_trunc = np.linalg.norm(Bk - B) / np.linalg.norm(B)
    e_more = np.linalg.norm(kr.compressed_B(o, tuple(min(n, r + 1) for r in ranks)) - B) / np.linalg.norm(B)
    assert 0 < e_more < e_trunc


def test_khatri_rao_pin_catches_a_planted_mistake(monkeypatch):
    """The projection pin above fails when U^(d) loses its singular values (u instead of u sigma),
    a plausible slip in eq. SVD."""
    from oracle import kr
    o = _kr_mol()
    ranks = (6, 6, 6)
    good = kr.compressed_B(o, ranks)

    def no_sigma(S, rank):
        u, sv, vt = np.linalg.svd(S, full_matrices=False)
        return u[:, :rank], vt[:rank].T, sv

    monkeypatch.setattr(kr, "truncated_factors", no_sigma)
    bad = kr.compressed_B(o, ranks)
    assert np.linalg.norm(bad - good) > 1e-3 * np.linalg.norm(good)


# ------------------------------------------ long-range exchange (appendix, eq. exchange) ----

def test_exchange_factored_equals_direct():
    """The appendix's factored exchange (through M and the node sum K) equals eq. exchange
    evaluated on Algorithm 1's B, for three orbitals of a contracted s/p/d molecule."""
    from oracle import exchange
    m = synth.random_molecule(4102, natoms=2, cube=3.0, nprim=2, alpha_range=(0.2, 20.0), omega=0.4, n=8, P=8)
    o = oracle.Oracle.from_molecule(m)
    Q = np.random.default_rng(5).standard_normal((3, o.nbf))
    Kd = exchange.exchange_direct(o, Q, threads=1)
    Kf = exchange.exchange_factored(o, Q, threads=1)
    assert np.linalg.norm(Kf - Kd) <= 1e-12 * np.linalg.norm(Kd)
    assert np.allclose(Kd, Kd.T, rtol=0, atol=1e-14 * np.abs(Kd).max())


def test_exchange_matches_closed_form_contracted_s():
    """Contracted s functions, two orbitals: eq. exchange against the erf-Boys closed forms,
    K(mu, nu) = 2 sum_j sum_{lambda, kappa} q_{j lambda} q_{j kappa} (mu lambda | kappa nu)."""
    from oracle import exchange
    centers = ((0.0, 0.0, 0.0), (1.1, 0.4, -0.7), (-0.6, 0.9, 0.5))
    raw = [((0.8, 2.0), (0.7, 0.3)), ((1.5,), (1.0,)), ((1.1, 3.0), (0.5, 0.5))]
    o = small_mol(ls=(0, 0, 0), nprim=(2, 1, 2), exps=(0.8, 2.0, 1.5, 1.1, 3.0), coefs=(0.7, 0.3, 1.0, 0.5, 0.5),
                  centers=centers, omega=0.3, n=32, P=24)
    bf = [(centers[i], (0, 0, 0), raw[i][0], raw[i][1]) for i in range(3)]
    Q = np.array([[0.6, -0.3, 0.5], [0.2, 0.8, -0.4]])
    ints = np.zeros((3, 3, 3, 3))
    for q in itertools.product(range(3), repeat=4):
        ints[q] = cf.contracted_entry([bf[i] for i in q], 0.3)
    ref = np.zeros((3, 3))
    for mu, nu in itertools.product(range(3), repeat=2):
        ref[mu, nu] = 2.0 * sum(Q[j, l] * Q[j, k] * ints[mu, l, k, nu] for j in range(2) for l in range(3)
                                for k in range(3))
    got = exchange.exchange_direct(o, Q, threads=1)
    assert np.max(np.abs(got - ref)) <= 1e-11 * np.abs(ref).max()


def test_exchange_single_function_is_twice_J():
    """One basis function, one orbital q: K = 2 q q B(00,00) and J(D = q^2) = q^2 B(00,00), so
    K = 2 J (the factor 2 and the orbital sum of eq. exchange)."""
    from oracle import exchange
    o = small_mol(ls=(0,), nprim=(2,), exps=(0.9, 2.5), coefs=(0.6, 0.5), centers=((0.2, -0.1, 0.3),),
                  omega=0.4, n=16, P=16)
    q = 0.7
    K = exchange.exchange_factored(o, np.array([[q]]), threads=1)
    J = o.jbuild_factored(np.array([[[q * q]]]), threads=1)
    assert abs(K[0, 0] - 2.0 * J.reshape(-1)[0]) <= 1e-14 * abs(K[0, 0])
