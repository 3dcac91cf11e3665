"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle, element by element.

Tolerances (relative Frobenius norm unless stated):
  FP64 path       1e-12   (both forms of Theorem 1)
  FP32 CUDA-core  1e-5
Sizes: the small s-only workload in full, scaled-down s/p/d contracted instances (several
tiles and a ragged tail), and sampled rows of the full-size 180-function instance.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2210_13069_gb300 import synth

pytestmark = pytest.mark.gpu


def rel_fro(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def lib():
    import torch
    from paper_2210_13069_gb300 import build_lib, lrtei
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build_lib.build()
    lrtei.load()
    return lrtei


def mol_spd_small(seed=2001, natoms=2, nprim=3, n=12, P=12, omega=0.4):
    return synth.random_molecule(seed, natoms=natoms, cube=4.0, nprim=nprim, alpha_range=(0.1, 50.0), omega=omega,
                                 n=n, P=P)


def mol_ragged(seed=2002):
    """Shells with different contraction lengths (ragged I_mu I_nu) and l up to 2; N_b = 45."""
    m = synth.random_molecule(seed, natoms=3, cube=5.0, nprim=2, alpha_range=(0.2, 30.0), omega=0.5, n=10, P=10)
    rng = np.random.default_rng(seed)
    for i, sh in enumerate(m.shells):
        k = 1 + (i % 3)
        sh.exps = np.sort(np.exp(rng.uniform(np.log(0.2), np.log(30.0), size=k)))[::-1].copy()
        sh.coefs = rng.uniform(0.1, 1.0, size=k)
    return m


@pytest.mark.parametrize("form", ["hadamard", "factored"])
def test_small_s_full_B_fp64(lib, form):
    m = synth.workload_small_s()
    ref = oracle.Oracle.from_molecule(m).assemble_B()
    pl = lib.Plan(m, "fp64")
    B = pl.assemble_B(form).cpu().numpy()
    pl.status()
    assert rel_fro(B, ref) <= 1e-12
    assert np.max(np.abs(B - ref)) <= 1e-12 * np.abs(ref).max()


def test_factors_match_oracle(lib):
    m = mol_ragged()
    o = oracle.Oracle.from_molecule(m)
    pl = lib.Plan(m, "fp64")
    S, C, s, w, c = [t.cpu().numpy() for t in pl.factors()]
    so, wo = o.nodes()
    assert np.max(np.abs(s - so)) <= 1e-15 * m.omega
    assert np.max(np.abs(w - wo) / wo) <= 1e-13
    for d in range(3):
        for p in range(m.P):
            A = o.cheb(d, p)
            assert np.max(np.abs(C[d, p] - A)) <= 1e-14 * np.abs(A).max()
    # moments: rows ordered by unique pair (mu <= nu) then j = j1 * I_nu + j2
    nbf = m.nbf
    row = 0
    for mu in range(nbf):
        for nu in range(mu, nbf):
            Wd = [o.moments(mu, nu, d) for d in range(3)]
            I = Wd[0].shape[0]
            for d in range(3):
                got = S[d, row:row + I]
                scale = np.abs(Wd[d]).max(axis=1, keepdims=True)
                assert np.all(np.abs(got - Wd[d]) <= 1e-13 * scale + 1e-300), (mu, nu, d)
            row += I
    assert row == S.shape[1]


def mol_high_order(n, P, half, seed=2100):
    """Two atoms with an s, a p and a d shell each (N_b = 20), exponents from 0.05 to 800, in an
    explicit cube of half-width `half` around the atoms' centre (2.5 bohr cuts the diffuse
    functions; 25 bohr holds them), at the Chebyshev and quadrature orders the selector reaches."""
    m = synth.random_molecule(seed, natoms=2, cube=1.5, shells_per_atom=(("s", 1), ("p", 1), ("d", 1)), nprim=2,
                              alpha_range=(0.05, 800.0), omega=0.6, n=n, P=P)
    c = m.atoms.mean(axis=0)
    m.box_lo, m.box_hi = c - half, c + half
    return m


@pytest.mark.parametrize("n,P,half", [(40, 96, 2.5), (40, 96, 25.0), (56, 128, 2.5), (64, 128, 25.0)])
def test_factors_and_B_rows_at_high_orders(lib, n, P, half):
    """Nodes, weights, Chebyshev coefficients and every moment row against the oracle (pinned at
    n = 64 by QUADPACK) at n = 40..64 and P = 96..128, and sampled rows of the FP64 B within 1e-12:
    by both forms at n = 40, by the Hadamard form above (the FP64 factored form's mode products
    cost 6 P n^4 per row: minutes at n = 64)."""
    m = mol_high_order(n, P, half)
    o = oracle.Oracle.from_molecule(m)
    pl = lib.Plan(m, "fp64")
    S, C, s, w, c = [t.cpu().numpy() for t in pl.factors()]
    so, wo = o.nodes()
    e_s = float(np.max(np.abs(s - so)) / m.omega)
    # weights: relative to the bound one ulp of a node sets next to z = +-1 (the oracle's pin
    # against 40-digit roots uses the same bound, 2e-14 + 4e-16 / (1 - |z|)), for both sides
    z = 2.0 * so / m.omega - 1.0
    e_w = float(np.max(np.abs(w - wo) / wo / (2.0 * (2e-14 + 4e-16 / (1.0 - np.abs(z))))))
    worst_c = 0.0
    for d in range(3):
        for p in range(m.P):
            A = o.cheb(d, p)
            worst_c = max(worst_c, np.max(np.abs(C[d, p] - A)) / np.abs(A).max())
    worst_s, row = 0.0, 0
    for mu in range(m.nbf):
        for nu in range(mu, m.nbf):
            Wd = [o.moments(mu, nu, d) for d in range(3)]
            I = Wd[0].shape[0]
            for d in range(3):
                scale = np.abs(Wd[d]).max(axis=1)
                worst_s = max(worst_s, float(np.max(np.abs(S[d, row:row + I] - Wd[d]).max(axis=1) / scale)))
            row += I
    rows = [0, 7 * m.nbf + 12, (m.nbf - 1) * m.nbf + m.nbf - 1]
    ref = o.B_rows(rows)
    errs = {}
    for form in ("hadamard", "factored") if n <= 40 else ("hadamard",):
        B = pl.assemble_B(form)
        errs[form] = rel_fro(B[rows].cpu().numpy(), ref)
        del B
    pl.status()
    print(f"n={n} P={P} box half-width {half}: nodes {e_s:.1e}, weights {e_w:.2f} of the bound, Chebyshev coefficients "
          f"{worst_c:.1e}, moments {worst_s:.1e} (of each row's maximum), B rows "
          + ", ".join(f"{k} {v:.1e}" for k, v in errs.items()), flush=True)
    assert e_s <= 1e-15 and e_w <= 1.0
    assert worst_c <= 1e-14
    assert worst_s <= 1e-13
    assert max(errs.values()) <= 1e-12
    pl.close()


@pytest.mark.parametrize("form", ["hadamard", "factored"])
def test_contracted_spd_full_B_fp64(lib, form):
    m = mol_spd_small()
    ref = oracle.Oracle.from_molecule(m).assemble_B()
    pl = lib.Plan(m, "fp64")
    B = pl.assemble_B(form).cpu().numpy()
    assert rel_fro(B, ref) <= 1e-12


@pytest.mark.parametrize("form", ["hadamard", "factored"])
def test_ragged_full_B_fp64(lib, form):
    """N_b = 45 -> 1035 unique pairs: spans many 64-wide GEMM tiles with a ragged tail."""
    m = mol_ragged()
    ref = oracle.Oracle.from_molecule(m).assemble_B()
    pl = lib.Plan(m, "fp64")
    B = pl.assemble_B(form).cpu().numpy()
    assert rel_fro(B, ref) <= 1e-12
    assert pl.info["npair"] == 1035


def test_entries_algorithm1(lib):
    m = mol_ragged()
    o = oracle.Oracle.from_molecule(m)
    rng = np.random.default_rng(5)
    idx = rng.integers(0, m.nbf, size=(3000, 4)).astype(np.int32)
    ref = o.entries(idx)
    pl = lib.Plan(m, "fp64")
    got = pl.entries(idx).cpu().numpy()
    assert rel_fro(got, ref) <= 1e-12
    scale = np.abs(ref).max()
    assert np.max(np.abs(got - ref)) <= 1e-12 * scale


def test_entries_empty_and_single_function(lib):
    import torch
    m = synth.random_molecule(9, natoms=1, cube=1.0, shells_per_atom=(("s", 1),), nprim=1, alpha_range=(0.5, 0.5),
                              omega=0.3, n=6, P=4)
    pl = lib.Plan(m, "fp64")
    assert pl.nbf == 1
    out = torch.empty(0, dtype=torch.float64, device="cuda")
    idx = torch.empty((0, 4), dtype=torch.int32, device="cuda")
    lib.lrtei_entries(pl.plan, idx, 0, out)
    B = pl.assemble_B("hadamard").cpu().numpy()
    ref = oracle.Oracle.from_molecule(m).assemble_B()
    assert rel_fro(B, ref) <= 1e-13


def test_explicit_box_and_n1_P1(lib):
    """Degenerate orders n = 1, P = 1 and an explicit, non-cubic box."""
    m = mol_spd_small(n=1, P=1)
    m.box_lo = np.array([-3.0, -2.5, -4.0])
    m.box_hi = np.array([7.0, 6.5, 5.0])
    ref = oracle.Oracle.from_molecule(m).assemble_B()
    pl = lib.Plan(m, "fp64")
    for form in ("hadamard", "factored"):
        B = pl.assemble_B(form).cpu().numpy()
        assert rel_fro(B, ref) <= 1e-12


def test_jbuild_fp64(lib):
    import torch
    m = mol_ragged()
    o = oracle.Oracle.from_molecule(m)
    D = synth.random_densities(11, m.nbf, 5)
    ref = o.jbuild_factored(D)
    pl = lib.Plan(m, "fp64")
    J = pl.jbuild(torch.as_tensor(D, device="cuda")).cpu().numpy()
    assert rel_fro(J, ref) <= 1e-12
    assert np.max(np.abs(J - J.transpose(0, 2, 1))) <= 1e-14 * np.abs(J).max()


def test_fp32_path_error_stated(lib):
    m = mol_spd_small()
    ref = oracle.Oracle.from_molecule(m).assemble_B()
    pl = lib.Plan(m, "fp32")
    B = pl.assemble_B("factored").cpu().numpy()
    err = rel_fro(B, ref)
    print(f"fp32 CUDA-core factored form: rel. Frobenius error {err:.3e}")
    assert err <= 1e-5


def test_full_size_180_sampled_rows(lib):
    """The 180-function s/p/d instance at full size: sampled rows of B_u, both forms."""
    m = synth.workload_spd()
    o = oracle.Oracle.from_molecule(m)
    pl = lib.Plan(m, "fp64")
    nbf = m.nbf
    rng = np.random.default_rng(17)
    picks = [(0, 0), (int(rng.integers(0, nbf)), int(rng.integers(0, nbf))), (nbf - 1, nbf - 1)]
    for mu, nu in picks:
        mu, nu = min(mu, nu), max(mu, nu)
        r = mu * nbf - mu * (mu - 1) // 2 + (nu - mu)
        full = o.B_rows([mu * nbf + nu])[0]
        # unique columns in pair order
        cols = [ka * nbf + la for ka in range(nbf) for la in range(ka, nbf)]
        ref = full[cols]
        for form in ("hadamard", "factored"):
            got = pl.Bu_rows(r, r + 1, form).cpu().numpy()[0]
            assert rel_fro(got, ref) <= 1e-12, (mu, nu, form)


# ------------------------------------------------------------------ tensor-core (split BF16) path

@pytest.mark.parametrize("maker", ["small_s", "spd_small", "ragged"])
def test_split_f16_full_B(lib, maker):
    """tcgen05 path (8+12+12-bit integer slices, exact leading products): rel. Frobenius <= 1e-7."""
    m = {"small_s": synth.workload_small_s, "spd_small": mol_spd_small, "ragged": mol_ragged}[maker]()
    ref = oracle.Oracle.from_molecule(m).assemble_B()
    pl = lib.Plan(m, "split_f16")
    B = pl.assemble_B("auto").cpu().numpy()
    pl.status()
    err = rel_fro(B, ref)
    print(f"split_f16 {maker}: N_b={m.nbf} rel. Frobenius error {err:.3e}")
    assert err <= 1e-7
    # the factored form on the tensor cores is exactly symmetric (mirrored tiles)
    assert np.array_equal(B, B.T)


@pytest.mark.parametrize("maker", ["small_s", "spd_small", "ragged"])
def test_split_f16_8_full_B(lib, maker):
    """Eight products in three accumulators (the next-order slice products kept, the small terms
    accumulated at their own scale): rel. Frobenius <= 1e-8, B exactly symmetric."""
    m = {"small_s": synth.workload_small_s, "spd_small": mol_spd_small, "ragged": mol_ragged}[maker]()
    ref = oracle.Oracle.from_molecule(m).assemble_B()
    pl = lib.Plan(m, "split_f16_8")
    B = pl.assemble_B("auto").cpu().numpy()
    pl.status()
    err = rel_fro(B, ref)
    print(f"split_f16_8 {maker}: N_b={m.nbf} rel. Frobenius error {err:.3e}")
    assert err <= 1e-8
    assert np.array_equal(B, B.T)


@pytest.mark.parametrize("cfg", ["0", "1"])
def test_split_f16_8_each_tile_config_and_jbuild(lib, cfg, monkeypatch):
    """The eight-product kernel configurations (128x64 tiles for B and for J-builds of 40
    densities, 128x32 for 7 densities, both K depths) on the ragged 45-function instance."""
    import torch
    monkeypatch.setenv("LRTEI_TC_CONFIG", cfg)
    m = mol_ragged()
    o = oracle.Oracle.from_molecule(m)
    pl = lib.Plan(m, "split_f16_8")
    B = pl.assemble_B().cpu().numpy()
    pl.status()
    assert rel_fro(B, o.assemble_B()) <= 1e-8
    for R in (40, 7):
        D = synth.random_densities(14, m.nbf, R)
        J = pl.jbuild(torch.as_tensor(D, device="cuda")).cpu().numpy()
        err = rel_fro(J, o.jbuild_factored(D))
        print(f"split_f16_8 J-build R={R}: {err:.3e}")
        assert err <= 1e-8, R


@pytest.mark.parametrize("maker", ["spd_small", "ragged"])
def test_plain_bf16_error_stated(lib, maker):
    """Plain BF16 operands with FP32 accumulation: rel. Frobenius <= 1e-3."""
    m = {"spd_small": mol_spd_small, "ragged": mol_ragged}[maker]()
    ref = oracle.Oracle.from_molecule(m).assemble_B()
    pl = lib.Plan(m, "bf16")
    B = pl.assemble_B().cpu().numpy()
    err = rel_fro(B, ref)
    print(f"plain bf16 {maker}: rel. Frobenius error {err:.3e}")
    assert err <= 1e-3


def test_split_f16_jbuild(lib):
    import torch
    m = mol_ragged()
    o = oracle.Oracle.from_molecule(m)
    D = synth.random_densities(12, m.nbf, 7)
    ref = o.jbuild_factored(D)
    pl = lib.Plan(m, "split_f16")
    J = pl.jbuild(torch.as_tensor(D, device="cuda")).cpu().numpy()
    pl.status()
    err = rel_fro(J, ref)
    print(f"split_f16 J-build: rel. Frobenius error {err:.3e}")
    assert err <= 1e-7


def test_split_f16_full_size_180(lib):
    """Full-size 180-function instance: sampled rows of B (tensor-core row path and the full
    symmetric assembly) against the oracle, the banded assembly into pinned host memory against
    the device one (bit for bit), the whole B against the FP64 GPU path (within 1e-12 of the
    oracle on sampled rows above), and a 32-density J-build against the FP64 GPU path."""
    import torch
    m = synth.workload_spd()
    o = oracle.Oracle.from_molecule(m)
    nbf = m.nbf
    pl = lib.Plan(m, "split_f16")
    full = pl.assemble_B()
    rng = np.random.default_rng(23)
    picks = [(0, 0), (int(rng.integers(0, nbf)), int(rng.integers(0, nbf))), (nbf - 1, nbf - 1), (3, 170)]
    cols = [ka * nbf + la for ka in range(nbf) for la in range(ka, nbf)]
    refs, rows_tc, rows_full = [], [], []
    for mu, nu in picks:
        mu, nu = min(mu, nu), max(mu, nu)
        r = mu * nbf - mu * (mu - 1) // 2 + (nu - mu)
        ref_full = o.B_rows([mu * nbf + nu])[0]
        refs.append(ref_full)
        rows_tc.append(pl.Bu_rows(r, r + 1).cpu().numpy()[0])
        rows_full.append(full[mu * nbf + nu].cpu().numpy())
    refs = np.array(refs)
    e_rows = rel_fro(np.array(rows_tc), refs[:, cols])
    e_full_rows = rel_fro(np.array(rows_full), refs)
    print(f"split_f16 180 functions, sampled rows: rel. Frobenius {e_rows:.3e} (row path), {e_full_rows:.3e} (assembly)")
    assert e_rows <= 1e-7 and e_full_rows <= 1e-7
    # the same B into pinned host memory (16 bands, copy-engine transfers) is bit-identical
    Bh = torch.empty((nbf * nbf, nbf * nbf), dtype=torch.float64, pin_memory=True)
    pl.assemble_B(out=Bh)
    torch.cuda.synchronize()
    pl.status()
    step = 2048
    for i in range(0, nbf * nbf, step):
        assert torch.equal(full[i:i + step].cpu(), Bh[i:i + step]), i
    del Bh
    p64 = lib.Plan(m, "fp64")
    B64 = p64.assemble_B()
    e_all = float(torch.linalg.norm(full - B64) / torch.linalg.norm(B64))
    print(f"split_f16 180 functions, whole B vs FP64 GPU path: rel. Frobenius {e_all:.3e}")
    assert e_all <= 1e-7
    del full, B64
    D = torch.as_tensor(synth.random_densities(31, nbf, 32), device="cuda")
    J = pl.jbuild(D)
    J64 = p64.jbuild(D)
    err = float(torch.linalg.norm(J - J64) / torch.linalg.norm(J64))
    print(f"split_f16 J-build, 180 functions, 32 densities: rel. error vs FP64 {err:.3e}")
    assert err <= 1e-7


@pytest.mark.parametrize("cfg", ["0", "1", "2"])
def test_split_f16_each_tile_config(lib, cfg, monkeypatch):
    """Every kernel configuration the tuner may pick (64- and 32-deep K stages; 128x128 tiles
    for B, 128x64 and 128x32 tiles for J-builds of 40 and 7 densities; the CTA-pair kernel for the
    non-symmetric G product, configuration 2, which the J-build shapes do not have) gives the same
    accuracy on B and J; the 45-function instance leaves ragged tails in every tile shape."""
    import torch
    monkeypatch.setenv("LRTEI_TC_CONFIG", cfg)
    m = mol_ragged()
    o = oracle.Oracle.from_molecule(m)
    ref = o.assemble_B()
    pl = lib.Plan(m, "split_f16")
    B = pl.assemble_B().cpu().numpy()
    pl.status()
    assert rel_fro(B, ref) <= 1e-7
    assert np.array_equal(B, B.T)
    for R in (40, 7):
        D = synth.random_densities(13, m.nbf, R)
        J = pl.jbuild(torch.as_tensor(D, device="cuda")).cpu().numpy()
        assert rel_fro(J, o.jbuild_factored(D)) <= 1e-7, R


@pytest.mark.parametrize("precision,bands,chunk", [
    ("fp64", None, None), ("split_f16", None, None), ("split_f16_8", None, None), ("bf16", None, None),
    ("split_f16", "1", None), ("split_f16", "3", "7"), ("split_f16_8", "4", "50")])
def test_assemble_B_into_pinned_host_memory(lib, precision, bands, chunk, monkeypatch):
    """B assembled into pinned host memory equals B in device memory, bit for bit: on the
    tensor-core path through bands of the upper triangle (N_b = 45: 1035 unique pairs, nine
    128-row blocks, so the default runs nine bands) with copy-engine transfers of the completed
    rows, also as one band, and as three or four bands with ragged transfer chunks; also with a
    leading dimension above N_b^2.  Pageable host memory is refused before any launch."""
    import torch
    if bands:
        monkeypatch.setenv("LRTEI_HOST_BANDS", bands)
    if chunk:
        monkeypatch.setenv("LRTEI_HOST_CHUNK_ROWS", chunk)
    m = mol_ragged()
    pl = lib.Plan(m, precision)
    Bd = pl.assemble_B().cpu()
    nb2 = m.nbf * m.nbf
    Bh = torch.full((nb2, nb2), float("nan"), dtype=torch.float64, pin_memory=True)
    pl.assemble_B(out=Bh)
    torch.cuda.synchronize()
    pl.status()
    assert torch.equal(Bd, Bh)
    wide = torch.full((nb2, nb2 + 3), float("nan"), dtype=torch.float64, pin_memory=True)
    lib.lrtei_assemble_B(pl.plan, 0, wide, nb2 + 3)
    torch.cuda.synchronize()
    pl.status()
    assert torch.equal(Bd, wide[:, :nb2])
    assert torch.isnan(wide[:, nb2:]).all()
    pageable = torch.empty((nb2, nb2), dtype=torch.float64)
    with pytest.raises(ValueError):
        pl.assemble_B(out=pageable)
    with pytest.raises(lib.LrteiError) as ei:
        lib.lrtei_assemble_B(pl.plan, 0, pageable, nb2)
    assert ei.value.status == 1
    pl.close()


@pytest.mark.parametrize("precision", ["split_f16", "split_f16_8", "bf16"])
@pytest.mark.parametrize("nshell", [1, 2])
def test_tensor_core_paths_on_one_and_few_functions(lib, precision, nshell):
    """Degenerate sizes through the tensor-core GEMMs: one s function (one unique pair, a 1 x 1
    B_u inside a 128 x 128 tile) and an s plus a p shell (N_b = 4); B and a J-build against the
    oracle within the precision's bound."""
    import torch
    shells = [synth.Shell(center=np.array([0.1, -0.2, 0.3]), l=0, exps=np.array([3.0, 0.4]),
                          coefs=np.array([0.6, 0.5]))]
    if nshell == 2:
        shells.append(synth.Shell(center=np.array([1.2, 0.4, -0.7]), l=1, exps=np.array([1.1]),
                                  coefs=np.array([1.0])))
    atoms = np.array([sh.center for sh in shells])
    m = synth.Molecule(atoms=atoms, shells=shells, omega=0.5, n=12, P=16, name=f"tiny{nshell}")
    o = oracle.Oracle.from_molecule(m)
    ref = o.assemble_B()
    pl = lib.Plan(m, precision)
    B = pl.assemble_B().cpu().numpy()
    pl.status()
    tol = {"split_f16": 1e-7, "split_f16_8": 1e-8, "bf16": 1e-3}[precision]
    assert rel_fro(B, ref) <= tol
    D = synth.random_densities(3, m.nbf, 2)
    J = pl.jbuild(torch.as_tensor(D, device="cuda")).cpu().numpy()
    assert rel_fro(J, o.jbuild_factored(D)) <= tol
    pl.close()


@pytest.mark.parametrize("precision", ["fp64", "split_f16", "split_f16_8", "bf16"])
def test_streamed_jbuild_matches_one_pass(lib, precision, monkeypatch):
    """The streamed J-build (F_u built in blocks of unique pairs, node sum by mode products) on
    the ragged 45-function instance, with 200-pair blocks (a ragged last block) and with one
    block: against the one-pass J-build and the oracle."""
    import torch
    m = mol_ragged()
    o = oracle.Oracle.from_molecule(m)
    D = synth.random_densities(21, m.nbf, 9)
    ref = o.jbuild_factored(D)
    tol = {"fp64": 1e-12, "split_f16": 1e-7, "split_f16_8": 1e-8, "bf16": 1e-3}[precision]
    pl = lib.Plan(m, precision)
    Dt = torch.as_tensor(D, device="cuda")
    J1 = pl.jbuild(Dt).cpu().numpy()
    for block in ("200", "5000"):
        monkeypatch.setenv("LRTEI_JBUILD_BLOCK", block)
        J = pl.jbuild(Dt).cpu().numpy()
        pl.status()
        err = rel_fro(J, ref)
        print(f"streamed J-build {precision}, blocks of {block} pairs: {err:.3e} (one pass {rel_fro(J1, ref):.3e})")
        assert err <= tol
        if precision == "fp64":
            assert rel_fro(J, J1) <= 1e-13
    pl.close()


def _K_rows(omega, n, w, C, rows):
    """Rows (a1 n + a2) n + a3 of (omega / sqrt(pi)) sum_p w_p A_x^p (x) A_y^p (x) A_z^p from the
    weights w[p] and the Chebyshev coefficient matrices C[d][p] (n x n)."""
    out = np.zeros((len(rows), n ** 3))
    for i, row in enumerate(rows):
        a1, a2, a3 = row // (n * n), (row // n) % n, row % n
        for p in range(len(w)):
            out[i] += w[p] * np.kron(C[0][p][a1], np.kron(C[1][p][a2], C[2][p][a3]))
    return out * omega / np.sqrt(np.pi)


@pytest.mark.parametrize("n,P", [(12, 12), (7, 40), (6, 60), (24, 32)])
def test_dense_K_matches_oracle_factors(lib, n, P):
    """The dense node sum K of the factored form (pairs of FP32 numbers, any P; P = 60 spans
    more nodes than one 32-wide pass).  Its arithmetic: against K formed in FP64 from the plan's
    own weights and coefficients, every
    entry within 2e-13 of its row's largest entry.  Against the oracle's weights and coefficients
    within 1e-11: the weights agree to 1e-13 relative and an entry sums terms up to ~18 times the
    row maximum.  Full K for small n, sampled rows at n = 24."""
    m = mol_spd_small(n=n, P=P)
    o = oracle.Oracle.from_molecule(m)
    pl = lib.Plan(m, "split_f16")
    K = pl.dense_K()
    _, Cg, _, wg, _ = [t.cpu().numpy() for t in pl.factors()]
    pl.status()
    n3 = n ** 3
    rows = list(range(n3)) if n3 <= 2000 else [0, 1, n3 // 3, n3 // 2 + 7, n3 - 1]
    got = K[rows].cpu().numpy() if n3 > 2000 else K.cpu().numpy()
    _, wo = o.nodes()
    Co = [[o.cheb(d, p) for p in range(P)] for d in range(3)]
    ref_plan = _K_rows(m.omega, n, wg, Cg, rows)
    ref_oracle = _K_rows(o.omega, n, wo, Co, rows)
    scale = np.abs(ref_oracle).max(axis=1, keepdims=True)
    err_plan = float((np.abs(got - ref_plan) / scale).max())
    err_oracle = float((np.abs(got - ref_oracle) / scale).max())
    print(f"dense K n={n} P={P}: max |error| / row max = {err_plan:.2e} (plan factors), {err_oracle:.2e} (oracle)")
    assert err_plan <= 2e-13
    assert err_oracle <= 1e-11
    if n3 <= 2000:
        assert np.allclose(got, got.T, rtol=0, atol=1e-12 * np.abs(ref_oracle).max())
    pl.close()


def _kept_primitive_pairs(m, tau):
    """Per unique pair (mu <= nu), the kept primitive pairs (j1, j2) under the screening criterion
    of Section 6, exp(-a b / (a + b) |A - B|^2) <= tau discards, evaluated here from the shells."""
    import math
    shell_of = [s for s, sh in enumerate(m.shells) for _ in range(sh.ncart)]
    out = []
    for mu in range(len(shell_of)):
        for nu in range(mu, len(shell_of)):
            A, B = m.shells[shell_of[mu]], m.shells[shell_of[nu]]
            d2 = sum((A.center[l] - B.center[l]) ** 2 for l in range(3))
            out.append([(j1, j2) for j1, a in enumerate(A.exps) for j2, b in enumerate(B.exps)
                        if not (tau > 0 and math.exp(-(a * b / (a + b)) * d2) <= tau)])
    return out


@pytest.mark.parametrize("precision", ["fp64", "split_f16"])
def test_screening_matches_screened_oracle(lib, precision):
    """Primitive-pair screening (Section 6) with tau = 1e-3 on the contracted s/p/d instance: the
    plan keeps exactly the primitive pairs the criterion keeps (counted here from the shells), the
    moments of the kept rows are the oracle's for those primitive pairs, and B and a J-build match
    the screened oracle within the precision's bound; tau = 0 changes nothing."""
    import torch
    m = mol_spd_small()
    tau = 1e-3
    kept = _kept_primitive_pairs(m, tau)
    nkept = sum(len(k) for k in kept)
    nall = sum(len(k) for k in _kept_primitive_pairs(m, 0.0))
    assert 0 < nkept < nall
    o = oracle.Oracle.from_molecule(m, tau_screening=tau)
    ref = o.assemble_B()
    ref0 = oracle.Oracle.from_molecule(m).assemble_B()
    assert rel_fro(ref, ref0) > 1e-9  # screening changes B at this tau
    pl = lib.Plan(m, precision, tau_screening=tau)
    assert pl.info["nrows"] == nkept and pl.info["tau_screening"] == tau
    tol = 1e-13 if precision == "fp64" else 1e-7
    B = pl.assemble_B().cpu().numpy()
    pl.status()
    err = rel_fro(B, ref)
    D = synth.random_densities(17, m.nbf, 5)
    J = pl.jbuild(torch.as_tensor(D, device="cuda")).cpu().numpy()
    errJ = rel_fro(J, o.jbuild_factored(D))
    print(f"screening tau={tau} {precision}: rows {nkept}/{nall}, B {err:.2e}, J {errJ:.2e}")
    assert err <= tol and errJ <= tol
    if precision == "fp64":
        S = pl.factors()[0].cpu().numpy()
        Smax = np.abs(S).max(axis=(1, 2))  # the plan's largest moment in each dimension
        shell_of = [s for s, sh in enumerate(m.shells) for _ in range(sh.ncart)]
        row, nbf = 0, m.nbf
        for r, (mu, nu) in enumerate((mu, nu) for mu in range(nbf) for nu in range(mu, nbf)):
            Kn = m.shells[shell_of[nu]].exps.size
            for d in range(3):
                if not kept[r]:
                    continue
                W = o.moments(mu, nu, d)
                want = np.array([W[j1 * Kn + j2] for j1, j2 in kept[r]])
                got = S[d, row:row + len(kept[r])]
                scale = np.abs(want).max(axis=1, keepdims=True)
                # the two quadratures agree to 1e-13 of the row maximum; a row whose largest moment
                # is many orders below the plan's largest (a pair far from the box centre, with a
                # small K_AB) enters B in that proportion, so its error is bounded against the plan's
                # largest moment in this dimension instead (1e-16 of it: rounding)
                floor = 1e-16 * Smax[d]
                assert np.all(np.abs(got - want) <= 1e-13 * scale + floor), (mu, nu, d)
            row += len(kept[r])
        assert row == S.shape[1]
        p0 = lib.Plan(m, precision, tau_screening=0.0)
        pd = lib.Plan(m, precision)
        assert p0.info["nrows"] == pd.info["nrows"] == nall
        assert np.array_equal(p0.assemble_B().cpu().numpy(), pd.assemble_B().cpu().numpy())
        p0.close()
        pd.close()
    pl.close()
