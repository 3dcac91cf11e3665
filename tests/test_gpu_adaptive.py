"""Adaptive choice of the integration domain on the GPU (Section 6) against the adaptive oracle
(oracle/adaptive.py, pinned on the CPU by interpolation identities, the single-box oracle and the
Table 3 trend against the erf-Boys closed form).

The partitions (an integer decision from FP64 supports, taken on both sides with the same
formula) must agree exactly; B (both precisions), Algorithm 1 entries and J-builds must match the
oracle: FP64 1e-12, split-F16 1e-7.
"""
import numpy as np
import pytest

from oracle import adaptive as ad
from paper_2210_13069_gb300 import synth

pytestmark = pytest.mark.gpu


def rel_fro(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


@pytest.fixture(scope="module")
def lib():
    import torch
    from paper_2210_13069_gb300 import build_lib, lrtei
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build_lib.build()
    lrtei.load()
    return lrtei


def mol_spd():
    """Three atoms, s/p/d shells of 1-3 primitives, exponents 0.08..60 (N_b = 30)."""
    m = synth.random_molecule(3101, natoms=3, cube=6.0, shells_per_atom=(("s", 2), ("p", 1), ("d", 1)), nprim=2,
                              alpha_range=(0.08, 60.0), omega=0.4, n=12, P=12)
    rng = np.random.default_rng(3101)
    for i, sh in enumerate(m.shells):
        k = 1 + (i % 3)
        sh.exps = np.sort(np.exp(rng.uniform(np.log(0.08), np.log(60.0), size=k)))[::-1].copy()
        sh.coefs = rng.uniform(0.2, 1.0, size=k)
    return m


TAU = 1e-20


@pytest.fixture(scope="module")
def case():
    m = mol_spd()
    a = ad.Adaptive(m, m.omega, m.n, m.P, TAU, 3)
    return m, a, a.assemble_B()


def test_partitions_agree(lib, case):
    m, a, _ = case
    pl = lib.Plan(m, "fp64", adaptive=(TAU, 3))
    info = pl.info
    assert info["npartitions"] == a.npart == 3
    assert np.allclose(info["partition_b"], a.bs, rtol=1e-15, atol=0)
    pl.close()


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("split_f16", 1e-7)])
def test_B_and_jbuild_match_the_adaptive_oracle(lib, case, precision, tol):
    import torch
    m, a, ref = case
    pl = lib.Plan(m, precision, adaptive=(TAU, 3))
    B = pl.assemble_B().cpu().numpy()
    D = synth.random_densities(8, m.nbf, 4)
    J = pl.jbuild(torch.as_tensor(D, device="cuda")).cpu().numpy()
    Jref = np.einsum("rc,qc->qr", ref, D.reshape(4, -1)).reshape(D.shape)
    pl.status()
    e_b, e_j = rel_fro(B, ref), rel_fro(J, Jref)
    print(f"adaptive ({a.npart} boxes {np.round(a.bs, 2)}) {precision}: B {e_b:.2e}, J {e_j:.2e}")
    assert e_b <= tol
    assert e_j <= 1e-12  # the J-build runs in FP64 for every precision
    pl.close()


def test_entries_match_the_adaptive_oracle(lib, case):
    m, a, ref = case
    pl = lib.Plan(m, "fp64", adaptive=(TAU, 3))
    rng = np.random.default_rng(9)
    idx = rng.integers(0, m.nbf, size=(400, 4)).astype(np.int32)
    got = pl.entries(idx).cpu().numpy()
    pl.status()
    want = ref[idx[:, 0] * m.nbf + idx[:, 1], idx[:, 2] * m.nbf + idx[:, 3]]
    assert np.max(np.abs(got - want)) <= 1e-12 * np.abs(ref).max()
    pl.close()


def test_unsupported_calls_are_refused(lib, case):
    import torch
    m, _, _ = case
    pl = lib.Plan(m, "fp64", adaptive=(TAU, 2))
    K = torch.empty(1, dtype=torch.float64, device="cuda")
    for call in (lambda: lib.lrtei_dense_K(pl.plan, K), lambda: pl.compress(1e-6),
                 lambda: lib.lrtei_assemble_Bu_rows(pl.plan, 0, 0, 1, K, pl.npair)):
        with pytest.raises(lib.LrteiError) as ei:
            call()
        assert ei.value.status == 6
    for tau, npart in ((0.0, 2), (1.0, 2), (1e-20, 0), (1e-20, 9)):
        with pytest.raises(lib.LrteiError) as ei:
            lib.lrtei_plan_create_adaptive(pl.basis, 0.4, 8, 8, tau, npart)
        assert ei.value.status == 1
    pl.close()
