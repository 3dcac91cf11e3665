"""Khatri-Rao low-rank compression on the GPU (Section 6, eq. SVD and eq. approxepsilon) against
the oracle's numpy form of the same equations (oracle/kr.py).

- Full rank (eps = 0): the compressed plan reproduces the oracle's uncompressed B (FP64, 1e-12),
  and the device singular values match a direct SVD of the oracle's moment matrices.
- Truncated ranks: the ranks the device picks equal the oracle's eps rule, and B, entries and
  J-builds of the compressed plan match the oracle's compressed B with the same ranks (FP64 1e-11:
  the kept subspaces agree to rounding; split-F16 1e-7).
- The 180-function workload at the eps the benchmark uses: sampled rows of the compressed B in
  the eight-product split (the precision the compressed leg runs) against the oracle's
  uncompressed B within 1e-7 (the metric's bound), the whole B and a J-build against the
  uncompressed FP64 GPU path, and the compression error alone (FP64), stated.  The six-product
  split on compressed factors is stated too: its rows are graded (their weight sits in the few
  columns of the largest singular values), which per-row fixed-point slices represent less well
  than the flat rows of the uncompressed factors (9e-8 measured, at the edge of the bound).
"""
import numpy as np
import pytest

import oracle
from oracle import kr
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


def mol_spd(seed=2001):
    return synth.random_molecule(seed, natoms=3, cube=5.0, nprim=3, alpha_range=(0.1, 50.0), omega=0.4, n=16, P=12)


def test_full_rank_reproduces_uncompressed_B(lib):
    m = mol_spd()
    o = oracle.Oracle.from_molecule(m)
    ref = o.assemble_B()
    S, _, _ = kr.moment_rows(o)
    for form in ("factored", "hadamard"):
        pl = lib.Plan(m, "fp64")
        sig, ranks = pl.compress(0.0)
        assert list(ranks) == [m.n] * 3 and pl.info["kr_rank"] == m.n and pl.info["cheb_n"] == m.n
        for d in range(3):
            sv = np.linalg.svd(S[d], compute_uv=False)
            assert np.max(np.abs(sig[d] - sv)) <= 1e-12 * sv[0], d
        B = pl.assemble_B(form).cpu().numpy()
        pl.status()
        err = rel_fro(B, ref)
        print(f"KR full rank ({form}): rel. Frobenius vs uncompressed oracle {err:.3e}")
        assert err <= 1e-12
        pl.close()


@pytest.mark.parametrize("eps", [1e-4, 1e-6])
def test_truncated_matches_oracle_compressed_B(lib, eps):
    import torch
    m = mol_spd()
    o = oracle.Oracle.from_molecule(m)
    ranks_o = kr.ranks_for_eps(o, eps)
    R = max(ranks_o)
    assert R < m.n
    ref = kr.compressed_B(o, [R, R, R])
    unc = o.assemble_B()
    pl = lib.Plan(m, "fp64")
    _, ranks = pl.compress(eps)
    assert list(ranks) == ranks_o and pl.info["n"] == R
    B = pl.assemble_B("factored").cpu().numpy()
    Bh = pl.assemble_B("hadamard").cpu().numpy()
    # Algorithm 1 entries on the compressed factors
    rng = np.random.default_rng(3)
    idx = rng.integers(0, m.nbf, size=(500, 4)).astype(np.int32)
    ent = pl.entries(idx).cpu().numpy()
    rows = idx[:, 0] * m.nbf + idx[:, 1]
    cols = idx[:, 2] * m.nbf + idx[:, 3]
    # J-build on the compressed factored form
    D = synth.random_densities(5, m.nbf, 3)
    J = pl.jbuild(torch.as_tensor(D, device="cuda")).cpu().numpy()
    Jref = np.einsum("rc,qc->qr", ref, D.reshape(3, -1)).reshape(D.shape)
    pl.status()
    e_b, e_h, e_e, e_j = rel_fro(B, ref), rel_fro(Bh, ref), rel_fro(ent, ref[rows, cols]), rel_fro(J, Jref)
    print(f"KR eps={eps:g} R={R}: B {e_b:.2e}, Hadamard {e_h:.2e}, entries {e_e:.2e}, J {e_j:.2e}; "
          f"compression error vs uncompressed {rel_fro(ref, unc):.2e}")
    assert max(e_b, e_h, e_e, e_j) <= 1e-11
    pl.close()
    ps = lib.Plan(m, "split_f16")
    ps.compress(eps)
    Bs = ps.assemble_B().cpu().numpy()
    Js = ps.jbuild(torch.as_tensor(D, device="cuda")).cpu().numpy()
    ps.status()
    e_bs, e_js = rel_fro(Bs, ref), rel_fro(Js, Jref)
    print(f"KR eps={eps:g} split_f16: B {e_bs:.2e}, J {e_js:.2e}")
    assert e_bs <= 1e-7 and e_js <= 1e-7
    ps.close()


def test_compress_arguments_and_once(lib):
    m = mol_spd()
    pl = lib.Plan(m, "fp64")
    for eps, mr in ((-1.0, 0), (1.0, 0), (0.1, m.n + 1), (0.1, -1)):
        with pytest.raises(lib.LrteiError) as ei:
            lib.lrtei_plan_compress(pl.plan, eps, mr)
        assert ei.value.status == 1
    _, ranks = pl.compress(1e-3, max_rank=4)
    assert pl.info["n"] == 4 and max(ranks) >= 4
    with pytest.raises(lib.LrteiError) as ei:
        pl.compress(1e-3)
    assert ei.value.status == 6
    pl.close()


KR_EPS_180 = 1e-8  # the benchmark's compression threshold on the 180-function workload


def test_full_size_180_compressed_within_metric_bound(lib):
    import torch
    m = synth.workload_spd()
    o = oracle.Oracle.from_molecule(m)
    nbf = m.nbf
    pl = lib.Plan(m, "split_f16_8")
    sig, ranks = pl.compress(KR_EPS_180)
    R = pl.info["n"]
    full = pl.assemble_B()
    rng = np.random.default_rng(23)
    picks = [(0, 0), (int(rng.integers(0, nbf)), int(rng.integers(0, nbf))), (nbf - 1, nbf - 1), (3, 170), (40, 41)]
    refs, rows = [], []
    for mu, nu in picks:
        refs.append(o.B_rows([mu * nbf + nu])[0])
        rows.append(full[mu * nbf + nu].cpu().numpy())
    e_rows = rel_fro(np.array(rows), np.array(refs))
    p64 = lib.Plan(m, "fp64")
    B64 = p64.assemble_B()
    e_all = float(torch.linalg.norm(full - B64) / torch.linalg.norm(B64))
    del full
    pc = lib.Plan(m, "fp64")
    pc.compress(KR_EPS_180)
    Bc = pc.assemble_B()
    e_comp = float(torch.linalg.norm(Bc - B64) / torch.linalg.norm(B64))
    del Bc
    D = torch.as_tensor(synth.random_densities(31, nbf, 32), device="cuda")
    J = pl.jbuild(D)
    J64 = p64.jbuild(D)
    e_j = float(torch.linalg.norm(J - J64) / torch.linalg.norm(J64))
    pl.status()
    p64.status()
    p6 = lib.Plan(m, "split_f16")
    p6.compress(KR_EPS_180)
    B6 = p6.assemble_B()
    e_six = float(torch.linalg.norm(B6 - B64) / torch.linalg.norm(B64))
    del B6
    p6.status()
    print(f"KR 180 functions eps={KR_EPS_180:g}: ranks {[int(r) for r in ranks]} -> R={R}; split_f16_8 sampled rows vs "
          f"oracle {e_rows:.3e}, whole B vs uncompressed FP64 GPU {e_all:.3e} (compression alone {e_comp:.3e}; "
          f"six products {e_six:.3e}), J (32 densities) {e_j:.3e}")
    assert R < m.n
    assert e_comp <= 1e-8
    assert e_rows <= 1e-7 and e_all <= 1e-7 and e_j <= 1e-7
    for p in (pl, p64, pc, p6):
        p.close()
