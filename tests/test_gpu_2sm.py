"""The 2-SM tensor-core GEMM (cta_group::2: a CTA pair computes 256 x 128 tiles, each SM loading
half of B), against the one-SM kernel and the oracle.  LRTEI_TC_2SM=1 selects it for the
non-symmetric six-product GEMMs with 128-column tiles (G = F_u K), =2 for the symmetric B_u = G F_u^T
too; LRTEI_TC_2SM_BK=32 gives it five 32-deep operand stages instead of two 64-deep ones.  Without
the variable the tuner times the pair kernel beside the one-SM configurations."""
import numpy as np
import pytest

import oracle
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


def mol_ragged(seed=2002):
    m = synth.random_molecule(seed, natoms=3, cube=5.0, nprim=2, alpha_range=(0.2, 30.0), omega=0.5, n=10, P=10)
    rng = np.random.default_rng(seed)
    for i, sh in enumerate(m.shells):
        k = 1 + (i % 3)
        sh.exps = np.sort(np.exp(rng.uniform(np.log(0.2), np.log(30.0), size=k)))[::-1].copy()
        sh.coefs = rng.uniform(0.1, 1.0, size=k)
    return m


def mol_spd4():
    return synth.workload_spd(natoms=4)  # N_b = 60, n = 24: G is 1830 x 13 824 (eight 256-row tiles)


@pytest.mark.parametrize("bk", ["32", "64"])
@pytest.mark.parametrize("flag", ["1", "2"])
@pytest.mark.parametrize("maker", [mol_ragged, mol_spd4])
def test_two_sm_assembly_matches_oracle_and_one_sm(lib, maker, flag, bk, monkeypatch):
    m = maker()
    o = oracle.Oracle.from_molecule(m)
    nbf = m.nbf
    rows = [0, nbf + 3, (nbf // 2) * nbf + nbf // 3, nbf * nbf - 1]
    ref = o.B_rows(rows)
    monkeypatch.delenv("LRTEI_TC_2SM", raising=False)
    monkeypatch.setenv("LRTEI_TC_CONFIG", "0")  # the one-SM kernel, not the tuner's choice
    p1 = lib.Plan(m, "split_f16")
    B1 = p1.assemble_B().cpu().numpy()
    p1.status()
    p1.close()
    monkeypatch.delenv("LRTEI_TC_CONFIG")
    monkeypatch.setenv("LRTEI_TC_2SM", flag)
    monkeypatch.setenv("LRTEI_TC_2SM_BK", bk)
    p2 = lib.Plan(m, "split_f16")
    B2 = p2.assemble_B().cpu().numpy()
    p2.status()
    p2.close()
    e2, e1 = rel_fro(B2[rows], ref), rel_fro(B1[rows], ref)
    d = float(np.max(np.abs(B2 - B1)) / np.abs(B1).max())
    print(f"2-SM GEMM ({flag}, BK {bk}), N_b={nbf}: rows vs oracle {e2:.2e} (one SM {e1:.2e}); max |2-SM - one SM| / max "
          f"{d:.1e}; symmetric {np.abs(B2 - B2.T).max():.1e}")
    assert e2 <= 1e-7
    assert np.array_equal(B2, B1)  # each element's chunk sums are the one-SM kernel's, bit for bit
    assert np.array_equal(B2, B2.T)  # the symmetric walk mirrors every block exactly


def test_two_sm_full_size_180(lib, monkeypatch):
    import time
    import torch
    m = synth.workload_spd()
    o = oracle.Oracle.from_molecule(m)
    nbf = m.nbf
    rows = [0, 37 * nbf + 101, nbf * nbf - 1]
    ref = o.B_rows(rows)
    out = {}
    runs = [("0", "32"), ("1", "32"), ("1", "64"), ("2", "32"), ("2", "64")]
    for flag, bk in runs:
        monkeypatch.setenv("LRTEI_TC_2SM", flag)
        monkeypatch.setenv("LRTEI_TC_2SM_BK", bk)
        if flag == "0":
            monkeypatch.setenv("LRTEI_TC_CONFIG", "0")  # the one-SM kernel, not the tuner's choice
        else:
            monkeypatch.delenv("LRTEI_TC_CONFIG", raising=False)
        pl = lib.Plan(m, "split_f16")
        B = pl.assemble_B()
        pl.assemble_B(out=B)
        torch.cuda.synchronize()
        lib.lrtei_profile_reset()
        lib.lrtei_profile_enable(True)
        t0 = time.perf_counter()
        for _ in range(3):
            pl.assemble_B(out=B)
        torch.cuda.synchronize()
        dt = (time.perf_counter() - t0) / 3
        g_ms, g_n = lib.lrtei_profile_get("tc_gemm")
        lib.lrtei_profile_enable(False)
        lib.lrtei_profile_reset()
        pl.status()
        out[flag, bk] = (B[rows].cpu().numpy(), dt, g_ms / max(g_n, 1))
        pl.close()
        del B
        torch.cuda.empty_cache()
    one = out["0", "32"]
    for key in runs[1:]:
        e = rel_fro(out[key][0], ref)
        print(f"2-SM ({key[0]}, BK {key[1]}) full size: {out[key][1] * 1e3:.1f} ms per B (one SM {one[1] * 1e3:.1f} "
              f"ms); tc_gemm per launch {out[key][2]:.2f} ms (one SM {one[2]:.2f} ms); rows vs oracle {e:.2e}")
        assert e <= 1e-7
