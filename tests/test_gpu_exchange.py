"""Long-range exchange on the GPU (appendix "The Hartree-Fock exchange", eq. exchange) against the
oracle's direct route (oracle/exchange.py: the dense B^lr of Algorithm 1 contracted with the
orbital coefficients), which the CPU pins tie to the erf-Boys closed forms.

Tolerances (relative Frobenius): FP64 path 1e-12; split-F16 1e-7.  Orbitals in one block and in
several (LRTEI_EXCHANGE_BLOCK); a Khatri-Rao compressed plan against the same contraction of the
oracle's compressed B; the 180-function workload with 90 orbitals against the FP64 GPU path
(six and eight products within 1e-7).
"""
import numpy as np
import pytest

import oracle
from oracle import exchange as ex, kr
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


def orbitals(seed, norb, nbf):
    rng = np.random.default_rng(seed)
    return rng.normal(0.0, 1.0 / np.sqrt(nbf), size=(norb, nbf))


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("split_f16", 1e-7)])
@pytest.mark.parametrize("block", [0, 3])
def test_exchange_matches_oracle(lib, precision, tol, block, monkeypatch):
    import torch
    m = mol_ragged()
    o = oracle.Oracle.from_molecule(m)
    Q = orbitals(5, 8, m.nbf)
    ref = ex.exchange_direct(o, Q)
    if block:
        monkeypatch.setenv("LRTEI_EXCHANGE_BLOCK", str(block))
    pl = lib.Plan(m, precision)
    K = pl.exchange(torch.as_tensor(Q, device="cuda")).cpu().numpy()
    pl.status()
    err = rel_fro(K, ref)
    print(f"exchange {precision} (block {block or 'all'}): rel. Frobenius vs oracle {err:.3e}; "
          f"symmetry {np.abs(K - K.T).max() / np.abs(K).max():.1e}")
    assert err <= tol
    pl.close()


def test_exchange_on_a_compressed_plan(lib):
    import torch
    m = synth.random_molecule(2001, natoms=3, cube=5.0, nprim=3, alpha_range=(0.1, 50.0), omega=0.4, n=16, P=12)
    o = oracle.Oracle.from_molecule(m)
    R = max(kr.ranks_for_eps(o, 1e-6))
    B4 = kr.compressed_B(o, [R, R, R]).reshape((m.nbf,) * 4)
    Q = orbitals(6, 5, m.nbf)
    ref = 2.0 * np.einsum("mlkn,lk->mn", B4, Q.T @ Q)
    pl = lib.Plan(m, "fp64")
    pl.compress(1e-6)
    assert pl.info["n"] == R
    K = pl.exchange(torch.as_tensor(Q, device="cuda")).cpu().numpy()
    pl.status()
    err = rel_fro(K, ref)
    print(f"exchange on the compressed plan (R={R}): rel. Frobenius vs oracle {err:.3e}")
    assert err <= 1e-11
    pl.close()


def test_exchange_full_size_180_with_90_orbitals(lib):
    """Six and eight products meet 1e-7 against the FP64 path (six: 8.6e-8 measured with the
    8/12/12-bit slices and 128-deep drains, 1.6e-7 with 8/11/11-bit slices and 256-deep ones: the
    contraction over 90 orbitals x n^3 cancels more than B's)."""
    import time
    import torch
    m = synth.workload_spd()
    Q = torch.as_tensor(orbitals(7, 90, m.nbf), device="cuda")
    res = {}
    for prec in ("split_f16", "split_f16_8", "fp64"):
        pl = lib.Plan(m, prec)
        pl.exchange(Q)  # builds the operands
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        K = pl.exchange(Q)
        torch.cuda.synchronize()
        res[prec] = (K.cpu().numpy(), time.perf_counter() - t0)
        pl.status()
        pl.close()
        torch.cuda.empty_cache()
    err6 = rel_fro(res["split_f16"][0], res["fp64"][0])
    err8 = rel_fro(res["split_f16_8"][0], res["fp64"][0])
    print(f"exchange, 180 functions, 90 orbitals: split_f16 {res['split_f16'][1] * 1e3:.1f} ms (rel. error "
          f"{err6:.3e}), split_f16_8 {res['split_f16_8'][1] * 1e3:.1f} ms ({err8:.3e}), FP64 {res['fp64'][1] * 1e3:.1f} ms")
    assert err8 <= 1e-7 and err6 <= 1e-7
