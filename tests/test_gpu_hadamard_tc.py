"""The Hadamard form of Theorem 1 / Algorithm 1 on the tensor cores (k_tc_hadamard.cu), for bases
whose unique pairs hold one primitive pair each: full B against the oracle, the FP64 path and the
tensor-core factored form; bands of B_u rows; the form the library chooses; pinned host output;
degenerate and ragged sizes; the 180-function uncontracted workload."""
import numpy as np
import pytest

import oracle
from paper_2210_13069_gb300 import synth

pytestmark = pytest.mark.gpu

HADAMARD, FACTORED = 1, 2


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


def mol_unc(seed, natoms, shells, n, P, cube=5.0, omega=0.5, alpha=(0.1, 80.0)):
    return synth.random_molecule(seed, natoms=natoms, cube=cube, shells_per_atom=shells, nprim=1,
                                 alpha_range=alpha, omega=omega, n=n, P=P)


CASES = {
    # s functions only (the 20-function instance of the small plain-TA configuration)
    "nb20_s": lambda: synth.workload_small_s(),
    # s, p, d on three atoms: N_b = 33, 561 unique pairs (a ragged last 128-row block and 64-column block)
    "spd33": lambda: mol_unc(2201, 3, (("s", 2), ("p", 1), ("d", 1)), n=12, P=10),
    # n above 32: two 32-deep steps per product
    "spd33_n40": lambda: mol_unc(2202, 3, (("s", 2), ("p", 1), ("d", 1)), n=40, P=16),
    # one node, one Chebyshev polynomial
    "n1_P1": lambda: mol_unc(2203, 2, (("s", 2), ("p", 1)), n=1, P=1),
    # one basis function: a 1 x 1 B_u
    "one_function": lambda: mol_unc(2204, 1, (("s", 1),), n=8, P=6),
}


@pytest.mark.parametrize("case", list(CASES))
def test_full_B_against_oracle_fp64_and_factored(lib, case):
    m = CASES[case]()
    o = oracle.Oracle.from_molecule(m)
    Bo = o.assemble_B()
    pl = lib.Plan(m, "split_f16")
    B = pl.assemble_B("hadamard").cpu().numpy()
    assert pl.info["last_form"] == HADAMARD
    pl.status()
    msg = ""
    if m.n ** 3 <= 32768:  # the factored form's symmetric product takes K = n^3 in one pass
        Bf = pl.assemble_B("factored").cpu().numpy()
        assert pl.info["last_form"] == FACTORED
        pl.status()
        msg = f"; factored vs oracle {rel_fro(Bf, Bo):.2e}"
    pl.close()
    p64 = lib.Plan(m, "fp64")
    B64 = p64.assemble_B().cpu().numpy()
    p64.close()
    e_o, e_64 = rel_fro(B, Bo), rel_fro(B, B64)
    print(f"{case} (N_b = {m.nbf}, n = {m.n}, P = {m.P}): tensor-core Hadamard vs oracle {e_o:.2e}, vs FP64 GPU "
          f"{e_64:.2e}{msg}")
    assert np.array_equal(B, B.T)  # every off-diagonal element is stored with its mirror
    assert e_o <= 2e-8 and e_64 <= 2e-8


def test_row_bands_match_the_symmetric_pass(lib):
    """lrtei_assemble_Bu_rows on bands that start and end inside 128-row blocks: the elements on
    and above the diagonal are computed by the same tile products as in the full pass (bit for
    bit); below it the band computes G(r, c) = T(r) . S(c) where the full pass mirrors T(c) . S(r)."""
    m = CASES["spd33"]()
    pl = lib.Plan(m, "split_f16")
    npair = m.nbf * (m.nbf + 1) // 2
    full = pl.Bu_rows(0, npair).cpu().numpy()
    assert pl.info["last_form"] == HADAMARD
    for r0, r1 in ((0, 17), (5, 130), (128, npair), (200, 201), (npair - 1, npair)):
        band = pl.Bu_rows(r0, r1).cpu().numpy()
        ref = full[r0:r1]
        upper = np.triu(np.ones((npair, npair), dtype=bool))[r0:r1]
        assert np.array_equal(band[upper], ref[upper]), (r0, r1)
        assert rel_fro(band, ref) <= 1e-8, (r0, r1)
    pl.status()
    pl.close()


def test_form_choice(lib):
    """Uncontracted split plans take the tensor-core Hadamard form where the cost model favours
    it (P (6n + 3) <= 2 n^3); contracted and eight-product plans take the factored form."""
    unc = CASES["spd33"]()
    pl = lib.Plan(unc, "split_f16")
    pl.assemble_B()
    assert pl.info["last_form"] == HADAMARD
    pl.close()
    pl = lib.Plan(unc, "split_f16_8")
    pl.assemble_B()
    assert pl.info["last_form"] == FACTORED
    pl.close()
    tiny = CASES["n1_P1"]()  # n = 1: the cost model picks the factored form unless asked
    pl = lib.Plan(tiny, "split_f16")
    pl.assemble_B()
    assert pl.info["last_form"] == FACTORED
    pl.assemble_B("hadamard")
    assert pl.info["last_form"] == HADAMARD
    pl.close()
    con = synth.random_molecule(2205, natoms=2, cube=4.0, nprim=2, omega=0.5, n=10, P=8)
    pl = lib.Plan(con, "split_f16")
    pl.assemble_B("hadamard")  # not available with contracted pairs: the factored form runs
    assert pl.info["last_form"] == FACTORED
    pl.close()


def test_pinned_host_output(lib):
    import torch
    m = CASES["spd33"]()
    pl = lib.Plan(m, "split_f16")
    Bd = pl.assemble_B().cpu()
    nb2 = m.nbf * m.nbf
    Bh = torch.full((nb2, nb2), float("nan"), dtype=torch.float64, pin_memory=True)
    pl.assemble_B(out=Bh)
    torch.cuda.synchronize()
    pl.status()
    assert pl.info["last_form"] == HADAMARD
    assert torch.equal(Bd, Bh)
    pl.close()


def test_full_size_uncontracted_180(lib):
    """The 180-function s/p/d workload with one primitive per shell: sampled rows against the
    oracle, and the time per B against the tensor-core factored form."""
    import time
    import torch
    m = synth.workload_spd(nprim=1)
    o = oracle.Oracle.from_molecule(m)
    nbf = m.nbf
    rows = [0, 37 * nbf + 101, 90 * nbf + 3, nbf * nbf - 1]
    ref = o.B_rows(rows)
    pl = lib.Plan(m, "split_f16")
    times = {}
    out = {}
    for form in ("hadamard", "factored"):
        B = pl.assemble_B(form)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(3):
            pl.assemble_B(form, out=B)
        torch.cuda.synchronize()
        times[form] = (time.perf_counter() - t0) / 3
        out[form] = B[rows].cpu().numpy()
        pl.status()
        del B
        torch.cuda.empty_cache()
    pl.close()
    e_h, e_f = rel_fro(out["hadamard"], ref), rel_fro(out["factored"], ref)
    print(f"uncontracted N_b = {nbf}: tensor-core Hadamard {times['hadamard'] * 1e3:.1f} ms per B (rows vs oracle "
          f"{e_h:.2e}); factored {times['factored'] * 1e3:.1f} ms ({e_f:.2e})")
    assert e_h <= 2e-8 and e_f <= 1e-7
    assert times["hadamard"] < times["factored"]
