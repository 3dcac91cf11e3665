"""The 360-function instance (24 atoms, omega = 0.33, n = 24, P = 32) through the split-F16
tensor-core path, with eight and with six products: the full 129 600 x 129 600 FP64 B (134 GB)
is assembled, its sampled rows are checked against the oracle (two rows) and against the FP64
GPU path (four rows), and its exact symmetry on sampled entries.  Tolerance: relative Frobenius
1e-7 per set of rows."""
import numpy as np
import pytest

import oracle
from paper_2210_13069_gb300 import synth

pytestmark = pytest.mark.gpu


def rel_fro(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


@pytest.mark.parametrize("precision", ["split_f16_8", "split_f16"])
def test_split_full_size_360(precision):
    import torch
    from paper_2210_13069_gb300 import build_lib, lrtei
    assert torch.cuda.is_available(), "GPU test"
    build_lib.build()
    lrtei.load()
    m = synth.workload_spd_large()
    nbf = m.nbf
    assert nbf == 360
    pl = lrtei.Plan(m, precision)
    B = pl.assemble_B()
    torch.cuda.synchronize()
    pl.status()
    pl.close()
    rng = np.random.default_rng(360)
    picks = [(0, 0), (int(rng.integers(0, nbf)), int(rng.integers(0, nbf))), (nbf - 1, nbf - 1), (7, 331)]
    picks = [(min(a, b), max(a, b)) for a, b in picks]
    rows = {pk: B[pk[0] * nbf + pk[1]].cpu().numpy() for pk in picks}
    idx = torch.as_tensor(rng.integers(0, nbf * nbf, size=(2, 4096)), device="cuda")
    assert torch.equal(B[idx[0], idx[1]], B[idx[1], idx[0]])
    del B
    torch.cuda.empty_cache()
    p64 = lrtei.Plan(m, "fp64")
    cols = np.array([ka * nbf + la for ka in range(nbf) for la in range(ka, nbf)])
    got, ref = [], []
    for mu, nu in picks:
        r = mu * nbf - mu * (mu - 1) // 2 + (nu - mu)
        ref.append(p64.Bu_rows(r, r + 1).cpu().numpy()[0])
        got.append(rows[(mu, nu)][cols])
    p64.close()
    e64 = rel_fro(got, ref)
    o = oracle.Oracle.from_molecule(m)
    oref = o.B_rows([picks[1][0] * nbf + picks[1][1], picks[3][0] * nbf + picks[3][1]])
    eor = rel_fro([rows[picks[1]], rows[picks[3]]], oref)
    print(f"{precision} 360 functions: sampled rows vs FP64 GPU {e64:.3e}, vs oracle {eor:.3e}")
    assert e64 <= 1e-7 and eor <= 1e-7
