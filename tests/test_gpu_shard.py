"""The sharded J-build and B rows on one GPU: the ranks of paper_2210_13069_gb300.shard emulated in
one process (each rank's halves run in turn through lrtei_jbuild_partial_x / lrtei_jbuild_apply_x
and lrtei_assemble_Bu_rows, the all-reduce a sum over the emulated ranks), against the oracle."""
import numpy as np
import pytest

import oracle
from paper_2210_13069_gb300 import shard, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import torch
    from paper_2210_13069_gb300 import build_lib, lrtei
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build_lib.build()
    lrtei.load()
    return lrtei


def mol():
    return synth.random_molecule(4301, natoms=3, cube=5.0, nprim=2, alpha_range=(0.2, 30.0), omega=0.5, n=10, P=10)


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("split_f16", 1e-7)])
@pytest.mark.parametrize("world", [1, 2, 3])
def test_sharded_jbuild_and_b_rows(lib, precision, tol, world):
    import torch
    m = mol()
    o = oracle.Oracle.from_molecule(m)
    D = synth.random_densities(21, m.nbf, 5)
    ref_J = o.jbuild_factored(D)
    pl = lib.Plan(m, precision)
    Dd = torch.as_tensor(D, device="cuda")
    partial_x, apply_x = shard.gpu_halves(pl, Dd)
    npair = pl.npair
    # emulated ranks: the all-reduce of rank k's value is the sum over all ranks' values
    Xs = [partial_x(*shard.pair_ranges(npair, world)[k]) for k in range(world)]
    X = sum(Xs)
    J = sum(apply_x(X, *shard.pair_ranges(npair, world)[k]) for k in range(world))
    Jfull = pl.jbuild(Dd)
    pl.status()
    e_j = float(np.linalg.norm(J.cpu().numpy() - ref_J) / np.linalg.norm(ref_J))
    e_jf = float(np.linalg.norm(Jfull.cpu().numpy() - ref_J) / np.linalg.norm(ref_J))
    rows = []
    for k in range(world):
        r0, r1, blk = shard.b_rows_sharded(shard.gpu_b_rows(pl, "factored"), npair, k, world)
        rows.append(blk.cpu().numpy())
    Bu = np.concatenate(rows)
    nb = m.nbf
    pairs = [(mu, nu) for mu in range(nb) for nu in range(mu, nb)]
    sample = [0, 7, len(pairs) // 2, len(pairs) - 1]
    ref_rows = o.B_rows([pairs[r][0] * nb + pairs[r][1] for r in sample])
    cols = [mu * nb + nu for mu, nu in pairs]
    e_b = float(np.linalg.norm(Bu[sample] - ref_rows[:, cols]) / np.linalg.norm(ref_rows[:, cols]))
    pl.status()
    print(f"sharded over {world} ({precision}): J {e_j:.2e} (one-rank J-build {e_jf:.2e}), B_u rows {e_b:.2e}")
    assert Bu.shape == (len(pairs), len(pairs))
    assert e_j <= tol and e_b <= tol
    pl.close()
