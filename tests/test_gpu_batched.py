"""Batched J-builds: many molecules of uneven size, several omega, n and P, in one captured CUDA
graph (molecules spread over concurrent capture streams), against single-molecule J-builds and
the FP64 oracle."""
import numpy as np
import pytest

import oracle
from paper_2210_13069_gb300 import synth

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


@pytest.fixture(scope="module")
def lib():
    import torch
    from paper_2210_13069_gb300 import build_lib, lrtei
    assert torch.cuda.is_available()
    build_lib.build()
    lrtei.load()
    return lrtei


def small_batch():
    specs = [(1, 0.2, 10, 8, 2), (2, 0.33, 12, 10, 3), (1, 0.5, 9, 12, 1), (3, 1.0, 11, 9, 2), (2, 0.5, 8, 14, 3),
             (1, 0.33, 13, 11, 2)]
    mols = []
    for i, (natoms, omega, n, P, nprim) in enumerate(specs):
        mols.append(synth.random_molecule(5000 + i, natoms=natoms, cube=4.0, nprim=nprim, alpha_range=(0.2, 20.0),
                                          omega=omega, n=n, P=P))
    return mols


@pytest.mark.parametrize("precision,tol", [("split_f16", 1e-7), ("fp64", 1e-12)])
def test_batched_matches_single_and_oracle(lib, precision, tol):
    import torch
    mols = small_batch()
    plans = [lib.Plan(m, precision) for m in mols]
    Rs = [3 + (i % 4) for i in range(len(mols))]
    Ds = [torch.as_tensor(synth.random_densities(600 + i, m.nbf, Rs[i]), device="cuda") for i, m in enumerate(mols)]
    Js = [torch.full_like(D, float("nan")) for D in Ds]
    singles = [pl.jbuild(D) for pl, D in zip(plans, Ds)]
    for call in range(3):  # first call runs and captures, later calls replay the graph
        for J in Js:
            J.fill_(float("nan"))
        lib.lrtei_jbuild_batched([p.plan for p in plans], Ds, Rs, Js)
        torch.cuda.synchronize()
        for i in range(len(mols)):
            assert torch.equal(Js[i], singles[i]), (call, i)
    for i in (0, 3):
        ref = oracle.Oracle.from_molecule(mols[i]).jbuild_factored(Ds[i].cpu().numpy())
        assert rel(Js[i].cpu().numpy(), ref) <= tol
    # the graph reads the densities at replay time
    Ds[1].mul_(-0.5)
    lib.lrtei_jbuild_batched([p.plan for p in plans], Ds, Rs, Js)
    torch.cuda.synchronize()
    assert torch.equal(Js[1], plans[1].jbuild(Ds[1]))
    for p in plans:
        p.status()
        p.close()


def test_batched_graph_after_operands_rebuilt(lib):
    """A six-product plan keeps F_u and K without the fourth slice plane until a B assembly needs
    it; the assembly rebuilds both, so a J-build graph captured before it is dropped and captured
    again: the next batched call still equals single J-builds."""
    import torch
    mols = small_batch()[:3]
    plans = [lib.Plan(m, "split_f16") for m in mols]
    Rs = [4, 2, 5]
    Ds = [torch.as_tensor(synth.random_densities(700 + i, m.nbf, Rs[i]), device="cuda") for i, m in enumerate(mols)]
    Js = [torch.empty_like(D) for D in Ds]
    for _ in range(2):  # run and capture, then replay
        lib.lrtei_jbuild_batched([p.plan for p in plans], Ds, Rs, Js)
    torch.cuda.synchronize()
    first = [J.clone() for J in Js]
    B = plans[0].assemble_B()  # rebuilds the slices of F_u and K with the t1 / 2^12 plane
    for _ in range(2):
        for J in Js:
            J.fill_(float("nan"))
        lib.lrtei_jbuild_batched([p.plan for p in plans], Ds, Rs, Js)
        torch.cuda.synchronize()
        for i in range(len(plans)):
            assert torch.equal(Js[i], plans[i].jbuild(Ds[i])), i
            assert rel(Js[i].cpu().numpy(), first[i].cpu().numpy()) <= 1e-12, i
    del B
    for p in plans:
        p.status()
        p.close()


def test_graph_cache_keeps_at_most_32_and_recaptures(lib):
    """Thirty-five distinct J-build calls (one plan, one density batch, 35 output buffers) each
    leave a captured graph; the cache keeps the 32 most recent, so the first calls' graphs are
    dropped and recaptured when they come again, with the same results."""
    import torch
    m = small_batch()[1]
    pl = lib.Plan(m, "split_f16")
    D = torch.as_tensor(synth.random_densities(810, m.nbf, 3), device="cuda")
    ref = pl.jbuild(D)
    outs = [torch.empty_like(D) for _ in range(35)]
    for rep in range(3):  # run and capture, then replay (with evictions in between)
        for J in outs:
            J.fill_(float("nan"))
            pl.jbuild(D, out=J)
        torch.cuda.synchronize()
        for J in outs:
            assert torch.equal(J, ref), rep
    pl.status()
    pl.close()
