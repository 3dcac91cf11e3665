"""Golden entries (tests/golden/*_entries.txt, written by tests/golden/make_golden.py from the
oracle alone): the oracle still reproduces them (a change to its arithmetic shows here), and the
GPU path's Algorithm 1 entries (FP64) match them."""
import importlib.util
import os

import numpy as np
import pytest

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))
_spec = importlib.util.spec_from_file_location("make_golden", os.path.join(HERE, "golden", "make_golden.py"))
make_golden = importlib.util.module_from_spec(_spec)
_spec.loader.exec_module(make_golden)

NAMES = ["nb20_s", "spd2"]


@pytest.mark.parametrize("name", NAMES)
def test_oracle_reproduces_golden_entries(name):
    mol, _ = make_golden.cases()[name]
    params, idx, vals = make_golden.read(name)
    o = oracle.Oracle.from_molecule(mol)
    assert (int(params["nbf"]), float(params["omega"]), int(params["n"]), int(params["P"])) == \
        (o.nbf, o.omega, o.n, o.P)
    got = o.entries(idx, threads=1)
    assert np.max(np.abs(got - vals)) <= 1e-15 * np.max(np.abs(vals))


@pytest.mark.gpu
@pytest.mark.parametrize("name", NAMES)
def test_gpu_entries_match_golden(name):
    import torch
    from paper_2210_13069_gb300 import build_lib, lrtei
    assert torch.cuda.is_available()
    build_lib.build()
    mol, _ = make_golden.cases()[name]
    _, idx, vals = make_golden.read(name)
    pl = lrtei.Plan(mol, "fp64")
    got = pl.entries(idx).cpu().numpy()
    pl.status()
    pl.close()
    err = float(np.max(np.abs(got - vals)) / np.max(np.abs(vals)))
    print(f"golden {name}: max |GPU - golden| / max |golden| = {err:.2e}")
    assert err <= 1e-13
