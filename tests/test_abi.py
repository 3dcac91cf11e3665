"""The C-ABI library builds, loads and exports every symbol include/lrtei.h declares; host-side
validation rejects bad input before any device work (no GPU needed)."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

from paper_2210_13069_gb300 import build_lib, lrtei, synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build_lib.build()
    return lrtei.load()


def declared_symbols():
    hdr = open(os.path.join(ROOT, "include", "lrtei.h")).read()
    hdr = re.sub(r"/\*.*?\*/", "", hdr, flags=re.S)
    return sorted(set(re.findall(r"\b(lrtei_[A-Za-z0-9_]+)\s*\(", hdr)))


def test_header_declares_the_boundary():
    names = declared_symbols()
    for must in ["lrtei_basis_create", "lrtei_plan_create", "lrtei_assemble_B", "lrtei_entries", "lrtei_factors",
                 "lrtei_jbuild", "lrtei_jbuild_batched", "lrtei_plan_status", "lrtei_last_error"]:
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", lrtei.library_path()], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r"\bT (lrtei_[A-Za-z0-9_]+)\b", out))
    missing = [s for s in declared_symbols() if s not in exported]
    assert not missing, missing
    for s in declared_symbols():
        assert hasattr(lib, s)


def test_basis_validation_on_host(lib):
    m = synth.workload_spd(natoms=2)
    c, l, k, e, cf = m.packed()
    b = lrtei.lrtei_basis_create(c, l, k, e, cf)
    assert lrtei.lrtei_basis_nbf(b) == m.nbf == 30
    lrtei.lrtei_basis_destroy(b)
    bad = e.copy()
    bad[3] = -1.0
    with pytest.raises(lrtei.LrteiError) as ei:
        lrtei.lrtei_basis_create(c, l, k, bad, cf)
    assert ei.value.status == 1 and "exponent" in str(ei.value)
    badl = l.copy()
    badl[0] = 7
    with pytest.raises(lrtei.LrteiError):
        lrtei.lrtei_basis_create(c, badl, k, e, cf)


def test_plan_arguments_validated_before_device(lib):
    m = synth.workload_small_s()
    c, l, k, e, cf = m.packed()
    b = lrtei.lrtei_basis_create(c, l, k, e, cf)
    try:
        for kw in [dict(omega=-1.0, n=8, P=8), dict(omega=0.5, n=0, P=8), dict(omega=0.5, n=65, P=8),
                   dict(omega=0.5, n=8, P=0)]:
            with pytest.raises(lrtei.LrteiError) as ei:
                lrtei.lrtei_plan_create(b, kw["omega"], kw["n"], kw["P"], stream=0)
            assert ei.value.status == 1
    finally:
        lrtei.lrtei_basis_destroy(b)


def test_no_cpu_fallback_without_device(lib):
    """On a machine without a CUDA device the library refuses to compute (no CPU fallback)."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    m = synth.workload_small_s()
    c, l, k, e, cf = m.packed()
    b = lrtei.lrtei_basis_create(c, l, k, e, cf)
    try:
        with pytest.raises(lrtei.LrteiError) as ei:
            lrtei.lrtei_plan_create(b, 0.5, 16, 20, stream=0)
        assert ei.value.status == 3
    finally:
        lrtei.lrtei_basis_destroy(b)
