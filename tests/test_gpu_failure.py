"""Device-side failure reporting, exercised without faulting the GPU.

- A bounded wait of the tensor-core GEMM that runs out: the test hook LRTEI_TEST_STALL_CYCLES
  makes every CTA's MMA thread wait on a barrier that nothing completes; the wait gives up, the
  kernel leaves through its bounded drain path, lrtei_plan_status reports LRTEI_ERR_TIMEOUT, and
  the next call on the same plan is correct again.  The same for the tensor-core Hadamard kernel.
- An index list with a basis-function index outside [0, N_b): the device check gives that entry
  NaN and reads nothing for it, the other entries are unchanged, and the plan reports
  LRTEI_ERR_ARG (both entry points).
- A density holding a NaN: the J-build's unpacking kernel sees a non-finite J and the plan
  reports LRTEI_ERR_NUMERIC.
"""
import os

import numpy as np
import pytest

from paper_2210_13069_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import torch
    from paper_2210_13069_gb300 import build_lib, lrtei
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build_lib.build()
    lrtei.load()
    return lrtei


def test_gemm_wait_that_runs_out_reports_timeout_then_recovers(lib):
    import torch
    m = synth.workload_small_s()
    ref_plan = lib.Plan(m, "fp64")
    ref = ref_plan.assemble_B("factored").cpu().numpy()
    ref_plan.close()
    pl = lib.Plan(m, "split_f16")
    os.environ["LRTEI_TEST_STALL_CYCLES"] = "200000"  # ~0.1 ms, then the abort path
    try:
        pl.assemble_B("factored")
        torch.cuda.synchronize()
    finally:
        del os.environ["LRTEI_TEST_STALL_CYCLES"]
    with pytest.raises(lib.LrteiError) as ei:
        pl.status()
    assert ei.value.status == 4, ei.value
    # the context is intact and the same plan computes correctly afterwards
    B = pl.assemble_B("factored").cpu().numpy()
    pl.status()
    err = np.linalg.norm(B - ref) / np.linalg.norm(ref)
    assert err <= 1e-7, err
    pl.close()


def test_hadamard_kernel_wait_that_runs_out_reports_timeout_then_recovers(lib):
    """The same bounded-wait failure path in the tensor-core Hadamard kernel (uncontracted s
    functions): its MMA thread waits on a barrier nothing completes, every role leaves through
    its bounded drain, the plan reports LRTEI_ERR_TIMEOUT, and the next call is correct."""
    import torch
    m = synth.workload_small_s()
    ref_plan = lib.Plan(m, "fp64")
    ref = ref_plan.assemble_B("hadamard").cpu().numpy()
    ref_plan.close()
    pl = lib.Plan(m, "split_f16")
    os.environ["LRTEI_TEST_STALL_CYCLES"] = "200000"
    try:
        pl.assemble_B("hadamard")
        torch.cuda.synchronize()
    finally:
        del os.environ["LRTEI_TEST_STALL_CYCLES"]
    with pytest.raises(lib.LrteiError) as ei:
        pl.status()
    assert ei.value.status == 4, ei.value
    B = pl.assemble_B("hadamard").cpu().numpy()
    pl.status()
    assert pl.info["last_form"] == 1
    err = np.linalg.norm(B - ref) / np.linalg.norm(ref)
    assert err <= 2e-8, err
    pl.close()


@pytest.mark.parametrize("entry_point", ["lrtei_entries", "lrtei_entries_noalloc"])
def test_out_of_range_index_gives_nan_and_arg_status(lib, entry_point):
    import torch
    m = synth.workload_small_s()
    pl = lib.Plan(m, "fp64")
    rng = np.random.default_rng(5)
    idx = rng.integers(0, m.nbf, size=(300, 4)).astype(np.int32)
    good = torch.empty(len(idx), dtype=torch.float64, device="cuda")
    lib.lrtei_entries(pl.plan, torch.as_tensor(idx, device="cuda"), len(idx), good)
    pl.status()
    bad = idx.copy()
    bad[17, 2] = m.nbf          # one past the end
    bad[250, 0] = -3            # negative
    d_bad = torch.as_tensor(bad, device="cuda")
    out = torch.zeros(len(idx), dtype=torch.float64, device="cuda")
    getattr(lib, entry_point)(pl.plan, d_bad, len(idx), out)
    torch.cuda.synchronize()
    with pytest.raises(lib.LrteiError) as ei:
        pl.status()
    assert ei.value.status == 1 and "outside" in str(ei.value)
    o, g = out.cpu().numpy(), good.cpu().numpy()
    assert np.isnan(o[17]) and np.isnan(o[250])
    keep = np.ones(len(idx), bool)
    keep[[17, 250]] = False
    assert np.all(np.isfinite(o[keep]))
    assert np.max(np.abs(o[keep] - g[keep])) <= 1e-13 * np.abs(g).max()
    pl.status()  # the status was cleared by the read above
    pl.close()


def test_nonfinite_density_reports_numeric(lib):
    import torch
    m = synth.workload_small_s()
    pl = lib.Plan(m, "fp64")
    D = torch.as_tensor(synth.random_densities(11, m.nbf, 2), device="cuda")
    J = pl.jbuild(D)
    pl.status()
    assert torch.isfinite(J).all()
    D[1, 3, 4] = float("nan")
    D[1, 4, 3] = float("nan")
    pl.jbuild(D, out=J)
    torch.cuda.synchronize()
    with pytest.raises(lib.LrteiError) as ei:
        pl.status()
    assert ei.value.status == 5, ei.value
    pl.close()
