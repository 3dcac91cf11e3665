"""lrtei_entries_noalloc: Algorithm 1 entries for callers that cannot allocate device memory.

The call is checked through the C ABI against lrtei_entries (same plan, same index list) on
two calls in a row, within the FP64 tolerance of the other parity tests (1e-12 relative
Frobenius and max-norm), on a plain and on a screened plan; around each call the library's own
allocation counter (lrtei_profile_get("alloc")) and the device's free memory must not move,
which is the property the call exists for.  Its size limit is checked to be refused before any
launch.  This file is collected last on purpose; it passes alone in a fresh process too.
"""
import numpy as np
import pytest

from paper_2210_13069_gb300 import synth

pytestmark = pytest.mark.gpu


def _mol():
    m = synth.random_molecule(2002, natoms=3, cube=5.0, nprim=2, alpha_range=(0.2, 30.0), omega=0.5, n=10, P=10)
    rng = np.random.default_rng(2002)
    for i, sh in enumerate(m.shells):
        k = 1 + (i % 3)
        sh.exps = np.sort(np.exp(rng.uniform(np.log(0.2), np.log(30.0), size=k)))[::-1].copy()
        sh.coefs = rng.uniform(0.1, 1.0, size=k)
    return m


@pytest.mark.parametrize("tau", [0.0, 1e-3])
def test_noalloc_entries_match_lrtei_entries_twice(tau):
    import torch
    from paper_2210_13069_gb300 import build_lib, lrtei
    assert torch.cuda.is_available(), "GPU test"
    build_lib.build()
    lrtei.load()
    m = _mol()
    pl = lrtei.Plan(m, "fp64", tau_screening=tau)
    if tau > 0:
        assert pl.info["nrows"] < lrtei.Plan(m, "fp64").info["nrows"]  # some pairs were screened out
    rng = np.random.default_rng(77)
    for call, count in enumerate((4000, 9000)):
        idx = torch.as_tensor(rng.integers(0, m.nbf, size=(count, 4)).astype(np.int32), device="cuda")
        ref = torch.empty(count, dtype=torch.float64, device="cuda")
        lrtei.lrtei_entries(pl.plan, idx, count, ref)
        got = torch.full((count,), float("nan"), dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        allocs0 = lrtei.lrtei_profile_get("alloc")[1]
        free0 = torch.cuda.mem_get_info()[0]
        lrtei.lrtei_entries_noalloc(pl.plan, idx, count, got)
        torch.cuda.synchronize()
        assert lrtei.lrtei_profile_get("alloc")[1] == allocs0, "the no-allocation call requested device memory"
        assert torch.cuda.mem_get_info()[0] == free0
        pl.status()
        r, g = ref.cpu().numpy(), got.cpu().numpy()
        assert np.all(np.isfinite(g)), call
        assert np.linalg.norm(g - r) <= 1e-12 * np.linalg.norm(r), call
        assert np.max(np.abs(g - r)) <= 1e-12 * np.abs(r).max(), call
    pl.close()


def test_noalloc_rejects_oversized_request():
    import torch
    from paper_2210_13069_gb300 import build_lib, lrtei
    build_lib.build()
    m = _mol()
    pl = lrtei.Plan(m, "fp64")
    too_many = (1 << 18) + 1
    idx = torch.zeros((too_many, 4), dtype=torch.int32, device="cuda")
    out = torch.empty(too_many, dtype=torch.float64, device="cuda")
    with pytest.raises(lrtei.LrteiError) as ei:
        lrtei.lrtei_entries_noalloc(pl.plan, idx, too_many, out)
    assert ei.value.status == 6 and "at most 262144" in str(ei.value)
    pl.close()
