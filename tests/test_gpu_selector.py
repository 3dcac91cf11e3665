"""The learned (n, P) selector: the device MLP kernels against the FP64 CPU reference network,
training by the device Adam kernel, the selection policy and checkpoints through the C ABI, and
the selector judged by the FP64 oracle on held-out instances.

Training data are error sweeps of the plain method computed by the CUDA library
(lrtei_entries_orders); the held-out instances are drawn with other seeds.  The error of the
chosen (n, P) on a held-out instance is that of the library's entries (a fresh plan at that
(n, P), lrtei_entries) against the FP64 oracle's entries at the reference orders (64, 128) on the
same sampled indices: the oracle is the judge, not the library.
"""
import os

import numpy as np
import pytest

import oracle
from oracle import mlp as mlp_ref

pytestmark = pytest.mark.gpu

# Sweeps the test itself trains on (exercising sweeps and training on the GPU); the held-out
# evaluation judges the committed network trained on 20 000 sweeps by
# `python -m paper_2210_13069_gb300.selector --sweeps 20000` (seeds 10000..29999).
N_SWEEPS = int(os.environ.get("LRTEI_TEST_SELECTOR_SWEEPS", "300"))
CHECKPOINT = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2210_13069_gb300",
                          "selector_20k.bin")


@pytest.fixture(scope="module")
def lib():
    import torch
    from paper_2210_13069_gb300 import build_lib, lrtei
    assert torch.cuda.is_available()
    build_lib.build()
    lrtei.load()
    return lrtei


def test_mlp_forward_and_gradient_match_cpu_reference(lib):
    import torch
    H = 64
    sel = lib.lrtei_selector_create(H, 5)
    try:
        theta = lib.lrtei_selector_get_params(sel).astype(np.float64)
        rng = np.random.default_rng(1)
        X = rng.normal(0, 1, (777, 6)).astype(np.float32)
        T = rng.normal(0, 1, (777, 2)).astype(np.float32)
        dX, dT = torch.as_tensor(X, device="cuda"), torch.as_tensor(T, device="cuda")
        out = torch.empty((777, 2), dtype=torch.float32, device="cuda")
        lib.lrtei_selector_forward(sel, dX, out, 777)
        y_ref = mlp_ref.forward(theta, H, X.astype(np.float64))
        assert np.max(np.abs(out.cpu().numpy() - y_ref)) <= 1e-4 * max(1.0, np.abs(y_ref).max())
        g = torch.empty(lib.lrtei_selector_nparams(sel), dtype=torch.float32, device="cuda")
        loss = lib.lrtei_selector_grad(sel, dX, dT, 777, g)
        L_ref, g_ref = mlp_ref.loss_and_grad(theta, H, X.astype(np.float64), T.astype(np.float64))
        assert abs(loss - L_ref) <= 1e-5 * L_ref
        gg = g.cpu().numpy()
        assert np.linalg.norm(gg - g_ref) <= 1e-4 * np.linalg.norm(g_ref)
    finally:
        lib.lrtei_selector_destroy(sel)


def test_adam_training_fits_a_smooth_map(lib):
    from paper_2210_13069_gb300.selector import Selector
    rng = np.random.default_rng(2)
    X = rng.uniform(-1, 1, (4096, 6)).astype(np.float32)
    Y = np.stack([0.5 * np.sin(X[:, 0] * 2) + 0.2 * X[:, 1] * X[:, 2], 0.3 * X[:, 3] ** 2 - 0.1 * X[:, 4]], 1)
    s = Selector(64, seed=3)
    hist = s.train(X, Y.astype(np.float32), epochs=120, batch=256, lr=3e-3)
    assert hist[-1] < 0.05 * hist[0]
    assert hist[-1] < 2e-3


def test_selection_policy_through_the_c_abi(lib, tmp_path):
    """Range check and fallback, grid rounding with margins, checkpoint round trip, and rejection
    of a corrupted or foreign checkpoint: all inside the library."""
    sel = lib.lrtei_selector_create(64, 9)
    try:
        # outside the trained ranges (omega 3, box 50 bohr, target 1e-12): the fixed (32, 48)
        for raw in ([3.0, 10.0, 0.1, 100.0, 1, 1e-6], [0.5, 50.0, 0.1, 100.0, 1, 1e-6],
                    [0.5, 10.0, 0.1, 100.0, 1, 1e-12], [0.5, 10.0, 0.1, 100.0, 3, 1e-6]):
            assert lib.lrtei_select_np(sel, raw) == (32, 48, True)
        n, P, fb = lib.lrtei_select_np(sel, [0.5, 10.0, 0.1, 100.0, 1, 1e-6])
        assert not fb and n in (8, 12, 16, 20, 24, 28, 32, 40, 48, 56, 64) and P in (8, 12, 16, 20, 24, 28, 32, 40,
                                                                                    48, 64, 80, 96, 128)
        for bad in ([0.0, 10.0, 0.1, 100.0, 1, 1e-6], [0.5, 10.0, -0.1, 100.0, 1, 1e-6],
                    [0.5, 10.0, 0.1, 100.0, 1, float("nan")]):
            with pytest.raises(lib.LrteiError) as ei:
                lib.lrtei_select_np(sel, bad)
            assert ei.value.status == 1
        f = lib.lrtei_selector_features([0.5, 12.0, 0.1, 1000.0, 2, 1e-6])
        assert np.allclose(f, [0.5, 0.4, -1.0, 0.75, 1.0, 0.6], atol=1e-7)
        assert np.allclose(lib.lrtei_selector_encode(64, 128), [1.0, 1.0])
        path = str(tmp_path / "sel.bin")
        lib.lrtei_selector_save(sel, path, '{"note": "test"}')
        h2, meta = lib.lrtei_selector_load(path)
        assert meta == '{"note": "test"}'
        assert np.array_equal(lib.lrtei_selector_get_params(sel), lib.lrtei_selector_get_params(h2))
        assert lib.lrtei_select_np(h2, [0.5, 10.0, 0.1, 100.0, 1, 1e-6]) == (n, P, False)
        lib.lrtei_selector_destroy(h2)
        raw = bytearray(open(path, "rb").read())
        raw[40] ^= 1
        bad = str(tmp_path / "bad.bin")
        open(bad, "wb").write(bytes(raw))
        with pytest.raises(lib.LrteiError) as ei:
            lib.lrtei_selector_load(bad)
        assert "checksum" in str(ei.value)
        raw = bytearray(open(path, "rb").read())
        raw[8] = 7  # another version
        open(bad, "wb").write(bytes(raw))
        with pytest.raises(lib.LrteiError) as ei:
            lib.lrtei_selector_load(bad)
        assert "version" in str(ei.value)
    finally:
        lib.lrtei_selector_destroy(sel)


def test_sweep_orders_match_fresh_plans(lib):
    """lrtei_entries_orders (one plan, moments shared across n) against a fresh plan per (n, P)."""
    import torch
    from paper_2210_13069_gb300 import selector as S
    mol, _, _ = S.sweep_molecule(123)
    idx = torch.as_tensor(S.sweep_indices(123, mol.nbf, 40), device="cuda")
    ns, Ps = [8, 24, 56, 64, 64], [128, 128, 128, 12, 128]
    pl = lib.Plan(mol, "fp64")
    out = torch.empty((len(ns), 40), dtype=torch.float64, device="cuda")
    lib.lrtei_entries_orders(pl.plan, ns, Ps, idx, 40, out)
    got = out.cpu().numpy()
    pl.status()
    pl.close()
    for k, (n, P) in enumerate(zip(ns, Ps)):
        ref = S._entries(mol, n, P, idx)
        assert np.max(np.abs(got[k] - ref)) <= 1e-13 * np.abs(ref).max(), (n, P)


def test_training_on_sweeps(lib):
    """Sweeps of the plain method and training on them, on the GPU (a short run)."""
    from paper_2210_13069_gb300 import selector as S
    sel, rows, hist = S.train_from_sweeps(N_SWEEPS, epochs=120)
    assert rows > 2 * N_SWEEPS
    assert hist[-1] < 0.5 * hist[0]
    sel.close()


@pytest.fixture(scope="module")
def trained(lib):
    """The committed selector, trained on 20 000 error sweeps of the plain method."""
    from paper_2210_13069_gb300 import selector as S
    sel = S.Selector.load(CHECKPOINT)
    assert sel.meta.get("sweeps") == 20_000
    print(f"selector checkpoint: {sel.meta}")
    return sel, None, None


def test_selector_meets_target_judged_by_the_oracle(lib, trained):
    """Held-out instances: the chosen (n, P) reaches the requested error against the FP64
    oracle's entries at (64, 128) in at least 90 % of the cases where the plain method can reach
    it, and where the fixed (32, 48) also reaches it the chosen one is cheaper on average (cost of
    a J-build ~ n^3)."""
    import torch
    from paper_2210_13069_gb300 import selector as S
    sel, _, _ = trained
    met = tried = 0
    gains, fixed_fail, worst = [], 0, 0.0
    for i in range(24):
        seed = 90_000 + i
        mol, half, omega = S.sweep_molecule(seed)
        idx_h = S.sweep_indices(seed, mol.nbf, 96)
        idx = torch.as_tensor(idx_h, device="cuda")
        ref = oracle.Oracle.from_molecule(mol, n=S.N_REF, P=S.P_REF).entries(idx_h)  # the judge
        nrm = np.linalg.norm(ref)
        amin, amax, lmax = S.molecule_features(mol)
        err_at = {}

        def err(n, P):
            if (n, P) not in err_at:
                err_at[(n, P)] = float(np.linalg.norm(S._entries(mol, n, P, idx) - ref) / nrm)
            return err_at[(n, P)]

        for t in (1e-4, 1e-6, 1e-8):
            if err(56, 96) > t / 4:  # the plain method's grid cannot reach t on this instance
                continue
            n, P, fb = sel.select(omega, half, amin, amax, lmax, t)
            e = err(n, P)
            tried += 1
            met += e <= t
            worst = max(worst, e / t)
            if err(*S.FALLBACK) <= t:
                gains.append((32 ** 3) / (n ** 3))
            else:
                fixed_fail += 1
    print(f"selector judged by the oracle: met {met}/{tried}; fixed (32, 48) failed {fixed_fail}/{tried}; "
          f"mean cost gain where both meet the target {np.mean(gains):.2f}x; worst error / target {worst:.2f}")
    assert tried >= 40
    assert met >= 0.9 * tried
    assert np.mean(gains) > 1.0


@pytest.mark.parametrize("seed,omega", [(5000, 0.3), (5001, 0.8)])
def test_selector_on_a_600_function_molecule(lib, trained, seed, omega):
    """A 40-atom, 600-function s/p/d molecule (cube side 12 (40/12)^(1/3) bohr, omega = 0.3 or 0.8),
    eight densities, target 1e-6: the factored J-build at the selected (n, P) and at the fixed (32, 48),
    both split-F16 on the tensor cores, against an FP64 J-build at a larger (n, P).  F_u does not
    fit in device memory at these orders, so the J-builds stream it in blocks of unique pairs.
    The selected (n, P) meets the target."""
    import time
    import torch
    from paper_2210_13069_gb300 import selector as S, synth
    sel, _, _ = trained
    target, R = 1e-6, 8
    m = synth.random_molecule(seed, natoms=40, cube=12.0 * (40 / 12) ** (1 / 3), omega=omega, n=32, P=48,
                              name="nb600_spd")
    assert m.nbf == 600
    amin, amax, lmax = S.molecule_features(m)
    probe = lib.Plan(m, "fp64", n=8, P=8)
    half = 0.5 * max(probe.info["box_hi"][d] - probe.info["box_lo"][d] for d in range(3))
    probe.close()
    n_sel, P_sel, fb = sel.select(m.omega, half, amin, amax, lmax, target)
    assert not fb, "the 600-function molecule lies inside the trained feature ranges"
    n_ref, P_ref = min(max(n_sel, 32) + 8, 64), max(P_sel, 48) + 16
    D = torch.as_tensor(synth.random_densities(600, m.nbf, R), device="cuda")

    def jbuild(prec, n, P):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        pl = lib.Plan(m, prec, n=n, P=P)
        J = pl.jbuild(D)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        pl.status()
        pl.close()
        out = J.cpu().numpy()
        del J
        torch.cuda.empty_cache()
        return out, dt

    J_sel, t_sel = jbuild("split_f16", n_sel, P_sel)
    J_fix, t_fix = jbuild("split_f16", 32, 48)
    J_ref, t_ref = jbuild("fp64", n_ref, P_ref)
    e_sel = float(np.linalg.norm(J_sel - J_ref) / np.linalg.norm(J_ref))
    e_fix = float(np.linalg.norm(J_fix - J_ref) / np.linalg.norm(J_ref))
    print(f"selector N_b=600 (omega {omega}, box half-width {half:.1f}): selected (n, P) = ({n_sel}, {P_sel}): error "
          f"{e_sel:.2e}, plan + J-build {t_sel:.1f} s; fixed (32, 48): error {e_fix:.2e}, {t_fix:.1f} s; "
          f"reference FP64 ({n_ref}, {P_ref}) {t_ref:.1f} s")
    assert e_sel <= target
