"""Learned choice of the Chebyshev order n and the quadrature size P: sweep orchestration and
marshalling around the library's selector calls.

The paper picks the number of interpolation nodes per quadrature node with chebfun2 and shows
how the error trades n against P (Section 3.1, Section 6.1).  Here a small MLP (6 -> 64 -> 64
-> 2, trained on the GPU by the library's own forward/backward/Adam kernels) maps
    (omega, box half-width, alpha_min, alpha_max, max l, target)
to the cheapest (n, P) that reached the target error in error sweeps of the plain method.
Feature normalisation, the training ranges, the fallback to the conservative fixed (32, 48),
the margins and the rounding to the grids, training and checkpoints all live in the library
(lrtei_selector_features / _encode / lrtei_select_np / lrtei_selector_train / _save / _load);
this module draws the sweep instances, runs the sweeps through lrtei_entries_orders and builds
the labels.

Every number here comes from the CUDA library; nothing calls the CPU oracle.
"""
from __future__ import annotations

import json
from typing import List, Optional, Sequence, Tuple

import numpy as np

from . import lrtei, synth

N_GRID = [8, 12, 16, 20, 24, 28, 32, 40, 48, 56]
P_GRID = [8, 12, 16, 20, 24, 28, 32, 40, 48, 64, 80, 96]
N_REF, P_REF = 64, 128
TARGETS = [10.0 ** -k for k in range(3, 10)]
FALLBACK = (32, 48)


def features(omega: float, half: float, amin: float, amax: float, lmax: int, target: float) -> np.ndarray:
    """Normalised feature vector of one instance (computed by the library)."""
    return lrtei.lrtei_selector_features([omega, half, amin, amax, lmax, target])


def encode_targets(n: float, P: float) -> np.ndarray:
    return lrtei.lrtei_selector_encode(int(n), int(P))


def molecule_features(mol) -> Tuple[float, float, int]:
    amin = min(float(np.min(s.exps)) for s in mol.shells)
    amax = max(float(np.max(s.exps)) for s in mol.shells)
    lmax = max(s.l for s in mol.shells)
    return amin, amax, lmax


# ------------------------------------------------------------------ error sweeps on the GPU

def sweep_molecule(seed: int):
    """A random small instance spanning the feature ranges: 2-3 atoms inside an explicit box of
    half-width 3..32 bohr, one contracted shell per atom (l up to 2), omega in [0.2, 1]."""
    rng = np.random.Generator(np.random.Philox(seed))
    half = float(np.exp(rng.uniform(np.log(3.0), np.log(32.0))))
    omega = float(rng.uniform(0.2, 1.0))
    lmax = int(rng.integers(0, 3))
    amin = float(10 ** rng.uniform(-1.3, 0.0))
    amax = float(10 ** rng.uniform(max(np.log10(amin) + 0.5, -0.3), 3.3))
    natoms = int(rng.integers(2, 4))
    atoms = rng.uniform(-0.4 * half, 0.4 * half, size=(natoms, 3))
    shells = []
    for a in range(natoms):
        l = lmax if a == 0 else int(rng.integers(0, lmax + 1))
        k = int(rng.integers(1, 3))
        e = np.sort(np.exp(rng.uniform(np.log(amin), np.log(amax), size=k)))[::-1].copy()
        e[-1] = amin if a == 0 else e[-1]
        e[0] = amax if a == natoms - 1 else e[0]
        shells.append(synth.Shell(center=atoms[a].copy(), l=l, exps=e, coefs=rng.uniform(0.3, 1.0, size=k)))
    mol = synth.Molecule(atoms=atoms, shells=shells, omega=omega, n=N_REF, P=P_REF, name=f"sweep{seed}",
                         box_lo=np.full(3, -half), box_hi=np.full(3, half))
    return mol, half, omega


def sweep_indices(seed: int, nbf: int, nent: int) -> np.ndarray:
    rng = np.random.Generator(np.random.Philox(seed + 7))
    return rng.integers(0, nbf, size=(nent, 4)).astype(np.int32)


def _entries(mol, n: int, P: int, idx_dev) -> np.ndarray:
    """Algorithm 1 entries of a fresh plan at (n, P) (lrtei_entries)."""
    import torch
    pl = lrtei.Plan(mol, "fp64", n=n, P=P)
    out = torch.empty(idx_dev.shape[0], dtype=torch.float64, device="cuda")
    lrtei.lrtei_entries(pl.plan, idx_dev, idx_dev.shape[0], out)
    res = out.cpu().numpy()
    pl.close()
    return res


def sweep(seed: int, nent: int = 32) -> dict:
    """Errors of sampled entries at every n of N_GRID (P = P_REF) and every P of P_GRID
    (n = N_REF), relative (Frobenius over the sample) to the entries at (N_REF, P_REF): one plan
    at the reference orders, every order evaluated by lrtei_entries_orders."""
    import torch
    mol, half, omega = sweep_molecule(seed)
    idx = torch.as_tensor(sweep_indices(seed, mol.nbf, nent), device="cuda")
    ns = N_GRID + [N_REF] * len(P_GRID) + [N_REF]
    Ps = [P_REF] * len(N_GRID) + P_GRID + [P_REF]
    pl = lrtei.Plan(mol, "fp64")
    out = torch.empty((len(ns), nent), dtype=torch.float64, device="cuda")
    lrtei.lrtei_entries_orders(pl.plan, ns, Ps, idx, nent, out)
    res = out.cpu().numpy()
    pl.status()
    pl.close()
    ref = res[-1]
    nrm = np.linalg.norm(ref)
    err = [float(np.linalg.norm(r - ref) / nrm) for r in res[:-1]]
    amin, amax, lmax = molecule_features(mol)
    return {"seed": seed, "omega": omega, "half": half, "amin": amin, "amax": amax, "lmax": lmax,
            "err_n": err[:len(N_GRID)], "err_P": err[len(N_GRID):]}


def label(sw: dict, target: float) -> Optional[Tuple[int, int]]:
    """Cheapest grid (n, P) with both error components at most target/4; None if unreachable."""
    n = next((g for g, e in zip(N_GRID, sw["err_n"]) if e <= target / 4), None)
    P = next((g for g, e in zip(P_GRID, sw["err_P"]) if e <= target / 4), None)
    if n is None or P is None:
        return None
    return n, P


def dataset(sweeps: Sequence[dict]):
    X, Y = [], []
    for sw in sweeps:
        for t in TARGETS:
            lab = label(sw, t)
            if lab is None:
                continue
            X.append(features(sw["omega"], sw["half"], sw["amin"], sw["amax"], sw["lmax"], t))
            Y.append(encode_targets(*lab))
    return np.array(X, dtype=np.float32), np.array(Y, dtype=np.float32)


# ------------------------------------------------------------------ the selector object

class Selector:
    """A handle on the library's selector (network on the GPU, policy in the library)."""

    def __init__(self, hidden: int = 64, seed: int = 1, handle: Optional[int] = None):
        self.hidden = hidden
        self.handle = handle if handle is not None else lrtei.lrtei_selector_create(hidden, seed)

    def close(self):
        if getattr(self, "handle", None):
            lrtei.lrtei_selector_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def train(self, X: np.ndarray, Y: np.ndarray, epochs: int = 300, batch: int = 256, lr: float = 2e-3):
        import torch
        dX = torch.as_tensor(np.ascontiguousarray(X, dtype=np.float32), device="cuda")
        dY = torch.as_tensor(np.ascontiguousarray(Y, dtype=np.float32), device="cuda")
        return list(lrtei.lrtei_selector_train(self.handle, dX, dY, len(X), epochs, batch, lr))

    def predict_raw(self, X: np.ndarray) -> np.ndarray:
        import torch
        dX = torch.as_tensor(np.ascontiguousarray(X, dtype=np.float32), device="cuda")
        out = torch.empty((len(X), 2), dtype=torch.float32, device="cuda")
        lrtei.lrtei_selector_forward(self.handle, dX, out, len(X))
        return out.cpu().numpy()

    def select(self, omega, half, amin, amax, lmax, target) -> Tuple[int, int, bool]:
        """(n, P, used_fallback) from lrtei_select_np."""
        return lrtei.lrtei_select_np(self.handle, [omega, half, amin, amax, lmax, target])

    def save(self, path: str, meta: Optional[dict] = None):
        lrtei.lrtei_selector_save(self.handle, path, json.dumps(meta or {}))

    @classmethod
    def load(cls, path: str) -> "Selector":
        h, meta = lrtei.lrtei_selector_load(path)
        npar = lrtei.lrtei_selector_nparams(h)  # H^2 + 10 H + 2 parameters for width H
        hidden = int(round((-10 + (100 - 4 * (2 - npar)) ** 0.5) / 2))
        sel = cls(hidden=hidden, handle=h)
        sel.meta = json.loads(meta) if meta else {}
        return sel


# ------------------------------------------------------------------ training run

DEFAULT_CHECKPOINT = "selector_20k.bin"


def train_from_sweeps(nsweeps: int, seed0: int = 10_000, epochs: int = 60, hidden: int = 64, net_seed: int = 11,
                      log=print):
    """Error sweeps of instances seed0 .. seed0 + nsweeps - 1, their labels, and a network trained
    on them; returns (selector, number of labelled rows, loss history)."""
    import time
    t0 = time.perf_counter()
    sweeps = []
    for i in range(nsweeps):
        sweeps.append(sweep(seed0 + i))
        if log and (i + 1) % 1000 == 0:
            log(f"  {i + 1} sweeps, {time.perf_counter() - t0:.0f} s")
    X, Y = dataset(sweeps)
    sel = Selector(hidden, seed=net_seed)
    hist = sel.train(X, Y, epochs=epochs, batch=256, lr=2e-3)
    if log:
        log(f"{nsweeps} sweeps in {time.perf_counter() - t0:.0f} s, {len(X)} labelled rows, loss {hist[0]:.2e} -> "
            f"{hist[-1]:.2e}")
    return sel, len(X), hist


def main(argv=None):
    """python -m paper_2210_13069_gb300.selector --sweeps N --out FILE: train on N sweeps (seeds
    10000..) and write the checkpoint (the library's versioned, checksummed format)."""
    import argparse
    import os
    ap = argparse.ArgumentParser()
    ap.add_argument("--sweeps", type=int, default=20_000)
    ap.add_argument("--epochs", type=int, default=60)
    ap.add_argument("--out", default=os.path.join(os.path.dirname(os.path.abspath(__file__)), DEFAULT_CHECKPOINT))
    a = ap.parse_args(argv)
    from . import build_lib
    build_lib.build()
    sel, rows, hist = train_from_sweeps(a.sweeps, epochs=a.epochs)
    sel.save(a.out, meta={"sweeps": a.sweeps, "first_seed": 10_000, "rows": rows, "epochs": a.epochs,
                          "final_loss": float(hist[-1]), "n_grid": N_GRID, "p_grid": P_GRID,
                          "reference": [N_REF, P_REF]})
    print(f"wrote {a.out}")


if __name__ == "__main__":
    main()
