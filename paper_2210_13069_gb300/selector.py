"""Learned choice of the Chebyshev order n and the quadrature size P.

The paper picks the number of interpolation nodes per quadrature node with chebfun2 and shows
how the error trades n against P (Section 3.1, Section 6.1).  Here a small MLP (6 -> 64 -> 64
-> 2, trained on the GPU by the library's own forward/backward/Adam kernels) maps
    (omega, box half-width, log10 alpha_min, log10 alpha_max, max l, log10 target)
to the cheapest (n, P) that reached the target error in error sweeps of the plain method:
entries of B computed by the library at each (n, P) against the same entries at a high
reference order.  Out of the trained range, or if asked, the conservative fixed (32, 48) is
used instead.

Every number here comes from the CUDA library (Algorithm 1 entries); nothing calls the CPU
oracle.
"""
from __future__ import annotations

import hashlib
import io
import json
import math
from dataclasses import dataclass
from typing import List, Optional, Sequence, Tuple

import numpy as np

from . import lrtei, synth

N_GRID = [8, 12, 16, 20, 24, 28, 32, 40, 48, 56]
P_GRID = [8, 12, 16, 20, 24, 28, 32, 40, 48, 64, 80, 96]
N_REF, P_REF = 64, 128
TARGETS = [10.0 ** -k for k in range(3, 10)]
FALLBACK = (32, 48)
N_MAX, P_MAX = 64, 128
# training ranges of the features (inference outside them falls back)
RANGES = {"omega": (0.2, 1.0), "half": (3.0, 34.0), "lamin": (-1.4, 0.1), "lamax": (-0.4, 3.4), "lmax": (0, 2),
          "ltarget": (-9.0, -3.0)}


def features(omega: float, half: float, amin: float, amax: float, lmax: int, target: float) -> np.ndarray:
    """Normalised feature vector of one instance."""
    return np.array([omega, half / 30.0, math.log10(amin), math.log10(amax) / 4.0, lmax / 2.0,
                     -math.log10(target) / 10.0], dtype=np.float32)


def in_range(omega, half, amin, amax, lmax, target) -> bool:
    r = RANGES
    vals = {"omega": omega, "half": half, "lamin": math.log10(amin), "lamax": math.log10(amax), "lmax": lmax,
            "ltarget": math.log10(target)}
    return all(r[k][0] - 1e-9 <= v <= r[k][1] + 1e-9 for k, v in vals.items())


def encode_targets(n: float, P: float) -> np.ndarray:
    return np.array([(n - 8.0) / 56.0, (P - 8.0) / 120.0], dtype=np.float32)


def decode(y: np.ndarray) -> Tuple[float, float]:
    return 8.0 + 56.0 * float(y[0]), 8.0 + 120.0 * float(y[1])


def molecule_features(mol) -> Tuple[float, float, float, int]:
    amin = min(float(np.min(s.exps)) for s in mol.shells)
    amax = max(float(np.max(s.exps)) for s in mol.shells)
    lmax = max(s.l for s in mol.shells)
    return amin, amax, lmax


# ------------------------------------------------------------------ error sweeps on the GPU

def sweep_molecule(seed: int):
    """A random small instance spanning the feature ranges: 2-3 atoms inside an explicit box of
    half-width 3..34 bohr, one contracted shell per atom (l up to 2), omega in [0.2, 1]."""
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


def _entries(mol, n: int, P: int, idx_dev) -> np.ndarray:
    import torch
    pl = lrtei.Plan(mol, "fp64", n=n, P=P)
    out = torch.empty(idx_dev.shape[0], dtype=torch.float64, device="cuda")
    lrtei.lrtei_entries(pl.plan, idx_dev, idx_dev.shape[0], out)
    res = out.cpu().numpy()
    pl.close()
    return res


def sweep(seed: int, nent: int = 96) -> dict:
    """Errors of sampled entries at every n of N_GRID (P = P_REF) and every P of P_GRID
    (n = N_REF), relative (Frobenius over the sample) to the entries at (N_REF, P_REF)."""
    import torch
    mol, half, omega = sweep_molecule(seed)
    rng = np.random.Generator(np.random.Philox(seed + 7))
    idx = rng.integers(0, mol.nbf, size=(nent, 4)).astype(np.int32)
    idx_dev = torch.as_tensor(idx, device="cuda")
    ref = _entries(mol, N_REF, P_REF, idx_dev)
    nrm = np.linalg.norm(ref)
    err_n = [float(np.linalg.norm(_entries(mol, n, P_REF, idx_dev) - ref) / nrm) for n in N_GRID]
    err_P = [float(np.linalg.norm(_entries(mol, N_REF, P, idx_dev) - ref) / nrm) for P in P_GRID]
    amin, amax, lmax = molecule_features(mol)
    return {"seed": seed, "omega": omega, "half": half, "amin": amin, "amax": amax, "lmax": lmax, "err_n": err_n,
            "err_P": err_P}


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
    """An MLP on the GPU (library kernels) plus the fallback rule."""

    VERSION = 1

    def __init__(self, hidden: int = 64, seed: int = 1):
        self.hidden = hidden
        self.handle = lrtei.lrtei_selector_create(hidden, seed)

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
        dX = torch.as_tensor(X, device="cuda")
        dY = torch.as_tensor(Y, device="cuda")
        hist = []
        for ep in range(epochs):
            cur = lr if ep < epochs * 2 // 3 else lr * 0.1
            hist.append(lrtei.lrtei_selector_train_epoch(self.handle, dX, dY, len(X), batch, cur))
        return hist

    def predict_raw(self, X: np.ndarray) -> np.ndarray:
        import torch
        dX = torch.as_tensor(np.ascontiguousarray(X, dtype=np.float32), device="cuda")
        out = torch.empty((len(X), 2), dtype=torch.float32, device="cuda")
        lrtei.lrtei_selector_forward(self.handle, dX, out, len(X))
        return out.cpu().numpy()

    def select(self, omega, half, amin, amax, lmax, target, margin: Tuple[int, int] = (4, 8)) -> Tuple[int, int, bool]:
        """(n, P, used_fallback): the network's choice rounded up to the grids plus a margin, or
        the fixed conservative (32, 48) outside the trained range."""
        if not in_range(omega, half, amin, amax, lmax, target):
            return FALLBACK[0], FALLBACK[1], True
        n, P = decode(self.predict_raw(features(omega, half, amin, amax, lmax, target)[None, :])[0])
        n = next((g for g in N_GRID + [N_MAX] if g >= n + margin[0]), N_MAX)
        P = next((g for g in P_GRID + [P_MAX] if g >= P + margin[1]), P_MAX)
        return int(n), int(P), False

    # checkpoint: versioned, with a checksum of the parameter bytes
    def save(self, path: str, meta: Optional[dict] = None):
        params = lrtei.lrtei_selector_get_params(self.handle)
        digest = hashlib.sha256(params.tobytes()).hexdigest()
        header = {"version": self.VERSION, "hidden": self.hidden, "sha256": digest, "meta": meta or {}}
        with open(path, "wb") as f:
            np.savez(f, params=params, header=np.frombuffer(json.dumps(header).encode(), dtype=np.uint8))

    @classmethod
    def load(cls, path: str) -> "Selector":
        with open(path, "rb") as f:
            z = np.load(io.BytesIO(f.read()))
        header = json.loads(bytes(z["header"]).decode())
        if header.get("version") != cls.VERSION:
            raise ValueError(f"selector checkpoint version {header.get('version')} != {cls.VERSION}")
        params = z["params"].astype(np.float32)
        if hashlib.sha256(params.tobytes()).hexdigest() != header["sha256"]:
            raise ValueError("selector checkpoint checksum mismatch")
        sel = cls(hidden=int(header["hidden"]))
        lrtei.lrtei_selector_set_params(sel.handle, params)
        return sel
