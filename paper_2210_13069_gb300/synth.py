"""Seeded synthetic inputs: molecules (Gaussian basis sets) and density matrices.

This module only draws random inputs.  It holds none of the tensorized-approximation
arithmetic and is the one piece of code that both the CUDA path and the CPU oracle
consume (the oracle never imports the CUDA binding and vice versa).

The paper evaluates on quantum-package cc-pVDZ molecules (Section 6).  Those files are
not available here, so seeded stand-ins with the same role are drawn instead: atoms at
uniform positions in a cube, per atom a fixed list of contracted Cartesian shells
(s/p/d), exponents log-uniform in a range, contraction coefficients uniform.

Every generator uses numpy's counter-based Philox bit generator with an explicit seed.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Sequence, Tuple

import numpy as np

L_OF = {"s": 0, "p": 1, "d": 2}


@dataclass
class Shell:
    """One contracted Cartesian shell: center (bohr), angular momentum l, exponents, coefficients."""

    center: np.ndarray
    l: int
    exps: np.ndarray
    coefs: np.ndarray

    @property
    def ncart(self) -> int:
        return (self.l + 1) * (self.l + 2) // 2


@dataclass
class Molecule:
    """A synthetic molecule plus the TA parameters (omega, n, P) it is run with."""

    atoms: np.ndarray
    shells: List[Shell]
    omega: float
    n: int
    P: int
    name: str = ""
    box_lo: np.ndarray | None = None
    box_hi: np.ndarray | None = None

    @property
    def nbf(self) -> int:
        return sum(s.ncart for s in self.shells)

    def packed(self) -> Tuple[np.ndarray, np.ndarray, np.ndarray, np.ndarray, np.ndarray]:
        """Flat arrays (centers[ns,3], l[ns], nprim[ns], exps[sum nprim], coefs[sum nprim])."""
        centers = np.ascontiguousarray(np.array([s.center for s in self.shells], dtype=np.float64).reshape(-1, 3))
        ls = np.array([s.l for s in self.shells], dtype=np.int32)
        nprim = np.array([len(s.exps) for s in self.shells], dtype=np.int32)
        exps = np.ascontiguousarray(np.concatenate([s.exps for s in self.shells]).astype(np.float64))
        coefs = np.ascontiguousarray(np.concatenate([s.coefs for s in self.shells]).astype(np.float64))
        return centers, ls, nprim, exps, coefs


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(int(seed)))


def random_molecule(seed: int, natoms: int, cube: float,
                    shells_per_atom: Sequence[Tuple[str, int]] = (("s", 3), ("p", 2), ("d", 1)),
                    nprim: int = 3, alpha_range: Tuple[float, float] = (0.05, 2.0e3),
                    coef_range: Tuple[float, float] = (0.1, 1.0),
                    omega: float = 0.4, n: int = 24, P: int = 32, name: str = "") -> Molecule:
    """Atoms uniform in [0, cube]^3; each atom carries ``shells_per_atom`` contracted shells.

    Exponents are log-uniform in ``alpha_range`` (sorted descending inside a shell, as in
    tabulated basis sets); coefficients are uniform in ``coef_range`` (1.0 when nprim == 1).
    """
    rng = _rng(seed)
    atoms = rng.uniform(0.0, cube, size=(natoms, 3))
    lo, hi = np.log(alpha_range[0]), np.log(alpha_range[1])
    shells: List[Shell] = []
    for a in range(natoms):
        for kind, count in shells_per_atom:
            for _ in range(count):
                e = np.sort(np.exp(rng.uniform(lo, hi, size=nprim)))[::-1].copy()
                c = np.ones(nprim) if nprim == 1 else rng.uniform(coef_range[0], coef_range[1], size=nprim)
                shells.append(Shell(center=atoms[a].copy(), l=L_OF[kind], exps=e, coefs=c))
    return Molecule(atoms=atoms, shells=shells, omega=omega, n=n, P=P, name=name)


def random_densities(seed: int, nbf: int, R: int, rank: int | None = None) -> np.ndarray:
    """R symmetric PSD densities D_r = X_r X_r^T, X_r in R^{nbf x rank}, entries N(0, 1/nbf).

    Returns an array of shape (R, nbf, nbf), float64, C order.
    """
    rng = _rng(seed)
    k = max(1, nbf // 4) if rank is None else rank
    X = rng.normal(0.0, 1.0 / np.sqrt(nbf), size=(R, nbf, k))
    D = np.einsum("rik,rjk->rij", X, X)
    return np.ascontiguousarray(0.5 * (D + D.transpose(0, 2, 1)))


# ---------------------------------------------------------------------------------------
# Named workloads.  Seeds are 1000 + workload index; molecule index is mixed in for the
# batched and selector sets.
# ---------------------------------------------------------------------------------------

def workload_small_s(seed: int = 1001) -> Molecule:
    """4 atoms in a 6 bohr cube, 5 uncontracted s functions per atom (N_b = 20),
    exponents log-uniform in [0.1, 50]; omega = 0.5, n = 16, P = 20."""
    return random_molecule(seed, natoms=4, cube=6.0, shells_per_atom=(("s", 5),), nprim=1,
                           alpha_range=(0.1, 50.0), omega=0.5, n=16, P=20, name="nb20_s")


def workload_spd(seed: int = 1002, natoms: int = 12, cube: float = 12.0, omega: float = 0.4,
                 n: int = 24, P: int = 32, nprim: int = 3) -> Molecule:
    """12 atoms in a 12 bohr cube, 3s+2p+1d contracted shells per atom (N_b = 180)."""
    return random_molecule(seed, natoms=natoms, cube=cube, nprim=nprim, omega=omega, n=n, P=P,
                           name=f"nb{15 * natoms}_spd")


def workload_spd_large(seed: int = 1003) -> Molecule:
    """24 atoms in a cube of side 12 * 2**(1/3) bohr (N_b = 360), omega = 0.33."""
    return random_molecule(seed, natoms=24, cube=12.0 * 2.0 ** (1.0 / 3.0), omega=0.33, n=24, P=32,
                           name="nb360_spd")


def workload_batch(seed: int = 1004, nmol: int = 64) -> List[Molecule]:
    """64 molecules, 2..20 atoms each (N_b = 15 * atoms), cube side 12 * (atoms/12)^(1/3),
    omega in {0.2, 0.33, 0.5, 1.0}, n in [20, 28], P in [24, 40]."""
    rng = _rng(seed)
    mols = []
    for i in range(nmol):
        natoms = int(rng.integers(2, 21))
        omega = float(rng.choice([0.2, 0.33, 0.5, 1.0]))
        n = int(rng.integers(20, 29))
        P = int(rng.integers(24, 41))
        cube = 12.0 * (natoms / 12.0) ** (1.0 / 3.0)
        mols.append(random_molecule(seed * 1000 + i, natoms=natoms, cube=cube, omega=omega, n=n, P=P,
                                    name=f"batch{i}"))
    return mols
