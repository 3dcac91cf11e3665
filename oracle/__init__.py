"""ctypes wrapper of the FP64 CPU oracle (``lrtei_oracle.c``).

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may import this package.  It never imports the CUDA binding, and the
CUDA binding never imports it.  Inputs are plain numpy arrays (as drawn by the seeded
generator module); nothing here is a fallback of the product path.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liblrtei_oracle.so")
_SRC = os.path.join(_HERE, "lrtei_oracle.c")

_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain -O2, no fast-math, no FMA contraction, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "lrtei_oracle.h"))):
        tmp = _SO + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
               "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    if _lib is None:
        build()
        _lib = load_library(_SO)
    return _lib


def load_library(path: str):
    """Load an oracle shared library from ``path`` and declare its signatures."""
    lib = ctypes.CDLL(path)
    D = ctypes.POINTER(ctypes.c_double)
    I = ctypes.POINTER(ctypes.c_int)
    lib.orc_create.restype = ctypes.c_void_p
    lib.orc_create.argtypes = [ctypes.c_int, D, I, I, D, D, ctypes.c_double, ctypes.c_int, ctypes.c_int, D, D]
    lib.orc_destroy.argtypes = [ctypes.c_void_p]
    lib.orc_set_screening.argtypes = [ctypes.c_void_p, ctypes.c_double]
    lib.orc_nbf.argtypes = [ctypes.c_void_p]
    lib.orc_nbf.restype = ctypes.c_int
    lib.orc_box.argtypes = [ctypes.c_void_p, D, D]
    lib.orc_basis_function.argtypes = [ctypes.c_void_p, ctypes.c_int, D, I, I, D, D]
    lib.orc_gauss_legendre.argtypes = [ctypes.c_int, D, D]
    lib.orc_nodes.argtypes = [ctypes.c_void_p, D, D]
    lib.orc_cheb_coeff.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, D]
    lib.orc_moments.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, D]
    lib.orc_entry.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int]
    lib.orc_entry.restype = ctypes.c_double
    lib.orc_entries.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int32), ctypes.c_int64, D, ctypes.c_int]
    lib.orc_assemble_B.argtypes = [ctypes.c_void_p, D, ctypes.c_int]
    lib.orc_B_rows.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64), ctypes.c_int64, D, ctypes.c_int]
    lib.orc_jbuild_factored.argtypes = [ctypes.c_void_p, D, ctypes.c_int, D, ctypes.c_int]
    lib.orc_factor_M.argtypes = [ctypes.c_void_p, D, ctypes.c_int]
    return lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def default_threads() -> int:
    return max(1, os.cpu_count() or 1)


def gauss_legendre(N: int, lib=None):
    lib = lib or _load()
    z = np.zeros(N)
    w = np.zeros(N)
    lib.orc_gauss_legendre(N, _dp(z), _dp(w))
    return z, w


class Oracle:
    """One molecule + (omega, n, P, box) on the CPU, FP64."""

    def __init__(self, centers, ls, nprim, exps, coefs, omega: float, n: int, P: int,
                 box_lo: Optional[Sequence[float]] = None, box_hi: Optional[Sequence[float]] = None, lib=None,
                 tau_screening: float = 0.0):
        lib = lib or _load()
        self._lib = lib
        self._keep = [np.ascontiguousarray(centers, dtype=np.float64).reshape(-1, 3),
                      np.ascontiguousarray(ls, dtype=np.int32), np.ascontiguousarray(nprim, dtype=np.int32),
                      np.ascontiguousarray(exps, dtype=np.float64), np.ascontiguousarray(coefs, dtype=np.float64)]
        c, l, k, e, cf = self._keep
        blo = bhi = None
        if box_lo is not None:
            blo = np.ascontiguousarray(box_lo, dtype=np.float64)
            bhi = np.ascontiguousarray(box_hi, dtype=np.float64)
        self._h = lib.orc_create(len(l), _dp(c), _ip(l), _ip(k), _dp(e), _dp(cf), float(omega), int(n), int(P),
                                 _dp(blo) if blo is not None else None, _dp(bhi) if bhi is not None else None)
        if not self._h:
            raise ValueError("oracle rejected the input")
        self.omega, self.n, self.P = float(omega), int(n), int(P)
        self.nbf = lib.orc_nbf(self._h)
        self.tau_screening = float(tau_screening)
        if tau_screening:
            lib.orc_set_screening(self._h, float(tau_screening))

    @classmethod
    def from_molecule(cls, mol, **kw):
        centers, ls, nprim, exps, coefs = mol.packed()
        lo = kw.pop("box_lo", mol.box_lo)
        hi = kw.pop("box_hi", mol.box_hi)
        return cls(centers, ls, nprim, exps, coefs, kw.pop("omega", mol.omega), kw.pop("n", mol.n),
                   kw.pop("P", mol.P), box_lo=lo, box_hi=hi, tau_screening=kw.pop("tau_screening", 0.0))

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._lib.orc_destroy(h)
            self._h = None

    def box(self):
        lo = np.zeros(3)
        hi = np.zeros(3)
        self._lib.orc_box(self._h, _dp(lo), _dp(hi))
        return lo, hi

    def basis_function(self, mu: int):
        c = np.zeros(3)
        pw = np.zeros(3, dtype=np.int32)
        k = ctypes.c_int(0)
        e = np.zeros(16)
        cf = np.zeros(16)
        self._lib.orc_basis_function(self._h, mu, _dp(c), _ip(pw), ctypes.byref(k), _dp(e), _dp(cf))
        return c, pw, e[:k.value].copy(), cf[:k.value].copy()

    def nodes(self):
        s = np.zeros(self.P)
        w = np.zeros(self.P)
        self._lib.orc_nodes(self._h, _dp(s), _dp(w))
        return s, w

    def cheb(self, d: int, p: int) -> np.ndarray:
        A = np.zeros((self.n, self.n))
        self._lib.orc_cheb_coeff(self._h, d, p, _dp(A))
        return A

    def moments(self, mu: int, nu: int, d: int) -> np.ndarray:
        I = len(self.basis_function(mu)[2]) * len(self.basis_function(nu)[2])
        W = np.zeros((I, self.n))
        self._lib.orc_moments(self._h, mu, nu, d, _dp(W))
        return W

    def entry(self, mu: int, nu: int, ka: int, la: int) -> float:
        return self._lib.orc_entry(self._h, mu, nu, ka, la)

    def entries(self, idx4: np.ndarray, threads: Optional[int] = None) -> np.ndarray:
        idx = np.ascontiguousarray(idx4, dtype=np.int32).reshape(-1, 4)
        out = np.zeros(len(idx))
        self._lib.orc_entries(self._h, idx.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), len(idx), _dp(out),
                              threads or default_threads())
        return out

    def assemble_B(self, threads: Optional[int] = None) -> np.ndarray:
        nb2 = self.nbf * self.nbf
        B = np.zeros((nb2, nb2))
        self._lib.orc_assemble_B(self._h, _dp(B), threads or default_threads())
        return B

    def B_rows(self, rows, threads: Optional[int] = None) -> np.ndarray:
        r = np.ascontiguousarray(rows, dtype=np.int64)
        out = np.zeros((len(r), self.nbf * self.nbf))
        self._lib.orc_B_rows(self._h, r.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), len(r), _dp(out),
                             threads or default_threads())
        return out

    def factor_M(self, threads: Optional[int] = None) -> np.ndarray:
        M = np.zeros((self.nbf * self.nbf, self.n ** 3))
        self._lib.orc_factor_M(self._h, _dp(M), threads or default_threads())
        return M

    def jbuild_factored(self, D: np.ndarray, threads: Optional[int] = None) -> np.ndarray:
        D = np.ascontiguousarray(D, dtype=np.float64).reshape(-1, self.nbf, self.nbf)
        J = np.zeros_like(D)
        self._lib.orc_jbuild_factored(self._h, _dp(D), D.shape[0], _dp(J), threads or default_threads())
        return J
