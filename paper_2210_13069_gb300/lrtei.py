"""Thin ctypes binding of ``liblrtei.so`` (include/lrtei.h): argument marshalling only.

Every function named ``lrtei_*`` here calls the C function of the same name.  Device
buffers are passed as raw pointers (``int``) or as CUDA tensors (their ``data_ptr()``);
streams as ``torch.cuda.Stream``, raw handles or ``None`` (the current torch stream).
If the library is missing or cannot be loaded, every call raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_build", "liblrtei.so")

LRTEI_OK = 0
STATUS_NAMES = {0: "OK", 1: "ERR_ARG", 2: "ERR_ALLOC", 3: "ERR_CUDA", 4: "ERR_TIMEOUT", 5: "ERR_NUMERIC",
                6: "ERR_UNSUPPORTED"}
LRTEI_FP64, LRTEI_FP32, LRTEI_SPLIT_F16, LRTEI_BF16, LRTEI_SPLIT_F16_8 = 0, 1, 2, 3, 4
LRTEI_FORM_AUTO, LRTEI_FORM_HADAMARD, LRTEI_FORM_FACTORED = 0, 1, 2

PRECISIONS = {"fp64": LRTEI_FP64, "fp32": LRTEI_FP32, "split_f16": LRTEI_SPLIT_F16, "bf16": LRTEI_BF16,
              "split_f16_8": LRTEI_SPLIT_F16_8}
FORMS = {"auto": LRTEI_FORM_AUTO, "hadamard": LRTEI_FORM_HADAMARD, "factored": LRTEI_FORM_FACTORED}


class LrteiError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class PlanInfo(ctypes.Structure):
    _fields_ = [("nbf", ctypes.c_int), ("npair", ctypes.c_int64), ("nrows", ctypes.c_int64), ("n", ctypes.c_int),
                ("P", ctypes.c_int), ("omega", ctypes.c_double), ("box_lo", ctypes.c_double * 3),
                ("box_hi", ctypes.c_double * 3), ("precision", ctypes.c_int), ("last_form", ctypes.c_int),
                ("workspace_bytes", ctypes.c_size_t), ("tau_screening", ctypes.c_double), ("cheb_n", ctypes.c_int),
                ("kr_rank", ctypes.c_int), ("npartitions", ctypes.c_int), ("partition_b", ctypes.c_double * 8)]


_lib = None
VP = ctypes.c_void_p
DP = ctypes.POINTER(ctypes.c_double)
IP = ctypes.POINTER(ctypes.c_int)


def library_path() -> str:
    return _SO


def load():
    """Load liblrtei.so (built by ``paper_2210_13069_gb300.build_lib.build()``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_SO):
        raise LrteiError(3, f"CUDA library not built: {_SO} is missing (run build_lib.build())")
    lib = ctypes.CDLL(_SO)
    S = ctypes.c_int
    sig = {
        "lrtei_basis_create": (S, [ctypes.c_int, DP, IP, IP, DP, DP, ctypes.POINTER(VP)]),
        "lrtei_basis_destroy": (None, [VP]),
        "lrtei_basis_nbf": (ctypes.c_int, [VP]),
        "lrtei_plan_create": (S, [VP, ctypes.c_double, ctypes.c_int, ctypes.c_int, DP, DP, ctypes.c_int, VP,
                                  ctypes.POINTER(VP)]),
        "lrtei_plan_create_ex": (S, [VP, ctypes.c_double, ctypes.c_int, ctypes.c_int, DP, DP, ctypes.c_int,
                                     ctypes.c_double, VP, ctypes.POINTER(VP)]),
        "lrtei_plan_create_adaptive": (S, [VP, ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                           ctypes.c_int, ctypes.c_int, VP, ctypes.POINTER(VP)]),
        "lrtei_plan_destroy": (None, [VP]),
        "lrtei_plan_info_get": (S, [VP, ctypes.POINTER(PlanInfo)]),
        "lrtei_plan_status": (S, [VP]),
        "lrtei_assemble_B": (S, [VP, ctypes.c_int, VP, ctypes.c_int64, VP]),
        "lrtei_assemble_Bu_rows": (S, [VP, ctypes.c_int, ctypes.c_int64, ctypes.c_int64, VP, ctypes.c_int64, VP]),
        "lrtei_entries": (S, [VP, VP, ctypes.c_int64, VP, VP]),
        "lrtei_entries_noalloc": (S, [VP, VP, ctypes.c_int64, VP, VP]),
        "lrtei_entries_orders": (S, [VP, ctypes.c_int, IP, IP, VP, ctypes.c_int64, VP, VP]),
        "lrtei_factors": (S, [VP, VP, VP, VP, VP, VP, VP]),
        "lrtei_dense_K": (S, [VP, VP, VP]),
        "lrtei_plan_compress": (S, [VP, ctypes.c_double, ctypes.c_int, DP, IP, VP]),
        "lrtei_jbuild": (S, [VP, VP, ctypes.c_int, VP, VP]),
        "lrtei_exchange": (S, [VP, VP, ctypes.c_int, VP, VP]),
        "lrtei_jbuild_partial_x": (S, [VP, VP, ctypes.c_int, ctypes.c_int64, ctypes.c_int64, VP, VP]),
        "lrtei_jbuild_apply_x": (S, [VP, VP, ctypes.c_int, ctypes.c_int64, ctypes.c_int64, VP, VP]),
        "lrtei_jbuild_batched": (S, [ctypes.POINTER(VP), ctypes.c_int, ctypes.POINTER(VP), IP, ctypes.POINTER(VP),
                                     VP]),
        "lrtei_selector_create": (S, [ctypes.c_int, ctypes.c_uint64, ctypes.POINTER(VP)]),
        "lrtei_selector_destroy": (None, [VP]),
        "lrtei_selector_train_epoch": (S, [VP, VP, VP, ctypes.c_int, ctypes.c_int, ctypes.c_float,
                                           ctypes.POINTER(ctypes.c_float), VP]),
        "lrtei_selector_forward": (S, [VP, VP, VP, ctypes.c_int, VP]),
        "lrtei_selector_grad": (S, [VP, VP, VP, ctypes.c_int, VP, ctypes.POINTER(ctypes.c_float), VP]),
        "lrtei_selector_nparams": (ctypes.c_int64, [VP]),
        "lrtei_selector_get_params": (S, [VP, ctypes.POINTER(ctypes.c_float)]),
        "lrtei_selector_set_params": (S, [VP, ctypes.POINTER(ctypes.c_float)]),
        "lrtei_selector_features": (S, [DP, ctypes.POINTER(ctypes.c_float)]),
        "lrtei_selector_encode": (S, [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_float)]),
        "lrtei_select_np": (S, [VP, DP, IP, IP, IP]),
        "lrtei_selector_train": (S, [VP, VP, VP, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_float,
                                     ctypes.POINTER(ctypes.c_float), VP]),
        "lrtei_selector_save": (S, [VP, ctypes.c_char_p, ctypes.c_char_p]),
        "lrtei_selector_load": (S, [ctypes.c_char_p, ctypes.POINTER(VP), ctypes.c_char_p, ctypes.c_size_t]),
        "lrtei_profile_enable": (S, [ctypes.c_int]),
        "lrtei_profile_get": (S, [ctypes.c_char_p, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64)]),
        "lrtei_profile_reset": (None, []),
        "lrtei_measure_fma_peak": (S, [ctypes.c_int, ctypes.POINTER(ctypes.c_double), VP]),
        "lrtei_last_error": (ctypes.c_char_p, []),
        "lrtei_version": (ctypes.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _check(status: int):
    if status != LRTEI_OK:
        raise LrteiError(status, load().lrtei_last_error().decode())


def _ptr(x) -> Optional[int]:
    if x is None:
        return None
    if isinstance(x, int):
        return x
    return int(x.data_ptr())


def _stream(s) -> Optional[int]:
    if s is None:
        import torch
        return int(torch.cuda.current_stream().cuda_stream)
    if isinstance(s, int):
        return s
    return int(s.cuda_stream)


def _np(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


# ------------------------------------------------------------------ C-ABI named calls

def lrtei_basis_create(centers, l, nprim, exps, coefs) -> int:
    lib = load()
    c, L, K, e, cf = _np(centers, np.float64).reshape(-1), _np(l, np.int32), _np(nprim, np.int32), \
        _np(exps, np.float64), _np(coefs, np.float64)
    out = VP()
    _check(lib.lrtei_basis_create(len(L), c.ctypes.data_as(DP), L.ctypes.data_as(IP), K.ctypes.data_as(IP),
                                  e.ctypes.data_as(DP), cf.ctypes.data_as(DP), ctypes.byref(out)))
    return out.value


def lrtei_basis_destroy(basis: int):
    load().lrtei_basis_destroy(basis)


def lrtei_basis_nbf(basis: int) -> int:
    return load().lrtei_basis_nbf(basis)


def lrtei_plan_create(basis: int, omega: float, n: int, P: int, box_lo=None, box_hi=None,
                      precision: int = LRTEI_FP64, stream=None) -> int:
    lib = load()
    lo = hi = None
    if box_lo is not None:
        lo = _np(box_lo, np.float64)
        hi = _np(box_hi, np.float64)
    out = VP()
    _check(lib.lrtei_plan_create(basis, float(omega), int(n), int(P), lo.ctypes.data_as(DP) if lo is not None else None,
                                 hi.ctypes.data_as(DP) if hi is not None else None, int(precision), _stream(stream),
                                 ctypes.byref(out)))
    return out.value


def lrtei_plan_create_ex(basis: int, omega: float, n: int, P: int, box_lo=None, box_hi=None,
                         precision: int = LRTEI_FP64, tau_screening: float = 0.0, stream=None) -> int:
    lib = load()
    lo = hi = None
    if box_lo is not None:
        lo = _np(box_lo, np.float64)
        hi = _np(box_hi, np.float64)
    out = VP()
    _check(lib.lrtei_plan_create_ex(basis, float(omega), int(n), int(P),
                                    lo.ctypes.data_as(DP) if lo is not None else None,
                                    hi.ctypes.data_as(DP) if hi is not None else None, int(precision),
                                    float(tau_screening), _stream(stream), ctypes.byref(out)))
    return out.value


def lrtei_plan_create_adaptive(basis: int, omega: float, n: int, P: int, tau_adaptive: float, npartitions: int,
                               precision: int = LRTEI_FP64, stream=None) -> int:
    out = VP()
    _check(load().lrtei_plan_create_adaptive(basis, float(omega), int(n), int(P), float(tau_adaptive),
                                             int(npartitions), int(precision), _stream(stream), ctypes.byref(out)))
    return out.value


def lrtei_plan_destroy(plan: int):
    load().lrtei_plan_destroy(plan)


def lrtei_plan_info_get(plan: int) -> dict:
    info = PlanInfo()
    _check(load().lrtei_plan_info_get(plan, ctypes.byref(info)))
    return {"nbf": info.nbf, "npair": info.npair, "nrows": info.nrows, "n": info.n, "P": info.P,
            "omega": info.omega, "box_lo": list(info.box_lo), "box_hi": list(info.box_hi),
            "precision": info.precision, "last_form": info.last_form, "workspace_bytes": info.workspace_bytes,
            "tau_screening": info.tau_screening, "cheb_n": info.cheb_n, "kr_rank": info.kr_rank,
            "npartitions": info.npartitions, "partition_b": list(info.partition_b)[:info.npartitions]}


def lrtei_plan_status(plan: int):
    _check(load().lrtei_plan_status(plan))


def lrtei_assemble_B(plan: int, form: int, d_B, ld: int, stream=None):
    _check(load().lrtei_assemble_B(plan, int(form), _ptr(d_B), int(ld), _stream(stream)))


def lrtei_assemble_Bu_rows(plan: int, form: int, row_begin: int, row_end: int, d_Bu, ld: int, stream=None):
    _check(load().lrtei_assemble_Bu_rows(plan, int(form), int(row_begin), int(row_end), _ptr(d_Bu), int(ld),
                                         _stream(stream)))


def lrtei_entries(plan: int, d_idx4, count: int, d_out, stream=None):
    _check(load().lrtei_entries(plan, _ptr(d_idx4), int(count), _ptr(d_out), _stream(stream)))


def lrtei_entries_noalloc(plan: int, d_idx4, count: int, d_out, stream=None):
    """Algorithm 1 entries without any device allocation (fixed 4 MiB scratch per device,
    at most 262144 entries per call; calls that overlap on the GPU race on the scratch)."""
    _check(load().lrtei_entries_noalloc(plan, _ptr(d_idx4), int(count), _ptr(d_out), _stream(stream)))


def lrtei_entries_orders(plan: int, ns, Ps, d_idx4, count: int, d_out, stream=None):
    n = _np(ns, np.int32)
    P = _np(Ps, np.int32)
    if n.size != P.size:
        raise LrteiError(1, "ns and Ps differ in length")
    _check(load().lrtei_entries_orders(plan, int(n.size), n.ctypes.data_as(IP), P.ctypes.data_as(IP), _ptr(d_idx4),
                                       int(count), _ptr(d_out), _stream(stream)))


def lrtei_factors(plan: int, d_S=None, d_C=None, d_s=None, d_w=None, d_c=None, stream=None):
    _check(load().lrtei_factors(plan, _ptr(d_S), _ptr(d_C), _ptr(d_s), _ptr(d_w), _ptr(d_c), _stream(stream)))


def lrtei_plan_compress(plan: int, eps: float, max_rank: int = 0, n: Optional[int] = None, stream=None):
    """Khatri-Rao compression of the plan's factors; returns (singular values 3 x n, ranks R_d)."""
    n = n if n is not None else lrtei_plan_info_get(plan)["n"]
    sig = np.zeros(3 * n, dtype=np.float64)
    ranks = np.zeros(3, dtype=np.int32)
    _check(load().lrtei_plan_compress(plan, float(eps), int(max_rank), sig.ctypes.data_as(DP),
                                      ranks.ctypes.data_as(IP), _stream(stream)))
    return sig.reshape(3, n), ranks


def lrtei_dense_K(plan: int, d_K, stream=None):
    _check(load().lrtei_dense_K(plan, _ptr(d_K), _stream(stream)))


def lrtei_jbuild(plan: int, d_D, R: int, d_J, stream=None):
    _check(load().lrtei_jbuild(plan, _ptr(d_D), int(R), _ptr(d_J), _stream(stream)))


def lrtei_jbuild_partial_x(plan: int, d_D, R: int, pair_begin: int, pair_end: int, d_X, stream=None):
    _check(load().lrtei_jbuild_partial_x(plan, _ptr(d_D), int(R), int(pair_begin), int(pair_end), _ptr(d_X),
                                         _stream(stream)))


def lrtei_jbuild_apply_x(plan: int, d_X, R: int, pair_begin: int, pair_end: int, d_J, stream=None):
    _check(load().lrtei_jbuild_apply_x(plan, _ptr(d_X), int(R), int(pair_begin), int(pair_end), _ptr(d_J),
                                       _stream(stream)))


def lrtei_exchange(plan: int, d_Q, norb: int, d_K, stream=None):
    _check(load().lrtei_exchange(plan, _ptr(d_Q), int(norb), _ptr(d_K), _stream(stream)))


def lrtei_jbuild_batched(plans: Sequence[int], d_D: Sequence, R: Sequence[int], d_J: Sequence, stream=None):
    m = len(plans)
    P = (VP * m)(*plans)
    Dp = (VP * m)(*[_ptr(x) for x in d_D])
    Jp = (VP * m)(*[_ptr(x) for x in d_J])
    Rr = (ctypes.c_int * m)(*[int(r) for r in R])
    _check(load().lrtei_jbuild_batched(P, m, Dp, Rr, Jp, _stream(stream)))


def lrtei_profile_enable(on: bool):
    _check(load().lrtei_profile_enable(1 if on else 0))


def lrtei_profile_reset():
    load().lrtei_profile_reset()


def lrtei_measure_fma_peak(fp64: bool, stream=None) -> float:
    """Measured CUDA-core FMA rate in TFLOP/s (FP64 or FP32), all SMs of the current device."""
    tf = ctypes.c_double(0.0)
    _check(load().lrtei_measure_fma_peak(1 if fp64 else 0, ctypes.byref(tf), _stream(stream)))
    return tf.value


def lrtei_profile_get(kernel: str):
    """(total device ms, launches) of one kernel name since the last reset (synchronises)."""
    ms = ctypes.c_double(0.0)
    cnt = ctypes.c_int64(0)
    _check(load().lrtei_profile_get(kernel.encode(), ctypes.byref(ms), ctypes.byref(cnt)))
    return ms.value, cnt.value


# ------------------------------------------------------------------ selector (MLP) calls

FP = ctypes.POINTER(ctypes.c_float)


def lrtei_selector_create(hidden: int = 64, seed: int = 1) -> int:
    out = VP()
    _check(load().lrtei_selector_create(int(hidden), int(seed), ctypes.byref(out)))
    return out.value


def lrtei_selector_destroy(sel: int):
    load().lrtei_selector_destroy(sel)


def lrtei_selector_nparams(sel: int) -> int:
    return int(load().lrtei_selector_nparams(sel))


def lrtei_selector_forward(sel: int, d_X, d_Yhat, N: int, stream=None):
    _check(load().lrtei_selector_forward(sel, _ptr(d_X), _ptr(d_Yhat), int(N), _stream(stream)))


def lrtei_selector_grad(sel: int, d_X, d_Y, N: int, d_grad, stream=None) -> float:
    loss = ctypes.c_float(0.0)
    _check(load().lrtei_selector_grad(sel, _ptr(d_X), _ptr(d_Y), int(N), _ptr(d_grad), ctypes.byref(loss),
                                      _stream(stream)))
    return float(loss.value)


def lrtei_selector_train_epoch(sel: int, d_X, d_Y, N: int, batch: int, lr: float, stream=None) -> float:
    loss = ctypes.c_float(0.0)
    _check(load().lrtei_selector_train_epoch(sel, _ptr(d_X), _ptr(d_Y), int(N), int(batch), float(lr),
                                             ctypes.byref(loss), _stream(stream)))
    return float(loss.value)


def lrtei_selector_get_params(sel: int) -> np.ndarray:
    out = np.zeros(lrtei_selector_nparams(sel), dtype=np.float32)
    _check(load().lrtei_selector_get_params(sel, out.ctypes.data_as(FP)))
    return out


def lrtei_selector_set_params(sel: int, params: np.ndarray):
    p = np.ascontiguousarray(params, dtype=np.float32)
    if p.size != lrtei_selector_nparams(sel):
        raise LrteiError(1, "parameter count mismatch")
    _check(load().lrtei_selector_set_params(sel, p.ctypes.data_as(FP)))


def lrtei_selector_features(raw) -> np.ndarray:
    r = _np(raw, np.float64).reshape(6)
    out = np.zeros(6, dtype=np.float32)
    _check(load().lrtei_selector_features(r.ctypes.data_as(DP), out.ctypes.data_as(FP)))
    return out


def lrtei_selector_encode(n: int, P: int) -> np.ndarray:
    out = np.zeros(2, dtype=np.float32)
    _check(load().lrtei_selector_encode(int(n), int(P), out.ctypes.data_as(FP)))
    return out


def lrtei_select_np(sel: int, raw):
    """(n, P, used_fallback) for raw features (omega, half-width, alpha_min, alpha_max, l, target)."""
    r = _np(raw, np.float64).reshape(6)
    n, P, fb = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_int(0)
    _check(load().lrtei_select_np(sel, r.ctypes.data_as(DP), ctypes.byref(n), ctypes.byref(P), ctypes.byref(fb)))
    return n.value, P.value, bool(fb.value)


def lrtei_selector_train(sel: int, d_X, d_Y, N: int, epochs: int, batch: int, lr: float, stream=None) -> np.ndarray:
    hist = np.zeros(int(epochs), dtype=np.float32)
    _check(load().lrtei_selector_train(sel, _ptr(d_X), _ptr(d_Y), int(N), int(epochs), int(batch), float(lr),
                                       hist.ctypes.data_as(FP), _stream(stream)))
    return hist


def lrtei_selector_save(sel: int, path: str, meta: str = ""):
    _check(load().lrtei_selector_save(sel, path.encode(), meta.encode() if meta else None))


def lrtei_selector_load(path: str, meta_cap: int = 1 << 16):
    """(selector handle, meta text)."""
    out = VP()
    buf = ctypes.create_string_buffer(meta_cap)
    _check(load().lrtei_selector_load(path.encode(), ctypes.byref(out), buf, meta_cap))
    return out.value, buf.value.decode()


def lrtei_last_error() -> str:
    return load().lrtei_last_error().decode()


def lrtei_version() -> str:
    return load().lrtei_version().decode()


# ------------------------------------------------------------------ convenience wrapper

class Plan:
    """A basis plus a plan on the current CUDA device (owns both handles)."""

    def __init__(self, mol, precision: str = "fp64", stream=None, n=None, P=None, omega=None,
                 tau_screening: float = 0.0, adaptive=None):
        """adaptive=(tau_adaptive, npartitions) creates an adaptive-box plan (no explicit box)."""
        import torch
        centers, ls, nprim, exps, coefs = mol.packed()
        self.basis = lrtei_basis_create(centers, ls, nprim, exps, coefs)
        if adaptive is not None:
            self.plan = lrtei_plan_create_adaptive(self.basis, omega or mol.omega, n or mol.n, P or mol.P,
                                                   adaptive[0], adaptive[1], PRECISIONS[precision], stream)
        else:
            self.plan = lrtei_plan_create_ex(self.basis, omega or mol.omega, n or mol.n, P or mol.P, mol.box_lo,
                                             mol.box_hi, PRECISIONS[precision], tau_screening, stream)
        info = lrtei_plan_info_get(self.plan)
        self.nbf = info["nbf"]
        self.npair = info["npair"]
        self._torch = torch

    @property
    def info(self) -> dict:
        """lrtei_plan_info_get, read at each access (last_form follows the last assembly)."""
        return lrtei_plan_info_get(self.plan)

    def close(self):
        if getattr(self, "plan", None):
            lrtei_plan_destroy(self.plan)
            self.plan = None
        if getattr(self, "basis", None):
            lrtei_basis_destroy(self.basis)
            self.basis = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def assemble_B(self, form: str = "auto", out=None, stream=None):
        """B into `out`: a CUDA tensor, or a pinned CPU tensor (written directly by the device)."""
        torch = self._torch
        nb2 = self.nbf * self.nbf
        if out is None:
            out = torch.empty((nb2, nb2), dtype=torch.float64, device="cuda")
        elif not out.is_cuda and not out.is_pinned():
            raise ValueError("assemble_B: a host output must be pinned (page-locked) memory")
        lrtei_assemble_B(self.plan, FORMS[form], out, out.stride(0), stream)
        return out

    def Bu_rows(self, r0: int, r1: int, form: str = "auto", out=None, stream=None):
        torch = self._torch
        if out is None:
            out = torch.empty((r1 - r0, self.npair), dtype=torch.float64, device="cuda")
        lrtei_assemble_Bu_rows(self.plan, FORMS[form], r0, r1, out, out.stride(0), stream)
        return out

    def entries(self, idx4, stream=None):
        torch = self._torch
        idx = torch.as_tensor(np.ascontiguousarray(idx4, dtype=np.int32).reshape(-1, 4), device="cuda")
        out = torch.empty(idx.shape[0], dtype=torch.float64, device="cuda")
        lrtei_entries(self.plan, idx, idx.shape[0], out, stream)
        return out

    def factors(self, stream=None):
        torch = self._torch
        n, P, nrows = self.info["n"], self.info["P"], self.info["nrows"]
        S = torch.empty((3, nrows, n), dtype=torch.float64, device="cuda")
        C = torch.empty((3, P, n, n), dtype=torch.float64, device="cuda")
        s = torch.empty(P, dtype=torch.float64, device="cuda")
        w = torch.empty(P, dtype=torch.float64, device="cuda")
        c = torch.empty(nrows, dtype=torch.float64, device="cuda")
        lrtei_factors(self.plan, S, C, s, w, c, stream)
        return S, C, s, w, c

    def dense_K(self, stream=None):
        torch = self._torch
        n3 = self.info["n"] ** 3
        K = torch.empty((n3, n3), dtype=torch.float64, device="cuda")
        lrtei_dense_K(self.plan, K, stream)
        return K

    def jbuild(self, D, out=None, stream=None):
        torch = self._torch
        D = D.contiguous()
        if out is None:
            out = torch.empty_like(D)
        lrtei_jbuild(self.plan, D, D.shape[0], out, stream)
        return out

    def compress(self, eps: float, max_rank: int = 0, stream=None):
        """Khatri-Rao compression (eq. approxepsilon); returns (singular values, ranks R_d)."""
        sig, ranks = lrtei_plan_compress(self.plan, eps, max_rank, self.info["n"], stream)
        return sig, ranks

    def exchange(self, Q, out=None, stream=None):
        """K^lr (N_b x N_b) for orbital coefficients Q (norb x N_b), eq. exchange."""
        torch = self._torch
        Q = Q.contiguous()
        if out is None:
            out = torch.empty((self.nbf, self.nbf), dtype=torch.float64, device="cuda")
        lrtei_exchange(self.plan, Q, Q.shape[0], out, stream)
        return out

    def status(self):
        lrtei_plan_status(self.plan)
