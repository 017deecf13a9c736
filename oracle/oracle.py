"""Python face of the FP64 CPU oracle for segmented NCC (arXiv 2502.01286).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg use this module; the product path never does.
It does not import the CUDA package and the CUDA package does not import it.

Everything is double precision.  Images are numpy arrays indexed ``f[y, x]``
(rows y, columns x, paper Section 2), i.e. shape (N, M) for an M x N source
and (H, W) for a W x H template.  Offset maps are indexed ``rho[v, u]`` with
shape (N-H+1, M-W+1).
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass, field
from typing import Iterable, Optional, Sequence

import numpy as np

from . import build as _build

_lib = None


class _Seg(C.Structure):
    _fields_ = [("x", C.c_int), ("y", C.c_int), ("w", C.c_int), ("h", C.c_int), ("mu", C.c_double)]


def _load():
    global _lib
    if _lib is not None:
        return _lib
    path = _build.build()
    lib = C.CDLL(path)
    dp = C.POINTER(C.c_double)
    ip = C.POINTER(C.c_int)
    sp = C.POINTER(_Seg)
    lib.orc_sum_tables.argtypes = [dp, C.c_int, C.c_int, dp, dp]
    lib.orc_box_sum.argtypes = [dp, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int]
    lib.orc_box_sum.restype = C.c_double
    lib.orc_ncc_exact_map.argtypes = [dp, C.c_int, C.c_int, dp, C.c_int, C.c_int, ip, C.c_int, dp, C.c_int]
    lib.orc_ncc_exact_at.argtypes = [dp, C.c_int, C.c_int, dp, C.c_int, C.c_int, ip, ip, C.c_int, dp]
    lib.orc_precompute_template_approximation.argtypes = [
        dp, C.c_int, C.c_int, C.c_double, C.c_int, C.c_int, C.POINTER(sp), dp]
    lib.orc_precompute_template_approximation.restype = C.c_int
    lib.orc_split_only.argtypes = [dp, C.c_int, C.c_int, C.c_double, C.POINTER(sp)]
    lib.orc_split_only.restype = C.c_int
    lib.orc_merge_only.argtypes = [sp, C.c_int, C.POINTER(sp)]
    lib.orc_merge_only.restype = C.c_int
    lib.orc_free.argtypes = [C.c_void_p]
    lib.orc_segncc_map.argtypes = [dp, C.c_int, C.c_int, sp, C.c_int, C.c_int, C.c_int,
                                   C.c_double, C.c_double, C.c_int, ip, C.c_int, dp, C.c_int]
    _lib = lib
    return lib


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _iptr(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_int))


def _as_f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def default_threads() -> int:
    return max(1, os.cpu_count() or 1)


def _rows_arg(rows: Optional[Iterable[int]], V: int) -> np.ndarray:
    if rows is None:
        return np.arange(V, dtype=np.int32)
    r = np.asarray(list(rows) if not isinstance(rows, np.ndarray) else rows, dtype=np.int32)
    if r.size and (r.min() < 0 or r.max() >= V):
        raise ValueError("offset row out of range")
    return np.ascontiguousarray(r)


# --------------------------------------------------------------------------
# Sum tables (Eq. 10, Eq. 14) and box sums (Eq. 11)
# --------------------------------------------------------------------------
def sum_tables(f) -> tuple[np.ndarray, np.ndarray]:
    """Padded sum tables of f and f^2, each (N+1, M+1) float64 with a zero
    first row and column: ``s[y+1, x+1]`` is s(x, y) of Eq. 10."""
    lib = _load()
    f = _as_f64(f)
    N, M = f.shape
    s = np.empty((N + 1, M + 1), np.float64)
    s2 = np.empty((N + 1, M + 1), np.float64)
    lib.orc_sum_tables(_dptr(f), M, N, _dptr(s), _dptr(s2))
    return s, s2


def box_sum(s: np.ndarray, X: int, Y: int, w: int, h: int) -> float:
    """Eq. 11 on a table returned by :func:`sum_tables`."""
    lib = _load()
    s = _as_f64(s)
    M = s.shape[1] - 1
    return lib.orc_box_sum(_dptr(s), M, X, Y, w, h)


# --------------------------------------------------------------------------
# Exact NCC (Eq. 1)
# --------------------------------------------------------------------------
def ncc_exact_map(f, t, rows: Optional[Iterable[int]] = None, nthreads: Optional[int] = None) -> np.ndarray:
    """Exact NCC by Eq. 1 at every offset of the listed rows (all rows by
    default).  Rows that are not listed are NaN."""
    lib = _load()
    f = _as_f64(f)
    t = _as_f64(t)
    N, M = f.shape
    H, W = t.shape
    U, V = M - W + 1, N - H + 1
    if U <= 0 or V <= 0:
        raise ValueError("template larger than source")
    r = _rows_arg(rows, V)
    out = np.full((V, U), np.nan)
    lib.orc_ncc_exact_map(_dptr(f), M, N, _dptr(t), W, H, _iptr(r), int(r.size), _dptr(out),
                          nthreads or default_threads())
    return out


def ncc_exact_at(f, t, u: Sequence[int], v: Sequence[int]) -> np.ndarray:
    """Exact NCC by Eq. 1 at the offsets (u[i], v[i])."""
    lib = _load()
    f = _as_f64(f)
    t = _as_f64(t)
    N, M = f.shape
    H, W = t.shape
    uu = np.ascontiguousarray(np.asarray(u, np.int32))
    vv = np.ascontiguousarray(np.asarray(v, np.int32))
    if uu.shape != vv.shape:
        raise ValueError("u and v differ in length")
    if uu.size and (uu.min() < 0 or uu.max() > M - W or vv.min() < 0 or vv.max() > N - H):
        raise ValueError("offset out of range")
    out = np.empty(uu.size, np.float64)
    lib.orc_ncc_exact_at(_dptr(f), M, N, _dptr(t), W, H, _iptr(uu), _iptr(vv), int(uu.size), _dptr(out))
    return out


# --------------------------------------------------------------------------
# Template approximation (Section 3, Section 5)
# --------------------------------------------------------------------------
@dataclass
class Approximation:
    """Result of precompute_template_approximation.

    segments: int array (K, 4) of (x, y, w, h), in the order the merge leaves
    them (ascending (y, x)); mu: float64 (K,) segment values k_i (Eq. 4)."""
    segments: np.ndarray
    mu: np.ndarray
    W: int
    H: int
    k_split: int
    sigma_used: float
    kbar: float
    ek: float
    tbar: float
    rho_max: float
    weighted: bool = True
    extra: dict = field(default_factory=dict)

    @property
    def K(self) -> int:
        return int(self.segments.shape[0])

    def render(self) -> np.ndarray:
        """The approximate template k of Eq. 3 as an (H, W) image."""
        k = np.full((self.H, self.W), np.nan)
        for (x, y, w, h), m in zip(self.segments, self.mu):
            k[y:y + h, x:x + w] = m
        return k


def _take_segs(p, n: int) -> tuple[np.ndarray, np.ndarray]:
    lib = _load()
    segs = np.empty((n, 4), np.int64)
    mu = np.empty(n, np.float64)
    for i in range(n):
        s = p[i]
        segs[i] = (s.x, s.y, s.w, s.h)
        mu[i] = s.mu
    lib.orc_free(p)
    return segs, mu


def precompute_template_approximation(t, sigma_max: float, k_max: int = 0, weighted: bool = True) -> Approximation:
    """Section 5, precompute_template_approximation: split with sigma_max
    (raised by one until K <= k_max when k_max > 0), merge, then kbar, tbar
    and rho_max = NCC(t, k)."""
    lib = _load()
    t = _as_f64(t)
    H, W = t.shape
    p = C.POINTER(_Seg)()
    info = np.zeros(7, np.float64)
    n = lib.orc_precompute_template_approximation(_dptr(t), W, H, float(sigma_max), int(k_max),
                                                  1 if weighted else 0, C.byref(p), _dptr(info))
    segs, mu = _take_segs(p, n)
    return Approximation(segments=segs, mu=mu, W=W, H=H, k_split=int(info[1]), sigma_used=float(info[2]),
                         kbar=float(info[3]), ek=float(info[4]), tbar=float(info[5]), rho_max=float(info[6]),
                         weighted=weighted)


def split_segments(t, sigma_max: float) -> tuple[np.ndarray, np.ndarray]:
    """split_segment on the whole template, without merging, in emission order."""
    lib = _load()
    t = _as_f64(t)
    H, W = t.shape
    p = C.POINTER(_Seg)()
    n = lib.orc_split_only(_dptr(t), W, H, float(sigma_max), C.byref(p))
    return _take_segs(p, n)


def merge_segments(segs, mu) -> tuple[np.ndarray, np.ndarray]:
    """merge_redundant_segments on a given list."""
    lib = _load()
    segs = np.asarray(segs, np.int64)
    mu = np.asarray(mu, np.float64)
    n = segs.shape[0]
    arr = (_Seg * max(n, 1))()
    for i in range(n):
        arr[i] = _Seg(int(segs[i, 0]), int(segs[i, 1]), int(segs[i, 2]), int(segs[i, 3]), float(mu[i]))
    p = C.POINTER(_Seg)()
    m = lib.orc_merge_only(arr, n, C.byref(p))
    return _take_segs(p, m)


# --------------------------------------------------------------------------
# Segmented NCC (Eq. 9 - Eq. 18)
# --------------------------------------------------------------------------
def _seg_array(ap: Approximation):
    arr = (_Seg * max(ap.K, 1))()
    for i in range(ap.K):
        x, y, w, h = (int(v) for v in ap.segments[i])
        arr[i] = _Seg(x, y, w, h, float(ap.mu[i]))
    return arr


def segmented_ncc_map(f, ap: Approximation, method: str = "sat", rows: Optional[Iterable[int]] = None,
                      nthreads: Optional[int] = None) -> np.ndarray:
    """rho(u, v; f, k) of Eq. 18 at every offset of the listed rows.

    method="direct": Eq. 9 summed pixel by pixel over each segment.
    method="sat":    Eq. 10 - Eq. 18 through sum tables (the paper's route).
    Rows not listed are NaN."""
    lib = _load()
    f = _as_f64(f)
    N, M = f.shape
    U, V = M - ap.W + 1, N - ap.H + 1
    if U <= 0 or V <= 0:
        raise ValueError("template larger than source")
    r = _rows_arg(rows, V)
    out = np.full((V, U), np.nan)
    lib.orc_segncc_map(_dptr(f), M, N, _seg_array(ap), ap.K, ap.W, ap.H, ap.kbar, ap.ek,
                       1 if method == "sat" else 0, _iptr(r), int(r.size), _dptr(out),
                       nthreads or default_threads())
    return out


# --------------------------------------------------------------------------
# Main algorithm, step 7, with the exact second stage
# --------------------------------------------------------------------------
def candidates(rho_map: np.ndarray, tau: float) -> np.ndarray:
    """Linear offset indices v*U + u with rho >= tau (step 7f keeps exactly
    those), ascending.  NaN entries (rows not computed) never qualify."""
    V, U = rho_map.shape
    with np.errstate(invalid="ignore"):
        keep = rho_map >= tau
    return np.flatnonzero(keep.ravel()).astype(np.int64)


def refine(f, t, cand: np.ndarray, U: int, tau_exact: float) -> tuple[np.ndarray, np.ndarray]:
    """Exact NCC (Eq. 1) at each candidate; keep those with rho >= tau_exact.
    Returns (indices ascending, rho)."""
    cand = np.asarray(cand, np.int64)
    u = (cand % U).astype(np.int32)
    v = (cand // U).astype(np.int32)
    rho = ncc_exact_at(f, t, u, v)
    keep = rho >= tau_exact
    return cand[keep], rho[keep]


def main_algorithm(f, t, precision: float = 0.9, fast: float = 0.99, slow: float = 0.1, k_max: int = 5000,
                   weighted: bool = True):
    """Section 5 main algorithm as printed: k_fast and k_slow from
    precompute_template_approximation with sigma_max = fast * sigma_t and
    slow * sigma_t (sigma_t the template's std, same definition as Eq. 2),
    thresholds precision * rho_fast and precision * rho_slow (step 5), the
    coarse pass at every offset (steps 7a-7f) and the fine pass at the
    offsets that survive it (steps 7g-7j).

    Returns a dict with both approximations, thresholds, the coarse map, the
    candidate indices, the fine rho at each candidate and the matches
    (indices, rho)."""
    t64 = _as_f64(t)
    sigma_t = float(np.sqrt(np.mean((t64 - t64.mean()) ** 2)))
    ap_f = precompute_template_approximation(t64, fast * sigma_t, k_max, weighted)
    ap_s = precompute_template_approximation(t64, slow * sigma_t, k_max, weighted)
    thr_f = precision * ap_f.rho_max
    thr_s = precision * ap_s.rho_max
    rho_f = segmented_ncc_map(f, ap_f, "sat")
    cand = candidates(rho_f, thr_f)
    U = rho_f.shape[1]
    rows = np.unique(cand // U)
    rho_s_map = segmented_ncc_map(f, ap_s, "sat", rows=rows) if rows.size else np.full_like(rho_f, np.nan)
    rho_s = rho_s_map.ravel()[cand] if cand.size else np.zeros(0)
    keep = rho_s >= thr_s
    return {"fast": ap_f, "slow": ap_s, "thr_fast": thr_f, "thr_slow": thr_s, "rho_fast": rho_f,
            "cand": cand, "rho_slow_at_cand": rho_s, "idx": cand[keep], "rho": rho_s[keep]}
