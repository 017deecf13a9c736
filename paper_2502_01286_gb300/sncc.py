"""Thin Python binding of libsncc.so (the C ABI declared in include/sncc.h).

Argument marshalling only: every step of the path runs in the library's CUDA
kernels or its host segmentation.  PyTorch supplies device memory and the
current stream.  The library is loaded from this package's ``_build``
directory; if it has not been built, importing this module raises.

Names follow the C ABI: build_segments, integral, match, refine, exact_map.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libsncc.so")

if not os.path.exists(LIB_PATH):
    raise ImportError("libsncc.so is not built (%s); run paper_2502_01286_gb300/build.py or "
                      "__graft_entry__.build()" % LIB_PATH)
_lib = C.CDLL(LIB_PATH)

# Return codes and status bits (include/sncc.h).
OK = 0
ERR_ARG, ERR_UNIFORM, ERR_DTYPE, ERR_CAPACITY, ERR_CUDA, ERR_WORKSPACE, ERR_NOMEM, ERR_UNSUPPORTED = \
    -1, -2, -3, -4, -5, -6, -7, -8
STATUS_CAND_OVERFLOW, STATUS_MATCH_OVERFLOW, STATUS_WAIT_TIMEOUT, STATUS_SORT_OVERFLOW = 1, 2, 4, 8

EXPORTED = ["sncc_error_string", "sncc_version", "sncc_build_segments", "sncc_free_segments", "sncc_template_sigma",
            "sncc_sat_pitch",
            "sncc_integral_workspace_bytes", "sncc_integral", "sncc_plan_bytes", "sncc_plan_upload", "sncc_match",
            "sncc_match_multi", "sncc_pipeline_create", "sncc_pipeline_submit", "sncc_pipeline_flush",
            "sncc_pipeline_fused", "sncc_pipeline_compute_stream", "sncc_pipeline_destroy",
            "sncc_refine_workspace_bytes", "sncc_refine", "sncc_exact_map", "sncc_get_plan_info",
            "sncc_probe_smem_read", "sncc_probe_alu", "sncc_probe_wait_timeout", "sncc_probe_hbm_write", "sncc_integral_noalloc", "sncc_refine_segmented", "sncc_refine_segmented_tiles",
            "sncc_refine_segmented_tiles_workspace_bytes", "sncc_batch_create",
            "sncc_batch_destroy", "sncc_batch_device_bytes", "sncc_batch_upload", "sncc_batch_set_variant",
            "sncc_batch_get_info", "sncc_batch_match", "sncc_batch_autotune", "sncc_batch_refine_workspace_bytes",
            "sncc_batch_set_bucket_variant", "sncc_batch_get_bucket",
            "sncc_batch_refine", "sncc_diff_workspace_bytes", "sncc_diff_forward", "sncc_diff_backward"]
NOALLOC_SCRATCH_BYTES = 16 << 20


class SnccError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        self.code = code
        super().__init__("%s: %s (%d)" % (what, _lib.sncc_error_string(code).decode(), code))


class _Seg(C.Structure):
    _fields_ = [("x", C.c_int32), ("y", C.c_int32), ("w", C.c_int32), ("h", C.c_int32),
                ("sum", C.c_int64), ("mean", C.c_double)]


class _Segments(C.Structure):
    _fields_ = [("seg", C.POINTER(_Seg)), ("K", C.c_int32), ("K_split", C.c_int32), ("W", C.c_int32),
                ("H", C.c_int32), ("sigma_used", C.c_double), ("kbar", C.c_double), ("Ek", C.c_double),
                ("rho_max", C.c_double), ("T", C.c_int64), ("T2", C.c_int64), ("err_bound", C.c_double),
                ("plan", C.c_void_p), ("sigma_t", C.c_double)]


class PlanInfo(C.Structure):
    _fields_ = [("F", C.c_int32), ("blocks", C.c_int32), ("block_w", C.c_int32), ("block_h", C.c_int32),
                ("corners", C.c_int32), ("max_corners", C.c_int32), ("Q0", C.c_int64), ("runs8", C.c_int32),
                ("runs4", C.c_int32), ("runs2", C.c_int32), ("runs1", C.c_int32), ("template_corners", C.c_int32),
                ("wide_blocks", C.c_int32), ("wide_corners", C.c_int32), ("pairs", C.c_int32),
                ("sum_records", C.c_int32), ("sum_extra_rows", C.c_int64), ("strided8", C.c_int32),
                ("strided4", C.c_int32), ("strided3", C.c_int32), ("t023", C.c_int32)]


class MatchT(C.Structure):
    _fields_ = [("u", C.c_int32), ("v", C.c_int32), ("rho", C.c_float)]


_vp = C.c_void_p
_lib.sncc_error_string.restype = C.c_char_p
_lib.sncc_error_string.argtypes = [C.c_int]
_lib.sncc_version.restype = C.c_char_p
_lib.sncc_build_segments.argtypes = [_vp, C.c_int, C.c_int, C.c_int, C.c_double, C.c_int, C.POINTER(_Segments)]
_lib.sncc_free_segments.argtypes = [C.POINTER(_Segments)]
_lib.sncc_template_sigma.argtypes = [_vp, C.c_int, C.c_int, C.c_int, C.POINTER(C.c_double)]
_lib.sncc_free_segments.restype = None
_lib.sncc_sat_pitch.argtypes = [C.c_int]
_lib.sncc_integral_workspace_bytes.argtypes = [C.c_int, C.c_int]
_lib.sncc_integral_workspace_bytes.restype = C.c_size_t
_lib.sncc_integral.argtypes = [_vp, C.c_int, C.c_int, C.c_int, _vp, C.c_int, _vp, C.c_int, _vp, C.c_size_t, _vp]
_lib.sncc_integral_noalloc.argtypes = [_vp, C.c_int, C.c_int, C.c_int, _vp, C.c_int, _vp, C.c_int, _vp]
_lib.sncc_plan_bytes.argtypes = [C.POINTER(_Segments)]
_lib.sncc_plan_bytes.restype = C.c_size_t
_lib.sncc_plan_upload.argtypes = [C.POINTER(_Segments), _vp, C.c_size_t, _vp]
_lib.sncc_match.argtypes = [C.POINTER(_Segments), _vp, _vp, C.c_int, _vp, C.c_int, C.c_int, C.c_int, C.c_float,
                            _vp, C.c_int, _vp, C.c_int, _vp, _vp, _vp]
_lib.sncc_match_multi.argtypes = [C.POINTER(C.POINTER(_Segments)), C.POINTER(_vp), C.c_int, _vp, C.c_int, _vp,
                                  C.c_int, C.c_int, C.c_int, C.POINTER(C.c_float), C.POINTER(_vp), C.c_int,
                                  C.POINTER(_vp), C.c_int, C.POINTER(_vp), C.POINTER(_vp), _vp]


class _PipelineSlot(C.Structure):
    _fields_ = [("d_frame", _vp), ("d_s", _vp), ("d_s2", _vp), ("d_ws", _vp), ("ws_bytes", C.c_size_t),
                ("d_rho", _vp * 4), ("d_cand", _vp * 4), ("d_count", _vp * 4), ("d_status", _vp * 4),
                ("d_out", _vp * 4), ("d_nout", _vp * 4), ("d_rws", _vp * 4), ("rws_bytes", C.c_size_t)]


_lib.sncc_pipeline_create.argtypes = [C.POINTER(C.POINTER(_Segments)), C.POINTER(_vp), C.c_int, _vp, C.c_int,
                                      C.c_int, C.c_int, C.c_int, C.c_int, C.POINTER(C.c_float), C.c_float, C.c_int,
                                      C.c_int, C.c_int, C.POINTER(_PipelineSlot), C.POINTER(_vp)]
_lib.sncc_pipeline_submit.argtypes = [_vp, _vp, C.POINTER(_vp), C.POINTER(C.c_int32), C.POINTER(C.c_int32)]
_lib.sncc_pipeline_flush.argtypes = [_vp, C.POINTER(_vp), C.POINTER(C.c_int32), C.POINTER(C.c_int32)]
_lib.sncc_pipeline_fused.argtypes = [_vp]
_lib.sncc_pipeline_compute_stream.argtypes = [_vp]
_lib.sncc_pipeline_compute_stream.restype = _vp
_lib.sncc_pipeline_destroy.argtypes = [_vp]
_lib.sncc_pipeline_destroy.restype = None
_lib.sncc_refine_workspace_bytes.argtypes = [C.c_int] * 5
_lib.sncc_refine_workspace_bytes.restype = C.c_size_t
_lib.sncc_refine.argtypes = [_vp, C.c_int, C.c_int, C.c_int, _vp, C.c_int, C.c_int, C.c_int, C.c_int64, C.c_int64,
                             _vp, _vp, C.c_int, C.c_float, _vp, C.c_int, _vp, _vp, C.c_size_t, _vp, _vp]
_lib.sncc_refine_segmented.argtypes = [C.POINTER(_Segments), _vp, _vp, C.c_int, _vp, C.c_int, C.c_int, C.c_int,
                                       _vp, _vp, C.c_int, C.c_float, _vp, C.c_int, _vp, _vp, C.c_size_t, _vp, _vp]
_lib.sncc_refine_segmented_tiles.argtypes = _lib.sncc_refine_segmented.argtypes
_lib.sncc_refine_segmented_tiles_workspace_bytes.argtypes = [C.c_int] * 5
_lib.sncc_refine_segmented_tiles_workspace_bytes.restype = C.c_size_t
class BatchInfo(C.Structure):
    _fields_ = [("n_templates", C.c_int32), ("n_sources", C.c_int32), ("tile_rows", C.c_int32),
                ("tiles", C.c_int32), ("offsets", C.c_double), ("corner_offsets", C.c_double)]


BATCH_BUCKETS, BATCH_VARIANTS = 9, 6


class BatchBucket(C.Structure):
    _fields_ = [("templates", C.c_int32), ("pairs", C.c_int32), ("size_class", C.c_int32),
                ("density_class", C.c_int32), ("tile_rows", C.c_int32), ("block", C.c_int32),
                ("corner_offsets", C.c_double), ("ms", C.c_float * BATCH_VARIANTS)]


_pp = C.POINTER(C.c_void_p)
_lib.sncc_batch_create.argtypes = [C.POINTER(C.POINTER(_Segments)), _pp, C.POINTER(C.c_int), C.POINTER(C.c_float),
                                   C.POINTER(C.c_float), C.c_int, C.c_int, C.c_int, C.c_int, C.POINTER(C.c_void_p)]
_lib.sncc_batch_destroy.argtypes = [_vp]
_lib.sncc_batch_destroy.restype = None
_lib.sncc_batch_device_bytes.argtypes = [_vp]
_lib.sncc_batch_device_bytes.restype = C.c_size_t
_lib.sncc_batch_upload.argtypes = [_vp, _vp, C.c_size_t, _vp]
_lib.sncc_batch_set_variant.argtypes = [_vp, C.c_int]
_lib.sncc_batch_set_bucket_variant.argtypes = [_vp, C.c_int, C.c_int, C.c_int]
_lib.sncc_batch_get_bucket.argtypes = [_vp, C.c_int, C.POINTER(BatchBucket)]
_lib.sncc_batch_get_info.argtypes = [_vp, C.POINTER(BatchInfo)]
_lib.sncc_batch_match.argtypes = [_vp, _vp, _pp, _pp, C.c_int, C.c_int, _vp, C.c_int, _vp, _vp, _vp, _vp]
_lib.sncc_batch_autotune.argtypes = [_vp, _vp, _pp, _pp, C.c_int, C.c_int, _vp, C.c_int, _vp, _vp, _vp, C.c_int,
                                     _vp, C.POINTER(C.c_float)]
_lib.sncc_batch_refine_workspace_bytes.argtypes = [_vp, C.c_int]
_lib.sncc_batch_refine_workspace_bytes.restype = C.c_size_t
_lib.sncc_batch_refine.argtypes = [_vp, _vp, _pp, C.c_int, _vp, _vp, C.c_int, _vp, C.c_int, _vp, _vp, C.c_size_t,
                                   _vp, _vp]
_lib.sncc_diff_workspace_bytes.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int]
_lib.sncc_diff_workspace_bytes.restype = C.c_size_t
_lib.sncc_diff_forward.argtypes = [_vp, C.c_int, C.c_int, C.c_int, _vp, C.c_int, C.c_int, _vp, _vp, C.c_int, _vp,
                                   _vp, _vp, _vp, C.c_size_t, _vp]
_lib.sncc_diff_backward.argtypes = [_vp, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, _vp, _vp, C.c_int, _vp, _vp,
                                    _vp, _vp, C.c_int, _vp, _vp, C.c_size_t, _vp]
_lib.sncc_get_plan_info.argtypes = [C.POINTER(_Segments), C.POINTER(PlanInfo)]
_lib.sncc_probe_smem_read.argtypes = [_vp, C.c_int, C.c_int, _vp]
_lib.sncc_probe_alu.argtypes = [C.c_int, _vp, C.c_int, C.c_int, _vp]
_lib.sncc_probe_wait_timeout.argtypes = [_vp, _vp]
_lib.sncc_probe_hbm_write.argtypes = [_vp, C.c_size_t, _vp]
_lib.sncc_exact_map.argtypes = [_vp, C.c_int, C.c_int, C.c_int, _vp, C.c_int, C.c_int, C.c_int, C.c_int64,
                                C.c_int64, _vp, C.c_int, _vp, C.c_int, _vp, C.c_int, _vp]


def lib() -> C.CDLL:
    return _lib


def _check(code: int, what: str):
    if code != OK:
        raise SnccError(code, what)


def version() -> str:
    return _lib.sncc_version().decode()


# ---------------------------------------------------------------------------
# Template preparation
# ---------------------------------------------------------------------------
class Segments:
    """Owns an sncc_segments (host); exposes the table as numpy arrays."""

    def __init__(self, t: np.ndarray, sigma_max: float, k_max: int = 0):
        t = np.ascontiguousarray(np.asarray(t, dtype=np.uint8))
        if t.ndim != 2:
            raise ValueError("template must be 2-D (H, W)")
        H, W = t.shape
        self._s = _Segments()
        self._t = t
        _check(_lib.sncc_build_segments(t.ctypes.data, W, H, W, float(sigma_max), int(k_max), C.byref(self._s)),
               "sncc_build_segments")
        self.W, self.H = W, H
        self.sigma_max = float(sigma_max)
        self.k_max = int(k_max)

    def __del__(self):
        s = getattr(self, "_s", None)
        if s is not None and _lib is not None:
            _lib.sncc_free_segments(C.byref(s))

    def ref(self):
        return C.byref(self._s)

    K = property(lambda self: int(self._s.K))
    K_split = property(lambda self: int(self._s.K_split))
    sigma_used = property(lambda self: float(self._s.sigma_used))
    kbar = property(lambda self: float(self._s.kbar))
    Ek = property(lambda self: float(self._s.Ek))
    rho_max = property(lambda self: float(self._s.rho_max))
    T = property(lambda self: int(self._s.T))
    T2 = property(lambda self: int(self._s.T2))
    err_bound = property(lambda self: float(self._s.err_bound))
    sigma_t = property(lambda self: float(self._s.sigma_t))

    @property
    def table(self) -> np.ndarray:
        """(K, 4) int64 array of (x, y, w, h)."""
        return np.array([(self._s.seg[i].x, self._s.seg[i].y, self._s.seg[i].w, self._s.seg[i].h)
                         for i in range(self.K)], dtype=np.int64).reshape(-1, 4)

    @property
    def sums(self) -> np.ndarray:
        return np.array([self._s.seg[i].sum for i in range(self.K)], dtype=np.int64)

    @property
    def means(self) -> np.ndarray:
        return np.array([self._s.seg[i].mean for i in range(self.K)], dtype=np.float64)

    def plan_bytes(self) -> int:
        return int(_lib.sncc_plan_bytes(C.byref(self._s)))

    def plan_info(self) -> dict:
        pi = PlanInfo()
        _check(_lib.sncc_get_plan_info(C.byref(self._s), C.byref(pi)), "sncc_get_plan_info")
        return {k: int(getattr(pi, k)) for k, _ in PlanInfo._fields_}


def build_segments(t: np.ndarray, sigma_max: float, k_max: int = 0) -> Segments:
    return Segments(t, sigma_max, k_max)


def sat_pitch(M: int) -> int:
    return int(_lib.sncc_sat_pitch(M))


# ---------------------------------------------------------------------------
# Device calls (torch tensors for memory, current stream)
# ---------------------------------------------------------------------------
def _torch():
    import torch
    return torch


def _stream(stream=None):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _ptr(t) -> Optional[int]:
    return None if t is None else t.data_ptr()


@dataclass
class Tables:
    """Padded sum tables of one source: s (int32 or int64) and s2 (int64),
    each (N+1, pitch) on the device.  An int32 s holds the sums modulo 2^32
    (exact while 255*M*N < 2^31)."""
    s: "object"
    s2: "object"
    s_bits: int
    pitch: int
    M: int
    N: int


def choose_bits(M: int, N: int) -> int:
    """int32 where 255*M*N cannot overflow it, int64 otherwise: tables whose
    entries are the sums themselves."""
    return 32 if 255 * M * N < 2 ** 31 else 64


DIRECT_MAX_CORNERS = 64  # SNCC_DIRECT_MAX_CORNERS


def match_bits(M: int, N: int, segs=()) -> int:
    """Width of s for matching the approximations `segs` on an M x N source.

    The segment-sum kernels read s only through differences no larger than
    a template window (255*W*H < 2^31), which a 32-bit table holds exactly
    even where its entries wrap modulo 2^32: 32 bits (12 bytes per pixel
    written instead of 16, half the bytes per staged region word).  A
    template of at most DIRECT_MAX_CORNERS corners is summed from its
    corners' entries themselves, without staging; where a 32-bit table may
    wrap it would be staged instead, so such a matcher keeps 64 bits."""
    if 255 * M * N < 2 ** 31:
        return 32
    sparse = any(sg.plan_info()["template_corners"] <= DIRECT_MAX_CORNERS for sg in segs)
    return 64 if sparse else 32


def alloc_tables(M: int, N: int, s_bits: Optional[int] = None, device="cuda") -> Tables:
    torch = _torch()
    bits = s_bits or choose_bits(M, N)
    P = sat_pitch(M)
    s = torch.empty((N + 1, P), dtype=torch.int32 if bits == 32 else torch.int64, device=device)
    s2 = torch.empty((N + 1, P), dtype=torch.int64, device=device)
    return Tables(s, s2, bits, P, M, N)


def integral_workspace(M: int, N: int, device="cuda"):
    torch = _torch()
    return torch.empty(int(_lib.sncc_integral_workspace_bytes(M, N)), dtype=torch.uint8, device=device)


# kernels one sncc_integral call launches: column sums of bands, band scan,
# band emit
INTEGRAL_KERNELS = 3
# kernels one sncc_refine launches: the exact NCC at the candidates, then the
# sorted write-out (mark or rank, scan, scatter)
REFINE_KERNELS = 4


def integral(f, tables: Optional[Tables] = None, s_bits: Optional[int] = None, workspace=None, stream=None) -> Tables:
    """sncc_integral on a (N, M) uint8 CUDA tensor (row stride = its stride)."""
    torch = _torch()
    if f.dtype != torch.uint8 or f.dim() != 2 or not f.is_cuda or f.stride(1) != 1:
        raise ValueError("f must be a 2-D uint8 CUDA tensor with unit column stride")
    N, M = f.shape
    tb = tables or alloc_tables(M, N, s_bits, f.device)
    ws = workspace if workspace is not None else integral_workspace(M, N, f.device)
    _check(_lib.sncc_integral(f.data_ptr(), M, N, f.stride(0), tb.s.data_ptr(), tb.s_bits, tb.s2.data_ptr(),
                              tb.pitch, ws.data_ptr(), ws.numel(), _stream(stream)), "sncc_integral")
    return tb


def integral_noalloc(f, tables: Optional[Tables] = None, s_bits: Optional[int] = None, stream=None) -> Tables:
    """sncc_integral_noalloc: the same sum tables with no workspace argument;
    the library's fixed scratch array is used instead (see include/sncc.h)."""
    torch = _torch()
    if f.dtype != torch.uint8 or f.dim() != 2 or not f.is_cuda or f.stride(1) != 1:
        raise ValueError("f must be a 2-D uint8 CUDA tensor with unit column stride")
    N, M = f.shape
    tb = tables or alloc_tables(M, N, s_bits, f.device)
    _check(_lib.sncc_integral_noalloc(f.data_ptr(), M, N, f.stride(0), tb.s.data_ptr(), tb.s_bits,
                                      tb.s2.data_ptr(), tb.pitch, _stream(stream)), "sncc_integral_noalloc")
    return tb


def upload_plan(seg: Segments, device="cuda", stream=None):
    torch = _torch()
    nbytes = seg.plan_bytes()
    buf = torch.empty(max(16, (nbytes + 15) // 16 * 16), dtype=torch.uint8, device=device)
    _check(_lib.sncc_plan_upload(seg.ref(), buf.data_ptr(), buf.numel(), _stream(stream)), "sncc_plan_upload")
    return buf


@dataclass
class MatchBuffers:
    cand: "object"
    count: "object"
    status: "object"
    rho: "object"


def alloc_match(M: int, N: int, W: int, H: int, cand_cap: int, with_rho: bool = True, device="cuda") -> MatchBuffers:
    torch = _torch()
    U, V = M - W + 1, N - H + 1
    return MatchBuffers(cand=torch.empty(max(cand_cap, 1), dtype=torch.int32, device=device),
                        count=torch.zeros(1, dtype=torch.int32, device=device),
                        status=torch.zeros(1, dtype=torch.int32, device=device),
                        rho=torch.empty((V, U), dtype=torch.float32, device=device) if with_rho else None)


def match(seg: Segments, plan, tables: Tables, tau: float, bufs: MatchBuffers, cand_cap: Optional[int] = None,
          stream=None) -> None:
    """sncc_match: fills bufs.rho (if allocated), bufs.cand, bufs.count, bufs.status."""
    cap = bufs.cand.numel() if cand_cap is None else cand_cap
    rho_pitch = bufs.rho.stride(0) if bufs.rho is not None else 0
    _check(_lib.sncc_match(seg.ref(), plan.data_ptr(), tables.s.data_ptr(), tables.s_bits, tables.s2.data_ptr(),
                           tables.pitch, tables.M, tables.N, float(tau), _ptr(bufs.rho), rho_pitch,
                           bufs.cand.data_ptr(), cap, bufs.count.data_ptr(), bufs.status.data_ptr(),
                           _stream(stream)), "sncc_match")


MULTI_MAX = 4  # SNCC_MULTI_MAX


def match_multi(segs, plans, tables: Tables, taus, bufs, cand_cap: Optional[int] = None, stream=None) -> None:
    """sncc_match_multi: sncc_match for up to MULTI_MAX approximations of one
    template size in one launch; bufs[q] receives what match() would write
    for segs[q] (including bufs[q].status).  Raises
    SnccError with code ERR_UNSUPPORTED when the approximations do not fit
    one fused launch (then call match() for each)."""
    n = len(segs)
    if not (len(plans) == len(taus) == len(bufs) == n):
        raise ValueError("segs, plans, taus and bufs must have the same length")
    cap = min(b.cand.numel() for b in bufs) if cand_cap is None else cand_cap
    with_rho = [b.rho is not None for b in bufs]
    rho_pitch = next((b.rho.stride(0) for b in bufs if b.rho is not None), 0)
    if any(b.rho is not None and b.rho.stride(0) != rho_pitch for b in bufs):
        raise ValueError("all rho maps must have the same row pitch")
    seg_arr = (C.POINTER(_Segments) * n)(*[C.pointer(sg._s) for sg in segs])
    plan_arr = (_vp * n)(*[pl.data_ptr() for pl in plans])
    tau_arr = (C.c_float * n)(*[float(t) for t in taus])
    rho_arr = (_vp * n)(*[_ptr(b.rho) for b in bufs]) if any(with_rho) else None
    cand_arr = (_vp * n)(*[b.cand.data_ptr() for b in bufs])
    count_arr = (_vp * n)(*[b.count.data_ptr() for b in bufs])
    status_arr = (_vp * n)(*[b.status.data_ptr() for b in bufs])
    _check(_lib.sncc_match_multi(seg_arr, plan_arr, n, tables.s.data_ptr(), tables.s_bits, tables.s2.data_ptr(),
                                 tables.pitch, tables.M, tables.N, tau_arr, rho_arr, rho_pitch, cand_arr, cap,
                                 count_arr, status_arr, _stream(stream)), "sncc_match_multi")


@dataclass
class RefineBuffers:
    out: "object"      # (out_cap, 3) int32 view of sncc_match_t records
    nout: "object"
    ws: "object"
    cap: int


def alloc_refine(M: int, N: int, W: int, H: int, out_cap: int, device="cuda") -> RefineBuffers:
    """Match records and workspace of sncc_refine / sncc_refine_segmented for
    an M x N source and a W x H template (the workspace holds the records
    before sorting and one bit per offset for the sort)."""
    torch = _torch()
    nbytes = int(_lib.sncc_refine_workspace_bytes(M, N, W, H, out_cap))
    if nbytes == 0:
        raise SnccError(ERR_ARG, "sncc_refine_workspace_bytes")
    return RefineBuffers(out=torch.empty((max(out_cap, 1), 3), dtype=torch.int32, device=device),
                         nout=torch.zeros(1, dtype=torch.int32, device=device),
                         ws=torch.empty(nbytes, dtype=torch.uint8, device=device),
                         cap=out_cap)


def refine(f, t_dev, seg: Segments, bufs: MatchBuffers, tau: float, rb: RefineBuffers, cand_cap: Optional[int] = None,
           stream=None) -> None:
    """sncc_refine on the candidates in bufs; matches land in rb.out sorted by v*U+u."""
    N, M = f.shape
    H, W = t_dev.shape
    cap = bufs.cand.numel() if cand_cap is None else cand_cap
    _check(_lib.sncc_refine(f.data_ptr(), M, N, f.stride(0), t_dev.data_ptr(), W, H, t_dev.stride(0), seg.T, seg.T2,
                            bufs.cand.data_ptr(), bufs.count.data_ptr(), cap, float(tau), rb.out.data_ptr(), rb.cap,
                            rb.nout.data_ptr(), rb.ws.data_ptr(), rb.ws.numel(), bufs.status.data_ptr(),
                            _stream(stream)), "sncc_refine")


def refine_segmented(seg_fine: Segments, plan_fine, tables: Tables, bufs: MatchBuffers, tau: float,
                     rb: RefineBuffers, cand_cap: Optional[int] = None, stream=None) -> None:
    """sncc_refine_segmented: the paper's fine stage (k_slow) at the coarse
    candidates in bufs; matches land in rb.out sorted by v*U+u."""
    cap = bufs.cand.numel() if cand_cap is None else cand_cap
    _check(_lib.sncc_refine_segmented(seg_fine.ref(), plan_fine.data_ptr(), tables.s.data_ptr(), tables.s_bits,
                                      tables.s2.data_ptr(), tables.pitch, tables.M, tables.N, bufs.cand.data_ptr(),
                                      bufs.count.data_ptr(), cap, float(tau), rb.out.data_ptr(), rb.cap,
                                      rb.nout.data_ptr(), rb.ws.data_ptr(), rb.ws.numel(), bufs.status.data_ptr(),
                                      _stream(stream)), "sncc_refine_segmented")


def tiles_workspace(M: int, N: int, W: int, H: int, out_cap: int, device="cuda"):
    """Workspace for refine_segmented_tiles (256-byte aligned)."""
    torch = _torch()
    nbytes = int(_lib.sncc_refine_segmented_tiles_workspace_bytes(M, N, W, H, out_cap))
    if nbytes == 0:
        raise SnccError(ERR_ARG, "sncc_refine_segmented_tiles_workspace_bytes")
    raw = torch.empty(nbytes + 256, dtype=torch.uint8, device=device)
    off = (-raw.data_ptr()) % 256
    return raw[off:off + nbytes]


def refine_segmented_tiles(seg_fine: Segments, plan_fine, tables: Tables, bufs: MatchBuffers, tau: float,
                           rb: RefineBuffers, ws, cand_cap: Optional[int] = None, stream=None) -> None:
    """sncc_refine_segmented_tiles: the paper's fine stage evaluated on the
    tiles that hold coarse candidates; matches land in rb.out sorted by v*U+u."""
    cap = bufs.cand.numel() if cand_cap is None else cand_cap
    _check(_lib.sncc_refine_segmented_tiles(seg_fine.ref(), plan_fine.data_ptr(), tables.s.data_ptr(),
                                            tables.s_bits, tables.s2.data_ptr(), tables.pitch, tables.M, tables.N,
                                            bufs.cand.data_ptr(), bufs.count.data_ptr(), cap, float(tau),
                                            rb.out.data_ptr(), rb.cap, rb.nout.data_ptr(), ws.data_ptr(),
                                            ws.numel(), bufs.status.data_ptr(), _stream(stream)),
           "sncc_refine_segmented_tiles")


def matches_to_numpy(rb: RefineBuffers):
    """(u, v, rho) arrays of the stored matches (after the stream is synced)."""
    import torch
    n = min(int(rb.nout.item()), rb.cap)
    raw = rb.out[:n].cpu().numpy()
    u = raw[:, 0].astype(np.int64)
    v = raw[:, 1].astype(np.int64)
    rho = raw[:, 2].copy().view(np.float32)
    return u, v, rho


def exact_map(f, t_dev, T: int, T2: int, tables: Tables, rho=None, stream=None):
    """sncc_exact_map: exact NCC at every offset (FP32 map)."""
    torch = _torch()
    N, M = f.shape
    H, W = t_dev.shape
    U, V = M - W + 1, N - H + 1
    out = rho if rho is not None else torch.empty((V, U), dtype=torch.float32, device=f.device)
    _check(_lib.sncc_exact_map(f.data_ptr(), M, N, f.stride(0), t_dev.data_ptr(), W, H, t_dev.stride(0), int(T),
                               int(T2), tables.s.data_ptr(), tables.s_bits, tables.s2.data_ptr(), tables.pitch,
                               out.data_ptr(), out.stride(0), _stream(stream)), "sncc_exact_map")
    return out


def probe_smem_read(sink, ctas: int, iters: int, stream=None) -> int:
    """Launches the shared-memory read probe; returns the bytes it reads."""
    _check(_lib.sncc_probe_smem_read(sink.data_ptr(), ctas, iters, _stream(stream)), "sncc_probe_smem_read")
    return ctas * 256 * iters * 32 * 4


PROBE_DP4A, PROBE_IMAD_WIDE = 0, 1


def probe_hbm_write(buf, stream=None) -> int:
    """Launches the HBM write probe over the whole uint8 buffer; returns the
    bytes written."""
    n = buf.numel() * buf.element_size()
    _check(_lib.sncc_probe_hbm_write(buf.data_ptr(), n, _stream(stream)), "sncc_probe_hbm_write")
    return n


def probe_wait_timeout(status, stream=None) -> None:
    """Runs the bounded-wait test hook: a wait that nothing completes gives up
    after the library's limit and sets STATUS_WAIT_TIMEOUT in status."""
    _check(_lib.sncc_probe_wait_timeout(status.data_ptr(), _stream(stream)), "sncc_probe_wait_timeout")


def probe_alu(kind: int, sink, ctas: int, iters: int, stream=None) -> int:
    """Launches the instruction-rate probe; returns the instructions it issues
    (lane operations)."""
    _check(_lib.sncc_probe_alu(kind, sink.data_ptr(), ctas, iters, _stream(stream)), "sncc_probe_alu")
    return ctas * 256 * iters * 64


# ---------------------------------------------------------------------------
# The whole path, as a user calls it
# ---------------------------------------------------------------------------
def template_sigma(t: np.ndarray) -> float:
    """sigma_t of the paper's thresholds: the population std of the template
    (sncc_template_sigma, from its exact integer sums)."""
    t = np.ascontiguousarray(np.asarray(t, dtype=np.uint8))
    if t.ndim != 2:
        raise ValueError("template must be 2-D (H, W)")
    H, W = t.shape
    out = C.c_double()
    _check(_lib.sncc_template_sigma(t.ctypes.data, W, H, W, C.byref(out)), "sncc_template_sigma")
    return float(out.value)


class PaperMatcher:
    """The paper's own two-approximation search (Section 5 main algorithm):
    coarse k_fast (sigma_max = 0.99 sigma_t) at every offset, then the finer
    k_slow (sigma_max = 0.1 sigma_t, K_max = 5000) at the candidates,
    thresholds precision * rho_fast and precision * rho_slow.  The fine stage
    runs tile by tile on the tiles that hold candidates."""

    def __init__(self, t: np.ndarray, M: int, N: int, precision: float = 0.9, fast: float = 0.99,
                 slow: float = 0.1, k_max: int = 5000, cand_cap: int = 1 << 20, out_cap: int = 1 << 16,
                 keep_rho: bool = True, device="cuda"):
        st = template_sigma(t)
        self.fast = build_segments(t, fast * st, k_max)
        self.slow = build_segments(t, slow * st, k_max)
        if not (self.fast.Ek > 0 and self.slow.Ek > 0):
            raise SnccError(ERR_UNIFORM, "PaperMatcher")
        self.M, self.N = M, N
        self.W, self.H = self.fast.W, self.fast.H
        self.tau_fast = float(precision) * self.fast.rho_max
        self.tau_slow = float(precision) * self.slow.rho_max
        self.plan_fast = upload_plan(self.fast, device)
        self.plan_slow = upload_plan(self.slow, device)
        self.tables = alloc_tables(M, N, match_bits(M, N, (self.fast, self.slow)), device)
        self.ws = integral_workspace(M, N, device)
        self.mb = alloc_match(M, N, self.W, self.H, cand_cap, keep_rho, device)
        self.rb = alloc_refine(M, N, self.W, self.H, out_cap, device)
        self.tws = tiles_workspace(M, N, self.W, self.H, out_cap, device)

    def run(self, f, stream=None):
        integral(f, self.tables, workspace=self.ws, stream=stream)
        match(self.fast, self.plan_fast, self.tables, self.tau_fast, self.mb, stream=stream)
        refine_segmented_tiles(self.slow, self.plan_slow, self.tables, self.mb, self.tau_slow, self.rb, self.tws,
                               stream=stream)

    def status(self) -> int:
        return int(self.mb.status.item())


def capture_graph(launch):
    """Records the launches that launch() makes on the current stream into a
    CUDA graph, after one eager run on a side stream (which also performs the
    library's one-time setup outside the capture)."""
    torch = _torch()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        launch()
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        launch()
    return g


class Matcher:
    """Segmented-NCC template matcher for one template on one GPU.

    Prepares the approximation once (host), uploads its plan, and owns every
    device buffer, so that run() only launches kernels: sum tables, coarse
    pass, exact refine (Section 5 main algorithm with an exact second stage)."""

    def __init__(self, t: np.ndarray, sigma_max: float, M: int, N: int, precision: float = 0.9,
                 tau_exact: Optional[float] = None, k_max: int = 0, cand_cap: int = 1 << 20, out_cap: int = 1 << 16,
                 keep_rho: bool = True, device="cuda"):
        torch = _torch()
        self.seg = build_segments(t, sigma_max, k_max)
        if not self.seg.Ek > 0:
            raise SnccError(ERR_UNIFORM, "Matcher")
        self.M, self.N = M, N
        self.W, self.H = self.seg.W, self.seg.H
        self.U, self.V = M - self.W + 1, N - self.H + 1
        self.tau_c = float(precision) * self.seg.rho_max
        self.tau_e = float(precision) if tau_exact is None else float(tau_exact)
        self.device = device
        self.t_dev = torch.as_tensor(np.ascontiguousarray(t, np.uint8)).to(device)
        self.plan = upload_plan(self.seg, device)
        self.tables = alloc_tables(M, N, match_bits(M, N, (self.seg,)), device)
        self.ws = integral_workspace(M, N, device)
        self.mb = alloc_match(M, N, self.W, self.H, cand_cap, keep_rho, device)
        self.rb = alloc_refine(M, N, self.W, self.H, out_cap, device)

    def run(self, f, stream=None):
        """Launch the whole path on a (N, M) uint8 CUDA tensor (asynchronous)."""
        integral(f, self.tables, workspace=self.ws, stream=stream)
        match(self.seg, self.plan, self.tables, self.tau_c, self.mb, stream=stream)
        refine(f, self.t_dev, self.seg, self.mb, self.tau_e, self.rb, stream=stream)

    def capture(self, f):
        """Record run(f) in a CUDA graph (after one eager warm-up run); replay
        it after writing each new source into f."""
        return capture_graph(lambda: self.run(f))

    def status(self) -> int:
        return int(self.mb.status.item())


class MultiMatcher:
    """Segmented-NCC matching of one template at several std thresholds (one
    approximation each) on one GPU, e.g. the thresholds of a multi-threshold
    search.  run(): the sum tables once, the coarse passes of every
    approximation in one fused launch where the library accepts them
    (sncc_match_multi: same template, up to 64 x 64, more than 64 corners
    each), else one launch each, then the exact refine of each approximation.
    Output q lives in mbs[q] / rbs[q]."""

    def __init__(self, t: np.ndarray, sigmas, M: int, N: int, precision: float = 0.85,
                 tau_exact: Optional[float] = None, k_max: int = 0, cand_cap: int = 1 << 20, out_cap: int = 1 << 16,
                 keep_rho: bool = True, device="cuda"):
        torch = _torch()
        self.segs = [build_segments(t, sg, k_max) for sg in sigmas]
        if not all(sg.Ek > 0 for sg in self.segs):
            raise SnccError(ERR_UNIFORM, "MultiMatcher")
        self.M, self.N = M, N
        self.W, self.H = self.segs[0].W, self.segs[0].H
        self.taus = [float(precision) * sg.rho_max for sg in self.segs]
        self.tau_e = float(precision) if tau_exact is None else float(tau_exact)
        self.t_dev = torch.as_tensor(np.ascontiguousarray(t, np.uint8)).to(device)
        self.plans = [upload_plan(sg, device) for sg in self.segs]
        self.tables = alloc_tables(M, N, match_bits(M, N, self.segs), device)
        self.ws = integral_workspace(M, N, device)
        self.mbs = [alloc_match(M, N, self.W, self.H, cand_cap, keep_rho, device) for _ in self.segs]
        self.rbs = [alloc_refine(M, N, self.W, self.H, out_cap, device) for _ in self.segs]
        self.fused = None if len(self.segs) > 1 and MULTI_MAX >= len(self.segs) else False
        # the refines of the approximations are independent: all but the
        # first run on side streams (parallel branches of a captured graph)
        self.side = [torch.cuda.Stream(device) for _ in self.segs[1:]]

    def run(self, f, stream=None):
        """Launch the whole path on a (N, M) uint8 CUDA tensor (asynchronous).
        The first run finds out whether the coarse passes fuse (the library
        decides before it launches anything)."""
        integral(f, self.tables, workspace=self.ws, stream=stream)
        if self.fused is not False:
            try:
                match_multi(self.segs, self.plans, self.tables, self.taus, self.mbs, stream=stream)
                self.fused = True
            except SnccError as e:
                if e.code != ERR_UNSUPPORTED or self.fused:
                    raise
                self.fused = False
        if not self.fused:
            for sg, pl, tau, mb in zip(self.segs, self.plans, self.taus, self.mbs):
                match(sg, pl, self.tables, tau, mb, stream=stream)
        torch = _torch()
        main = torch.cuda.current_stream() if stream is None else stream
        for q, (sg, mb, rb) in enumerate(zip(self.segs, self.mbs, self.rbs)):
            if q == 0:
                refine(f, self.t_dev, sg, mb, self.tau_e, rb, stream=main)
                continue
            side = self.side[q - 1]
            side.wait_stream(main)
            refine(f, self.t_dev, sg, mb, self.tau_e, rb, stream=side)
        for side in self.side:
            main.wait_stream(side)

    def capture(self, f):
        """Record run(f) in a CUDA graph (after one eager warm-up run)."""
        return capture_graph(lambda: self.run(f))

    def status(self) -> int:
        s = 0
        for mb in self.mbs:
            s |= int(mb.status.item())
        return s


class StreamMatcher:
    """Pipelined matching of a stream of frames (pinned host uint8 tensors of
    N x M) with one template at one or more std thresholds, through the
    library's native frame pipeline (sncc_pipeline_*): two slots of device
    buffers, each slot's path captured in a CUDA graph, the next frame's copy
    and the previous frame's read-back overlapping the current frame's
    matching, one library call per frame.  submit(frame) returns the previous
    frame's lists (None on the first call); flush() returns the last one.  A
    list is one (u, v, rho) triple of numpy arrays per threshold."""

    def __init__(self, t: np.ndarray, sigmas, M: int, N: int, precision: float = 0.85,
                 tau_exact: Optional[float] = None, k_max: int = 0, cand_cap: int = 1 << 20, out_cap: int = 1 << 16,
                 keep_rho: bool = False, device="cuda"):
        torch = _torch()
        self.segs = [build_segments(t, sg, k_max) for sg in sigmas]
        n = len(self.segs)
        if not 1 <= n <= MULTI_MAX:
            raise ValueError("1 .. %d thresholds" % MULTI_MAX)
        if not all(sg.Ek > 0 for sg in self.segs):
            raise SnccError(ERR_UNIFORM, "StreamMatcher")
        self.M, self.N, self.n = M, N, n
        W, H = self.segs[0].W, self.segs[0].H
        self.taus = [float(precision) * sg.rho_max for sg in self.segs]
        self.tau_e = float(precision) if tau_exact is None else float(tau_exact)
        self.t_dev = torch.as_tensor(np.ascontiguousarray(t, np.uint8)).to(device)
        self.plans = [upload_plan(sg, device) for sg in self.segs]
        self._bufs = []
        slots = (_PipelineSlot * 2)()
        rho_pitch = 0
        for k in range(2):
            frame = torch.zeros((N, M), dtype=torch.uint8, device=device)
            tables = alloc_tables(M, N, match_bits(M, N, self.segs), device)
            ws = integral_workspace(M, N, device)
            mbs = [alloc_match(M, N, W, H, cand_cap, keep_rho, device) for _ in self.segs]
            rbs = [alloc_refine(M, N, W, H, out_cap, device) for _ in self.segs]
            sl = slots[k]
            sl.d_frame, sl.d_s, sl.d_s2 = frame.data_ptr(), tables.s.data_ptr(), tables.s2.data_ptr()
            sl.d_ws, sl.ws_bytes = ws.data_ptr(), ws.numel()
            for q in range(n):
                sl.d_rho[q] = _ptr(mbs[q].rho)
                sl.d_cand[q], sl.d_count[q] = mbs[q].cand.data_ptr(), mbs[q].count.data_ptr()
                sl.d_status[q] = mbs[q].status.data_ptr()
                sl.d_out[q], sl.d_nout[q], sl.d_rws[q] = rbs[q].out.data_ptr(), rbs[q].nout.data_ptr(), rbs[q].ws.data_ptr()
            sl.rws_bytes = rbs[0].ws.numel()
            if keep_rho:
                rho_pitch = mbs[0].rho.stride(0)
            self._bufs.append((frame, tables, ws, mbs, rbs))
        self.s_bits = self._bufs[0][1].s_bits
        torch.cuda.synchronize()  # the buffers are allocated and zeroed before the pipeline's streams use them
        seg_arr = (C.POINTER(_Segments) * n)(*[C.pointer(sg._s) for sg in self.segs])
        plan_arr = (_vp * n)(*[pl.data_ptr() for pl in self.plans])
        tau_arr = (C.c_float * n)(*self.taus)
        h = _vp()
        _check(_lib.sncc_pipeline_create(seg_arr, plan_arr, n, self.t_dev.data_ptr(), self.t_dev.stride(0), M, N,
                                         self.s_bits, self._bufs[0][1].pitch, tau_arr, self.tau_e, cand_cap, out_cap,
                                         rho_pitch, slots, C.byref(h)), "sncc_pipeline_create")
        self._h = h
        self.fused = bool(_lib.sncc_pipeline_fused(h))
        self.compute = torch.cuda.ExternalStream(_lib.sncc_pipeline_compute_stream(h), device=device)
        self.out_cap = out_cap
        self.h_out = [torch.empty((out_cap, 3), dtype=torch.int32, pin_memory=True) for _ in self.segs]
        self._h_out_ptrs = (_vp * n)(*[x.data_ptr() for x in self.h_out])
        self.h_count = np.zeros(n, np.int32)
        self.h_status = np.zeros(n, np.int32)
        self._pc = self.h_count.ctypes.data_as(C.POINTER(C.c_int32))
        self._ps = self.h_status.ctypes.data_as(C.POINTER(C.c_int32))
        self.frames = 0
        self.d2h_bytes = 0
        self.status_bits = 0

    def _lists(self):
        self.d2h_bytes += 8 * self.n
        out = []
        for q in range(self.n):
            m = min(int(self.h_count[q]), self.out_cap)
            self.status_bits |= int(self.h_status[q])
            self.d2h_bytes += 12 * m
            raw = self.h_out[q][:m].numpy()
            out.append((raw[:, 0].astype(np.int64), raw[:, 1].astype(np.int64), raw[:, 2].copy().view(np.float32)))
        return out

    def submit(self, frame):
        """Queue one frame; returns the previous frame's match lists."""
        torch = _torch()
        if frame.dtype != torch.uint8 or tuple(frame.shape) != (self.N, self.M) or frame.is_cuda or \
                not frame.is_contiguous():
            raise ValueError("frame must be a contiguous host uint8 tensor of shape (N, M)")
        rc = _lib.sncc_pipeline_submit(self._h, frame.data_ptr(), self._h_out_ptrs, self._pc, self._ps)
        if rc < 0:
            _check(rc, "sncc_pipeline_submit")
        self.frames += 1
        return self._lists() if rc == 1 else None

    def flush(self):
        """The match lists of the last submitted frame (None if there is none)."""
        rc = _lib.sncc_pipeline_flush(self._h, self._h_out_ptrs, self._pc, self._ps)
        if rc < 0:
            _check(rc, "sncc_pipeline_flush")
        return self._lists() if rc == 1 else None

    def status(self) -> int:
        """OR of the status words of every frame reported so far."""
        return self.status_bits

    def close(self):
        if getattr(self, "_h", None):
            _lib.sncc_pipeline_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()


# ---------------------------------------------------------------------------
# Batched matching: many templates x several sources in one persistent launch
# ---------------------------------------------------------------------------
class Batch:
    """Segmented NCC of every (source, template) pair of a batch.

    run() launches: the sum tables of every source, one persistent coarse
    pass over all pairs (sncc_batch_match), and the exact refine of every
    candidate (sncc_batch_refine).  capture() records that sequence in a CUDA
    graph; autotune() picks the tile height on the caller's data."""

    def __init__(self, templates, sigmas, M: int, N: int, n_sources: int, precision: float = 0.85,
                 tau_exact: Optional[float] = None, k_max: int = 0, cand_cap: int = 1 << 22, out_cap: int = 1 << 16,
                 device="cuda"):
        torch = _torch()
        self.templates = [np.ascontiguousarray(np.asarray(t, np.uint8)) for t in templates]
        self.segs = [build_segments(t, sg, k_max) for t, sg in zip(self.templates, sigmas)]
        nt = len(self.templates)
        self.M, self.N, self.ns, self.nt = M, N, n_sources, nt
        seg_ptrs = (C.POINTER(_Segments) * nt)(*[C.pointer(sg._s) for sg in self.segs])
        pix = (C.c_void_p * nt)(*[t.ctypes.data for t in self.templates])
        strides = (C.c_int * nt)(*[t.shape[1] for t in self.templates])
        self.tau_c = [float(precision) * sg.rho_max for sg in self.segs]
        te = float(precision) if tau_exact is None else float(tau_exact)
        self.tau_e = [te] * nt
        tc = (C.c_float * nt)(*self.tau_c)
        tx = (C.c_float * nt)(*self.tau_e)
        h = C.c_void_p()
        _check(_lib.sncc_batch_create(seg_ptrs, pix, strides, tc, tx, nt, n_sources, M, N, C.byref(h)),
               "sncc_batch_create")
        self._h = h
        nbytes = int(_lib.sncc_batch_device_bytes(h))
        self.image = torch.empty(max(16, nbytes), dtype=torch.uint8, device=device)
        _check(_lib.sncc_batch_upload(h, self.image.data_ptr(), self.image.numel(), _stream(None)),
               "sncc_batch_upload")
        self.tables = [alloc_tables(M, N, match_bits(M, N), device) for _ in range(n_sources)]
        self.ws = integral_workspace(M, N, device)
        self.cand_cap, self.out_cap = cand_cap, out_cap
        self.cand = torch.empty(2 * max(cand_cap, 1), dtype=torch.int32, device=device)
        self.count = torch.zeros(1, dtype=torch.int32, device=device)
        self.counter = torch.zeros(1, dtype=torch.int32, device=device)
        self.status = torch.zeros(1, dtype=torch.int32, device=device)
        self.out = torch.empty((max(out_cap, 1), 4), dtype=torch.int32, device=device)
        self.nout = torch.zeros(1, dtype=torch.int32, device=device)
        self.rws = torch.empty(int(_lib.sncc_batch_refine_workspace_bytes(h, out_cap)), dtype=torch.uint8,
                               device=device)
        self._s = (C.c_void_p * n_sources)(*[tb.s.data_ptr() for tb in self.tables])
        self._s2 = (C.c_void_p * n_sources)(*[tb.s2.data_ptr() for tb in self.tables])
        self.s_bits = self.tables[0].s_bits
        self.pitch = self.tables[0].pitch

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and _lib is not None:
            _lib.sncc_batch_destroy(h)

    def info(self) -> dict:
        bi = BatchInfo()
        _check(_lib.sncc_batch_get_info(self._h, C.byref(bi)), "sncc_batch_get_info")
        return {k: getattr(bi, k) for k, _ in BatchInfo._fields_}

    def set_tile_rows(self, R: int):
        """Every bucket to tile height R with 64 x 64 template blocks."""
        _check(_lib.sncc_batch_set_variant(self._h, int(R)), "sncc_batch_set_variant")

    def set_bucket_variant(self, bucket: int, R: int, block: int):
        _check(_lib.sncc_batch_set_bucket_variant(self._h, int(bucket), int(R), int(block)),
               "sncc_batch_set_bucket_variant")

    def buckets(self) -> list:
        """One dict per template bucket: templates, pairs, classes, the
        chosen variant (tile_rows, block) and the autotuner's times."""
        out = []
        for k in range(BATCH_BUCKETS):
            bb = BatchBucket()
            _check(_lib.sncc_batch_get_bucket(self._h, k, C.byref(bb)), "sncc_batch_get_bucket")
            d = {f: getattr(bb, f) for f, _ in BatchBucket._fields_ if f != "ms"}
            d["bucket"] = k
            d["ms"] = list(bb.ms)
            out.append(d)
        return out

    def _match_args(self):
        return (self._h, self.image.data_ptr(), self._s, self._s2, self.s_bits, self.pitch, self.cand.data_ptr(),
                self.cand_cap, self.count.data_ptr(), self.counter.data_ptr(), self.status.data_ptr())

    def run(self, sources, stream=None):
        """Launch the whole batched path (asynchronous) on (N, M) uint8 CUDA tensors."""
        if len(sources) != self.ns:
            raise ValueError("expected %d sources" % self.ns)
        for f, tb in zip(sources, self.tables):
            integral(f, tb, workspace=self.ws, stream=stream)
        _check(_lib.sncc_batch_match(*self._match_args(), _stream(stream)), "sncc_batch_match")
        fp = (C.c_void_p * self.ns)(*[f.data_ptr() for f in sources])
        _check(_lib.sncc_batch_refine(self._h, self.image.data_ptr(), fp, sources[0].stride(0), self.cand.data_ptr(),
                                      self.count.data_ptr(), self.cand_cap, self.out.data_ptr(), self.out_cap,
                                      self.nout.data_ptr(), self.rws.data_ptr(), self.rws.numel(),
                                      self.status.data_ptr(), _stream(stream)), "sncc_batch_refine")

    def autotune(self, sources, reps: int = 3, stream=None):
        """Time every variant of every bucket (the bucket alone) on these
        sources and keep the fastest per bucket; returns {bucket: {(R,
        block): ms}} for the buckets that hold pairs.  Synchronises."""
        for f, tb in zip(sources, self.tables):
            integral(f, tb, workspace=self.ws, stream=stream)
        ms = (C.c_float * (BATCH_BUCKETS * BATCH_VARIANTS))()
        _check(_lib.sncc_batch_autotune(*self._match_args(), int(reps), _stream(stream), ms), "sncc_batch_autotune")
        out = {}
        for k, bb in enumerate(self.buckets()):
            if bb["pairs"]:
                out[k] = {((8, 4, 2)[v % 3], 64 if v < 3 else 32): ms[k * BATCH_VARIANTS + v]
                          for v in range(BATCH_VARIANTS)}
        return out

    def capture(self, sources):
        """Record run(sources) in a CUDA graph (after one eager warm-up run)."""
        return capture_graph(lambda: self.run(sources))

    def candidates(self):
        """(pair, index) arrays of the stored candidates (after a sync)."""
        n = min(int(self.count.item()), self.cand_cap)
        c = self.cand[:2 * n].view(-1, 2).cpu().numpy()
        return c[:, 0].astype(np.int64), c[:, 1].astype(np.int64)

    def matches(self):
        """(pair, u, v, rho) arrays of the stored matches, sorted (after a sync)."""
        n = min(int(self.nout.item()), self.out_cap)
        raw = self.out[:n].cpu().numpy()
        return (raw[:, 0].astype(np.int64), raw[:, 1].astype(np.int64), raw[:, 2].astype(np.int64),
                raw[:, 3].copy().view(np.float32))


# ---------------------------------------------------------------------------
# Differentiation: L = sum_o (rho_k - rho_t)^2 with hand-written gradients
# ---------------------------------------------------------------------------
class DiffProblem:
    """Fixed segmentation (rectangles) of a float template t, with workspace,
    for the loss between segmented and exact NCC over a float source."""

    def __init__(self, t, rects, M: int, N: int, device="cuda"):
        torch = _torch()
        self.t = torch.as_tensor(np.ascontiguousarray(np.asarray(t, np.float32))).to(device)
        self.rects = torch.as_tensor(np.ascontiguousarray(np.asarray(rects, np.int32))).to(device)
        self.H, self.W = self.t.shape
        self.M, self.N = M, N
        self.K = self.rects.shape[0]
        nbytes = int(_lib.sncc_diff_workspace_bytes(M, N, self.W, self.H))
        if nbytes == 0:
            raise SnccError(ERR_ARG, "sncc_diff_workspace_bytes")
        self.ws = torch.empty(nbytes + 256, dtype=torch.uint8, device=device)
        off = (-self.ws.data_ptr()) % 256
        self.ws_ptr = self.ws.data_ptr() + off
        self.ws_bytes = nbytes
        self.U, self.V = M - self.W + 1, N - self.H + 1
        self._ws_holds = None  # (f, k) identity and versions of the forward the workspace holds

    def loss(self, f, k):
        """Differentiable L(f, k) (float64 scalar tensor)."""
        return _SegmentedNCCLoss.apply(f, k, self)


def _diff_forward(pb: DiffProblem, f, k):
    torch = _torch()
    rho_k = torch.empty((pb.V, pb.U), dtype=torch.float32, device=f.device)
    rho_t = torch.empty_like(rho_k)
    loss = torch.empty(1, dtype=torch.float64, device=f.device)
    _check(_lib.sncc_diff_forward(f.data_ptr(), pb.M, pb.N, f.stride(0), pb.t.data_ptr(), pb.W, pb.H,
                                  pb.rects.data_ptr(), k.data_ptr(), pb.K, rho_k.data_ptr(), rho_t.data_ptr(),
                                  loss.data_ptr(), pb.ws_ptr, pb.ws_bytes, _stream(None)), "sncc_diff_forward")
    pb._ws_holds = _ws_token(f, k)
    return rho_k, rho_t, loss


def _ws_token(f, k):
    """Identity of a forward's inputs: storage, layout and in-place version."""
    return (f.data_ptr(), f.stride(0), f._version, k.data_ptr(), k._version)


def _make_autograd():
    import torch

    class SegmentedNCCLoss(torch.autograd.Function):
        """L = sum_o (rho_k - rho_t)^2; backward by the library's kernels."""

        @staticmethod
        def forward(ctx, f, k, pb):
            if f.dtype != torch.float32 or k.dtype != torch.float32 or not f.is_cuda or f.stride(1) != 1:
                raise ValueError("f and k must be float32 CUDA tensors (f with unit column stride)")
            k = k.contiguous()
            rho_k, rho_t, loss = _diff_forward(pb, f, k)
            ctx.pb = pb
            ctx.save_for_backward(f, k, rho_k, rho_t)
            return loss[0]

        @staticmethod
        def backward(ctx, dloss):
            f, k, rho_k, rho_t = ctx.saved_tensors
            pb = ctx.pb
            # the workspace must hold this forward's intermediates; it still does
            # unless another forward ran on it or the inputs changed in place
            if pb._ws_holds != _ws_token(f, k):
                _diff_forward(pb, f, k)
            dl = dloss.reshape(1).to(torch.float64).contiguous()
            grad_f = torch.empty((pb.N, pb.M), dtype=torch.float32, device=f.device)
            grad_k = torch.empty(pb.K, dtype=torch.float32, device=f.device)
            _check(_lib.sncc_diff_backward(f.data_ptr(), pb.M, pb.N, f.stride(0), pb.W, pb.H, pb.rects.data_ptr(),
                                           k.data_ptr(), pb.K, rho_k.data_ptr(), rho_t.data_ptr(), dl.data_ptr(),
                                           grad_f.data_ptr(), pb.M, grad_k.data_ptr(), pb.ws_ptr, pb.ws_bytes,
                                           _stream(None)), "sncc_diff_backward")
            return grad_f, grad_k, None

    return SegmentedNCCLoss


class _LazyFn:
    fn = None

    @classmethod
    def apply(cls, *a):
        if cls.fn is None:
            cls.fn = _make_autograd()
        return cls.fn.apply(*a)


_SegmentedNCCLoss = _LazyFn


def refit_segment_values(pb: DiffProblem, f, k0, steps: int = 100, lr: float = 0.5):
    """Refits the segment values at a fixed segmentation so that segmented NCC
    tracks exact NCC (Adam on L); returns (k, losses)."""
    torch = _torch()
    k = torch.nn.Parameter(torch.as_tensor(np.asarray(k0, np.float32)).to(f.device).clone())
    opt = torch.optim.Adam([k], lr=lr)
    losses = []
    for _ in range(steps):
        opt.zero_grad()
        loss = pb.loss(f, k)
        loss.backward()
        opt.step()
        losses.append(float(loss.item()))
    return k.detach(), losses
