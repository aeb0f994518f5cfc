"""Python binding of the C ABI in include/omni.h (argument marshalling only).

Every step of the correlator runs in the CUDA library
paper_0909_0001_gb300/lib/libomni.so; this module only converts torch tensors
and numpy arrays to pointers and sizes.  There is no CPU fallback: if the
library is missing, loading fails with an error.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence, Tuple

import numpy as np
import torch

from .synth import Level

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "lib", "libomni.so")

OMNI_OK = 0
STATUS_NAMES = {0: "OMNI_OK", 1: "OMNI_ERR_INVALID_ARG", 2: "OMNI_ERR_COLLISION",
                3: "OMNI_ERR_UNSUPPORTED", 4: "OMNI_ERR_OOM", 5: "OMNI_ERR_CUDA",
                6: "OMNI_ERR_TIMEOUT"}
DTYPES = {"cf32": 0, "ci8": 1}
PRECISIONS = {"fp32": 0, "mixed": 1, "mixed_bf16": 2}

# every entry point include/omni.h declares
EXPORTS = (
    "omni_lattice_shape", "omni_baselines", "omni_plan_create", "omni_plan_destroy",
    "omni_plan_info", "omni_correlate", "omni_correlate_host", "omni_visibilities",
    "omni_visibilities_host", "omni_reset", "omni_sync", "omni_last_error",
    "omni_status_string", "omni_profile_enable", "omni_profile_read", "omni_correlate_noalloc",
    "omni_plan_create_batch", "omni_batch_info", "omni_radial_bins", "omni_unique_baselines",
    "omni_sum_groups", "omni_plan_create_beams", "omni_plan_create_tiles",
    "omni_fengine_scratch_bytes", "omni_fengine", "omni_plan_create_tuned", "omni_plan_knobs",
)


class OmniError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class omni_level(ctypes.Structure):
    _fields_ = [("n1", ctypes.c_int32), ("n2", ctypes.c_int32), ("A", ctypes.c_double * 4)]


class omni_kernel_stat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 64), ("launches", ctypes.c_int64),
                ("total_ms", ctypes.c_double), ("bytes", ctypes.c_double),
                ("flops", ctypes.c_double), ("tensor", ctypes.c_int32)]


_lib: Optional[ctypes.CDLL] = None


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise OSError(f"{path} not found: build it with paper_0909_0001_gb300.build.build()")
    L = ctypes.CDLL(path)
    vp, i64, i32, dbl = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_double
    P = ctypes.POINTER
    lv = P(omni_level)
    sig = {
        "omni_lattice_shape": (ctypes.c_int, [lv, ctypes.c_int, P(i64), P(i64)]),
        "omni_baselines": (ctypes.c_int, [lv, ctypes.c_int, P(i32), P(i64), P(dbl)]),
        "omni_plan_create": (ctypes.c_int, [lv, ctypes.c_int, i64, ctypes.c_int, ctypes.c_int,
                                            P(vp)]),
        "omni_plan_create_beams": (ctypes.c_int, [lv, ctypes.c_int, i64, ctypes.c_int, P(vp)]),
        "omni_plan_create_tiles": (ctypes.c_int, [lv, i64, P(dbl), i64, ctypes.c_int, ctypes.c_int, P(vp)]),
        "omni_fengine_scratch_bytes": (i64, [i64, i64, i32, i32]),
        "omni_plan_create_tuned": (ctypes.c_int, [lv, ctypes.c_int, i64, ctypes.c_int, ctypes.c_int, vp,
                                                  i64, ctypes.c_char_p, P(ctypes.c_int), P(vp)]),
        "omni_plan_knobs": (ctypes.c_int, [vp, P(i64), P(ctypes.c_int), P(ctypes.c_int), P(dbl)]),
        "omni_fengine": (ctypes.c_int, [vp, i64, i64, i32, i32, vp, vp, ctypes.c_float, ctypes.c_int,
                                        vp, vp, i64, P(i64), vp]),
        "omni_plan_destroy": (None, [vp]),
        "omni_plan_info": (ctypes.c_int, [vp, P(ctypes.c_int), P(i32), P(i32), P(i64), P(i64),
                                          P(i64)]),
        "omni_correlate": (ctypes.c_int, [vp, vp, i64, vp]),
        "omni_correlate_host": (ctypes.c_int, [vp, vp, i64, vp]),
        "omni_visibilities": (ctypes.c_int, [vp, vp, ctypes.c_int, vp]),
        "omni_visibilities_host": (ctypes.c_int, [vp, vp, ctypes.c_int, vp]),
        "omni_reset": (ctypes.c_int, [vp, vp]),
        "omni_sync": (ctypes.c_int, [vp, vp]),
        "omni_last_error": (ctypes.c_char_p, []),
        "omni_status_string": (ctypes.c_char_p, [ctypes.c_int]),
        "omni_profile_enable": (ctypes.c_int, [vp, ctypes.c_int]),
        "omni_plan_create_batch": (ctypes.c_int, [P(lv), P(ctypes.c_int), ctypes.c_int, i64,
                                                  ctypes.c_int, ctypes.c_int, P(vp)]),
        "omni_batch_info": (ctypes.c_int, [vp, P(ctypes.c_int), P(i64), P(i64)]),
        "omni_radial_bins": (ctypes.c_int, [lv, ctypes.c_int, dbl, i64, P(i32), P(i64)]),
        "omni_unique_baselines": (ctypes.c_int, [lv, ctypes.c_int, P(i64), P(i32), P(dbl), P(i64)]),
        "omni_sum_groups": (ctypes.c_int, [vp, i64, i64, vp, i64, vp, vp]),
        "omni_correlate_noalloc": (ctypes.c_int, [lv, ctypes.c_int, i64, ctypes.c_int, vp, i64,
                                                  vp, vp]),
        "omni_profile_read": (ctypes.c_int, [vp, P(omni_kernel_stat), ctypes.c_int,
                                             P(ctypes.c_int), ctypes.c_int]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def _check(status: int) -> None:
    if status != OMNI_OK:
        raise OmniError(status, load().omni_last_error().decode())


def _levels(levels: Sequence[Level]):
    arr = (omni_level * len(levels))()
    for k, lv in enumerate(levels):
        arr[k].n1, arr[k].n2 = int(lv.n1), int(lv.n2)
        for c in range(4):
            arr[k].A[c] = float(lv.A[c])
    return arr


def lattice_shape(levels: Sequence[Level]) -> Tuple[int, int]:
    """(n_antennas, n_lags) of a hierarchy (host only)."""
    N, Q = ctypes.c_int64(), ctypes.c_int64()
    _check(load().omni_lattice_shape(_levels(levels), len(levels), ctypes.byref(N),
                                     ctypes.byref(Q)))
    return N.value, Q.value


def baselines(levels: Sequence[Level]) -> Tuple[np.ndarray, np.ndarray, np.ndarray]:
    """(dm [Q][2n] int32, redundancy [Q] int64, dr [Q][2] float64), host only."""
    _, Q = lattice_shape(levels)
    D = 2 * len(levels)
    dm = np.zeros((Q, D), dtype=np.int32)
    red = np.zeros(Q, dtype=np.int64)
    dr = np.zeros((Q, 2), dtype=np.float64)
    _check(load().omni_baselines(
        _levels(levels), len(levels), dm.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
        red.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
        dr.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
    return dm, red, dr


def radial_bins(levels: Sequence[Level], bin_width: float, n_bins: int):
    """(bin_of_lag [Q] int32, -1 beyond the last bin; pairs_per_bin [n_bins] int64), host only."""
    _, Q = lattice_shape(levels)
    bins = np.zeros(Q, dtype=np.int32)
    pairs = np.zeros(max(n_bins, 1), dtype=np.int64)
    _check(load().omni_radial_bins(_levels(levels), len(levels), float(bin_width), int(n_bins),
                                   bins.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                   pairs.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))))
    return bins, pairs[:n_bins]


def unique_baselines(levels: Sequence[Level]):
    """(group_of_lag [Q] int32, dr_unique [G][2], pairs_unique [G] int64), host only."""
    _, Q = lattice_shape(levels)
    n = ctypes.c_int64()
    group = np.zeros(Q, dtype=np.int32)
    dr = np.zeros((Q, 2))
    pairs = np.zeros(Q, dtype=np.int64)
    _check(load().omni_unique_baselines(_levels(levels), len(levels), ctypes.byref(n),
                                        group.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                        dr.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                        pairs.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))))
    return group, dr[:n.value], pairs[:n.value]


def sum_groups(vis: torch.Tensor, groups: torch.Tensor, n_groups: int,
               out: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
    """out[c][g] = sum of vis[c][q] over q with groups[q] == g, on the GPU."""
    if vis.dtype != torch.complex128 or not vis.is_cuda or not vis.is_contiguous() or vis.dim() != 2:
        raise ValueError("vis must be a contiguous complex128 CUDA tensor [C][Q]")
    if groups.dtype != torch.int32 or not groups.is_cuda or groups.numel() != vis.shape[1]:
        raise ValueError("groups must be an int32 CUDA tensor of Q entries")
    C, Q = vis.shape
    if out is None:
        out = torch.empty((C, n_groups), dtype=torch.complex128, device=vis.device)
    _check(load().omni_sum_groups(ctypes.c_void_p(vis.data_ptr()), C, Q,
                                  ctypes.c_void_p(groups.contiguous().data_ptr()), int(n_groups),
                                  ctypes.c_void_p(out.data_ptr()), _stream_ptr(stream)))
    return out


def correlate_noalloc(levels: Sequence[Level], volts: torch.Tensor, dtype: str,
                      out: torch.Tensor, stream=None) -> torch.Tensor:
    """One integration through omni_correlate_noalloc, which allocates no device
    memory (for callers that cannot allocate; see include/omni.h).  volts:
    contiguous device [C][T][N][2] of dtype (int8 for "ci8", float32 or
    complex64 for "cf32"); out: contiguous device complex128 [C][Q] on the same
    device.  Every argument is checked here, before the library is called."""
    if dtype not in DTYPES:
        raise ValueError(f"dtype must be one of {sorted(DTYPES)}")
    want = torch.int8 if dtype == "ci8" else torch.float32
    if volts.dtype == torch.complex64 and dtype == "cf32":
        volts = torch.view_as_real(volts)
    if volts.dtype != want:
        raise TypeError(f"voltages must be {want} [C][T][N][2] for dtype {dtype}, got {volts.dtype}")
    N, Q = lattice_shape(levels)
    if volts.dim() != 4 or volts.shape[0] < 1 or volts.shape[2] != N or volts.shape[3] != 2:
        raise ValueError(f"voltages must have shape [C][T][{N}][2] with C >= 1, got {tuple(volts.shape)}")
    C, T = int(volts.shape[0]), int(volts.shape[1])
    if out.dtype != torch.complex128:
        raise TypeError("out must be complex128")
    if out.numel() != C * Q:
        raise ValueError(f"out must hold C x Q = {C} x {Q} values, got {out.numel()}")
    if not (volts.is_contiguous() and out.is_contiguous()):
        raise ValueError("volts and out must be contiguous")
    if not (volts.is_cuda and out.is_cuda):
        raise ValueError("volts and out must be CUDA tensors")
    if volts.device != out.device:
        raise ValueError("volts and out must be on the same device")
    with torch.cuda.device(volts.device):
        _check(load().omni_correlate_noalloc(_levels(levels), len(levels), C, DTYPES[dtype],
                                             ctypes.c_void_p(volts.data_ptr()), T,
                                             ctypes.c_void_p(out.data_ptr()), _stream_ptr(stream)))
    return out


def _stream_ptr(stream) -> ctypes.c_void_p:
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(int(stream.cuda_stream))


def fengine(raw: torch.Tensor, channels: int, taps: int = 1, window: Optional[torch.Tensor] = None,
            gains: Optional[torch.Tensor] = None, scale: float = 1.0, dtype: str = "ci8",
            out: Optional[torch.Tensor] = None, scratch: Optional[torch.Tensor] = None,
            stream=None) -> torch.Tensor:
    """F-engine (Appendix A step 2): channelise raw int8 samples [N][S] (device)
    into channel voltages [F][T][N][2] (int8 or float32), the layout Plan.correlate
    reads with C = F.  window: [taps * 2F] float32 (None: ones); gains: [F][N]
    complex64 (None: 1)."""
    if raw.dtype != torch.int8 or raw.dim() != 2 or not raw.is_cuda or not raw.is_contiguous():
        raise ValueError("raw must be a contiguous int8 CUDA tensor [N][S]")
    N, S = raw.shape
    L = load()
    need = L.omni_fengine_scratch_bytes(N, S, channels, taps)
    M = 2 * channels
    T = (S - (taps - 1) * M) // M if S >= (taps - 1) * M else 0   # frames, as the library counts them
    if out is None:
        out = torch.empty((channels, T, N, 2), dtype=torch.int8 if dtype == "ci8" else torch.float32,
                          device=raw.device)
    if scratch is None:
        scratch = torch.empty(max(1, need // 8), dtype=torch.float64, device=raw.device)
    wptr = None
    if window is not None:
        window = window.to(device=raw.device, dtype=torch.float32).contiguous()
        if window.numel() != taps * 2 * channels:
            raise ValueError("window must have taps * 2F values")
        wptr = ctypes.c_void_p(window.data_ptr())
    gptr = None
    if gains is not None:
        gains = torch.view_as_real(gains.to(device=raw.device, dtype=torch.complex64).contiguous())
        if gains.numel() != 2 * channels * N:
            raise ValueError("gains must be [F][N] complex")
        gptr = ctypes.c_void_p(gains.data_ptr())
    frames = ctypes.c_int64()
    _check(L.omni_fengine(ctypes.c_void_p(raw.data_ptr()), N, S, channels, taps, wptr, gptr,
                          float(scale), DTYPES[dtype], ctypes.c_void_p(out.data_ptr()),
                          ctypes.c_void_p(scratch.data_ptr()), scratch.numel() * scratch.element_size(),
                          ctypes.byref(frames), _stream_ptr(stream)))
    return out


class Plan:
    """A correlator plan for C channels of one hierarchy (owns device memory)."""

    def __init__(self, levels: Sequence[Level], channels: int, dtype: str = "cf32",
                 precision: str = "fp32"):
        self.levels = list(levels)
        self.channels = int(channels)
        self.dtype = dtype
        self.precision = precision
        h = self._create()
        self._h = h
        nd = ctypes.c_int()
        dims = (ctypes.c_int32 * 16)()
        pad = (ctypes.c_int32 * 16)()
        N, Q, C = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        _check(load().omni_plan_info(h, ctypes.byref(nd), dims, pad, ctypes.byref(N),
                                     ctypes.byref(Q), ctypes.byref(C)))
        self.dims = [dims[d] for d in range(nd.value)]
        self.padded = [pad[d] for d in range(nd.value)]
        self.n_antennas = N.value
        self.n_lags = Q.value

    def _create(self) -> ctypes.c_void_p:
        h = ctypes.c_void_p()
        tune = getattr(self, "_tune", None)
        if tune is not None:
            volts, cache = tune
            T = self._check_volts_shape(volts)
            hit = ctypes.c_int()
            _check(load().omni_plan_create_tuned(
                _levels(self.levels), len(self.levels), self.channels, DTYPES[self.dtype],
                PRECISIONS[self.precision], ctypes.c_void_p(volts.data_ptr()), T,
                None if cache is None else os.fsencode(cache), ctypes.byref(hit), ctypes.byref(h)))
            self.from_cache = bool(hit.value)
            return h
        _check(load().omni_plan_create(_levels(self.levels), len(self.levels), self.channels,
                                       DTYPES[self.dtype], PRECISIONS[self.precision],
                                       ctypes.byref(h)))
        return h

    @classmethod
    def tuned(cls, levels: Sequence[Level], channels: int, volts: torch.Tensor, dtype: str = "cf32",
              precision: str = "fp32", cache: Optional[str] = None) -> "Plan":
        """A plan whose chunking, overlap and pass structure were chosen by timing
        candidates on these device voltages [C][T][N][2] (cached in `cache`)."""
        self = cls.__new__(cls)
        self._tune = (volts, cache)
        cls.__init__(self, levels, channels, dtype=dtype, precision=precision)
        self._tune = None
        return self

    def knobs(self) -> dict:
        mb, ov, lp, sp = ctypes.c_int64(), ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
        _check(load().omni_plan_knobs(self._h, ctypes.byref(mb), ctypes.byref(ov), ctypes.byref(lp),
                                      ctypes.byref(sp)))
        return {"chunk_mb": mb.value, "overlap": bool(ov.value), "level_passes": bool(lp.value),
                "split_tc": sp.value}

    def _check_volts_shape(self, v: torch.Tensor) -> int:
        if not v.is_cuda or not v.is_contiguous() or v.dim() != 4 or v.shape[0] != self.channels:
            raise ValueError("tuning voltages must be contiguous CUDA [C][T][N][2]")
        return int(v.shape[1])

    # ---------------------------------------------------------------- checks
    def _check_volts(self, v: torch.Tensor) -> int:
        want = torch.int8 if self.dtype == "ci8" else torch.float32
        if v.dtype == torch.complex64 and self.dtype == "cf32":
            v = torch.view_as_real(v)
        if v.dtype != want:
            raise TypeError(f"voltages must be {want} [C][T][N][2] for dtype {self.dtype}")
        if v.dim() != 4 or v.shape[0] != self.channels or v.shape[2] != self.n_antennas \
                or v.shape[3] != 2:
            raise ValueError(f"voltages must have shape [{self.channels}][T][{self.n_antennas}][2],"
                             f" got {tuple(v.shape)}")
        if not v.is_contiguous():
            raise ValueError("voltages must be contiguous")
        return int(v.shape[1])

    # ---------------------------------------------------------------- calls
    def correlate(self, volts: torch.Tensor, stream=None) -> None:
        """Accumulate |F|^2 of device voltages [C][T][N][2] (async on stream)."""
        if not volts.is_cuda:
            raise ValueError("correlate() takes device voltages; use correlate_host()")
        T = self._check_volts(volts)
        _check(load().omni_correlate(self._h, ctypes.c_void_p(volts.data_ptr()), T,
                                     _stream_ptr(stream)))

    def correlate_host(self, volts: torch.Tensor, stream=None) -> None:
        """Accumulate host voltages (copied in chunks, overlapped with the transforms)."""
        if volts.is_cuda:
            raise ValueError("correlate_host() takes host voltages")
        T = self._check_volts(volts)
        _check(load().omni_correlate_host(self._h, ctypes.c_void_p(volts.data_ptr()), T,
                                          _stream_ptr(stream)))

    def visibilities(self, reset: bool = True, out: Optional[torch.Tensor] = None,
                     stream=None) -> torch.Tensor:
        """Visibilities [C][Q] complex128 on the device."""
        if out is None:
            out = torch.empty((self.channels, self.n_lags), dtype=torch.complex128, device="cuda")
        if out.dtype != torch.complex128 or not out.is_cuda or not out.is_contiguous() \
                or out.numel() != self.channels * self.n_lags:
            raise ValueError("out must be a contiguous complex128 CUDA tensor of C*Q elements")
        _check(load().omni_visibilities(self._h, ctypes.c_void_p(out.data_ptr()), int(reset),
                                        _stream_ptr(stream)))
        return out

    def visibilities_host(self, reset: bool = True, out: Optional[torch.Tensor] = None,
                          stream=None) -> torch.Tensor:
        """Visibilities [C][Q] complex128 copied into host memory."""
        if out is None:
            out = torch.empty((self.channels, self.n_lags), dtype=torch.complex128)
        if out.dtype != torch.complex128 or out.is_cuda or not out.is_contiguous() \
                or out.numel() != self.channels * self.n_lags:
            raise ValueError("out must be a contiguous complex128 host tensor of C*Q elements")
        _check(load().omni_visibilities_host(self._h, ctypes.c_void_p(out.data_ptr()),
                                             int(reset), _stream_ptr(stream)))
        return out

    def profile(self, enable: bool = True) -> None:
        """Record CUDA events around every kernel launch (per-pass timings)."""
        _check(load().omni_profile_enable(self._h, int(enable)))

    def kernel_stats(self, clear: bool = False) -> list:
        """Per-pass [{name, launches, total_ms, bytes, flops, tensor}] (waits for recorded events)."""
        n = ctypes.c_int()
        _check(load().omni_profile_read(self._h, None, 0, ctypes.byref(n), 0))
        arr = (omni_kernel_stat * max(1, n.value))()
        _check(load().omni_profile_read(self._h, arr, n.value, ctypes.byref(n), int(clear)))
        return [{"name": arr[i].name.decode(), "launches": arr[i].launches,
                 "total_ms": arr[i].total_ms, "bytes": arr[i].bytes, "flops": arr[i].flops,
                 "tensor": bool(arr[i].tensor)} for i in range(n.value)]

    def reset(self, stream=None) -> None:
        _check(load().omni_reset(self._h, _stream_ptr(stream)))

    def sync(self, stream=None) -> None:
        _check(load().omni_sync(self._h, _stream_ptr(stream)))

    def close(self) -> None:
        if getattr(self, "_h", None) is not None and self._h.value:
            load().omni_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class BeamPlan(Plan):
    """Beam-space correlator (Appendix A, steps 4-5): every level-1 block is
    Fourier transformed unpadded into n1 x n2 digital pointings, and each
    pointing is correlated over the axes of levels 2..n.  visibilities()
    returns [C][Q' * n1 * n2] complex128, the pointing index fastest; split()
    views it as [C][Q'][k_b][k_a], with the Q' lags of baselines(levels[1:])."""

    def __init__(self, levels: Sequence[Level], channels: int, dtype: str = "cf32"):
        super().__init__(levels, channels, dtype=dtype, precision="fp32")
        self.beam_shape = (int(self.levels[0].n1), int(self.levels[0].n2))
        self.n_beams = self.beam_shape[0] * self.beam_shape[1]
        self.n_coarse_lags = self.n_lags // self.n_beams

    def _create(self) -> ctypes.c_void_p:
        h = ctypes.c_void_p()
        _check(load().omni_plan_create_beams(_levels(self.levels), len(self.levels),
                                             self.channels, DTYPES[self.dtype], ctypes.byref(h)))
        return h

    def split(self, V: torch.Tensor) -> torch.Tensor:
        return V.reshape(self.channels, self.n_coarse_lags, self.beam_shape[1], self.beam_shape[0])


class TilePlan(Plan):
    """Tile hybrid (Sec. III): identical one-level tiles at arbitrary offsets,
    FFT-correlated within each tile and pairwise between tiles.  visibilities()
    returns [C][n_tiles * n_tiles * Q] complex128; split() views it as
    [C][i][j][Q] (lags of baselines([tile]) order)."""

    def __init__(self, tile: Level, offsets, channels: int, dtype: str = "cf32",
                 precision: str = "fp32"):
        self.offsets = np.ascontiguousarray(np.asarray(offsets, dtype=np.float64).reshape(-1, 2))
        self.n_tiles = int(self.offsets.shape[0])
        super().__init__([tile], channels, dtype=dtype, precision=precision)
        self.n_tile_lags = self.n_lags // (self.n_tiles * self.n_tiles)

    def _create(self) -> ctypes.c_void_p:
        h = ctypes.c_void_p()
        off = self.offsets.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        _check(load().omni_plan_create_tiles(_levels(self.levels), self.n_tiles, off,
                                             self.channels, DTYPES[self.dtype],
                                             PRECISIONS[self.precision], ctypes.byref(h)))
        return h

    def split(self, V: torch.Tensor) -> torch.Tensor:
        return V.reshape(self.channels, self.n_tiles, self.n_tiles, self.n_tile_lags)

    def baseline_vectors(self) -> np.ndarray:
        """Physical baseline o_i - o_j + A D of every output, [n_tiles][n_tiles][Q][2]."""
        _, _, dr = baselines(self.levels)
        o = self.offsets
        return (o[:, None, None, :] - o[None, :, None, :]) + dr[None, None, :, :]


class BatchPlan(Plan):
    """Several independent arrays (possibly of different hierarchies), C channels each.

    Voltages are passed as one flat tensor holding the arrays' [C][T][N_a][2]
    blocks one after another (see pack()); visibilities come back as one flat
    complex128 tensor of the arrays' [C][Q_a] blocks (see unpack())."""

    def __init__(self, arrays: Sequence[Sequence[Level]], channels: int, dtype: str = "cf32",
                 precision: str = "fp32"):
        self.arrays = [list(a) for a in arrays]
        self.channels = int(channels)
        self.dtype = dtype
        self.precision = precision
        n = len(self.arrays)
        keep = [_levels(a) for a in self.arrays]
        ptrs = (ctypes.POINTER(omni_level) * n)(*[ctypes.cast(k, ctypes.POINTER(omni_level))
                                                   for k in keep])
        nl = (ctypes.c_int * n)(*[len(a) for a in self.arrays])
        h = ctypes.c_void_p()
        _check(load().omni_plan_create_batch(ptrs, nl, n, self.channels, DTYPES[dtype],
                                             PRECISIONS[precision], ctypes.byref(h)))
        self._h = h
        na = ctypes.c_int()
        N = (ctypes.c_int64 * n)()
        Q = (ctypes.c_int64 * n)()
        _check(load().omni_batch_info(h, ctypes.byref(na), N, Q))
        self.antennas = list(N)
        self.lags = list(Q)
        self.n_antennas = sum(self.antennas)
        self.n_lags = sum(self.lags)

    def pack(self, volts: Sequence[torch.Tensor]) -> torch.Tensor:
        """Concatenate per-array voltages [C][T][N_a][2] into the flat batch layout."""
        if len(volts) != len(self.arrays):
            raise ValueError("one voltage tensor per array")
        T = int(volts[0].shape[1])
        for v, N in zip(volts, self.antennas):
            if tuple(v.shape) != (self.channels, T, N, 2):
                raise ValueError(f"expected [{self.channels}][{T}][{N}][2], got {tuple(v.shape)}")
        return torch.cat([v.reshape(-1) for v in volts])

    def samples_of(self, flat: torch.Tensor) -> int:
        per = self.channels * self.n_antennas * 2
        if flat.dim() != 1 or flat.numel() % per:
            raise ValueError("flat batch voltages must be 1-D with C * T * sum(N_a) * 2 values")
        return flat.numel() // per

    def unpack(self, vis: torch.Tensor) -> list:
        """Split flat visibilities into per-array [C][Q_a] views."""
        out, off = [], 0
        for Q in self.lags:
            out.append(vis[off:off + self.channels * Q].view(self.channels, Q))
            off += self.channels * Q
        return out

    def _flat(self, volts: torch.Tensor) -> int:
        want = torch.int8 if self.dtype == "ci8" else torch.float32
        if volts.dtype != want or not volts.is_contiguous():
            raise TypeError(f"flat batch voltages must be contiguous {want}")
        return self.samples_of(volts)

    def correlate(self, volts: torch.Tensor, stream=None) -> None:
        if not volts.is_cuda:
            raise ValueError("correlate() takes device voltages; use correlate_host()")
        T = self._flat(volts)
        _check(load().omni_correlate(self._h, ctypes.c_void_p(volts.data_ptr()), T,
                                     _stream_ptr(stream)))

    def correlate_host(self, volts: torch.Tensor, stream=None) -> None:
        if volts.is_cuda:
            raise ValueError("correlate_host() takes host voltages")
        T = self._flat(volts)
        _check(load().omni_correlate_host(self._h, ctypes.c_void_p(volts.data_ptr()), T,
                                          _stream_ptr(stream)))

    def visibilities(self, reset: bool = True, out: Optional[torch.Tensor] = None,
                     stream=None) -> torch.Tensor:
        if out is None:
            out = torch.empty(self.channels * self.n_lags, dtype=torch.complex128, device="cuda")
        if out.dtype != torch.complex128 or not out.is_cuda or not out.is_contiguous() \
                or out.numel() != self.channels * self.n_lags:
            raise ValueError("out must be a contiguous complex128 CUDA tensor of C*sum(Q_a)")
        _check(load().omni_visibilities(self._h, ctypes.c_void_p(out.data_ptr()), int(reset),
                                        _stream_ptr(stream)))
        return out

    def visibilities_host(self, reset: bool = True, out: Optional[torch.Tensor] = None,
                          stream=None) -> torch.Tensor:
        if out is None:
            out = torch.empty(self.channels * self.n_lags, dtype=torch.complex128)
        if out.dtype != torch.complex128 or out.is_cuda or not out.is_contiguous() \
                or out.numel() != self.channels * self.n_lags:
            raise ValueError("out must be a contiguous complex128 host tensor of C*sum(Q_a)")
        _check(load().omni_visibilities_host(self._h, ctypes.c_void_p(out.data_ptr()),
                                             int(reset), _stream_ptr(stream)))
        return out
