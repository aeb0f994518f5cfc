"""Python entry points of the CPU FP64 oracle (a ctypes wrapper over omni_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by tests/, by __graft_entry__.smoke() and by
bench.py's CPU-baseline leg, never by the product package.

What the oracle computes is the plain brute-force definition of the summed
visibilities (Eq. ConvolutionDefEq, Sec. II.C; Eq. ProofEq2, Sec. II.D):
V_c(D) = sum_t sum_m x_{c,t}(m+D) conj(x_{c,t}(m)), plus the lag table with
its redundancy counts (Sec. III), the geometry of Eq. GridEq, and the
beam-space variant of Appendix A (steps 4-5: direct DFT of each level-1
block into pointings, brute-force correlation over the coarser levels) and the
tile hybrid of Sec. III (brute-force correlation of every ordered tile pair at
every intra-tile offset), and the F-engine of Appendix A step 2 (polyphase
frames, direct DFT, gains, round-half-even int8 quantiser).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from typing import Sequence, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "omni_oracle.c")
_LIBDIR = os.path.join(_HERE, "lib")
_LIB = os.path.join(_LIBDIR, "libomni_oracle.so")

DTYPE_CODE = {"cf64": 0, "cf32": 1, "ci8": 2}

_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, OpenMP) into oracle/lib/."""
    os.makedirs(_LIBDIR, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        i32p = ctypes.POINTER(ctypes.c_int32)
        i64p = ctypes.POINTER(ctypes.c_int64)
        f64p = ctypes.POINTER(ctypes.c_double)
        L.oracle_n_antennas.restype = ctypes.c_int64
        L.oracle_n_antennas.argtypes = [ctypes.c_int, i32p]
        L.oracle_n_lags.restype = ctypes.c_int64
        L.oracle_n_lags.argtypes = [ctypes.c_int, i32p]
        L.oracle_lag_table.restype = None
        L.oracle_lag_table.argtypes = [ctypes.c_int, i32p, i32p, i64p]
        L.oracle_positions.restype = None
        L.oracle_positions.argtypes = [ctypes.c_int, i32p, f64p, f64p]
        L.oracle_baseline_vectors.restype = None
        L.oracle_baseline_vectors.argtypes = [ctypes.c_int, f64p, ctypes.c_int64, i32p, f64p]
        L.oracle_collides.restype = ctypes.c_int
        L.oracle_collides.argtypes = [ctypes.c_int64, f64p, ctypes.c_double]
        L.oracle_correlate.restype = None
        L.oracle_correlate.argtypes = [ctypes.c_int, i32p, ctypes.c_int64, ctypes.c_int64,
                                       ctypes.c_int, ctypes.c_void_p, f64p]
        L.oracle_correlate_selected.restype = None
        L.oracle_correlate_selected.argtypes = [ctypes.c_int, i32p, ctypes.c_int64,
                                                ctypes.c_int64, ctypes.c_int, ctypes.c_void_p,
                                                ctypes.c_int64, i64p, i64p, f64p]
        L.oracle_beam_correlate.restype = None
        L.oracle_beam_correlate.argtypes = [ctypes.c_int, i32p, ctypes.c_int64, ctypes.c_int64,
                                            ctypes.c_int, ctypes.c_void_p, f64p]
        L.oracle_tile_correlate.restype = None
        L.oracle_tile_correlate.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int64,
                                            ctypes.c_int64, ctypes.c_int, ctypes.c_void_p, f64p]
        L.oracle_fengine.restype = None
        L.oracle_fengine.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, ctypes.c_int,
                                     ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double,
                                     f64p]
        L.oracle_quantize.restype = None
        L.oracle_quantize.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p]
        L.oracle_max_dims.restype = ctypes.c_int
        _lib = L
    return _lib


def _i32(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.int32))


def _ptr(a: np.ndarray, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


def n_lags(dims: Sequence[int]) -> int:
    d = _i32(dims)
    return int(lib().oracle_n_lags(len(d), _ptr(d, ctypes.c_int32)))


def lag_table(dims: Sequence[int]) -> Tuple[np.ndarray, np.ndarray]:
    """(dm [Q][D] int32, redundancy [Q] int64), dimension 0 fastest."""
    d = _i32(dims)
    Q = n_lags(d)
    dm = np.zeros((Q, len(d)), dtype=np.int32)
    red = np.zeros(Q, dtype=np.int64)
    lib().oracle_lag_table(len(d), _ptr(d, ctypes.c_int32), _ptr(dm, ctypes.c_int32),
                           _ptr(red, ctypes.c_int64))
    return dm, red


def _level_arrays(levels) -> Tuple[np.ndarray, np.ndarray]:
    shape = _i32([v for lv in levels for v in (lv.n1, lv.n2)])
    A = np.ascontiguousarray(np.array([lv.A for lv in levels], dtype=np.float64).ravel())
    return shape, A


def positions(levels) -> np.ndarray:
    shape, A = _level_arrays(levels)
    N = int(np.prod(shape))
    r = np.zeros((N, 2))
    lib().oracle_positions(len(levels), _ptr(shape, ctypes.c_int32), _ptr(A, ctypes.c_double),
                           _ptr(r, ctypes.c_double))
    return r


def baseline_vectors(levels, dm: np.ndarray) -> np.ndarray:
    _, A = _level_arrays(levels)
    dm = np.ascontiguousarray(dm, dtype=np.int32)
    dr = np.zeros((dm.shape[0], 2))
    lib().oracle_baseline_vectors(len(levels), _ptr(A, ctypes.c_double), dm.shape[0],
                                  _ptr(dm, ctypes.c_int32), _ptr(dr, ctypes.c_double))
    return dr


def collides(levels, tol_rel: float = 1e-9) -> bool:
    r = np.ascontiguousarray(positions(levels))
    return bool(lib().oracle_collides(r.shape[0], _ptr(r, ctypes.c_double), tol_rel))


def _as_input(x) -> Tuple[np.ndarray, int]:
    """Accept a [C][T][N][2] array (float64/float32/int8) or complex [C][T][N]."""
    a = x.numpy() if hasattr(x, "numpy") else np.asarray(x)
    if np.iscomplexobj(a):
        a = np.stack([a.real, a.imag], axis=-1).astype(np.float64)
    a = np.ascontiguousarray(a)
    if a.dtype == np.float64:
        return a, 0
    if a.dtype == np.float32:
        return a, 1
    if a.dtype == np.int8:
        return a, 2
    raise TypeError(f"unsupported voltage dtype {a.dtype}")


def correlate(dims: Sequence[int], x) -> np.ndarray:
    """Brute-force visibilities, complex128 [C][Q] (lags dimension-0 fastest)."""
    d = _i32(dims)
    a, code = _as_input(x)
    C, T, N = a.shape[0], a.shape[1], a.shape[2]
    if N != int(np.prod(d)):
        raise ValueError("voltage length does not match the lattice")
    Q = n_lags(d)
    V = np.zeros((C, Q, 2))
    lib().oracle_correlate(len(d), _ptr(d, ctypes.c_int32), C, T, code,
                           a.ctypes.data_as(ctypes.c_void_p), _ptr(V, ctypes.c_double))
    return V[..., 0] + 1j * V[..., 1]


def correlate_selected(dims: Sequence[int], x, chans, lag_idx) -> np.ndarray:
    """Brute-force visibilities at selected (channel, lag index) pairs, complex128 [S]."""
    d = _i32(dims)
    a, code = _as_input(x)
    C, T = a.shape[0], a.shape[1]
    ch = np.ascontiguousarray(np.asarray(chans, dtype=np.int64))
    lq = np.ascontiguousarray(np.asarray(lag_idx, dtype=np.int64))
    V = np.zeros((len(ch), 2))
    lib().oracle_correlate_selected(len(d), _ptr(d, ctypes.c_int32), C, T, code,
                                    a.ctypes.data_as(ctypes.c_void_p), len(ch),
                                    _ptr(ch, ctypes.c_int64), _ptr(lq, ctypes.c_int64),
                                    _ptr(V, ctypes.c_double))
    return V[:, 0] + 1j * V[:, 1]


def beam_correlate(dims: Sequence[int], x) -> np.ndarray:
    """Beam-space visibilities (Appendix A steps 4-5), complex128 [C][Q'][n1*n2]:
    an unpadded direct DFT of every level-1 block (dims[0], dims[1]) into
    pointings, then the brute-force correlation of each pointing over the
    remaining dimensions (lags in lag_table(dims[2:]) order, pointing fastest)."""
    d = _i32(dims)
    if len(d) < 3:
        raise ValueError("the beam-space variant needs a coarser level")
    a, code = _as_input(x)
    C, T, N = a.shape[0], a.shape[1], a.shape[2]
    if N != int(np.prod(d)):
        raise ValueError("voltage length does not match the lattice")
    Qc = n_lags(d[2:])
    nb = int(d[0]) * int(d[1])
    B = np.zeros((C, Qc, nb, 2))
    lib().oracle_beam_correlate(len(d), _ptr(d, ctypes.c_int32), C, T, code,
                                a.ctypes.data_as(ctypes.c_void_p), _ptr(B, ctypes.c_double))
    return B[..., 0] + 1j * B[..., 1]


def tile_correlate(n1: int, n2: int, n_tiles: int, x) -> np.ndarray:
    """Tile-hybrid visibilities, complex128 [C][n_tiles][n_tiles][Q]: for each
    ordered tile pair (i, j) the brute-force sum of x_i(m + D) conj(x_j(m)) over
    the pairs of antennas with intra-tile offset D (lags dimension 0 fastest)."""
    a, code = _as_input(x)
    C, T, N = a.shape[0], a.shape[1], a.shape[2]
    if N != n1 * n2 * n_tiles:
        raise ValueError("voltage length does not match the tiles")
    Q = (2 * n1 - 1) * (2 * n2 - 1)
    V = np.zeros((C, n_tiles, n_tiles, Q, 2))
    lib().oracle_tile_correlate(n1, n2, n_tiles, C, T, code, a.ctypes.data_as(ctypes.c_void_p),
                                _ptr(V, ctypes.c_double))
    return V[..., 0] + 1j * V[..., 1]


def fengine(raw, F: int, P: int = 1, window=None, gains=None, scale: float = 1.0) -> np.ndarray:
    """F-engine channel voltages (Appendix A step 2) as complex128 [F][T][N]:
    polyphase sum of P frames of 2F samples, direct DFT, Nyquist bin dropped,
    times scale and the per-(channel, antenna) complex gain."""
    r = np.ascontiguousarray(np.asarray(raw.numpy() if hasattr(raw, "numpy") else raw, dtype=np.int8))
    N, S = r.shape
    M = 2 * F
    T = (S - (P - 1) * M) // M if S >= (P - 1) * M else 0
    w = None if window is None else np.ascontiguousarray(np.asarray(window, dtype=np.float64))
    g = None
    if gains is not None:
        gc = np.asarray(gains, dtype=np.complex128).reshape(F, N)
        g = np.ascontiguousarray(np.stack([gc.real, gc.imag], axis=-1))
    out = np.zeros((F, T, N, 2))
    lib().oracle_fengine(r.ctypes.data_as(ctypes.c_void_p), N, S, F, P,
                         None if w is None else w.ctypes.data_as(ctypes.c_void_p),
                         None if g is None else g.ctypes.data_as(ctypes.c_void_p), scale,
                         _ptr(out, ctypes.c_double))
    return out[..., 0] + 1j * out[..., 1]


def quantize(x) -> np.ndarray:
    """int8 codes of float32 values: round half to even, clip to [-127, 127]."""
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    q = np.zeros(a.shape, dtype=np.int8)
    lib().oracle_quantize(a.ctypes.data_as(ctypes.c_void_p), a.size, q.ctypes.data_as(ctypes.c_void_p))
    return q


# ---------------------------------------------------------------- physical baselines

def radial_bins(levels, bin_width: float, n_bins: int):
    """Radial bin of every lag, floor(|dr| / bin_width) (or -1 beyond n_bins), and
    the antenna pairs per bin: the radially binned baseline distribution of Sec. III."""
    dims = [v for lv in levels for v in (lv.n1, lv.n2)]
    dm, red = lag_table(dims)
    dr = baseline_vectors(levels, dm)
    b = np.floor(np.hypot(dr[:, 0], dr[:, 1]) / bin_width)
    b = np.where(b < n_bins, b, -1).astype(np.int64)
    pairs = np.zeros(n_bins, dtype=np.int64)
    for q in range(len(b)):
        if b[q] >= 0:
            pairs[b[q]] += red[q]
    return b.astype(np.int32), pairs


def unique_baselines(levels, tol_rel: float = 1e-9):
    """Lags grouped by coincident physical baseline (plain loop over existing groups)."""
    dims = [v for lv in levels for v in (lv.n1, lv.n2)]
    dm, red = lag_table(dims)
    dr = baseline_vectors(levels, dm)
    tol = tol_rel * float(np.max(np.hypot(dr[:, 0], dr[:, 1])))
    reps, pairs, group = [], [], np.zeros(len(dr), dtype=np.int32)
    for q in range(len(dr)):
        for g, r in enumerate(reps):
            if np.hypot(dr[q, 0] - r[0], dr[q, 1] - r[1]) <= tol:
                group[q] = g
                pairs[g] += red[q]
                break
        else:
            group[q] = len(reps)
            reps.append(dr[q])
            pairs.append(int(red[q]))
    return group, np.array(reps), np.array(pairs, dtype=np.int64)


def group_sum(V: np.ndarray, group: np.ndarray, n_groups: int) -> np.ndarray:
    """out[c][g] = sum of V[c][q] over q with group[q] == g (FP64)."""
    out = np.zeros((V.shape[0], n_groups), dtype=np.complex128)
    for q in range(V.shape[1]):
        if 0 <= group[q] < n_groups:
            out[:, group[q]] += V[:, q]
    return out
