"""Pins for the CPU FP64 oracle, each tied to something other than the oracle.

Every check here runs on the CPU.  The oracle is the brute-force definition of
the summed visibilities (Eq. ConvolutionDefEq / ProofEq2); these tests hold it
to the values the paper prints, to closed forms, to invariants, and to two
independent routes (a naive O(L^2) DFT and numpy.fft) that reach the same
numbers through the zero-padded FFT / square / inverse-FFT procedure of
Sec. II.C.
"""
import itertools
import math

import numpy as np
import pytest

from conftest import read_golden
from oracle import oracle
from paper_0909_0001_gb300 import synth


def _cplx(x):
    x = np.asarray(x, dtype=np.float64)
    return x[..., 0] + 1j * x[..., 1]


def _lags_per_dim(dims):
    return [np.arange(-(n - 1), n) for n in dims]


def _lag_vectors(dims):
    """All lag vectors, dimension 0 fastest (written independently of the oracle)."""
    rev = list(itertools.product(*[range(-(n - 1), n) for n in dims[::-1]]))
    return np.array([v[::-1] for v in rev], dtype=np.int64)


def fft_route(dims, x):
    """Sec. II.C: zero-pad to 2n_d, FFT, |.|^2, sum over t, inverse FFT, gather lags."""
    x = _cplx(x) if not np.iscomplexobj(x) else x
    C, T, N = x.shape
    shape_rev = tuple(dims[::-1])                    # numpy axis order: slowest first
    pad = tuple(2 * n if n > 1 else 1 for n in shape_rev)
    out = []
    for c in range(C):
        P = np.zeros(pad)
        for t in range(T):
            F = np.fft.fftn(x[c, t].reshape(shape_rev), s=pad, axes=tuple(range(len(pad))))
            P += np.abs(F) ** 2
        g = np.fft.ifftn(P)
        idx = np.ix_(*[np.arange(-(n - 1), n) % L for n, L in zip(shape_rev, pad)])
        out.append(g[idx].ravel())
    return np.array(out)


def naive_dft_route(dims, x):
    """The same route with the multidimensional DFT written as an explicit O(L^2) sum."""
    x = _cplx(x)
    C, T, N = x.shape
    Ls = [2 * n if n > 1 else 1 for n in dims]
    L = int(np.prod(Ls))
    # flattened lattice coordinates, dimension 0 fastest
    kk = np.array(list(itertools.product(*[range(l) for l in Ls[::-1]])))[:, ::-1]
    mm = np.array(list(itertools.product(*[range(n) for n in dims[::-1]])))[:, ::-1]
    phase = np.zeros((L, N))
    for d, Ld in enumerate(Ls):
        phase += np.outer(kk[:, d], mm[:, d]) / Ld
    W = np.exp(-2j * math.pi * phase)                 # forward DFT, e^{-}
    lags = _lag_vectors(dims)
    phase_inv = np.zeros((len(lags), L))
    for d, Ld in enumerate(Ls):
        phase_inv += np.outer(lags[:, d], kk[:, d]) / Ld
    Winv = np.exp(2j * math.pi * phase_inv) / L        # inverse DFT, e^{+}, 1/L
    out = []
    for c in range(C):
        P = np.zeros(L)
        for t in range(T):
            P += np.abs(W @ x[c, t]) ** 2
        out.append(Winv @ P)
    return np.array(out)


def relerr(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


# ---------------------------------------------------------------- paper values

def test_warmup_example_1d():
    g = read_golden("warmup_example.txt")
    f = g["voltages"][0]
    x = np.zeros((1, 1, 9, 2))
    x[0, 0, [0, 1, 2, 6, 7, 8], 0] = f                 # x = 1,2,3,7,8,9
    V = oracle.correlate([9, 1], x)
    np.testing.assert_array_equal(V.real[0], g["g_1d"][0])
    np.testing.assert_array_equal(V.imag[0], 0.0)


def test_warmup_example_two_level():
    g = read_golden("warmup_example.txt")
    x = np.zeros((1, 1, 6, 2))
    x[0, 0, :, 0] = g["voltages"][0]
    dims = synth.lattice_dims(synth.paper_fixture("warmup_2level"))
    assert dims == [3, 1, 2, 1]
    V = oracle.correlate(dims, x)[0]
    np.testing.assert_array_equal(V.real.reshape(3, 5), np.array(g["G_2d_row"]))
    # Mapping the 2-D lag (D1, D2) to the physical separation D1 + 6 D2 gives
    # back the 17-long 1-D result (zeros at the separations no pair has).
    dm, _ = oracle.lag_table(dims)
    g1 = np.zeros(17)
    for q in range(len(V)):
        g1[dm[q, 0] + 6 * dm[q, 2] + 8] += V[q].real
    np.testing.assert_array_equal(g1, g["g_1d"][0])


# ---------------------------------------------------------------- closed forms

@pytest.mark.parametrize("dims", [[4, 1], [3, 5], [4, 3, 2, 3], [2, 3, 1, 2, 3, 2]])
def test_all_ones_gives_redundancy(dims):
    T = 3
    x = synth.all_ones(dims, 1, T)
    V = oracle.correlate(dims, x)[0]
    lags = _lag_vectors(dims)
    expect = T * np.prod([n - np.abs(lags[:, d]) for d, n in enumerate(dims)], axis=0)
    np.testing.assert_array_equal(V.real, expect)
    np.testing.assert_array_equal(V.imag, 0.0)
    dm, red = oracle.lag_table(dims)
    np.testing.assert_array_equal(dm, lags)
    np.testing.assert_array_equal(red * T, expect)


def test_redundancy_counts_by_pair_enumeration():
    """Redundancy of each lag counted by visiting every antenna pair."""
    dims = [3, 2, 2, 3]
    m = synth.antenna_indices([synth.Level(3, 2), synth.Level(2, 3)])
    lags = _lag_vectors(dims)
    count = {tuple(v): 0 for v in lags}
    for i in range(len(m)):
        for j in range(len(m)):
            count[tuple(m[i] - m[j])] += 1
    _, red = oracle.lag_table(dims)
    np.testing.assert_array_equal(red, [count[tuple(v)] for v in lags])


def test_single_antenna_delta():
    dims = [3, 4, 2, 2]
    N = int(np.prod(dims))
    T = 5
    a = np.array([0.75, -1.25])
    x = np.zeros((1, T, N, 2))
    x[0, :, 17] = a
    V = oracle.correlate(dims, x)[0]
    zero = len(V) // 2                                 # lag 0 sits in the middle
    assert _lag_vectors(dims)[zero].tolist() == [0, 0, 0, 0]
    assert V[zero] == pytest.approx(T * (a @ a))
    V[zero] = 0
    assert np.all(V == 0)


def test_plane_wave_closed_form():
    """x_t(i) = a_t exp(2 pi i u.r_i):  V(D) = sum|a_t|^2 exp(2 pi i u.dr(D)) prod(n_d-|D_d|)."""
    levels = synth.hierarchy([(4, 3), (3, 2)], [0.3, 1.1], [0.1, -0.25])
    dims = synth.lattice_dims(levels)
    r = synth.antenna_positions(levels)
    u = np.array([0.137, -0.291])
    rng = np.random.default_rng(5)
    a = rng.normal(size=4) + 1j * rng.normal(size=4)
    x = a[:, None] * np.exp(2j * math.pi * (r @ u))[None, :]
    V = oracle.correlate(dims, x[None])[0]
    lags = _lag_vectors(dims)
    dr = np.zeros((len(lags), 2))
    for k, lv in enumerate(levels):
        dr += lags[:, 2 * k:2 * k + 2] @ np.asarray(lv.A).reshape(2, 2).T
    red = np.prod([n - np.abs(lags[:, d]) for d, n in enumerate(dims)], axis=0)
    expect = np.sum(np.abs(a) ** 2) * np.exp(2j * math.pi * (dr @ u)) * red
    assert relerr(V, expect) < 1e-13


# ---------------------------------------------------------------- invariants

def test_hermitian_parseval_dc():
    dims = [4, 3, 3, 2]
    x = synth.random_complex(dims, 2, 3, seed=11).numpy().astype(np.float64)
    V = oracle.correlate(dims, x)
    xc = _cplx(x)
    for c in range(2):
        # Hermitian: V(-D) = conj V(D)  (Sec. II.C palindrome for real input)
        np.testing.assert_allclose(V[c][::-1], np.conj(V[c]), rtol=0, atol=1e-12)
        zero = V.shape[1] // 2
        assert V[c, zero].real == pytest.approx(np.sum(np.abs(xc[c]) ** 2), rel=1e-13)
        assert abs(V[c, zero].imag) < 1e-12
        assert np.sum(V[c]) == pytest.approx(np.sum(np.abs(xc[c].sum(axis=1)) ** 2), rel=1e-12)


# ---------------------------------------------------------------- other routes

@pytest.mark.parametrize("dims", [[2, 2, 2, 2], [3, 2, 2, 1], [4, 3], [1, 3, 2, 1]])
def test_naive_dft_route(dims):
    x = synth.random_complex(dims, 2, 2, seed=3).numpy().astype(np.float64)
    assert relerr(oracle.correlate(dims, x), naive_dft_route(dims, x)) < 1e-12


@pytest.mark.parametrize("fixture", ["three_level", "blocks", "interleaved", "warmup_2level"])
def test_numpy_fft_route_on_paper_layouts(fixture):
    levels = synth.paper_fixture(fixture)
    dims = synth.lattice_dims(levels)
    T = 2 if fixture != "blocks" else 1
    x = synth.random_complex(dims, 1, T, seed=7).numpy().astype(np.float64)
    assert relerr(oracle.correlate(dims, x), fft_route(dims, x)) < 1e-12


def test_numpy_fft_route_medium():
    dims = [6, 4, 3, 5]
    x = synth.random_complex(dims, 2, 3, seed=9).numpy().astype(np.float64)
    assert relerr(oracle.correlate(dims, x), fft_route(dims, x)) < 1e-12


# ---------------------------------------------------------------- input types

def test_input_types_are_converted_exactly():
    dims = [4, 4, 2, 3]
    x8 = synth.random_complex(dims, 2, 2, seed=1, dtype="ci8", sigma=40.0)
    ref = oracle.correlate(dims, x8.numpy().astype(np.float64))
    np.testing.assert_array_equal(oracle.correlate(dims, x8), ref)
    np.testing.assert_array_equal(oracle.correlate(dims, x8.float()), ref)


def test_selected_lags_match_full():
    dims = [5, 3, 2, 2]
    x = synth.random_complex(dims, 3, 2, seed=2)
    V = oracle.correlate(dims, x)
    rng = np.random.default_rng(0)
    ch = rng.integers(0, 3, 40)
    q = rng.integers(0, V.shape[1], 40)
    np.testing.assert_array_equal(oracle.correlate_selected(dims, x, ch, q), V[ch, q])


# ---------------------------------------------------------------- geometry

def test_positions_match_generator_geometry():
    levels = synth.paper_fixture("three_level")
    np.testing.assert_allclose(oracle.positions(levels), synth.antenna_positions(levels),
                               rtol=0, atol=1e-12)
    # Fig. 1 numbers: antenna i_1 = 4, i_4 = 2 of block (0,0,0,0) sits at (4, 2);
    # level-2 step a_2 = (8, 0), a_5 = (2, 8); level-3 step a_3 = (40, 10), a_6 = (-10, 40)
    r = oracle.positions(levels)
    assert r[4 + 5 * 2].tolist() == [4.0, 2.0]
    assert r[15].tolist() == [8.0, 0.0]                  # m = (0,0,1,0,0,0)
    assert r[15 * 3].tolist() == [2.0, 8.0]              # m = (0,0,0,1,0,0)
    assert r[15 * 9].tolist() == [40.0, 10.0]            # m = (0,0,0,0,1,0)
    assert r[15 * 27].tolist() == [-10.0, 40.0]          # m = (0,0,0,0,0,1)


def test_baseline_vectors():
    levels = synth.hierarchy([(3, 2), (2, 3)], [0.4, 2.0], [0.2, -0.1])
    dims = synth.lattice_dims(levels)
    dm, _ = oracle.lag_table(dims)
    dr = oracle.baseline_vectors(levels, dm)
    r = synth.antenna_positions(levels)
    m = synth.antenna_indices(levels)
    lut = {tuple(v): i for i, v in enumerate(m)}
    for q in range(len(dm)):
        for i, mi in enumerate(m):
            j = lut.get(tuple(mi - dm[q]))
            if j is not None:                            # pair (i, j) has m_i - m_j = D
                np.testing.assert_allclose(dr[q], r[i] - r[j], atol=1e-12)
                break


def test_collision_check():
    assert not oracle.collides(synth.paper_fixture("interleaved"))
    assert not oracle.collides(synth.paper_fixture("three_level"))
    # a_1 = (1,0) with 4 points and a_2 = (2,0) with 2 points put two antennas at x = 2, 3
    clash = [synth.Level(4, 1, (1.0, 0.0, 0.0, 1.0)), synth.Level(2, 1, (2.0, 0.0, 0.0, 1.0))]
    assert oracle.collides(clash)


# ---------------------------------------------------------------- physical baselines

def _pair_separations(levels):
    r = synth.antenna_positions(levels)
    return (r[:, None, :] - r[None, :, :]).reshape(-1, 2)


def test_radial_profile_of_ones_is_the_pair_distance_histogram():
    """Sec. III: binning d = l * l^- radially gives the 1-D baseline distribution."""
    levels = synth.paper_fixture("three_level")
    w, nb = 5.0, 30
    _, pairs = oracle.radial_bins(levels, w, nb)
    d = np.hypot(*_pair_separations(levels).T)
    hist = np.bincount(np.floor(d / w).astype(int), minlength=nb)[:nb]
    np.testing.assert_array_equal(pairs, hist)


COINCIDENT = [synth.Level(4, 1, (2.0, 0.0, 0.0, 1.0)), synth.Level(2, 1, (5.0, 0.0, 0.0, 1.0))]


def test_unique_baselines_match_pair_enumeration():
    """x = 0,2,4,6 and +5: the lags (3,-1) and (-2,1) both mean a separation of 1."""
    assert not oracle.collides(COINCIDENT)
    group, reps, pairs = oracle.unique_baselines(COINCIDENT)
    sep = np.round(_pair_separations(COINCIDENT), 9)
    uniq, counts = np.unique(sep, axis=0, return_counts=True)
    assert len(reps) == len(uniq) < len(group)
    order = np.lexsort((reps[:, 1], reps[:, 0]))
    np.testing.assert_allclose(reps[order], uniq)
    np.testing.assert_array_equal(pairs[order], counts)


def test_group_sum_of_correlation_equals_pairs_by_physical_separation():
    group, reps, _ = oracle.unique_baselines(COINCIDENT)
    x = synth.random_complex(synth.lattice_dims(COINCIDENT), 1, 2, seed=4)
    V = oracle.correlate(synth.lattice_dims(COINCIDENT), x)
    merged = oracle.group_sum(V, group, len(reps))
    xc = x.numpy().astype(np.float64)
    xc = xc[..., 0] + 1j * xc[..., 1]
    r = synth.antenna_positions(COINCIDENT)
    expect = np.zeros(len(reps), dtype=complex)
    for t in range(xc.shape[1]):
        for i in range(len(r)):
            for j in range(len(r)):
                g = int(np.argmin(np.hypot(*(reps - (r[i] - r[j])).T)))
                expect[g] += xc[0, t, i] * np.conj(xc[0, t, j])
    np.testing.assert_allclose(merged[0], expect, rtol=0, atol=1e-10)


# ---------------------------------------------------------------- beam-space variant

BEAM_LAYOUTS = [
    [synth.Level(4, 2), synth.Level(3, 2, (5.0, 0.0, 0.0, 5.0))],
    [synth.Level(3, 3), synth.Level(2, 2, (4.0, 0.5, 0.0, 4.0)), synth.Level(2, 1, (10.0, 0.0, 0.0, 10.0))],
    [synth.Level(5, 1), synth.Level(1, 4, (7.0, 0.0, 0.0, 7.0))],
]


@pytest.mark.parametrize("levels", BEAM_LAYOUTS)
def test_beam_sum_is_the_zero_level1_lag_slice(levels):
    """Summed over pointings, |DFT|^2 is Parseval's n1 n2 sum over the block,
    so sum_k B(k; D') = n1 n2 V(0, 0, D') of the full 2n-D correlator."""
    dims = synth.lattice_dims(levels)
    x = synth.random_complex(dims, 2, 3, seed=41)
    B = oracle.beam_correlate(dims, x)
    V = oracle.correlate(dims, x)
    lags = _lag_vectors(dims)
    sel = np.where((lags[:, 0] == 0) & (lags[:, 1] == 0))[0]
    assert relerr(B.sum(axis=2), dims[0] * dims[1] * V[:, sel]) < 1e-12


@pytest.mark.parametrize("levels", BEAM_LAYOUTS)
def test_beam_all_ones(levels):
    """All-ones blocks put n1 n2 in pointing 0 only: B(0; D') = (n1 n2)^2 T prod (n_d - |D_d|)."""
    dims = synth.lattice_dims(levels)
    T = 2
    B = oracle.beam_correlate(dims, synth.all_ones(dims, 1, T))
    lags = _lag_vectors(dims[2:])
    red = np.prod([n - np.abs(lags[:, d]) for d, n in enumerate(dims[2:])], axis=0)
    nb = dims[0] * dims[1]
    np.testing.assert_allclose(B[0, :, 0].real, nb * nb * T * red, rtol=1e-12, atol=1e-9)
    assert np.abs(B[0, :, 0].imag).max() < 1e-9
    assert np.abs(B[0, :, 1:]).max() < 1e-9


def test_beam_separable_plane_wave():
    """x(a, b, m') = exp(2 pi i (ka a / n1 + kb b / n2)) g(m') lands in pointing
    (ka, kb) alone, with B = (n1 n2)^2 times the coarse lattice's own correlation of g."""
    levels = BEAM_LAYOUTS[0]
    dims = synth.lattice_dims(levels)
    n1, n2, cdims = dims[0], dims[1], dims[2:]
    ka, kb = 3, 1
    rng = np.random.default_rng(5)
    T, Nc = 3, int(np.prod(cdims))
    g = rng.standard_normal((1, T, Nc)) + 1j * rng.standard_normal((1, T, Nc))
    a = np.arange(n1)[None, :]
    b = np.arange(n2)[:, None]
    w = np.exp(2j * math.pi * (ka * a / n1 + kb * b / n2)).ravel()       # [n2 * n1], a fastest
    x = (g[:, :, :, None] * w[None, None, None, :]).reshape(1, T, Nc * n1 * n2)
    B = oracle.beam_correlate(dims, x)
    Vg = oracle.correlate(cdims, g)
    k = ka + n1 * kb
    assert relerr(B[:, :, k], (n1 * n2) ** 2 * Vg) < 1e-12
    others = np.delete(B, k, axis=2)
    assert np.abs(others).max() < 1e-9 * np.abs(B[:, :, k]).max()


def test_beam_numpy_route():
    """numpy: unpadded fft2 over each block, then the zero-padded FFT route of
    Sec. II.C over the remaining axes, per pointing."""
    levels = BEAM_LAYOUTS[1]
    dims = synth.lattice_dims(levels)
    x = _cplx(synth.random_complex(dims, 1, 2, seed=43).numpy())
    C, T, N = x.shape
    n1, n2, cdims = dims[0], dims[1], dims[2:]
    Nc = int(np.prod(cdims))
    blocks = x.reshape(C, T, Nc, n2, n1)
    y = np.fft.fft2(blocks, axes=(3, 4))                                  # [C][T][Nc][kb][ka]
    y = y.reshape(C, T, Nc, n1 * n2).transpose(0, 3, 1, 2)                 # [C][k][T][Nc]
    ref = np.stack([fft_route(cdims, y[:, k]) for k in range(n1 * n2)], axis=2)
    assert relerr(oracle.beam_correlate(dims, x), ref) < 1e-12


# ---------------------------------------------------------------- tile hybrid

def test_tile_diagonal_is_each_tile_alone():
    n1, n2, nt = 3, 2, 4
    x = synth.random_complex([n1, n2, nt], 2, 3, seed=51)
    V = oracle.tile_correlate(n1, n2, nt, x)
    for i in range(nt):
        Vi = oracle.correlate([n1, n2], x[:, :, i * n1 * n2:(i + 1) * n1 * n2])
        assert relerr(V[:, i, i], Vi) < 1e-14


def test_tiles_on_a_lattice_reduce_to_the_two_level_hypercube():
    """Tiles placed on a grid form a 2-level hierarchy; summing V_ij over the
    tile pairs with the same tile-grid offset gives the hypercube's visibility
    at (intra-tile lag, tile-grid lag)."""
    n1, n2, N1, N2 = 3, 2, 3, 2
    nt = N1 * N2
    x = synth.random_complex([n1, n2, N1, N2], 1, 2, seed=52)
    V = oracle.tile_correlate(n1, n2, nt, x)
    H = oracle.correlate([n1, n2, N1, N2], x)
    Q1, Q2 = 2 * n1 - 1, 2 * n2 - 1
    R1, R2 = 2 * N1 - 1, 2 * N2 - 1
    acc = np.zeros((Q1 * Q2, R1 * R2), dtype=complex)
    for i in range(nt):
        for j in range(nt):
            D1 = (i % N1) - (j % N1) + (N1 - 1)
            D2 = (i // N1) - (j // N1) + (N2 - 1)
            acc[:, D1 + R1 * D2] += V[0, i, j]
    # hypercube lag index: intra-tile lag fastest, then the tile-grid lag
    assert relerr(acc.T.ravel(), H[0]) < 1e-13


def test_tile_hermitian_and_all_ones():
    n1, n2, nt = 4, 3, 3
    x = synth.random_complex([n1, n2, nt], 1, 2, seed=53)
    V = oracle.tile_correlate(n1, n2, nt, x)
    Q = (2 * n1 - 1) * (2 * n2 - 1)
    for i in range(nt):
        for j in range(nt):
            np.testing.assert_allclose(V[0, j, i][::-1], np.conj(V[0, i, j]), rtol=0, atol=1e-12)
    T = 3
    W = oracle.tile_correlate(n1, n2, nt, synth.all_ones([n1, n2, nt], 1, T))
    lags = _lag_vectors([n1, n2])
    red = (n1 - np.abs(lags[:, 0])) * (n2 - np.abs(lags[:, 1]))
    assert W.shape == (1, nt, nt, Q)
    np.testing.assert_array_equal(W[0].real, np.broadcast_to(T * red, (nt, nt, Q)))


def test_tile_numpy_cross_spectrum_route():
    """numpy: zero-padded fft2 of every tile, cross-spectra summed over time,
    inverse fft2, gather the intra-tile lags."""
    n1, n2, nt = 4, 3, 3
    x = _cplx(synth.random_complex([n1, n2, nt], 1, 3, seed=54).numpy())
    Y = np.fft.fft2(x.reshape(1, 3, nt, n2, n1), s=(2 * n2, 2 * n1), axes=(3, 4))
    S = np.einsum("ctiab,ctjab->cijab", Y, np.conj(Y))
    g = np.fft.ifft2(S, axes=(3, 4))
    idx = np.ix_(np.arange(-(n2 - 1), n2) % (2 * n2), np.arange(-(n1 - 1), n1) % (2 * n1))
    ref = g[..., idx[0], idx[1]].reshape(1, nt, nt, -1)
    assert relerr(oracle.tile_correlate(n1, n2, nt, x), ref) < 1e-12


# ---------------------------------------------------------------- F-engine

def test_fengine_single_tap_is_numpy_rfft_per_frame():
    rng = np.random.default_rng(61)
    N, F, T = 3, 8, 5
    raw = rng.integers(-128, 128, size=(N, 2 * F * T)).astype(np.int8)
    X = oracle.fengine(raw, F)
    ref = np.fft.rfft(raw.reshape(N, T, 2 * F).astype(np.float64), axis=-1)[..., :F]
    assert X.shape == (F, T, N)
    assert relerr(X, ref.transpose(2, 1, 0)) < 1e-14


def test_fengine_polyphase_frames_and_gains():
    """P taps: the windowed sum of P consecutive frames, then the real FFT
    (numpy, a different route); gains and scale multiply each channel."""
    rng = np.random.default_rng(62)
    N, F, P, S = 2, 16, 4, 2 * 16 * 9 + 5
    raw = rng.integers(-100, 100, size=(N, S)).astype(np.int8)
    w = rng.standard_normal(P * 2 * F)
    g = rng.standard_normal((F, N)) + 1j * rng.standard_normal((F, N))
    X = oracle.fengine(raw, F, P, window=w, gains=g, scale=0.25)
    M = 2 * F
    T = (S - (P - 1) * M) // M
    frames = np.stack([raw[:, t * M:(t + P) * M].astype(np.float64) for t in range(T)], axis=1)
    u = (frames.reshape(N, T, P, M) * w.reshape(P, M)).sum(axis=2)
    ref = 0.25 * np.fft.rfft(u, axis=-1)[..., :F].transpose(2, 1, 0) * g[:, None, :]
    assert X.shape == (F, T, N)
    assert relerr(X, ref) < 1e-13


def test_fengine_tone_closed_form():
    """The period-4 sequence (A, 0, -A, 0) has all its power in channel F/2:
    X(F/2) = A F, every other channel 0."""
    N, F, T, A = 2, 32, 3, 100
    pattern = np.array([A, 0, -A, 0], dtype=np.int8)
    raw = np.tile(pattern, (N, 2 * F * T // 4))
    X = oracle.fengine(raw, F)
    expect = np.zeros((F, T, N), dtype=complex)
    expect[F // 2] = A * F
    np.testing.assert_allclose(X, expect, rtol=0, atol=1e-9)


def test_quantizer_rounds_half_to_even_and_clips():
    x = np.array([0.5, 1.5, 2.5, -0.5, -1.5, -2.5, 126.5, 127.49, 127.5, 300.0, -127.5, -1e9], dtype=np.float32)
    np.testing.assert_array_equal(oracle.quantize(x),
                                  np.array([0, 2, 2, 0, -2, -2, 126, 127, 127, 127, -127, -127], dtype=np.int8))
