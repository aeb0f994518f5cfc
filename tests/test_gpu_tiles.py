"""GPU parity of the tile-hybrid plan (Sec. III: FFT correlation within
identical tiles at arbitrary offsets, brute-force correlation between them)
against the CPU FP64 oracle.

Bar: relative Frobenius error per channel <= 1e-5 (FP32 path); all-ones
counts exact after rounding."""
import numpy as np
import pytest
import torch

from oracle import oracle
from paper_0909_0001_gb300 import omni, synth

pytestmark = pytest.mark.gpu

TOL = 1e-5


def offsets(n_tiles, seed, spread=200.0):
    rng = np.random.default_rng(seed)
    return rng.uniform(-spread, spread, size=(n_tiles, 2))


def tile_vis(tile, offs, x, dtype="cf32"):
    C = x.shape[0]
    with omni.TilePlan(tile, offs, C, dtype=dtype) as plan:
        plan.correlate(x.cuda())
        return plan.split(plan.visibilities()).cpu().numpy()


def relerr_per_channel(V, ref):
    num = np.linalg.norm((V - ref).reshape(V.shape[0], -1), axis=1)
    den = np.maximum(np.linalg.norm(ref.reshape(ref.shape[0], -1), axis=1), 1e-300)
    return float(np.max(num / den))


CASES = [(3, 2, 4), (4, 4, 5), (16, 16, 17), (5, 3, 3), (1, 1, 3), (32, 1, 2), (8, 8, 33)]


@pytest.mark.parametrize("n1, n2, nt", CASES)
@pytest.mark.parametrize("dtype", ["cf32", "ci8"])
def test_tiles_match_oracle(n1, n2, nt, dtype):
    tile = synth.Level(n1, n2, (1.0, 0.3, 0.0, 1.0))
    x = synth.random_complex([n1, n2, nt], 2, 5, seed=81, dtype=dtype,
                             sigma=30.0 if dtype == "ci8" else 1.0)
    V = tile_vis(tile, offsets(nt, 1), x, dtype)
    ref = oracle.tile_correlate(n1, n2, nt, x)
    assert relerr_per_channel(V, ref) <= TOL


def test_tiles_all_ones_exact():
    n1, n2, nt, T = 8, 8, 6, 3
    V = tile_vis(synth.Level(n1, n2), offsets(nt, 2), synth.all_ones([n1, n2, nt], 1, T, "ci8"), "ci8")
    _, red, _ = omni.baselines([synth.Level(n1, n2)])
    np.testing.assert_array_equal(np.rint(V[0].real).astype(np.int64),
                                  np.broadcast_to(T * red, (nt, nt, len(red))))


def test_tiles_many_chunks_and_split_calls(monkeypatch):
    monkeypatch.setenv("OMNI_CHUNK_MB", "1")
    n1, n2, nt = 16, 16, 9
    tile = synth.Level(n1, n2)
    x = synth.random_complex([n1, n2, nt], 3, 9, seed=82)
    with omni.TilePlan(tile, offsets(nt, 3), 3) as plan:
        plan.correlate(x[:, :5].contiguous().cuda())
        plan.correlate(x[:, 5:].contiguous().cuda())
        V = plan.split(plan.visibilities()).cpu().numpy()
    assert relerr_per_channel(V, oracle.tile_correlate(n1, n2, nt, x)) <= TOL


def test_tiles_sized_run_one_channel():
    """32 tiles of 8x8 at random offsets, 4 channels x 64 samples of int8;
    channel 2 checked in full (every tile pair and lag)."""
    n1, n2, nt = 8, 8, 32
    x = synth.random_complex([n1, n2, nt], 4, 64, seed=83, dtype="ci8", sigma=20.0)
    V = tile_vis(synth.Level(n1, n2, (1.0, 0.0, 0.0, 1.0)), offsets(nt, 4), x, "ci8")
    assert relerr_per_channel(V[2:3], oracle.tile_correlate(n1, n2, nt, x[2:3])) <= TOL


def test_tiles_hermitian_pairs_and_host_path():
    n1, n2, nt = 4, 3, 3
    x = synth.random_complex([n1, n2, nt], 1, 4, seed=84)
    with omni.TilePlan(synth.Level(n1, n2), offsets(nt, 5), 1) as plan:
        plan.correlate_host(x)
        Vh = plan.split(plan.visibilities_host()).numpy()
        dr = plan.baseline_vectors()
    for i in range(nt):
        for j in range(nt):
            np.testing.assert_allclose(Vh[0, j, i][::-1], np.conj(Vh[0, i, j]), rtol=0,
                                       atol=1e-5 * np.abs(Vh).max())
            np.testing.assert_allclose(dr[j, i][::-1], -dr[i, j], rtol=0, atol=1e-9)


def test_tiles_on_the_lattice_equal_the_hypercube():
    """The 2-level workload's blocks as tiles at their level-2 positions: the
    tile pairs with equal grid offset sum to the hypercube plan's visibilities."""
    w = synth.workload("hier2")
    lv1, lv2 = w.levels
    x = synth.voltages(w, channels=2, samples=8)
    A2 = np.array(lv2.A).reshape(2, 2)
    grid = np.array([(j1, j2) for j2 in range(lv2.n2) for j1 in range(lv2.n1)], dtype=float)
    Vt = tile_vis(lv1, grid @ A2.T, x, "ci8")                       # [C][i][j][Q]
    with omni.Plan(w.levels, 2, dtype="ci8") as plan:
        plan.correlate(x.cuda())
        H = plan.visibilities().cpu().numpy()
    N1, N2 = lv2.n1, lv2.n2
    R1 = 2 * N1 - 1
    acc = np.zeros((2, R1 * (2 * N2 - 1), Vt.shape[-1]), dtype=complex)
    for i in range(N1 * N2):
        for j in range(N1 * N2):
            g = (i % N1 - j % N1 + N1 - 1) + R1 * (i // N1 - j // N1 + N2 - 1)
            acc[:, g] += Vt[:, i, j]
    assert relerr_per_channel(acc.reshape(2, -1), H) <= TOL


# ---------------------------------------------------------------- mixed precision (tcgen05)

TOL_MIXED = 1e-4


def tile_vis_mixed(tile, offs, x):
    with omni.TilePlan(tile, offs, x.shape[0], dtype="ci8", precision="mixed") as plan:
        plan.correlate(x.cuda())
        return plan.split(plan.visibilities()).cpu().numpy()


@pytest.mark.parametrize("n1, n2, nt, T", [(3, 2, 4, 5), (4, 4, 5, 16), (16, 16, 17, 37),
                                           (8, 8, 33, 20), (5, 3, 3, 9), (32, 1, 2, 17),
                                           (4, 2, 64, 24)])
def test_tiles_mixed_match_oracle(n1, n2, nt, T):
    """Cross-spectra as tensor-core GEMMs over the samples (sample counts that
    are not multiples of the 16-sample step, up to the 64-tile limit)."""
    tile = synth.Level(n1, n2, (1.0, 0.3, 0.0, 1.0))
    x = synth.random_complex([n1, n2, nt], 2, T, seed=91, dtype="ci8", sigma=30.0)
    V = tile_vis_mixed(tile, offsets(nt, 6), x)
    ref = oracle.tile_correlate(n1, n2, nt, x)
    assert relerr_per_channel(V, ref) <= TOL_MIXED


def test_tiles_mixed_more_steps_than_stages():
    """100 samples: seven 16-sample steps, so every shared-memory ring wraps."""
    n1, n2, nt = 4, 4, 16
    x = synth.random_complex([n1, n2, nt], 2, 100, seed=93, dtype="ci8", sigma=30.0)
    V = tile_vis_mixed(synth.Level(n1, n2, (1.0, 0.3, 0.0, 1.0)), offsets(nt, 10), x)
    assert relerr_per_channel(V, oracle.tile_correlate(n1, n2, nt, x)) <= TOL_MIXED


def test_tiles_mixed_full_scale_and_all_ones():
    """+-127 everywhere (the largest spectra FP16 must hold after the 1/16 scale)
    and the layout map of ones, exact after rounding."""
    n1, n2, nt = 16, 16, 8
    x = torch.full((1, 6, n1 * n2 * nt, 2), 127, dtype=torch.int8)
    V = tile_vis_mixed(synth.Level(n1, n2), offsets(nt, 7), x)
    assert relerr_per_channel(V, oracle.tile_correlate(n1, n2, nt, x)) <= TOL_MIXED
    ones = synth.all_ones([n1, n2, nt], 1, 3, "ci8")
    V = tile_vis_mixed(synth.Level(n1, n2), offsets(nt, 7), ones)
    _, red, _ = omni.baselines([synth.Level(n1, n2)])
    np.testing.assert_array_equal(np.rint(V[0].real).astype(np.int64),
                                  np.broadcast_to(3 * red, (nt, nt, len(red))))


def test_tiles_mixed_chunks_and_split_calls(monkeypatch):
    """Several chunks per call and several calls: the accumulators restart per
    chunk and the FP64 fold adds them."""
    monkeypatch.setenv("OMNI_CHUNK_MB", "2")
    n1, n2, nt = 8, 8, 12
    x = synth.random_complex([n1, n2, nt], 3, 41, seed=92, dtype="ci8", sigma=20.0)
    with omni.TilePlan(synth.Level(n1, n2), offsets(nt, 8), 3, dtype="ci8", precision="mixed") as plan:
        plan.correlate(x[:, :19].contiguous().cuda())
        plan.correlate(x[:, 19:].contiguous().cuda())
        V = plan.split(plan.visibilities()).cpu().numpy()
    assert relerr_per_channel(V, oracle.tile_correlate(n1, n2, nt, x)) <= TOL_MIXED


def test_tiles_mixed_on_the_lattice_equal_the_hypercube():
    """64 tiles (the 2-level workload's blocks at their level-2 positions): the
    mixed tile plan agrees with the FP32 tile plan, and its tile pairs of equal
    grid offset sum to the FP32 hypercube's visibilities."""
    w = synth.workload("hier2")
    lv1, lv2 = w.levels
    x = synth.voltages(w, channels=2, samples=40)
    A2 = np.array(lv2.A).reshape(2, 2)
    grid = np.array([(j1, j2) for j2 in range(lv2.n2) for j1 in range(lv2.n1)], dtype=float)
    Vm = tile_vis_mixed(lv1, grid @ A2.T, x)
    Vf = tile_vis(lv1, grid @ A2.T, x, "ci8")
    assert relerr_per_channel(Vm, Vf) <= TOL_MIXED
    with omni.Plan(w.levels, 2, dtype="ci8") as plan:
        plan.correlate(x.cuda())
        H = plan.visibilities().cpu().numpy()
    N1, N2 = lv2.n1, lv2.n2
    R1 = 2 * N1 - 1
    acc = np.zeros((2, R1 * (2 * N2 - 1), Vm.shape[-1]), dtype=complex)
    for i in range(N1 * N2):
        for j in range(N1 * N2):
            g = (i % N1 - j % N1 + N1 - 1) + R1 * (i // N1 - j // N1 + N2 - 1)
            acc[:, g] += Vm[:, i, j]
    assert relerr_per_channel(acc.reshape(2, -1), H) <= TOL_MIXED


def test_tiles_mixed_rejects_what_it_does_not_support():
    tile = synth.Level(4, 4)
    with pytest.raises(omni.OmniError) as e:      # padded tile size 6 x 1: not a multiple of 4
        omni.TilePlan(synth.Level(3, 1), offsets(3, 9), 1, dtype="ci8", precision="mixed_bf16")
    assert e.value.status == 3
    with pytest.raises(omni.OmniError) as e:      # more than 64 tiles
        omni.TilePlan(tile, offsets(65, 9, spread=2000.0), 1, dtype="ci8", precision="mixed")
    assert e.value.status == 3
