"""GPU parity of the mixed-precision path beyond its tensor-core level-1 shape.

Any 2-level hierarchy of at most 64 level-1 blocks runs level 1 as the FP32 FFT
and level 2 in lag space on tensor cores: the block cross-spectra summed over
time as one tcgen05 GEMM per level-1 frequency, then summed over block pairs of
equal grid offset (Sec. II.D's convolution over the level-2 axes).  Operands are
FP16 hi/lo with a power-of-two scale (fixed from the block size for int8
voltages, per channel and chunk from the voltages' max |x| for float ones) or
BF16 split three ways (no scale).  Bar: relative Frobenius error per channel
<= 1e-4 against the CPU FP64 oracle (the mixed bar); the measured errors are
near 1e-6."""
import numpy as np
import pytest
import torch

from oracle import oracle
from paper_0909_0001_gb300 import omni, synth

pytestmark = pytest.mark.gpu

TOL_MIXED = 1e-4

SHAPES = {
    "8x8 on 4x4": ([(8, 8), (4, 4)], [0.0, 0.5], [0.0, 0.15]),
    "16x8 on 8x8": ([(16, 8), (8, 8)], [0.0, 0.2], [0.0, -0.1]),
    "4x4 on 16x4 (64 blocks)": ([(4, 4), (16, 4)], [0.0, 1.1], [0.0, 0.3]),
    "12x12 on 5x5 (24-point axes)": ([(12, 12), (5, 5)], [0.0, 2.0], [0.0, 0.0]),
    "6x4 on 3x7": ([(6, 4), (3, 7)], [0.3, 0.9], [0.1, -0.2]),
    "16x16 on 8x8": ([(16, 16), (8, 8)], [0.0, 0.5236], [0.0, 0.2]),
}


def vis(levels, x, dtype, precision, calls=None):
    with omni.Plan(levels, x.shape[0], dtype=dtype, precision=precision) as plan:
        xd = x.cuda()
        if calls is None:
            plan.correlate(xd)
        else:
            t0 = 0
            for t in calls:
                plan.correlate(xd[:, t0:t0 + t].contiguous())
                t0 += t
        return plan.visibilities().cpu().numpy()


def relerr_per_channel(V, ref):
    num = np.linalg.norm(V - ref, axis=1)
    den = np.maximum(np.linalg.norm(ref, axis=1), 1e-300)
    return num / den


@pytest.mark.parametrize("shape", list(SHAPES))
@pytest.mark.parametrize("dtype", ["ci8", "cf32"])
@pytest.mark.parametrize("precision", ["mixed", "mixed_bf16"])
def test_general_two_level_mixed_matches_oracle(shape, dtype, precision):
    levels = synth.hierarchy(*SHAPES[shape])
    dims = synth.lattice_dims(levels)
    # 21 samples: one full 16-sample step and a ragged one
    x = synth.random_complex(dims, 2, 21, seed=501, dtype=dtype, sigma=30.0 if dtype == "ci8" else 1.0)
    V = vis(levels, x, dtype, precision)
    err = relerr_per_channel(V, oracle.correlate(dims, x))
    assert err.max() <= TOL_MIXED, f"{shape} {dtype} {precision}: {err}"


def test_fp16_float_voltages_scaled_per_channel():
    """Channels 1e-4, 1 and 1e5 in amplitude in one plan: each gets its own
    power of two before the FP16 split (without it 1e5 overflows FP16 and 1e-4
    falls into its subnormals)."""
    w = synth.workload("hier2")
    x = synth.random_complex(w.dims, 3, 19, seed=502, dtype="cf32")
    x = x * torch.tensor([1e-4, 1.0, 1e5]).view(3, 1, 1, 1)
    V = vis(w.levels, x, "cf32", "mixed")
    err = relerr_per_channel(V, oracle.correlate(w.dims, x))
    assert err.max() <= TOL_MIXED, err


def test_bf16_float_voltages_over_a_wide_range():
    """BF16 keeps FP32's exponent range: 1e-12 and 1e12 without any scaling."""
    levels = synth.hierarchy(*SHAPES["8x8 on 4x4"])
    dims = synth.lattice_dims(levels)
    x = synth.random_complex(dims, 2, 17, seed=503, dtype="cf32")
    x = x * torch.tensor([1e-12, 1e12]).view(2, 1, 1, 1)
    V = vis(levels, x, "cf32", "mixed_bf16")
    err = relerr_per_channel(V, oracle.correlate(dims, x))
    assert err.max() <= TOL_MIXED, err


@pytest.mark.parametrize("precision", ["mixed", "mixed_bf16"])
def test_bf16_and_fp16_on_the_benchmark_shape(precision, monkeypatch):
    """16x16 blocks on 8x8, int8: FP16 with level 1 on tensor cores (default) or
    as the FP32 FFT, and BF16 (FP32 level 1); 37 samples, 3 channels."""
    w = synth.workload("hier2")
    x = synth.voltages(w, channels=3, samples=37)
    V = vis(w.levels, x, "ci8", precision)
    ref = oracle.correlate(w.dims, x)
    assert relerr_per_channel(V, ref).max() <= TOL_MIXED
    if precision == "mixed":
        monkeypatch.setenv("OMNI_TC_STAGE_A", "0")
        V2 = vis(w.levels, x, "ci8", precision)
        assert relerr_per_channel(V2, ref).max() <= TOL_MIXED


def test_scaled_float_chunks_and_split_calls(monkeypatch):
    """Small chunk buffers (several chunks, both overlap slots of the per-channel
    scale array reused) and split calls equal one call and the oracle."""
    monkeypatch.setenv("OMNI_CHUNK_MB", "2")
    monkeypatch.setenv("OMNI_OVERLAP", "1")
    levels = synth.hierarchy(*SHAPES["8x8 on 4x4"])
    dims = synth.lattice_dims(levels)
    x = synth.random_complex(dims, 5, 40, seed=504, dtype="cf32")
    x = x * torch.tensor([3e-3, 1.0, 7e2, 1.0, 5e4]).view(5, 1, 1, 1)
    ref = oracle.correlate(dims, x)
    one = vis(levels, x, "cf32", "mixed")
    split = vis(levels, x, "cf32", "mixed", calls=[13, 27])
    assert relerr_per_channel(one, ref).max() <= TOL_MIXED
    assert relerr_per_channel(split, ref).max() <= TOL_MIXED
    monkeypatch.setenv("OMNI_OVERLAP", "0")
    serial = vis(levels, x, "cf32", "mixed")
    assert relerr_per_channel(serial, one).max() <= 1e-6


def test_mixed_general_all_ones_exact_after_rounding():
    levels = synth.hierarchy(*SHAPES["4x4 on 16x4 (64 blocks)"])
    dims = synth.lattice_dims(levels)
    _, red, _ = omni.baselines(levels)
    for precision in ("mixed", "mixed_bf16"):
        V = vis(levels, synth.all_ones(dims, 1, 3, dtype="ci8"), "ci8", precision)
        np.testing.assert_array_equal(np.rint(V.real[0]).astype(np.int64), 3 * red)


@pytest.mark.parametrize("dtype, precision", [("cf32", "mixed"), ("ci8", "mixed_bf16"), ("cf32", "mixed_bf16")])
def test_tiles_other_mixed_forms_match_oracle(dtype, precision):
    n1, n2, nt = 8, 4, 13
    tile = synth.Level(n1, n2, (1.0, 0.3, 0.0, 1.0))
    rng = np.random.default_rng(505)
    offs = rng.uniform(-200.0, 200.0, size=(nt, 2))
    x = synth.random_complex([n1, n2, nt], 2, 19, seed=506, dtype=dtype, sigma=30.0 if dtype == "ci8" else 1.0)
    if dtype == "cf32":
        x = x * torch.tensor([2e-3, 4e3]).view(2, 1, 1, 1)
    with omni.TilePlan(tile, offs, 2, dtype=dtype, precision=precision) as plan:
        plan.correlate(x.cuda())
        V = plan.split(plan.visibilities()).cpu().numpy()
    ref = oracle.tile_correlate(n1, n2, nt, x)
    num = np.linalg.norm((V - ref).reshape(2, -1), axis=1)
    den = np.linalg.norm(ref.reshape(2, -1), axis=1)
    assert float(np.max(num / den)) <= TOL_MIXED
