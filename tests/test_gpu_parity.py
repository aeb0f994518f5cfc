"""GPU parity: the CUDA correlator (through the C ABI) against the CPU FP64 oracle.

Bar (FP32 path): relative Frobenius error of the visibilities <= 1e-5 per
channel; integer results (baseline indices, all-ones redundancy counts after
rounding, the paper's warm-up example) exact.
"""
import math

import numpy as np
import pytest
import torch

from conftest import read_golden
from oracle import oracle
from paper_0909_0001_gb300 import omni, synth

pytestmark = pytest.mark.gpu

TOL_FP32 = 1e-5


def gpu_vis(levels, x, dtype="cf32", calls=None, precision="fp32"):
    """Visibilities [C][Q] from the CUDA library for voltages x [C][T][N][2]."""
    C = x.shape[0]
    with omni.Plan(levels, C, dtype=dtype, precision=precision) as plan:
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
    return float(np.max(num / den))


def check(levels, x, dtype="cf32", tol=TOL_FP32, precision="fp32"):
    V = gpu_vis(levels, x, dtype, precision=precision)
    ref = oracle.correlate(synth.lattice_dims(levels), x)
    err = relerr_per_channel(V, ref)
    assert err <= tol, f"relative Frobenius error {err:.3e} > {tol:g}"
    return V, ref


# ---------------------------------------------------------------- paper values

def test_warmup_example_is_exact():
    g = read_golden("warmup_example.txt")
    f = np.array(g["voltages"][0], dtype=np.float32)
    x1 = torch.zeros((1, 1, 9, 2))
    x1[0, 0, [0, 1, 2, 6, 7, 8], 0] = torch.from_numpy(f)
    V1 = gpu_vis(synth.paper_fixture("warmup_1d"), x1)
    np.testing.assert_array_equal(np.rint(V1.real[0]), g["g_1d"][0])
    assert np.max(np.abs(V1[0] - np.array(g["g_1d"][0]))) < 1e-4
    x2 = torch.zeros((1, 1, 6, 2))
    x2[0, 0, :, 0] = torch.from_numpy(f)
    V2 = gpu_vis(synth.paper_fixture("warmup_2level"), x2)
    np.testing.assert_array_equal(np.rint(V2.real[0]).reshape(3, 5), np.array(g["G_2d_row"]))


@pytest.mark.parametrize("name,T", [("three_level", 3), ("blocks", 2), ("interleaved", 4),
                                    ("plank", 1), ("strips", 1), ("warmup_2level", 5)])
def test_paper_layouts(name, T):
    levels = synth.paper_fixture(name)
    x = synth.random_complex(synth.lattice_dims(levels), 1, T, seed=17)
    check(levels, x)


@pytest.mark.parametrize("levels", [
    synth.paper_fixture("blocks"),
    [synth.Level(16, 16)],
    synth.hierarchy([(4, 3), (3, 2), (2, 2)], [0.3, 1.0, 2.0], [0.1, 0.2, -0.2]),
    [synth.Level(1, 1)],
])
def test_all_ones_gives_exact_redundancy(levels):
    dims = synth.lattice_dims(levels)
    T = 2
    V = gpu_vis(levels, synth.all_ones(dims, 1, T))
    _, red, _ = omni.baselines(levels)
    np.testing.assert_array_equal(np.rint(V.real[0]).astype(np.int64), T * red)
    assert np.max(np.abs(V[0] - T * red)) < 1e-3 * max(1, T * red.max()) ** 0.5


# ---------------------------------------------------------------- workloads

def test_grid16_full_size():
    w = synth.workload("grid16")
    x = synth.voltages(w)
    check(w.levels, x)


def test_hier2_reduced_ragged_chunks_int8():
    w = synth.workload("hier2")
    x = synth.voltages(w, channels=3, samples=5)
    check(w.levels, x, dtype="ci8")


def test_hier3_small_six_dims():
    levels = synth.hierarchy([(4, 4), (4, 2), (2, 3)], [0.5, 1.5, 2.5], [0.2, -0.1, 0.3])
    x = synth.random_complex(synth.lattice_dims(levels), 2, 3, seed=5)
    check(levels, x)


def sampled_error(levels, x, V, chans, lags):
    """Frobenius error estimated from sampled lags: sqrt(Q mean|dV|^2) / ||V_gpu||."""
    ref = oracle.correlate_selected(synth.lattice_dims(levels), x, chans, lags)
    got = V[chans, lags]
    Q = V.shape[1]
    errs = []
    for c in np.unique(chans):
        m = chans == c
        est = math.sqrt(Q * np.mean(np.abs(got[m] - ref[m]) ** 2)) / np.linalg.norm(V[c])
        errs.append(est)
    return max(errs), got, ref


def property_checks(levels, x, V, tol=TOL_FP32):
    """Size-independent properties: V(0) = sum|x|^2 (Parseval), V(-D) = conj V(D)."""
    power = np.array([float((x[c].double() ** 2).sum()) for c in range(x.shape[0])])
    zero = V.shape[1] // 2
    np.testing.assert_allclose(V[:, zero].real, power, rtol=tol)
    herm = np.linalg.norm(V[:, ::-1] - np.conj(V), axis=1) / np.linalg.norm(V, axis=1)
    assert herm.max() <= tol


def test_hier3_full_lattice_sampled():
    w = synth.workload("hier3")
    x = synth.voltages(w, channels=1, samples=2)
    V = gpu_vis(w.levels, x)
    rng = np.random.default_rng(3)
    lags = np.concatenate([[V.shape[1] // 2, 0, V.shape[1] - 1], rng.integers(0, V.shape[1], 253)])
    err, _, _ = sampled_error(w.levels, x, V, np.zeros_like(lags), lags)
    assert err <= TOL_FP32, err
    property_checks(w.levels, x, V)


def test_grid1024_sampled():
    w = synth.workload("grid1024")
    x = synth.voltages(w, channels=1, samples=2)
    V = gpu_vis(w.levels, x)
    rng = np.random.default_rng(4)
    lags = np.concatenate([[V.shape[1] // 2], rng.integers(0, V.shape[1], 511)])
    err, _, _ = sampled_error(w.levels, x, V, np.zeros_like(lags), lags)
    assert err <= TOL_FP32, err
    property_checks(w.levels, x, V)


def test_hier2_full_size_sampled():
    """The benchmark configuration: 64 channels x 1024 samples of int8 voltages."""
    w = synth.workload("hier2")
    xd = synth.voltages(w, device="cuda")
    with omni.Plan(w.levels, w.channels, dtype=w.dtype) as plan:
        plan.correlate(xd)
        V = plan.visibilities().cpu().numpy()
    x = xd.cpu()
    del xd
    rng = np.random.default_rng(5)
    chans = np.repeat(np.array([0, 37, 63]), 96)
    lags = rng.integers(0, V.shape[1], chans.size)
    lags[::96] = V.shape[1] // 2
    err, _, _ = sampled_error(w.levels, x, V, chans, lags)
    assert err <= TOL_FP32, err
    property_checks(w.levels, x, V)


# ---------------------------------------------------------------- API semantics

def test_split_calls_equal_one_call_and_reset():
    levels = synth.hierarchy([(8, 4), (4, 4)], [0.0, 0.7], [0.0, 0.15])
    x = synth.random_complex(synth.lattice_dims(levels), 2, 12, seed=8)
    one = gpu_vis(levels, x)
    split = gpu_vis(levels, x, calls=[5, 0, 7])
    assert relerr_per_channel(split, one) <= 1e-6
    with omni.Plan(levels, 2) as plan:
        plan.correlate(synth.random_complex(synth.lattice_dims(levels), 2, 3, seed=99).cuda())
        plan.visibilities(reset=True)            # discards the first integration
        plan.correlate(x.cuda())
        again = plan.visibilities(reset=True).cpu().numpy()
    assert relerr_per_channel(again, one) <= 1e-6


def test_host_path_matches_device_path():
    w = synth.workload("hier2")
    x = synth.voltages(w, channels=2, samples=40)
    dev = gpu_vis(w.levels, x, dtype="ci8")
    with omni.Plan(w.levels, 2, dtype="ci8") as plan:
        plan.correlate_host(x.pin_memory())
        host = plan.visibilities_host().numpy()
        plan.correlate_host(x)                   # pageable memory works too
        host2 = plan.visibilities_host().numpy()
    np.testing.assert_array_equal(host, dev)
    np.testing.assert_array_equal(host2, dev)


@pytest.mark.parametrize("levels", [
    [synth.Level(1, 1)],
    [synth.Level(16, 1)],
    [synth.Level(1, 16)],
    [synth.Level(1, 1), synth.Level(5, 1, (3.0, 0.0, 0.0, 1.0))],
    [synth.Level(3, 5)],
    [synth.Level(7, 2), synth.Level(3, 1, (7.0, 0.0, 0.0, 2.0))],
    [synth.Level(100, 3)],
])
def test_degenerate_and_odd_shapes(levels):
    x = synth.random_complex(synth.lattice_dims(levels), 2, 3, seed=12)
    check(levels, x)


@pytest.mark.parametrize("n1, n2", [(64, 3), (3, 64), (256, 2), (2, 512), (128, 8), (60, 70)])
def test_four_step_axes_rows_and_columns(n1, n2):
    """Axes of 64..512 antennas (padded 128..1024, four-step passes): along the
    innermost axis W whole lines per CTA (forward and inverse), strided axes W
    inner indices per CTA."""
    levels = [synth.Level(n1, n2, (1.0, 0.1, 0.0, 1.0))]
    x = synth.random_complex([n1, n2], 2, 3, seed=79)
    check(levels, x)


@pytest.mark.parametrize("n1, n2", [(2048, 2), (2, 2048), (1024, 3), (3, 1024)])
def test_long_axes_three_step_passes(n1, n2):
    """Axes of 2048 and 1024 antennas (padded to 4096 and 2048): the forward
    three-step passes, with lines along the innermost axis (W whole rows per CTA)
    and along a strided axis (W inner indices per CTA, fewer than W here)."""
    levels = [synth.Level(n1, n2, (1.0, 0.2, 0.0, 1.0))]
    x = synth.random_complex([n1, n2], 2, 3, seed=77)
    check(levels, x)


def test_zero_samples_is_a_no_op():
    levels = [synth.Level(4, 4)]
    with omni.Plan(levels, 1) as plan:
        plan.correlate(torch.zeros((1, 0, 16, 2), device="cuda"))
        V = plan.visibilities().cpu().numpy()
    assert np.all(V == 0)


def test_wrong_input_is_rejected():
    with omni.Plan([synth.Level(4, 4)], 2) as plan:
        with pytest.raises(ValueError):
            plan.correlate(torch.zeros((1, 3, 16, 2), device="cuda"))
        with pytest.raises(TypeError):
            plan.correlate(torch.zeros((2, 3, 16, 2), dtype=torch.int8, device="cuda"))


# ---------------------------------------------------------------- pass families

@pytest.mark.parametrize("levels, T", [
    ([synth.Level(32, 32)], 3),                                            # one 64-point level, last
    (synth.hierarchy([(4, 4), (2, 2), (2, 2)], [0.2, 0.4, 0.6], [0.0, 0.1, 0.2]), 4),
    (synth.hierarchy([(8, 8), (32, 32)], [0.0, 1.0], [0.0, 0.3]), 1),     # 64-point coarse level
    (synth.hierarchy([(16, 16), (4, 4)], [0.0, 0.5], [0.0, 0.0]), 3),
])
def test_level_pass_shapes(levels, T):
    x = synth.random_complex(synth.lattice_dims(levels), 2, T, seed=21)
    check(levels, x)


def test_level_and_per_axis_paths_agree(monkeypatch):
    w = synth.workload("hier2")
    x = synth.voltages(w, channels=3, samples=20)
    fused = gpu_vis(w.levels, x, dtype="ci8")
    monkeypatch.setenv("OMNI_LEVEL_PASSES", "0")
    per_axis = gpu_vis(w.levels, x, dtype="ci8")
    assert relerr_per_channel(fused, per_axis) <= 2e-6


# ---------------------------------------------------------------- mixed precision

TOL_MIXED = 1e-4


def test_mixed_matches_oracle_ragged():
    w = synth.workload("hier2")
    x = synth.voltages(w, channels=3, samples=7)
    V, _ = check(w.levels, x, dtype="ci8", tol=TOL_MIXED, precision="mixed")
    fp32 = gpu_vis(w.levels, x, dtype="ci8")
    assert relerr_per_channel(V, fp32) <= TOL_MIXED


def test_mixed_extreme_int8_values():
    """Full-scale +-127 voltages: the FP16 operands must stay in range."""
    w = synth.workload("hier2")
    x = synth.random_complex(w.dims, 2, 3, seed=31, dtype="ci8", sigma=400.0)  # clipped to +-127
    assert int(x.abs().max()) == 127
    check(w.levels, x, dtype="ci8", tol=TOL_MIXED, precision="mixed")
    ones = torch.full_like(x, 127)
    check(w.levels, ones, dtype="ci8", tol=TOL_MIXED, precision="mixed")


def test_mixed_all_ones_exact_after_rounding():
    w = synth.workload("hier2")
    V = gpu_vis(w.levels, synth.all_ones(w.dims, 1, 2, dtype="ci8"), dtype="ci8", precision="mixed")
    _, red, _ = omni.baselines(w.levels)
    np.testing.assert_array_equal(np.rint(V.real[0]).astype(np.int64), 2 * red)


def test_mixed_full_size_sampled():
    w = synth.workload("hier2")
    xd = synth.voltages(w, device="cuda")
    with omni.Plan(w.levels, w.channels, dtype=w.dtype, precision="mixed") as plan:
        plan.correlate(xd)
        V = plan.visibilities().cpu().numpy()
    x = xd.cpu()
    del xd
    rng = np.random.default_rng(6)
    chans = np.repeat(np.array([1, 30, 62]), 96)
    lags = rng.integers(0, V.shape[1], chans.size)
    lags[::96] = V.shape[1] // 2
    err, _, _ = sampled_error(w.levels, x, V, chans, lags)
    assert err <= TOL_MIXED, err
    property_checks(w.levels, x, V, tol=TOL_MIXED)


def test_mixed_rejects_unsupported_shapes():
    """The lag-space mixed path needs exactly two levels, at most 64 level-1 blocks
    and a padded level-1 lattice whose size is a multiple of 4."""
    cases = [[synth.Level(16, 16)],                                          # one level
             synth.hierarchy([(4, 4), (2, 2), (2, 2)], [0, 0.3, 0.6], [0, 0.1, 0]),  # three
             synth.hierarchy([(4, 4), (9, 8)], [0, 0.4], [0, 0.1]),          # 72 blocks
             synth.hierarchy([(3, 1), (4, 4)], [0, 0.4], [0, 0.1])]          # 6 x 1 padded
    for levels in cases:
        for prec in ("mixed", "mixed_bf16"):
            with pytest.raises(omni.OmniError) as e:
                omni.Plan(levels, 1, dtype="ci8", precision=prec)
            assert e.value.status == 3


def test_mixed_tcgen05_variant(monkeypatch):
    """The tensor-memory (tcgen05) form of the per-sample level-2 DFT-GEMMs gives
    the same visibilities as the mma.sync form."""
    w = synth.workload("hier2")
    x = synth.voltages(w, channels=2, samples=9)
    monkeypatch.setenv("OMNI_MIXED_LAGSUM", "0")
    default = gpu_vis(w.levels, x, dtype="ci8", precision="mixed")
    monkeypatch.setenv("OMNI_TCGEN05", "1")
    V, _ = check(w.levels, x, dtype="ci8", tol=TOL_MIXED, precision="mixed")
    assert relerr_per_channel(V, default) <= 1e-6


@pytest.mark.parametrize("lagsum", ["1", "0"])
def test_mixed_level2_forms_agree(monkeypatch, lagsum):
    """Level 2 in lag space (block cross-spectra over time as a tcgen05 GEMM,
    summed by grid offset) and as per-sample DFT-GEMMs: each within the mixed
    bar of the oracle and of each other; sample counts off the 16-sample step."""
    w = synth.workload("hier2")
    x = synth.voltages(w, channels=3, samples=37)
    monkeypatch.setenv("OMNI_MIXED_LAGSUM", lagsum)
    V, _ = check(w.levels, x, dtype="ci8", tol=TOL_MIXED, precision="mixed")
    monkeypatch.setenv("OMNI_MIXED_LAGSUM", "0" if lagsum == "1" else "1")
    other = gpu_vis(w.levels, x, dtype="ci8", precision="mixed")
    assert relerr_per_channel(V, other) <= 2e-5


def test_mixed_lagsum_many_steps():
    """100 samples: seven 16-sample steps, more than the lag-sum kernel's rings."""
    w = synth.workload("hier2")
    x = synth.voltages(w, channels=2, samples=100)
    check(w.levels, x, dtype="ci8", tol=TOL_MIXED, precision="mixed")


@pytest.mark.parametrize("stage_a", ["0", "1"])
def test_mixed_level1_on_cuda_cores_or_tensor_cores(monkeypatch, stage_a):
    """Level 1 as the FP32 FFT (0) or as split-FP16 GEMMs (1); level 2 on tensor
    cores either way, with and without a split of the last pass."""
    w = synth.workload("hier2")
    x = synth.voltages(w, channels=5, samples=9)
    monkeypatch.setenv("OMNI_TC_STAGE_A", stage_a)
    check(w.levels, x, dtype="ci8", tol=TOL_MIXED, precision="mixed")
    monkeypatch.setenv("OMNI_SPLIT_TC", "0.4")
    check(w.levels, x, dtype="ci8", tol=TOL_MIXED, precision="mixed")


@pytest.mark.parametrize("frac", ["0", "0.3", "0.5", "0.8"])
def test_mixed_split_last_pass(monkeypatch, frac):
    """Channels of a chunk split between the tensor-core and the FP32 last pass
    (run concurrently) give the same visibilities as either alone."""
    w = synth.workload("hier2")
    x = synth.voltages(w, channels=11, samples=6)
    monkeypatch.setenv("OMNI_MIXED_LAGSUM", "0")
    monkeypatch.setenv("OMNI_SPLIT_TC", "0")
    tc_only = gpu_vis(w.levels, x, dtype="ci8", precision="mixed")
    monkeypatch.setenv("OMNI_SPLIT_TC", frac)
    V, _ = check(w.levels, x, dtype="ci8", tol=TOL_MIXED, precision="mixed")
    assert relerr_per_channel(V, tc_only) <= 2e-5
    # several chunks, so both stream slots and the split events are reused
    monkeypatch.setenv("OMNI_CHUNK_MB", "8")
    V2 = gpu_vis(w.levels, x, dtype="ci8", precision="mixed")
    assert relerr_per_channel(V2, V) <= 2e-5


def test_expired_tensor_core_wait_is_reported(monkeypatch):
    """A bounded device wait that runs out returns OMNI_ERR_TIMEOUT; the context stays usable.

    The test hook makes the first tcgen05 wait wait for a phase that never comes,
    with a budget of ~0.5 ms, so nothing hangs or faults."""
    w = synth.workload("hier2")
    x = synth.voltages(w, channels=1, samples=3).cuda()
    monkeypatch.setenv("OMNI_MIXED_LAGSUM", "0")
    monkeypatch.setenv("OMNI_TCGEN05", "1")
    monkeypatch.setenv("OMNI_TEST_FORCE_TIMEOUT", "1")
    with omni.Plan(w.levels, 1, dtype="ci8", precision="mixed") as plan:
        plan.correlate(x)
        with pytest.raises(omni.OmniError) as e:
            plan.visibilities()
        assert e.value.status == 6
    monkeypatch.delenv("OMNI_TEST_FORCE_TIMEOUT")
    V = gpu_vis(w.levels, x.cpu(), dtype="ci8", precision="mixed")
    assert np.isfinite(V).all()


@pytest.mark.parametrize("precision", ["mixed", "mixed_bf16"])
def test_expired_lag_sum_wait_is_reported(monkeypatch, precision):
    """The lag-sum kernel's bounded waits: with the test hook its converters wait for
    a phase that never comes (budget ~0.5 ms), every CTA gives up, drains its copies,
    frees its tensor memory and sets the error word; the host reports OMNI_ERR_TIMEOUT
    and the next plan on the same context is correct."""
    w = synth.workload("hier2")
    x = synth.voltages(w, channels=2, samples=40)
    monkeypatch.setenv("OMNI_TEST_FORCE_TIMEOUT", "1")
    with omni.Plan(w.levels, 2, dtype="ci8", precision=precision) as plan:
        plan.correlate(x.cuda())
        with pytest.raises(omni.OmniError) as e:
            plan.visibilities()
        assert e.value.status == 6
    monkeypatch.delenv("OMNI_TEST_FORCE_TIMEOUT")
    check(w.levels, x, dtype="ci8", tol=TOL_MIXED, precision=precision)


@pytest.mark.parametrize("precision, overlap", [("fp32", "1"), ("mixed", "1"), ("mixed", "0")])
def test_correlate_replays_from_a_cuda_graph(precision, overlap, monkeypatch):
    """omni_correlate (with and without the two streams of overlapped chunk
    passes) can be captured once and replayed: two replays accumulate twice one
    call's |F|^2."""
    monkeypatch.setenv("OMNI_OVERLAP", overlap)
    w = synth.workload("hier2")
    x = synth.voltages(w, channels=2, samples=30).cuda()
    with omni.Plan(w.levels, 2, dtype="ci8", precision=precision) as plan:
        plan.correlate(x)
        once = plan.visibilities(reset=True).cpu().numpy()
        torch.cuda.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            plan.correlate(x)
        graph.replay()
        graph.replay()
        twice = plan.visibilities(reset=True).cpu().numpy()
    assert relerr_per_channel(twice, 2 * once) <= 1e-6
