"""GPU parity of the beam-space plan (Appendix A, steps 4-5) against the CPU
FP64 oracle's direct-DFT-then-brute-force definition.

Bar: relative Frobenius error per channel <= 1e-5 (FP32 path); the all-ones
pointing power is exact after rounding."""
import numpy as np
import pytest
import torch

from oracle import oracle
from paper_0909_0001_gb300 import omni, synth

pytestmark = pytest.mark.gpu

TOL = 1e-5

LAYOUTS = {
    "4x2 on 3x2": [synth.Level(4, 2), synth.Level(3, 2, (5.0, 0.0, 0.0, 5.0))],
    "3x3 on 2x2 on 2x1": [synth.Level(3, 3), synth.Level(2, 2, (4.0, 0.5, 0.0, 4.0)),
                          synth.Level(2, 1, (10.0, 0.0, 0.0, 10.0))],
    "5x1 on 1x4": [synth.Level(5, 1), synth.Level(1, 4, (7.0, 0.0, 0.0, 7.0))],
    "16x16 on 3x5": [synth.Level(16, 16), synth.Level(3, 5, (20.0, 0.0, 0.0, 20.0))],
    "8x8 on 8x8": [synth.Level(8, 8), synth.Level(8, 8, (10.0, 0.0, 3.0, 10.0))],
    "128x2 on 2x2": [synth.Level(128, 2), synth.Level(2, 2, (200.0, 0.0, 0.0, 200.0))],
}


def beam_vis(levels, x, dtype="cf32"):
    C = x.shape[0]
    with omni.BeamPlan(levels, C, dtype=dtype) as plan:
        plan.correlate(x.cuda())
        V = plan.visibilities().cpu().numpy()
        return V.reshape(C, plan.n_coarse_lags, plan.n_beams)


def relerr_per_channel(V, ref):
    num = np.linalg.norm((V - ref).reshape(V.shape[0], -1), axis=1)
    den = np.maximum(np.linalg.norm(ref.reshape(ref.shape[0], -1), axis=1), 1e-300)
    return float(np.max(num / den))


@pytest.mark.parametrize("name", sorted(LAYOUTS))
@pytest.mark.parametrize("dtype", ["cf32", "ci8"])
def test_beams_match_oracle(name, dtype):
    levels = LAYOUTS[name]
    dims = synth.lattice_dims(levels)
    x = synth.random_complex(dims, 2, 5, seed=71, dtype=dtype, sigma=30.0 if dtype == "ci8" else 1.0)
    V = beam_vis(levels, x, dtype)
    ref = oracle.beam_correlate(dims, x)
    assert relerr_per_channel(V, ref) <= TOL


def test_beams_all_ones_exact():
    levels = LAYOUTS["8x8 on 8x8"]
    dims = synth.lattice_dims(levels)
    T = 3
    V = beam_vis(levels, synth.all_ones(dims, 1, T, dtype="ci8"), "ci8")
    _, red, _ = omni.baselines(levels[1:])
    nb = dims[0] * dims[1]
    np.testing.assert_array_equal(np.rint(V[0, :, 0].real).astype(np.int64), nb * nb * T * red)
    assert np.abs(V[0, :, 1:]).max() < 1e-6 * nb * nb * T


def test_beams_many_chunks_and_split_calls(monkeypatch):
    """Several chunks (tiny chunk buffers) and several correlate calls accumulate."""
    monkeypatch.setenv("OMNI_CHUNK_MB", "1")
    levels = LAYOUTS["16x16 on 3x5"]
    dims = synth.lattice_dims(levels)
    x = synth.random_complex(dims, 3, 7, seed=72)
    with omni.BeamPlan(levels, 3) as plan:
        plan.correlate(x[:, :4].contiguous().cuda())
        plan.correlate(x[:, 4:].contiguous().cuda())
        V = plan.split(plan.visibilities()).cpu().numpy()
    ref = oracle.beam_correlate(dims, x).reshape(V.shape)
    assert relerr_per_channel(V, ref) <= TOL


def test_beams_hier2_full_size_channel():
    """The 2-level workload at full size; one channel checked in full (all
    pointings and coarse lags) against the oracle at all 1024 samples."""
    w = synth.workload("hier2")
    xd = synth.voltages(w, device="cuda")
    with omni.BeamPlan(w.levels, w.channels, dtype=w.dtype) as plan:
        plan.correlate(xd)
        V = plan.visibilities().cpu().numpy().reshape(w.channels, plan.n_coarse_lags, plan.n_beams)
    x0 = xd[17:18].cpu()
    del xd
    ref = oracle.beam_correlate(w.dims, x0)
    assert relerr_per_channel(V[17:18], ref) <= TOL


def test_beams_host_path_and_layout():
    levels = LAYOUTS["4x2 on 3x2"]
    dims = synth.lattice_dims(levels)
    x = synth.random_complex(dims, 2, 4, seed=73)
    with omni.BeamPlan(levels, 2) as plan:
        assert plan.beam_shape == (4, 2) and plan.n_beams == 8
        assert plan.n_coarse_lags == len(omni.baselines(levels[1:])[1])
        assert plan.padded[:2] == [4, 2]
        plan.correlate_host(x)
        Vh = plan.visibilities_host().numpy()
        plan.correlate(x.cuda())
        Vd = plan.visibilities().cpu().numpy()
    np.testing.assert_array_equal(Vh, Vd)


def test_beams_reject_single_level_and_trivial_coarse_levels():
    with pytest.raises(omni.OmniError) as e:
        omni.BeamPlan([synth.Level(8, 8)], 1)
    assert e.value.status == 3
    with pytest.raises(omni.OmniError) as e:
        omni.BeamPlan([synth.Level(8, 8), synth.Level(1, 1)], 1)
    assert e.value.status == 3
