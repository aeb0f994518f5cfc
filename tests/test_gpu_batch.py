"""Batch plans: many independent arrays of uneven hierarchies in one plan."""
import numpy as np
import pytest
import torch

from oracle import oracle
from paper_0909_0001_gb300 import omni, synth

pytestmark = pytest.mark.gpu


def _arrays():
    return [
        [synth.Level(8, 8)],
        [synth.Level(8, 8, synth.sheared_rotation(1.0, 0.4, 0.1))],   # same shape: one run
        synth.hierarchy([(4, 4), (8, 8)], [0.1, 0.9], [0.0, 0.2]),
        [synth.Level(5, 3)],                                           # non-power-of-two
        [synth.Level(8, 8)],                                           # same shape, new run
        synth.hierarchy([(4, 4), (16, 16)], [0.3, 1.2], [0.1, -0.2]),
    ]


def _rel(a, b):
    return float(np.max(np.linalg.norm(a - b, axis=1) / np.linalg.norm(b, axis=1)))


@pytest.mark.parametrize("dtype", ["cf32", "ci8"])
def test_batch_matches_oracle_and_single_plans(dtype):
    arrays = _arrays()
    C, T = 2, 3
    volts = synth.batch_voltages(arrays, C, T, dtype=dtype)
    with omni.BatchPlan(arrays, C, dtype=dtype) as plan:
        assert plan.antennas == [int(np.prod(synth.lattice_dims(a))) for a in arrays]
        plan.correlate(plan.pack([v.cuda() for v in volts]))
        per_array = [v.cpu().numpy() for v in plan.unpack(plan.visibilities())]
    for a, (levels, v) in enumerate(zip(arrays, volts)):
        ref = oracle.correlate(synth.lattice_dims(levels), v)
        assert _rel(per_array[a], ref) <= 1e-5, a
        with omni.Plan(levels, C, dtype=dtype) as single:
            single.correlate(v.cuda())
            np.testing.assert_allclose(per_array[a], single.visibilities().cpu().numpy(),
                                       rtol=0, atol=1e-9 * np.abs(ref).max())


def test_batch_host_path_and_reset():
    arrays = _arrays()
    C = 3
    first = synth.batch_voltages(arrays, C, 4, dtype="ci8", seed=5)
    second = synth.batch_voltages(arrays, C, 6, dtype="ci8", seed=6)
    with omni.BatchPlan(arrays, C, dtype="ci8") as plan:
        plan.correlate_host(plan.pack(first))
        plan.visibilities_host(reset=True)
        plan.correlate_host(plan.pack(second).pin_memory())
        host = plan.unpack(plan.visibilities_host())
        plan.correlate(plan.pack([v.cuda() for v in second]))
        dev = plan.unpack(plan.visibilities().cpu())
    for h, d in zip(host, dev):
        np.testing.assert_array_equal(h.numpy(), d.numpy())


def test_batch_rejects_a_colliding_array():
    bad = [synth.Level(4, 1, (1.0, 0.0, 0.0, 1.0)), synth.Level(2, 1, (2.0, 0.0, 0.0, 1.0))]
    with pytest.raises(omni.OmniError) as e:
        omni.BatchPlan([[synth.Level(8, 8)], bad], 1)
    assert e.value.status == 2
    assert "array 1" in str(e.value)
