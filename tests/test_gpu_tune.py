"""The autotuner: candidates timed on the caller's voltages, the winner cached
in a JSON-lines file; tuned plans give the same visibilities as the oracle."""
import json

import numpy as np
import pytest

from oracle import oracle
from paper_0909_0001_gb300 import omni, synth

pytestmark = pytest.mark.gpu


def relerr_per_channel(V, ref):
    num = np.linalg.norm(V - ref, axis=1)
    den = np.maximum(np.linalg.norm(ref, axis=1), 1e-300)
    return float(np.max(num / den))


def test_tuned_fp32_plan_and_cache(tmp_path):
    levels = [synth.Level(8, 8), synth.Level(4, 4, (10.0, 1.0, -1.0, 10.0))]
    x = synth.random_complex(synth.lattice_dims(levels), 2, 16, seed=91)
    xd = x.cuda()
    cache = str(tmp_path / "tune.jsonl")
    plan = omni.Plan.tuned(levels, 2, xd, dtype="cf32", cache=cache)
    assert not plan.from_cache
    knobs = plan.knobs()
    plan.correlate(xd)
    V = plan.visibilities().cpu().numpy()
    plan.close()
    assert relerr_per_channel(V, oracle.correlate(synth.lattice_dims(levels), x)) <= 1e-5
    entries = [json.loads(line) for line in open(cache)]
    assert len(entries) == 1 and entries[0]["chunk_mb"] == knobs["chunk_mb"]
    again = omni.Plan.tuned(levels, 2, xd, dtype="cf32", cache=cache)
    assert again.from_cache and again.knobs() == knobs
    again.close()


def test_tuned_mixed_plan():
    w = synth.workload("hier2")
    x = synth.voltages(w, channels=1, samples=4)
    xd = x.cuda()
    plan = omni.Plan.tuned(w.levels, 1, xd, dtype="ci8", precision="mixed")
    plan.correlate(xd)
    V = plan.visibilities().cpu().numpy()
    knobs = plan.knobs()
    plan.close()
    assert knobs["chunk_mb"] in (384, 768, 1536, 3072)
    assert relerr_per_channel(V, oracle.correlate(w.dims, x)) <= 1e-4


def test_tuner_searches_the_radix_split_of_long_axes(tmp_path):
    """A 2048-point padded axis: the candidates include its three-step (16 x 16 x 8)
    and four-step (64 x 32) forms; the winner's split is in the cache and its
    visibilities match the oracle."""
    levels = [synth.Level(1024, 2, (1.0, 0.3, 0.0, 1.0))]
    dims = synth.lattice_dims(levels)
    x = synth.random_complex(dims, 1, 4, seed=92)
    xd = x.cuda()
    cache = str(tmp_path / "tune.jsonl")
    plan = omni.Plan.tuned(levels, 1, xd, dtype="cf32", cache=cache)
    plan.correlate(xd)
    V = plan.visibilities().cpu().numpy()
    plan.close()
    assert relerr_per_channel(V, oracle.correlate(dims, x)) <= 1e-5
    entries = [json.loads(line) for line in open(cache)]
    assert len(entries) == 1 and entries[0]["fft3"] in (0, 1)
    again = omni.Plan.tuned(levels, 1, xd, dtype="cf32", cache=cache)
    assert again.from_cache
    again.close()
