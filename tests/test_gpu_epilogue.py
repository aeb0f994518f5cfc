"""GPU epilogue: visibilities summed by physical-baseline group (radial bins,
coincident baselines) against the oracle's plain sums."""
import numpy as np
import pytest
import torch

from oracle import oracle
from paper_0909_0001_gb300 import omni, synth

pytestmark = pytest.mark.gpu

COINCIDENT = [synth.Level(4, 1, (2.0, 0.0, 0.0, 1.0)), synth.Level(2, 1, (5.0, 0.0, 0.0, 1.0))]


def _rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def test_radial_profile_matches_oracle():
    levels = synth.paper_fixture("three_level")
    dims = synth.lattice_dims(levels)
    x = synth.random_complex(dims, 3, 2, seed=13)
    with omni.Plan(levels, 3) as plan:
        plan.correlate(x.cuda())
        vis = plan.visibilities()
    bins, pairs = omni.radial_bins(levels, 2.5, 40)
    out = omni.sum_groups(vis, torch.from_numpy(bins).cuda(), 40).cpu().numpy()
    expect = oracle.group_sum(vis.cpu().numpy(), bins, 40)
    assert _rel(out, expect) < 1e-12
    # the layout map of ones: the radial profile is the pair-distance histogram
    T = 2
    with omni.Plan(levels, 1) as plan:
        plan.correlate(synth.all_ones(dims, 1, T).cuda())
        prof = omni.sum_groups(plan.visibilities(), torch.from_numpy(bins).cuda(), 40).cpu().numpy()
    np.testing.assert_array_equal(np.rint(prof.real[0]).astype(np.int64), T * pairs)


def test_coincident_baselines_merge():
    group, reps, _ = omni.unique_baselines(COINCIDENT)
    x = synth.random_complex(synth.lattice_dims(COINCIDENT), 2, 4, seed=14)
    with omni.Plan(COINCIDENT, 2) as plan:
        plan.correlate(x.cuda())
        vis = plan.visibilities()
    merged = omni.sum_groups(vis, torch.from_numpy(group).cuda(), len(reps)).cpu().numpy()
    ref = oracle.group_sum(oracle.correlate(synth.lattice_dims(COINCIDENT), x), group, len(reps))
    assert _rel(merged, ref) < 1e-5


def test_many_groups_path():
    """More groups than fit in shared memory: the global-atomics kernel."""
    C, Q, G = 3, 50000, 9000
    rng = np.random.default_rng(0)
    v = rng.normal(size=(C, Q)) + 1j * rng.normal(size=(C, Q))
    g = rng.integers(-1, G, Q).astype(np.int32)
    out = omni.sum_groups(torch.from_numpy(v).cuda(), torch.from_numpy(g).cuda(), G).cpu().numpy()
    expect = np.zeros((C, G), dtype=complex)
    for c in range(C):
        np.add.at(expect[c], g[g >= 0], v[c, g >= 0])
    assert _rel(out, expect) < 1e-12
