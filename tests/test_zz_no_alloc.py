"""omni_correlate_noalloc: the entry point for callers that cannot allocate
device memory (allocator hooks or pools owned by another framework, memory
reserved up front, real-time loops that forbid allocation).  It keeps its
scratch in a static device array inside the library; its results must match
the plan API's, call after call, because the array keeps the previous call's
contents and the accumulator has to be cleared each time.

Kept in a file of its own that pytest collects last.
"""
import numpy as np
import pytest
import torch

from oracle import oracle
from paper_0909_0001_gb300 import omni, synth

pytestmark = pytest.mark.gpu

TOL_FP32 = 1e-5


def plan_vis(levels, x, dtype):
    with omni.Plan(levels, x.shape[0], dtype=dtype) as plan:
        plan.correlate(x)
        return plan.visibilities().cpu().numpy()


def relerr(a, b):
    return float(np.max(np.linalg.norm(a - b, axis=1) / np.linalg.norm(b, axis=1)))


@pytest.mark.parametrize("levels, dtype, C, T", [
    (synth.workload("hier2").levels, "ci8", 2, 24),
    (synth.hierarchy([(8, 4), (4, 3), (2, 2)], [0.1, 0.9, 2.0], [0.0, 0.2, -0.1]), "cf32", 3, 5),
    (synth.paper_fixture("three_level"), "cf32", 1, 3),
    # a 3-point axis (padded to 6): its direct-DFT twiddles live in the static array
    (synth.hierarchy([(3, 4), (2, 2)], [0.0, 0.4], [0.0, 0.15]), "cf32", 2, 6),
])
def test_noalloc_matches_plan_api_and_oracle_on_consecutive_calls(levels, dtype, C, T):
    """Two calls in a row (the array keeps the first call's contents), each
    checked against the plan API and against the CPU FP64 oracle."""
    dims = synth.lattice_dims(levels)
    _, Q = omni.lattice_shape(levels)
    for call, seed in enumerate((101, 202)):
        x = synth.random_complex(dims, C, T, seed=seed, dtype=dtype, sigma=20.0).cuda()
        out = torch.empty((C, Q), dtype=torch.complex128, device="cuda")
        got = omni.correlate_noalloc(levels, x, dtype, out).cpu().numpy()
        ref = plan_vis(levels, x, dtype)
        err = relerr(got, ref)
        assert err <= TOL_FP32, f"call {call}: relative error {err:.3e} against the plan API"
        err_o = relerr(got, oracle.correlate(dims, x.cpu()))
        assert err_o <= TOL_FP32, f"call {call}: relative error {err_o:.3e} against the oracle"


def test_noalloc_zero_samples_gives_zero_visibilities():
    """T = 0 after a call with data: the cleared accumulator gives exact zeros."""
    levels = synth.hierarchy([(4, 4), (3, 2)], [0.0, 0.3], [0.0, 0.1])
    dims = synth.lattice_dims(levels)
    _, Q = omni.lattice_shape(levels)
    x = synth.random_complex(dims, 2, 4, seed=7, dtype="ci8", sigma=20.0).cuda()
    out = torch.empty((2, Q), dtype=torch.complex128, device="cuda")
    omni.correlate_noalloc(levels, x, "ci8", out)
    assert float(out.abs().max()) > 0
    out.fill_(1e300)
    omni.correlate_noalloc(levels, x[:, :0].contiguous(), "ci8", out)
    assert float(out.abs().max()) == 0.0


def test_noalloc_inverse_in_several_channel_groups():
    """20 channels of a 256 x 256 grid: 40 MiB of accumulator leave room for
    fewer than 20 channels of inverse buffer, so the inverse runs in groups."""
    levels = [synth.Level(256, 256)]
    dims = synth.lattice_dims(levels)
    _, Q = omni.lattice_shape(levels)
    C = 20
    for seed in (11, 12):
        x = synth.random_complex(dims, C, 2, seed=seed, dtype="ci8", sigma=20.0).cuda()
        out = torch.empty((C, Q), dtype=torch.complex128, device="cuda")
        got = omni.correlate_noalloc(levels, x, "ci8", out).cpu().numpy()
        assert relerr(got, plan_vis(levels, x, "ci8")) <= TOL_FP32


def test_noalloc_rejects_problems_beyond_its_scratch():
    w = synth.workload("hier2")            # 64 channels x 2 MiB of accumulator > 64 MiB
    x = torch.zeros((w.channels, 1, w.n_antennas, 2), dtype=torch.int8, device="cuda")
    out = torch.empty((w.channels, omni.lattice_shape(w.levels)[1]), dtype=torch.complex128,
                      device="cuda")
    with pytest.raises(omni.OmniError) as e:
        omni.correlate_noalloc(w.levels, x, "ci8", out)
    assert e.value.status == 3
    assert "static array holds" in str(e.value)
