"""CPU-only checks of the C ABI: the library loads, exports every declared entry
point, and its host-side tables match the oracle bit for bit."""
import os
import re

import numpy as np
import pytest

from oracle import oracle
from paper_0909_0001_gb300 import omni, synth
from paper_0909_0001_gb300.build import INCLUDE, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build()
    return omni.load()


def declared_entry_points():
    names = set()
    for h in os.listdir(INCLUDE):
        if h.endswith(".h"):
            text = open(os.path.join(INCLUDE, h)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(omni_[a-z_]+)\s*\(", text))
    return sorted(names)


def test_every_declared_symbol_is_exported(lib):
    names = declared_entry_points()
    assert "omni_correlate" in names and "omni_plan_create" in names
    for name in names:
        assert hasattr(lib, name), f"{name} declared in include/ but not exported"
    assert set(omni.EXPORTS) <= set(names)


LAYOUTS = {
    "warmup_2level": synth.paper_fixture("warmup_2level"),
    "three_level": synth.paper_fixture("three_level"),
    "blocks": synth.paper_fixture("blocks"),
    "interleaved": synth.paper_fixture("interleaved"),
    "sheared": synth.hierarchy([(5, 3), (3, 4), (2, 2)], [0.2, 1.3, 2.9], [0.1, -0.2, 0.25]),
    "hier2": synth.workload("hier2").levels,
}


@pytest.mark.parametrize("name", sorted(LAYOUTS))
def test_baseline_tables_match_oracle(lib, name):
    levels = LAYOUTS[name]
    dims = synth.lattice_dims(levels)
    dm, red, dr = omni.baselines(levels)
    odm, ored = oracle.lag_table(dims)
    np.testing.assert_array_equal(dm, odm)
    np.testing.assert_array_equal(red, ored)
    np.testing.assert_allclose(dr, oracle.baseline_vectors(levels, odm), rtol=0, atol=1e-9)
    N, Q = omni.lattice_shape(levels)
    assert N == int(np.prod(dims)) and Q == len(odm)


def test_collision_verdicts_match_oracle(lib):
    ok = [synth.paper_fixture("interleaved"), synth.paper_fixture("three_level"),
          synth.paper_fixture("warmup_2level"), [synth.Level(1, 1)]]
    bad = [[synth.Level(4, 1, (1, 0, 0, 1)), synth.Level(2, 1, (2, 0, 0, 1))],
           [synth.Level(3, 3, (1, 0, 0, 1)), synth.Level(2, 2, (0, 0, 0, 0))],
           [synth.Level(2, 1, (0, 0, 0, 0))]]
    for levels in ok + bad:
        expect = oracle.collides(levels)
        if expect:
            with pytest.raises(omni.OmniError) as e:
                omni.baselines(levels)
            assert e.value.status == 2
        else:
            omni.baselines(levels)
    assert not any(oracle.collides(lv) for lv in ok)
    assert all(oracle.collides(lv) for lv in bad)


@pytest.mark.parametrize("levels, status", [
    ([], 1),
    ([synth.Level(0, 3)], 1),
    ([synth.Level(3, -1)], 1),
    ([synth.Level(3, 3, (float("nan"), 0, 0, 1))], 1),
    ([synth.Level(4096, 2)], 3),        # padded axis 8192 > 4096
    ([synth.Level(513, 2)], 3),         # padded axis 1026: not a power of two and > 1024
    ([synth.Level(2, 2)] * 9, 1),       # more than 8 levels
])
def test_invalid_hierarchies_are_rejected(lib, levels, status):
    with pytest.raises(omni.OmniError) as e:
        omni.lattice_shape(levels)
    assert e.value.status == status
    assert omni.load().omni_last_error()


def test_status_strings(lib):
    for code, name in omni.STATUS_NAMES.items():
        assert lib.omni_status_string(code).decode() == name


def test_plan_create_rejects_bad_arguments_without_touching_the_gpu(lib):
    import ctypes
    h = ctypes.c_void_p()
    lv = omni._levels([synth.Level(4, 4)])
    assert lib.omni_plan_create(lv, 1, 0, 0, 0, ctypes.byref(h)) == 1       # no channels
    assert lib.omni_plan_create(lv, 1, 1, 7, 0, ctypes.byref(h)) == 1       # bad dtype
    assert lib.omni_plan_create(lv, 1, 1, 0, 9, ctypes.byref(h)) == 1       # bad precision
    assert lib.omni_plan_create(lv, 1, 1, 0, 0, None) == 1                  # no out pointer
    assert lib.omni_correlate(None, None, 1, None) == 1
    assert lib.omni_visibilities(None, None, 1, None) == 1


@pytest.mark.parametrize("name", ["three_level", "interleaved", "blocks"])
def test_radial_bins_match_oracle(lib, name):
    levels = synth.paper_fixture(name)
    for w, nb in ((1.0, 40), (7.5, 12)):
        b, pairs = omni.radial_bins(levels, w, nb)
        ob, opairs = oracle.radial_bins(levels, w, nb)
        np.testing.assert_array_equal(b, ob)
        np.testing.assert_array_equal(pairs, opairs)


@pytest.mark.parametrize("levels", [
    [synth.Level(4, 1, (2.0, 0.0, 0.0, 1.0)), synth.Level(2, 1, (5.0, 0.0, 0.0, 1.0))],
    synth.paper_fixture("interleaved"),
    synth.hierarchy([(3, 2), (2, 3)], [0.4, 2.0], [0.2, -0.1]),
    synth.paper_fixture("warmup_2level"),
])
def test_unique_baselines_match_oracle(lib, levels):
    g, dr, pairs = omni.unique_baselines(levels)
    og, odr, opairs = oracle.unique_baselines(levels)
    np.testing.assert_array_equal(g, og)
    np.testing.assert_allclose(dr, odr, rtol=0, atol=1e-9)
    np.testing.assert_array_equal(pairs, opairs)


def test_epilogue_rejects_bad_arguments(lib):
    with pytest.raises(omni.OmniError):
        omni.radial_bins([synth.Level(4, 4)], 0.0, 10)
    assert lib.omni_sum_groups(None, 1, 1, None, 1, None, None) == 1


def test_tile_plans_check_geometry_without_a_gpu(lib):
    tile = synth.Level(4, 4, (1.0, 0.0, 0.0, 1.0))
    with pytest.raises(omni.OmniError) as e:     # tile 1 overlaps tile 0 exactly
        omni.TilePlan(tile, [[0.0, 0.0], [2.0, 1.0]], 1)
    assert e.value.status == 2
    with pytest.raises(omni.OmniError) as e:
        omni.TilePlan(tile, [[0.0, 0.0], [float("nan"), 1.0]], 1)
    assert e.value.status == 1
    with pytest.raises(omni.OmniError) as e:
        omni.TilePlan(tile, np.zeros((0, 2)), 1)
    assert e.value.status == 1


def test_fengine_argument_checks_without_a_gpu(lib):
    f = lib.omni_fengine
    # (n_antennas, n_samples, F, taps, out dtype) -> status; no pointer is touched
    assert f(None, 4, 64, 3, 1, None, None, 1.0, 1, None, None, 0, None, None) == 1     # F not 2^k
    assert f(None, 4, 64, 8192, 1, None, None, 1.0, 1, None, None, 0, None, None) == 1  # F too large
    assert f(None, 4, 64, 8, 0, None, None, 1.0, 1, None, None, 0, None, None) == 1     # no taps
    assert f(None, 4, 64, 8, 1, None, None, 1.0, 7, None, None, 0, None, None) == 1     # bad dtype
    assert f(None, 4, 64, 32, 2, None, None, 1.0, 1, None, None, 0, None, None) == 0    # no frame
    assert f(None, 4, 64, 8, 1, None, None, 1.0, 1, None, None, 0, None, None) == 1     # NULL buffers
    assert lib.omni_fengine_scratch_bytes(4, 2 * 512 * 5 + 3, 512, 1) == 8 * 4 * 5 * 512
    assert lib.omni_fengine_scratch_bytes(4, 2 * 8 * 5 + 3, 8, 1) == 0       # fused pass, no scratch
    assert lib.omni_fengine_scratch_bytes(4, 100, 1024, 2) == 0              # no frame


def test_library_has_no_unresolved_internal_symbols(lib):
    """Every function the library calls inside itself is defined in it (an
    internal declaration in the wrong namespace links as an undefined symbol)."""
    import shutil
    import subprocess
    from paper_0909_0001_gb300.build import LIB
    if shutil.which("nm") is None:
        pytest.skip("nm not available")
    out = subprocess.run(["nm", "-D", "--undefined-only", LIB], capture_output=True, text=True).stdout
    bad = [l for l in out.splitlines() if "omni" in l or "_GLOBAL__N" in l]
    assert not bad, bad


def test_beam_and_tuned_plan_errors_without_a_gpu(lib):
    with pytest.raises(omni.OmniError) as e:          # one level: no coarser axes to correlate
        omni.BeamPlan([synth.Level(8, 8)], 1)
    assert e.value.status == 3
    import ctypes
    h = ctypes.c_void_p()
    with pytest.raises(omni.OmniError) as e:          # the tuner needs voltages to time
        omni._check(lib.omni_plan_create_tuned(omni._levels([synth.Level(4, 4)]), 1, 1, 0, 0, None, 1,
                                                None, None, ctypes.byref(h)))
    assert e.value.status == 1


def test_fengine_wrapper_rejects_host_tensors():
    import torch
    with pytest.raises(ValueError):
        omni.fengine(torch.zeros((4, 64), dtype=torch.int8), 8)
    with pytest.raises(ValueError):
        omni.fengine(torch.zeros((4, 64), dtype=torch.int16), 8)


def test_noalloc_wrapper_checks_arguments_before_the_library_call(lib):
    """correlate_noalloc rejects wrong shapes, element types, sizes and devices
    with ValueError/TypeError before it calls the library (CPU tensors here:
    every bad case must be caught by the shape and type checks first)."""
    import torch
    levels = synth.hierarchy([(4, 4), (2, 3)], [0.0, 0.5], [0.0, 0.1])
    N, Q = omni.lattice_shape(levels)
    good_ci8 = torch.zeros((2, 3, N, 2), dtype=torch.int8)
    out = torch.zeros((2, Q), dtype=torch.complex128)
    with pytest.raises(TypeError):     # int8 data passed as cf32 would be read 4x past its end
        omni.correlate_noalloc(levels, good_ci8, "cf32", out)
    with pytest.raises(TypeError):
        omni.correlate_noalloc(levels, good_ci8.float(), "ci8", out)
    with pytest.raises(ValueError):    # wrong antenna count
        omni.correlate_noalloc(levels, torch.zeros((2, 3, N + 1, 2), dtype=torch.int8), "ci8", out)
    with pytest.raises(ValueError):    # not [C][T][N][2]
        omni.correlate_noalloc(levels, torch.zeros((2, 3, N), dtype=torch.int8), "ci8", out)
    with pytest.raises(ValueError):    # out too small for C x Q
        omni.correlate_noalloc(levels, good_ci8, "ci8", torch.zeros((1, Q), dtype=torch.complex128))
    with pytest.raises(TypeError):
        omni.correlate_noalloc(levels, good_ci8, "ci8", out.real.contiguous())
    with pytest.raises(ValueError):    # unknown dtype string
        omni.correlate_noalloc(levels, good_ci8, "cf16", out)
    with pytest.raises(ValueError):    # host tensors: the last check, still before any launch
        omni.correlate_noalloc(levels, good_ci8, "ci8", out)
