"""GPU parity of the F-engine (Appendix A step 2) against the CPU FP64 oracle.

Bar: the FP32 channel voltages within relative Frobenius error 1e-5 of the
oracle's; the int8 codes bit-exact with the oracle's quantiser applied to the
same FP32 values (both sides decide on the same float)."""
import numpy as np
import pytest
import torch

from oracle import oracle
from paper_0909_0001_gb300 import omni

pytestmark = pytest.mark.gpu

TOL = 1e-5


def relerr(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def run(raw, F, P=1, window=None, gains=None, scale=1.0, dtype="cf32"):
    out = omni.fengine(raw.cuda(), F, P, window=None if window is None else torch.from_numpy(window),
                       gains=None if gains is None else torch.from_numpy(gains), scale=scale, dtype=dtype)
    torch.cuda.synchronize()
    o = out.cpu().numpy()
    return o[..., 0] + 1j * o[..., 1] if dtype == "cf32" else o


@pytest.mark.parametrize("N, F, P, extra", [(3, 8, 1, 0), (5, 64, 4, 17), (33, 256, 8, 3), (2, 2, 1, 1),
                                            (7, 4096, 2, 0), (40, 32, 3, 31),
                                            # F = 64 with 16-byte rows: the radix-8 x 8 kernel, a
                                            # partial 32-antenna group, one tap and eight
                                            (40, 64, 4, 0), (33, 64, 1, 16), (70, 64, 8, 32)])
def test_fengine_matches_oracle(N, F, P, extra):
    rng = np.random.default_rng(N * 1000 + F)
    T = 6
    S = (T + P - 1) * 2 * F + extra
    raw = torch.from_numpy(rng.integers(-128, 128, size=(N, S)).astype(np.int8))
    w = rng.standard_normal(P * 2 * F).astype(np.float32)
    g = (rng.standard_normal((F, N)) + 1j * rng.standard_normal((F, N))).astype(np.complex64)
    Y = run(raw, F, P, w, g, 0.125)
    ref = oracle.fengine(raw.numpy(), F, P, window=w.astype(np.float64), gains=g.astype(np.complex128),
                         scale=0.125)
    assert Y.shape == ref.shape
    assert relerr(Y, ref) <= TOL


@pytest.mark.parametrize("F", [64, 128, 512])  # the radix-8 x 8 pass, the fused pass, the two-kernel pass
def test_fengine_int8_codes_are_the_quantised_floats(F):
    rng = np.random.default_rng(7)
    N, P, T = 9, 4, 10
    raw = torch.from_numpy(rng.integers(-128, 128, size=(N, (T + P - 1) * 2 * F)).astype(np.int8))
    w = (np.hanning(P * 2 * F) * np.sinc(np.linspace(-P / 2, P / 2, P * 2 * F))).astype(np.float32)
    scale = 0.07 * (128 / F) ** 0.5
    Yf = run(raw, F, P, w, None, scale, "cf32")
    Yq = run(raw, F, P, w, None, scale, "ci8")
    f32 = np.stack([Yf.real, Yf.imag], axis=-1).astype(np.float32)
    np.testing.assert_array_equal(Yq, oracle.quantize(f32))
    assert np.abs(Yq).max() == 127                      # some codes clip
    assert (Yq != 0).mean() > 0.5


def test_fengine_feeds_the_correlator():
    """Channel voltages go straight into a plan: C = F channels, T frames."""
    from paper_0909_0001_gb300 import synth
    levels = [synth.Level(4, 4), synth.Level(2, 2, (6.0, 0.0, 0.0, 6.0))]
    N, F = 64, 16
    rng = np.random.default_rng(8)
    raw = torch.from_numpy(rng.integers(-60, 60, size=(N, 2 * F * 12)).astype(np.int8))
    volts = omni.fengine(raw.cuda(), F, 1, scale=0.1, dtype="ci8")
    with omni.Plan(levels, F, dtype="ci8") as plan:
        plan.correlate(volts)
        V = plan.visibilities().cpu().numpy()
    ref = oracle.correlate(synth.lattice_dims(levels), volts.cpu())
    assert relerr(V, ref) <= TOL


def test_fengine_rejects_bad_arguments():
    raw = torch.zeros((4, 64), dtype=torch.int8, device="cuda")
    for F, P in ((3, 1), (1, 1), (8192, 1), (8, 0), (8, 65)):
        with pytest.raises(omni.OmniError):
            omni.fengine(raw, F, P)
    # too few samples for one frame: no frames, nothing written
    out = omni.fengine(raw, 32, 2)
    assert out.shape[1] == 0
