"""Host-side logic of the surrogate (no GPU): the layer table and parameter
layout agree with the oracle, layout conversions round-trip, the learning-rate
schedule and the profile metric behave as defined."""
import math

import numpy as np
import pytest
import torch

from oracle import unet_oracle as U
from paper_2604_13929_gb300 import spnn, surrogate


@pytest.mark.parametrize("c0", [16, 32])
def test_layer_table_and_parameter_layout_match_the_oracle(c0):
    assert [t[:4] for t in U.layer_table(c0)] == spnn.layer_table(c0)
    P = U.init_params(c0, 3)
    flat = spnn.flatten_params(P, c0)
    assert flat.size == spnn.init_params(c0, 1).size
    back = spnn.unflatten_params(flat, U.layer_table(c0), c0)
    for name in list(P):
        np.testing.assert_array_equal(back[name][0], P[name][0])
        np.testing.assert_array_equal(back[name][1], P[name][1])


def test_init_params_scales():
    c0 = 16
    flat = spnn.init_params(c0, 5).astype(np.float64)
    off = 0
    for _, kind, ci, co in spnn.layer_table(c0):
        taps = 27 if kind == "conv3" else 8
        n = taps * ci * co
        w = flat[off:off + n]
        fan_in = ci if kind == "up" else taps * ci
        assert abs(w.std() / math.sqrt(2.0 / fan_in) - 1) < 0.1
        assert np.all(flat[off + n:off + n + co] == 0)
        off += n + co
    assert flat.size == off + c0 + 1


def test_plane_layout_round_trip():
    x = torch.randn(2, 3, 4, 5, 32)
    p = spnn.to_planes(x)
    assert p.shape == (4, 2, 3, 4, 5, 8)
    assert torch.equal(p[1, 0, 2, 3, 4], x[0, 2, 3, 4, 8:16])
    assert torch.equal(spnn.from_planes(p), x)


def test_cosine_schedule():
    lrs = [surrogate.cosine_lr(s, 200, 1e-3, 1e-5, warmup=20) for s in range(200)]
    assert lrs[0] == pytest.approx(1e-3 / 20)
    assert lrs[19] == pytest.approx(1e-3)
    assert lrs[-1] == pytest.approx(1e-5, rel=1e-2)
    assert all(a >= b for a, b in zip(lrs[19:], lrs[20:]))


def test_profile_rms_definition():
    rng = np.random.default_rng(0)
    ref = rng.uniform(0.5, 2.0, (3, 2, 64))
    assert np.all(surrogate.profile_rms(ref, ref) == 0)
    # a uniform 1 % error gives a fluence-weighted relative RMS of exactly 1 %
    np.testing.assert_allclose(surrogate.profile_rms(ref * 1.01, ref), 0.01, rtol=1e-12)
    # layers missing in one phase are skipped, not counted
    r2 = ref.copy()
    r2[0, 1, :10] = np.nan
    assert np.isfinite(surrogate.profile_rms(r2 * 1.02, r2)[0, 1])
