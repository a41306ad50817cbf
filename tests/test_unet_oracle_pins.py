"""Pins of the FP64 surrogate oracle against definitions it does not share code with:
brute-force loops, adjoint identities, closed forms and central finite differences."""
import itertools
import math

import numpy as np
import pytest

from oracle import unet_oracle as U


def _brute_conv3(x, w, b):
    B, D, H, W, C = x.shape
    y = np.zeros((B, D, H, W, w.shape[2]))
    for bb, z, yy, xx in itertools.product(range(B), range(D), range(H), range(W)):
        acc = b.copy()
        for kz, ky, kx in itertools.product(range(3), range(3), range(3)):
            zs, ys, xs = z + kz - 1, yy + ky - 1, xx + kx - 1
            if 0 <= zs < D and 0 <= ys < H and 0 <= xs < W:
                tap = kz * 9 + ky * 3 + kx
                for ci in range(C):
                    acc = acc + x[bb, zs, ys, xs, ci] * w[tap, ci]
        y[bb, z, yy, xx] = acc
    return y


def _brute_down(x, w, b):
    B, D, H, W, C = x.shape
    y = np.zeros((B, D // 2, H // 2, W // 2, w.shape[2]))
    for bb, z, yy, xx in itertools.product(range(B), range(D // 2), range(H // 2), range(W // 2)):
        acc = b.copy()
        for oz, oy, ox in itertools.product(range(2), range(2), range(2)):
            for ci in range(C):
                acc = acc + x[bb, 2 * z + oz, 2 * yy + oy, 2 * xx + ox, ci] * w[oz * 4 + oy * 2 + ox, ci]
        y[bb, z, yy, xx] = acc
    return y


def _brute_up(x, w, b):
    B, D, H, W, C = x.shape
    y = np.zeros((B, 2 * D, 2 * H, 2 * W, w.shape[2]))
    for bb, z, yy, xx in itertools.product(range(B), range(2 * D), range(2 * H), range(2 * W)):
        o = (z % 2) * 4 + (yy % 2) * 2 + (xx % 2)
        acc = b.copy()
        for ci in range(C):
            acc = acc + x[bb, z // 2, yy // 2, xx // 2, ci] * w[o, ci]
        y[bb, z, yy, xx] = acc
    return y


@pytest.fixture
def rng():
    return np.random.default_rng(11)


def test_conv3_matches_loops(rng):
    x = rng.standard_normal((2, 3, 4, 5, 2))
    w = rng.standard_normal((27, 2, 3))
    b = rng.standard_normal(3)
    np.testing.assert_allclose(U.conv3(x, w, b), _brute_conv3(x, w, b), rtol=1e-12, atol=1e-12)


def test_down_up_match_loops(rng):
    x = rng.standard_normal((2, 4, 2, 6, 3))
    w = rng.standard_normal((8, 3, 2))
    b = rng.standard_normal(2)
    np.testing.assert_allclose(U.down(x, w, b), _brute_down(x, w, b), rtol=1e-12, atol=1e-12)
    xs = rng.standard_normal((2, 2, 1, 3, 3))
    np.testing.assert_allclose(U.up(xs, w, b), _brute_up(xs, w, b), rtol=1e-12, atol=1e-12)


def test_conv3_single_taps_are_shifts(rng):
    x = rng.standard_normal((1, 4, 5, 6, 2))
    for tap, (dz, dy, dx) in enumerate(U._taps3()):
        w = np.zeros((27, 2, 2))
        w[tap] = np.eye(2)
        y = U.conv3(x, w)
        ref = np.zeros_like(x)
        D, H, W = x.shape[1:4]
        for z, yy, xx in itertools.product(range(D), range(H), range(W)):
            if 0 <= z + dz < D and 0 <= yy + dy < H and 0 <= xx + dx < W:
                ref[0, z, yy, xx] = x[0, z + dz, yy + dy, xx + dx]
        np.testing.assert_array_equal(y, ref)


def test_down_average_and_up_nearest(rng):
    x = rng.standard_normal((2, 4, 6, 2, 3))
    w = np.stack([np.eye(3) / 8.0] * 8)
    avg = x.reshape(2, 2, 2, 3, 2, 1, 2, 3).mean(axis=(2, 4, 6))
    np.testing.assert_allclose(U.down(x, w), avg, rtol=1e-14, atol=1e-15)
    w1 = np.stack([np.eye(3)] * 8)
    near = np.repeat(np.repeat(np.repeat(avg, 2, axis=1), 2, axis=2), 2, axis=3)
    np.testing.assert_allclose(U.up(avg, w1), near, rtol=1e-14, atol=1e-15)


def _inner(a, b):
    return float(np.sum(a * b))


def test_adjoint_identities(rng):
    """dgrad is the adjoint in x and wgrad the adjoint in W of each layer."""
    x = rng.standard_normal((2, 4, 6, 4, 3))
    w3 = rng.standard_normal((27, 3, 5))
    y3 = rng.standard_normal((2, 4, 6, 4, 5))
    lhs = _inner(U.conv3(x, w3), y3)
    assert math.isclose(lhs, _inner(x, U.conv3_dgrad(y3, w3)), rel_tol=1e-12)
    assert math.isclose(lhs, _inner(w3, U.conv3_wgrad(x, y3)[0]), rel_tol=1e-12)
    w2 = rng.standard_normal((8, 3, 5))
    yd = rng.standard_normal((2, 2, 3, 2, 5))
    lhs = _inner(U.down(x, w2), yd)
    assert math.isclose(lhs, _inner(x, U.down_dgrad(yd, w2)), rel_tol=1e-12)
    assert math.isclose(lhs, _inner(w2, U.down_wgrad(x, yd)[0]), rel_tol=1e-12)
    xu = rng.standard_normal((2, 2, 3, 2, 3))
    yu = rng.standard_normal((2, 4, 6, 4, 5))
    lhs = _inner(U.up(xu, w2), yu)
    assert math.isclose(lhs, _inner(xu, U.up_dgrad(yu, w2)), rel_tol=1e-12)
    assert math.isclose(lhs, _inner(w2, U.up_wgrad(xu, yu)[0]), rel_tol=1e-12)
    # bias gradients are the sums of the output gradients
    np.testing.assert_allclose(U.conv3_wgrad(x, y3)[1], y3.sum(axis=(0, 1, 2, 3)), rtol=1e-13)


def test_decoder_concatenation_order(rng):
    c0 = 2
    P = U.init_params(c0, 3)
    x = rng.standard_normal((1, 8, 8, 8, U.N_FEATURES))
    _, act = U.forward(P, x, c0)
    w, b = P["c0a"]
    # channels [0, c0) of c0a's input are u0, [c0, 2c0) the skip e0b
    ref = U.relu(U.conv3(act["u0"], w[:, :c0], b) + U.conv3(act["e0b"], w[:, c0:]))
    np.testing.assert_allclose(act["c0a"], ref, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("weighted", [False, True])
def test_network_gradients_match_finite_differences(rng, weighted):
    c0 = 2
    P = U.init_params(c0, 5)
    x = rng.standard_normal((2, 16, 16, 16, U.N_FEATURES))
    target = rng.standard_normal((2, 16, 16, 16))
    pred, act = U.forward(P, x, c0)
    grads = U.backward(P, act, pred, target, c0, fluence_weighted=weighted)

    def loss_now():
        return U.loss(U.forward(P, x, c0)[0], target, fluence_weighted=weighted)

    h = 1e-6
    checked = 0
    for name in [n for n, *_ in U.layer_table(c0)] + ["head"]:
        for which in (0, 1):
            arr = P[name][which]
            g = grads[name][which]
            for _ in range(2):
                idx = tuple(int(rng.integers(0, s)) for s in arr.shape)
                old = float(arr[idx])
                arr[idx] = old + h
                lp = loss_now()
                arr[idx] = old - h
                lm = loss_now()
                arr[idx] = old
                fd = (lp - lm) / (2 * h)
                assert abs(fd - g[idx]) <= 1e-6 * abs(fd) + 1e-9, (name, which, idx, fd, g[idx])
                checked += 1
    assert checked == 2 * 2 * 21


def test_fluence_weights_definition(rng):
    """Weights average to one per sample, are proportional to the fluence
    exp(target) within a sample, reduce to ones for a constant target, and
    make the loss the fluence-weighted mean of the squared log error."""
    target = rng.standard_normal((3, 4, 5, 6)) * 2.0
    w = U.loss_weights(target, True)
    np.testing.assert_allclose(w.reshape(3, -1).mean(axis=1), 1.0, rtol=1e-12)
    ratio = w / np.exp(target)
    for b in range(3):
        np.testing.assert_allclose(ratio[b], ratio[b].flat[0], rtol=1e-12)
    const = np.full((2, 3, 3, 3), 0.7)
    np.testing.assert_allclose(U.loss_weights(const, True), 1.0, rtol=1e-12)
    assert np.array_equal(U.loss_weights(target, False), np.ones_like(target))
    pred = target + rng.standard_normal(target.shape) * 0.1
    e = np.exp(target)
    by_hand = sum(float(np.sum(e[b] * (pred[b] - target[b]) ** 2) / np.sum(e[b])) for b in range(3)) / 3
    assert U.loss(pred, target, True) == pytest.approx(by_hand, rel=1e-12)


def test_adam_closed_form():
    """With a constant gradient the bias-corrected moments are exactly g and
    g^2, so every step moves by lr * g / (|g| + eps)."""
    g = np.array([0.3, -2.0, 1e-3])
    p = np.array([1.0, 2.0, 3.0])
    m = np.zeros(3)
    v = np.zeros(3)
    lr, eps = 0.01, 1e-8
    for t in range(1, 6):
        p_new, m, v = U.adam_step(p, g, m, v, t, lr, eps=eps)
        np.testing.assert_allclose(p - p_new, lr * g / (np.abs(g) + eps), rtol=1e-10)
        p = p_new
    # first step from zero moments with a different gradient follows Algorithm 1 by hand
    p1, m1, v1 = U.adam_step(np.zeros(1), np.array([4.0]), np.zeros(1), np.zeros(1), 1, 0.5)
    assert m1[0] == pytest.approx(0.4) and v1[0] == pytest.approx(0.016)
    assert p1[0] == pytest.approx(-0.5 * 4.0 / (4.0 + 1e-8))


def test_pack_input_and_targets():
    mask = np.zeros((2, 4, 2, 3), dtype=np.uint8)
    mask[1, 2, 1, 0] = 1
    x = U.pack_input(mask, [0.5, 2.0], [0.005, 0.01], [0.7, 0.0])
    assert x.shape == (2, 4, 2, 3, 16)
    assert x[1, 2, 1, 0, 0] == 1.0 and x[1, 2, 1, 0, 1] == 0.0 and x[0, 0, 0, 0, 1] == 1.0
    assert x[0, 3, 0, 0, 2] == pytest.approx(math.log(0.5))
    assert x[1, 0, 0, 0, 3] == pytest.approx(math.log(0.01) / 4)
    assert x[0, 1, 1, 2, 4] == pytest.approx(0.7)
    assert x[1, 3, 0, 1, 5] == pytest.approx(3.5 / 4)
    # sample 1 has one pore voxel of 24: phi = 1/24; diffusion attenuation of
    # the solid-fraction-scaled medium, mu_eff^2 = 3 mu_a' (mu_a' + mu_s'(1 - g))
    phi = 1 / 24
    ma, msp = (1 - phi) * 0.01, (1 - phi) * 2.0 * 1.0
    assert x[1, 2, 0, 0, 7] == pytest.approx(phi) and x[0, 0, 0, 0, 7] == 0
    assert x[1, 2, 1, 1, 6] == pytest.approx(-math.sqrt(3 * ma * (ma + msp)) * 2.5 / 8)
    assert x[0, 0, 0, 0, 6] == pytest.approx(-math.sqrt(3 * 0.005 * (0.005 + 0.5 * 0.3)) * 0.5 / 8)
    assert np.all(x[..., 8:] == 0)
    # an all-pore slab puts exactly one voxel of track per photon into each
    # layer, i.e. F = N / (nx ny) per voxel: Phi/S0 = 1 and ln Phi = 0
    nx, ny, n = 4, 2, 1000
    raw = np.full((3, ny, nx), n / (nx * ny) * 2.0 ** 32)
    np.testing.assert_allclose(U.log_fluence(raw, nx, ny, n), 0.0, atol=1e-15)
    assert U.log_fluence(np.zeros(1), nx, ny, n)[0] == pytest.approx(math.log(1e-6))


def test_phase_profiles():
    mask = np.zeros((1, 2, 2, 2), dtype=np.uint8)
    mask[0, 0, 0, 0] = 1
    lp = np.log(np.array([[[[2.0, 3.0], [5.0, 7.0]], [[1.0, 1.0], [1.0, 1.0]]]]))
    prof = U.phase_profiles(lp, mask)
    assert prof[0, 1, 0] == pytest.approx(2.0)
    assert prof[0, 0, 0] == pytest.approx(5.0)
    assert np.isnan(prof[0, 1, 1]) and prof[0, 0, 1] == pytest.approx(1.0)
