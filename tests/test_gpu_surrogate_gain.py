"""What the trained surrogate gains over the Monte Carlo alone.

A small U-Net (c0 = 16) is trained by the project's own tensor-core kernels
on Monte Carlo fields of the transport engine (64^3 Cahn-Hilliard masks,
random porosity and solid optics, fixed seeds), then judged on held-out masks
against a high-photon Monte Carlo reference of the same masks.

The gain is stated on the voxel field, the quantity the network predicts:
the RMS of ln(Phi/S0) over all held-out voxels.  The comparison is at equal
GPU time per field: Monte Carlo is given as many photons as it transports in
the time the network takes per field (forward pass plus depth profiles,
inputs resident), and scored against the same reference.  The network must
beat that Monte Carlo by GAIN_RMSE and deliver GAIN_SPEED times the fields
per second of the Monte Carlo run at 1e7 photons per 64^3 field (the
benchmark's definition of one Monte Carlo field).
"""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

N, C0, BATCH = 64, 16, 32
N_TRAIN, N_TEST = 512, 32
TRAIN_PHOTONS, REF_PHOTONS, FIELD_PHOTONS = 2_000_000, 20_000_000, 10_000_000
STEPS = 1500
GAIN_RMSE = 1.75         # equal-time MC voxel ln-RMSE over the surrogate's (measured 1.96)
GAIN_SPEED = 100.0       # surrogate fields/s over MC fields/s at 1e7 photons per field


@pytest.fixture(scope="module")
def mods():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_13929_gb300 import build
    build.build()
    from paper_2604_13929_gb300 import spnn, surrogate as sg
    return torch, spnn, sg


def _field_set(sg, count, seed, photons):
    masks, optics = sg.sample_problems(count, seed, n=N, ch_steps=500)
    target, mc_s = sg.simulate(masks, optics, photons)
    return sg.FieldSet(masks, optics, target, photons,
                       {"mc_s": mc_s, "mc_photons_per_s": count * photons / mc_s})


def test_surrogate_beats_equal_time_monte_carlo(mods):
    torch, spnn, sg = mods
    train = _field_set(sg, N_TRAIN, 101, TRAIN_PHOTONS)
    test = _field_set(sg, N_TEST, 202, REF_PHOTONS)
    net = spnn.UNet(C0, N, BATCH)
    net.set_params(spnn.init_params(C0, 7))
    losses, _ = sg.train(net, train, STEPS, BATCH, lr0=3e-3, lr1=3e-5, seed=3)
    assert np.isfinite(losses).all() and losses[-20:].mean() < 0.3 * losses[:5].mean()

    pred = sg.predict(net, test, BATCH)
    d = (pred - test.target).double()
    rmse_net = float(torch.sqrt((d * d).mean()).item())

    rate = sg.inference_rate(net, test, BATCH, reps=10)
    mc_rate = train.info["mc_photons_per_s"]
    eq_photons = max(100, int(mc_rate / rate["fields_per_s"]))
    eq_target, _ = sg.simulate(test.mask, test.optics, eq_photons, seed=sg.MC_SEED + 1)
    de = (eq_target - test.target).double()
    rmse_mc = float(torch.sqrt((de * de).mean()).item())
    speed = rate["fields_per_s"] / (mc_rate / FIELD_PHOTONS)
    net.close()
    info = dict(rmse_net=rmse_net, rmse_mc_equal_time=rmse_mc, eq_photons=eq_photons,
                fields_per_s=rate["fields_per_s"], mc_photons_per_s=mc_rate, speedup=speed,
                loss_first=float(losses[0]), loss_last=float(losses[-20:].mean()))
    print("surrogate gain", info)
    assert math.isfinite(rmse_net) and rmse_net * GAIN_RMSE <= rmse_mc, info
    assert speed >= GAIN_SPEED, info
