"""Training set, training loop and evaluation of the fluence surrogate.

The surrogate (``spnn.UNet``) learns ln(Phi/S0) per voxel from Monte Carlo
fields of the transport engine (``spmc``) on Cahn-Hilliard masks with random
porosity and solid optics, so that mask designs (Sec. 5 of arXiv 2604.13929)
can be screened without a photon run.  It is scored on held-out masks by the
fluence-weighted relative RMS deviation (Eq. RMSw) of its per-phase depth
profiles from the Monte Carlo ones, and by fields per second.

Every arithmetic step runs in the two CUDA libraries (transport, log-fluence
targets, input features, network, loss, Adam, profiles); this module only
sequences the calls and moves tensors.  The profile RMS is host FP64
post-processing of 2 x 64 numbers per mask (``diffusion.rms_weighted``).

Workload recipe (defaults): cubes of n = 64 voxels, Cahn-Hilliard fields of
1000 FP32 steps from noise seed ``seed * 100003 + i``, rank-thresholded to
porosity U[0.50, 0.95]; solid mu_s h log-uniform on [0.1, 2.0], mu_a h
U[0.001, 0.05], g U[0, 0.9]; 1e7 photons per field, periodic lateral faces.
"""
from __future__ import annotations

import math
import time
from dataclasses import dataclass, field

import numpy as np
import torch

from . import diffusion, inputs, spmc, spnn

MC_SEED = 20260809


@dataclass
class FieldSet:
    mask: torch.Tensor            # uint8 (N, n, n, n), 1 = pore
    optics: torch.Tensor          # float32 (N, 3): mu_s h, mu_a h, g
    target: torch.Tensor          # float32 (N, n, n, n): ln Phi/S0 from the Monte Carlo
    photons: int
    info: dict = field(default_factory=dict)

    def __len__(self):
        return self.mask.shape[0]


def sample_problems(count: int, seed: int, n: int = 64, ch_steps: int = 1000, chunk: int = 128):
    """Masks (uint8, cuda) and optics (float32, cuda) of `count` problems."""
    rng = np.random.default_rng(seed)
    phi = rng.uniform(0.50, 0.95, count)
    mus = np.exp(rng.uniform(math.log(0.1), math.log(2.0), count))
    mua = rng.uniform(0.001, 0.05, count)
    g = rng.uniform(0.0, 0.9, count)
    masks = torch.empty((count, n, n, n), dtype=torch.uint8, device="cuda")
    for c0 in range(0, count, chunk):
        idx = list(range(c0, min(count, c0 + chunk)))
        c = inputs.cahn_hilliard((n, n, n), ch_steps, device="cuda", dtype=torch.float32,
                                 seeds=[seed * 100003 + i for i in idx])
        for j, i in enumerate(idx):
            masks[i] = torch.from_numpy(inputs.rank_threshold(c[j], float(phi[i]))).cuda()
    optics = torch.tensor(np.stack([mus, mua, g], axis=1), dtype=torch.float32, device="cuda")
    return masks, optics


def simulate(masks, optics, photons: int, seed: int = MC_SEED, floor: float = 1e-6, chunk: int = 16):
    """Monte Carlo ln(Phi/S0) fields of every problem, batched launches of
    `chunk` masks; returns (targets float32 cuda, seconds of transport)."""
    count, n = masks.shape[0], masks.shape[1]
    target = torch.empty((count, n, n, n), dtype=torch.float32, device="cuda")
    raw = torch.empty((chunk, n, n, n), dtype=torch.int64, device="cuda")
    host_masks = masks.cpu().numpy()
    host_optics = optics.cpu().numpy().astype(np.float64)
    nph = torch.full((chunk,), float(photons), dtype=torch.float64, device="cuda")
    mc_s = 0.0
    for c0 in range(0, count, chunk):
        idx = list(range(c0, min(count, c0 + chunk)))
        problems = [(host_masks[i], host_optics[i, 0], host_optics[i, 1], host_optics[i, 2]) for i in idx]
        with spmc.Batch(problems) as b:
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            b.run([photons] * len(idx), seed)
            torch.cuda.synchronize()
            mc_s += time.perf_counter() - t0
            for j in range(len(idx)):
                b.raw_field_to(j, raw[j])
            torch.cuda.synchronize()
        k = len(idx)
        spnn.spnn_log_fluence(raw[:k], nph[:k], target[c0:c0 + k], floor=floor)
    torch.cuda.synchronize()
    return target, mc_s


def make_fields(count: int, seed: int, photons: int = 10 ** 7, n: int = 64) -> FieldSet:
    t0 = time.perf_counter()
    masks, optics = sample_problems(count, seed, n)
    t1 = time.perf_counter()
    target, mc_s = simulate(masks, optics, photons)
    return FieldSet(masks, optics, target, photons,
                    {"mask_s": t1 - t0, "mc_s": mc_s, "mc_fields_per_s": count / mc_s,
                     "mc_photons_per_s": count * photons / mc_s})


def features(fs: FieldSet, sel) -> torch.Tensor:
    """Input feature planes (2, b, n, n, n, 8) of the selected samples."""
    m = fs.mask[sel].contiguous()
    o = fs.optics[sel].contiguous()
    B, n = m.shape[0], m.shape[1]
    x = spnn.planes_empty(B, n, n, n, 16)
    spnn.spnn_pack_input(m, o, x)
    return x


def cosine_lr(step: int, steps: int, lr0: float, lr1: float, warmup: int = 20) -> float:
    if step < warmup:
        return lr0 * (step + 1) / warmup
    t = (step - warmup) / max(1, steps - warmup)
    return lr1 + 0.5 * (lr0 - lr1) * (1 + math.cos(math.pi * t))


def train(net: spnn.UNet, fs: FieldSet, steps: int, batch: int, lr0: float = 2e-3, lr1: float = 2e-5,
          seed: int = 0, log_every: int = 50, on_log=None):
    """Adam on the mean squared ln-fluence error over random minibatches.
    Returns the per-step losses and the seconds spent."""
    gen = torch.Generator(device="cpu").manual_seed(seed)
    N, n = len(fs), fs.mask.shape[1]
    pred = torch.empty((batch, n, n, n), dtype=torch.float32, device="cuda")
    loss = torch.zeros(steps, dtype=torch.float64, device="cuda")
    order = torch.randperm(N, generator=gen)
    pos = 0
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for step in range(steps):
        if pos + batch > N:
            order = torch.randperm(N, generator=gen)
            pos = 0
        sel = order[pos:pos + batch].cuda()
        pos += batch
        x = features(fs, sel)
        tgt = fs.target[sel].contiguous()
        net.forward(x, pred)
        net.backward(tgt, loss[step:step + 1])
        net.adam(cosine_lr(step, steps, lr0, lr1))
        if on_log and (step % log_every == 0 or step == steps - 1):
            on_log(step, float(loss[step].item()))
    torch.cuda.synchronize()
    spnn.spnn_status()
    return loss.cpu().numpy(), time.perf_counter() - t0


def predict(net: spnn.UNet, fs: FieldSet, batch: int) -> torch.Tensor:
    N, n = len(fs), fs.mask.shape[1]
    out = torch.empty((N, n, n, n), dtype=torch.float32, device="cuda")
    for c0 in range(0, N, batch):
        sel = torch.arange(c0, min(N, c0 + batch), device="cuda")
        if sel.numel() < batch:        # the network runs full batches; pad with repeats
            sel = torch.cat([sel, sel[-1].repeat(batch - sel.numel())])
        x = features(fs, sel)
        pred = torch.empty((batch, n, n, n), dtype=torch.float32, device="cuda")
        net.forward(x, pred)
        k = min(batch, N - c0)
        out[c0:c0 + k] = pred[:k]
    torch.cuda.synchronize()
    return out


def profiles(log_phi: torch.Tensor, mask: torch.Tensor) -> np.ndarray:
    """Per-phase depth profiles (N, 2, n) of exp(log_phi) (solid row 0, pore row 1)."""
    N, n = log_phi.shape[0], log_phi.shape[1]
    prof = torch.empty((N, 2, n), dtype=torch.float32, device="cuda")
    spnn.spnn_phase_profiles(log_phi.contiguous(), mask.contiguous(), prof)
    return prof.cpu().numpy().astype(np.float64)


def profile_rms(p_model: np.ndarray, p_ref: np.ndarray) -> np.ndarray:
    """Eq. RMSw of each mask's solid and pore profiles against the reference: (N, 2)."""
    N = p_ref.shape[0]
    out = np.full((N, 2), np.nan)
    for i in range(N):
        for ph in (0, 1):
            ok = np.isfinite(p_ref[i, ph]) & np.isfinite(p_model[i, ph])
            if ok.sum() >= 8:
                out[i, ph] = diffusion.rms_weighted(p_model[i, ph][ok], p_ref[i, ph][ok])
    return out


def evaluate(net: spnn.UNet, fs: FieldSet, batch: int) -> dict:
    pred = predict(net, fs, batch)
    pm = profiles(pred, fs.mask)
    pr = profiles(fs.target, fs.mask)
    rms = profile_rms(pm, pr)
    d = (pred - fs.target).double()
    return {"rms_w_solid_mean": float(np.nanmean(rms[:, 0])), "rms_w_pore_mean": float(np.nanmean(rms[:, 1])),
            "rms_w_mean": float(np.nanmean(rms)), "rms_w_median": float(np.nanmedian(rms)),
            "rms_w_p90": float(np.nanpercentile(rms, 90)), "rms_w_max": float(np.nanmax(rms)),
            "frac_masks_rms_w_le_2pct": float(np.mean(np.nanmax(rms, axis=1) <= 0.02)),
            "voxel_ln_rmse": float(torch.sqrt((d * d).mean()).item()),
            "voxel_rel_rmse": float(torch.sqrt(((torch.exp(d) - 1) ** 2).mean()).item())}


def inference_rate(net: spnn.UNet, fs: FieldSet, batch: int, reps: int = 5) -> dict:
    """Fields per second of forward + depth profiles at the given batch, inputs resident."""
    n = fs.mask.shape[1]
    sel = torch.arange(batch, device="cuda") % len(fs)
    x = features(fs, sel)
    m = fs.mask[sel].contiguous()
    pred = torch.empty((batch, n, n, n), dtype=torch.float32, device="cuda")
    prof = torch.empty((batch, 2, n), dtype=torch.float32, device="cuda")

    def once():
        net.forward(x, pred)
        spnn.spnn_phase_profiles(pred, m, prof)

    once()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        once()
    e1.record()
    torch.cuda.synchronize()
    spnn.spnn_status()
    ms = e0.elapsed_time(e1) / reps
    return {"ms_per_batch": ms, "fields_per_s": batch / (ms / 1e3)}
