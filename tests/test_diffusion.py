"""The diffusion-approximation and kinetic post-processing against the
paper's printed values, and the DA solution against its own equations."""
import math
import os

import numpy as np

from paper_2604_13929_gb300 import diffusion as d

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_da_kinetics.txt")
H, NZ = 1.45e-6, 384
MUA_SHELL, MUSP_SHELL = 5159.0, 20118.0
MC_MEAN = {0.70: {"MC3D": 6.17e19, "MC1D": 4.07e19}, 0.90: {"MC3D": 1.238e20}}


def _computed(key, phi):
    L = NZ * H
    s0 = d.incident_photon_flux(45.0, 365e-9)
    da = d.CollimatedDA(d.ema(MUA_SHELL, phi), d.ema(MUSP_SHELL, phi), L, s0)
    s_acc = d.accessible_surface(0.25, phi, 7.25e-9)
    k_app = 0.0052 / 60.0
    mua = d.ema(MUA_SHELL, phi)
    est = key.split("_")[-1]
    mean = da.mean_fluence if est == "DA" else MC_MEAN[phi].get(est)
    return {
        "S0": s0, "D_eff": da.D, "kappa_eff": da.kappa, "kappaL": da.kappa * L,
        "z_b_um": da.z_b * 1e6, "L_opt_DA_um": da.optical_length * 1e6,
        "Phi_DA": da.mean_fluence, "S_acc": s_acc,
        "L_opt_MC3D_um": (MC_MEAN[phi]["MC3D"] * L / s0 * 1e6) if phi in MC_MEAN else None,
        "ksKads_MC3D": d.ks_kads(k_app, s_acc, 0.25, mua, MC_MEAN[phi]["MC3D"]),
        "ksKads_MC1D": d.ks_kads(k_app, s_acc, 0.25, mua, MC_MEAN[phi].get("MC1D", 1.0)),
        "ksKads_DA": d.ks_kads(k_app, s_acc, 0.25, mua, da.mean_fluence),
        "rV_MC3D": d.mean_volumetric_rate(7.25e-9, s_acc, 0.25, mua, MC_MEAN[phi]["MC3D"]),
        "rV_DA": d.mean_volumetric_rate(7.25e-9, s_acc, 0.25, mua, da.mean_fluence),
    }[key] if mean is not None or est not in ("MC1D",) else None


def test_printed_da_and_kinetic_values():
    rows = [l.split() for l in open(GOLDEN) if l.strip() and not l.startswith("#")]
    assert len(rows) >= 20
    for key, phi, value, tol in rows:
        got = _computed(key, float(phi))
        assert abs(got / float(value) - 1) < float(tol), (key, phi, got, value)


def test_da_solution_satisfies_its_equation_and_boundaries():
    da = d.CollimatedDA(1548.0, 6035.0, 556.8e-6, 1.0)
    z = np.linspace(0, da.thickness, 2001)
    h = z[1] - z[0]
    f = da.diffuse(z)
    lap = (f[2:] - 2 * f[1:-1] + f[:-2]) / h ** 2
    lhs = da.D * lap - da.mu_a * f[1:-1]
    rhs = -da.mu_sp * np.exp(-da.mu_t * z[1:-1])
    assert np.max(np.abs(lhs - rhs)) < 1e-4 * np.max(np.abs(rhs))
    assert abs(da.diffuse(-da.z_b)) < 1e-12 and abs(da.diffuse(da.thickness + da.z_b)) < 1e-12


def test_closed_form_integral_matches_quadrature():
    da = d.CollimatedDA(515.9, 2011.8, 556.8e-6, 3.0)
    x, w = np.polynomial.legendre.leggauss(200)
    z = 0.5 * da.thickness * (x + 1)
    quad = 0.5 * da.thickness * np.sum(w * da.fluence(z))
    assert abs(da.integral(0, da.thickness) / quad - 1) < 1e-12
    edges = np.linspace(0, da.thickness, 9)
    assert abs(np.sum(da.layer_means(edges) * np.diff(edges)) / quad - 1) < 1e-12


def test_rms_metrics():
    da = np.array([4.0, 2.0, 1.0, 0.5])
    assert d.rms_weighted(da, da) == 0.0 and d.rms_unweighted(da, da) == 0.0
    mc = da * 1.1
    assert abs(d.rms_weighted(mc, da) - 0.1) < 1e-12
    assert abs(d.rms_unweighted(mc, da) - 0.1) < 1e-12
    assert abs(d.rms_log(mc, da) - math.log(1.1)) < 1e-12
    # the weighted form emphasises the bright (shallow) points
    mc2 = da.copy(); mc2[-1] *= 2.0
    assert d.rms_weighted(mc2, da) < d.rms_unweighted(mc2, da)
