"""Host FP64 post-processing of the Monte Carlo results (arXiv 2604.13929).

* the collimated diffusion approximation for a planar source on a slab
  (Sec. 2.4: Eq. DA_total, DA_diff_eq, Cpm, Phi_diff) with extrapolated
  boundaries at -z_b and L + z_b, z_b = 2 l*/3;
* the effective optical length and depth-averaged fluence (Eq. Lopt_DA);
* the fluence-weighted relative RMS deviation between two depth profiles
  (Eq. RMSw) and its unweighted and log-ratio variants (Sec. 2.7);
* the effective-medium scaling mu_eff = mu (1 - phi) (Eq. EMA_scaling);
* the kinetic chain: incident photon flux S0 = I0 / (h nu) (Eq. S0), the
  accessible catalytic surface S_acc (Eq. Sacc), k_V,mono (Eq. kV and its
  compact DA form Eq. kV_compact) and k_surf K_ads from a measured apparent
  rate constant (Eq. ksKads).

All lengths in metres unless stated; fluences in the units of S0.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

PLANCK = 6.62607015e-34      # J s
LIGHT = 299792458.0          # m / s


def incident_photon_flux(irradiance_w_m2: float, wavelength_m: float) -> float:
    """S0 = I0 / (h nu) for a monochromatic collimated source (Eq. S0)."""
    return irradiance_w_m2 * wavelength_m / (PLANCK * LIGHT)


def ema(mu: float, porosity: float) -> float:
    """Effective-medium scaling of a solid coefficient (Eq. EMA_scaling)."""
    return mu * (1.0 - porosity)


@dataclass
class CollimatedDA:
    """Collimated diffusion approximation on a slab of thickness L.

    mu_a, mu_sp: absorption and reduced scattering coefficients of the
    (effective) medium; s0: incident flux.  Phi(z) = S0 exp(-mu_t z) +
    Phi_diff(z), Phi_diff = A exp(-mu_t z) + C+ sinh[k (z + z_b)]
    + C- sinh[k (L + z_b - z)], vanishing at z = -z_b and z = L + z_b.
    """
    mu_a: float
    mu_sp: float
    thickness: float
    s0: float = 1.0

    def __post_init__(self):
        self.mu_t = self.mu_a + self.mu_sp
        self.D = 1.0 / (3.0 * (self.mu_a + self.mu_sp))
        self.kappa = math.sqrt(self.mu_a / self.D)
        self.l_star = 1.0 / self.mu_sp
        self.z_b = 2.0 / 3.0 * self.l_star
        L, zb, mt, k = self.thickness, self.z_b, self.mu_t, self.kappa
        self.L_e = L + 2.0 * zb
        self.A = self.mu_sp * self.s0 / (self.D * (k * k - mt * mt))
        sh = math.sinh(k * self.L_e)
        self.c_plus = -self.A * math.exp(-mt * (L + zb)) / sh
        self.c_minus = -self.A * math.exp(mt * zb) / sh

    def diffuse(self, z):
        z = np.asarray(z, dtype=np.float64)
        k, zb, L = self.kappa, self.z_b, self.thickness
        return (self.A * np.exp(-self.mu_t * z) + self.c_plus * np.sinh(k * (z + zb))
                + self.c_minus * np.sinh(k * (L + zb - z)))

    def fluence(self, z):
        """Phi_DA(z) = S0 exp(-mu_t z) + Phi_diff(z) (Eq. DA_total)."""
        z = np.asarray(z, dtype=np.float64)
        return self.s0 * np.exp(-self.mu_t * z) + self.diffuse(z)

    def integral(self, z0: float, z1: float) -> float:
        """Closed-form integral of Phi_DA over [z0, z1]."""
        k, zb, L, mt = self.kappa, self.z_b, self.thickness, self.mu_t
        e = lambda z: -math.exp(-mt * z) / mt  # noqa: E731
        ballistic = self.s0 * (e(z1) - e(z0))
        part = self.A * (e(z1) - e(z0))
        plus = self.c_plus * (math.cosh(k * (z1 + zb)) - math.cosh(k * (z0 + zb))) / k
        minus = -self.c_minus * (math.cosh(k * (L + zb - z1)) - math.cosh(k * (L + zb - z0))) / k
        return ballistic + part + plus + minus

    @property
    def optical_length(self) -> float:
        """L_opt = (1/S0) int_0^L Phi_DA dz (Eq. Lopt_DA)."""
        return self.integral(0.0, self.thickness) / self.s0

    @property
    def mean_fluence(self) -> float:
        """<Phi>_DA = S0 L_opt / L (Eq. Lopt_DA)."""
        return self.s0 * self.optical_length / self.thickness

    def layer_means(self, edges):
        """Mean of Phi_DA over each interval [edges[i], edges[i+1]]."""
        edges = np.asarray(edges, dtype=np.float64)
        return np.array([self.integral(a, b) / (b - a) for a, b in zip(edges[:-1], edges[1:])])


def rms_weighted(phi_mc, phi_da) -> float:
    """Fluence-weighted relative RMS deviation (Eq. RMSw)."""
    mc = np.asarray(phi_mc, dtype=np.float64)
    da = np.asarray(phi_da, dtype=np.float64)
    ok = np.isfinite(mc) & np.isfinite(da) & (da > 0)
    mc, da = mc[ok], da[ok]
    return float(np.sqrt(np.sum(da * (mc - da) ** 2 / da ** 2) / np.sum(da)))


def rms_unweighted(phi_mc, phi_da) -> float:
    """Relative RMS deviation with unit weights."""
    mc = np.asarray(phi_mc, dtype=np.float64)
    da = np.asarray(phi_da, dtype=np.float64)
    ok = np.isfinite(mc) & np.isfinite(da) & (da > 0)
    return float(np.sqrt(np.mean(((mc[ok] - da[ok]) / da[ok]) ** 2)))


def rms_log(phi_mc, phi_da) -> float:
    """RMS of the natural-log ratio ln(Phi_MC / Phi_DA)."""
    mc = np.asarray(phi_mc, dtype=np.float64)
    da = np.asarray(phi_da, dtype=np.float64)
    ok = np.isfinite(mc) & np.isfinite(da) & (da > 0) & (mc > 0)
    return float(np.sqrt(np.mean(np.log(mc[ok] / da[ok]) ** 2)))


def accessible_surface(f_np: float, porosity: float, a_np: float) -> float:
    """S_acc = f_NP (1 - phi) 3 / a_np (Eq. Sacc), per metre."""
    return f_np * (1.0 - porosity) * 3.0 / a_np


def kv_mono(k_surf: float, s_acc: float, phi_int: float, optical_length: float) -> float:
    """k_V,mono = k_surf S_acc phi_int L_opt (Eq. kV)."""
    return k_surf * s_acc * phi_int * optical_length


def kv_mono_compact(k_surf: float, s_acc: float, phi_int: float, l_star: float,
                    thickness: float) -> float:
    """The compact DA form of k_V,mono (Eq. kV_compact), z_b = 2 l*/3."""
    z_b = 2.0 / 3.0 * l_star
    return k_surf * s_acc * phi_int * l_star / (1.0 + thickness / (2.0 * l_star) + z_b / l_star)


def ks_kads(k_app: float, s_acc: float, phi_int: float, mu_a: float, mean_fluence: float) -> float:
    """k_surf K_ads = k_app / (S_acc phi_int mu_a <Phi>) (Eq. ksKads), m^4/photon."""
    return k_app / (s_acc * phi_int * mu_a * mean_fluence)


def mean_volumetric_rate(k_surf: float, s_acc: float, phi_int: float, mu_a: float,
                         mean_fluence: float) -> float:
    """r_V,mean = k_surf S_acc phi_int mu_a <Phi> (below Eq. kapp)."""
    return k_surf * s_acc * phi_int * mu_a * mean_fluence
