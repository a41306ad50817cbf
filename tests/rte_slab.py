"""Independent plane-parallel radiative-transfer solver used to pin the MC.

A homogeneous all-solid slab with periodic lateral faces and a laterally
uniform collimated source is an exact 1D plane-parallel problem, so the
steady radiative transfer equation in optical depth tau = (mu_s + mu_a) z

    mu dJ/dtau = -J + (omega/2) int p(mu, mu') J(mu') dmu'
                    + (omega/2) p(mu, 1) exp(-tau),

(J = 2 pi times the azimuthally averaged diffuse radiance, unit incident flux
along mu = 1, no incoming diffuse light at either face, n = 1) fixes the
reflectance, transmittance, absorptance and the depth profile of the fluence
that the MC estimates.

Method (not Monte Carlo): double-Gauss discrete ordinates, the azimuthally
averaged Henyey-Greenstein kernel from its Legendre moments g^l, and the
exact solution of the resulting linear ODE system by eigen-decomposition
(homogeneous part scaled so no exponential grows) plus the particular
solution for the exponential beam source.  No spatial discretisation error.
"""
from __future__ import annotations

import numpy as np
from numpy.polynomial import legendre as L


def _legendre_table(x: np.ndarray, lmax: int) -> np.ndarray:
    """P_l(x) for l = 0..lmax by the three-term recurrence."""
    P = np.zeros((lmax + 1, x.size))
    P[0] = 1.0
    if lmax >= 1:
        P[1] = x
    for l in range(1, lmax):
        P[l + 1] = ((2 * l + 1) * x * P[l] - l * P[l - 1]) / (l + 1)
    return P


class SlabSolution:
    def __init__(self, mus: float, mua: float, g: float, thickness: float,
                 n_half: int = 48, lmax: int | None = None):
        self.mut = mus + mua
        self.omega = mus / self.mut
        self.tau_L = self.mut * thickness
        self.thickness = thickness
        xg, wg = L.leggauss(n_half)
        mu_h = 0.5 * (xg + 1.0)             # nodes on (0, 1)
        w_h = 0.5 * wg
        self.mu = np.concatenate([-mu_h[::-1], mu_h])
        self.w = np.concatenate([w_h[::-1], w_h])      # sums to 2
        lmax = 2 * n_half - 1 if lmax is None else lmax
        P = _legendre_table(self.mu, lmax)
        P1 = _legendre_table(np.array([1.0]), lmax)[:, 0]
        coef = (2 * np.arange(lmax + 1) + 1) * g ** np.arange(lmax + 1)
        pm = (P * coef[:, None]).T @ P                 # p(mu_i, mu_j)
        # discrete energy conservation: (1/2) sum_j w_j p_ij = 1
        pm = pm / (0.5 * (pm * self.w[None, :]).sum(axis=1))[:, None]
        ps = (P * coef[:, None]).T @ P1                # p(mu_i, 1)
        n = self.mu.size
        M = np.diag(1.0 / self.mu)
        A = M @ (-np.eye(n) + 0.5 * self.omega * pm * self.w[None, :])
        b = M @ (0.5 * self.omega * ps)
        self.c = -np.linalg.solve(A + np.eye(n), b)     # particular: c exp(-tau)
        lam, V = np.linalg.eig(A)
        self.lam = lam.real
        self.V = V.real
        pos = self.lam > 0
        E0 = np.where(pos, np.exp(-self.lam * self.tau_L), 1.0)   # E_k(0)
        EL = np.where(pos, 1.0, np.exp(self.lam * self.tau_L))    # E_k(tau_L)
        down = self.mu > 0
        up = ~down
        rows = np.vstack([self.V[down] * E0[None, :], self.V[up] * EL[None, :]])
        rhs = np.concatenate([-self.c[down], -self.c[up] * np.exp(-self.tau_L)])
        self.alpha = np.linalg.solve(rows, rhs)
        self._pos = pos

    def J(self, tau: np.ndarray) -> np.ndarray:
        tau = np.atleast_1d(np.asarray(tau, dtype=np.float64))
        E = np.where(self._pos[None, :], np.exp(self.lam[None, :] * (tau[:, None] - self.tau_L)),
                     np.exp(self.lam[None, :] * tau[:, None]))
        return (E * self.alpha[None, :]) @ self.V.T + np.exp(-tau)[:, None] * self.c[None, :]

    def fluence(self, z: np.ndarray) -> np.ndarray:
        """Total fluence per unit incident flux at depth z (voxel units)."""
        tau = self.mut * np.asarray(z, dtype=np.float64)
        return self.J(tau) @ self.w + np.exp(-np.atleast_1d(tau))

    def layer_means(self, nz: int, order: int = 16) -> np.ndarray:
        xg, wg = L.leggauss(order)
        out = np.empty(nz)
        for iz in range(nz):
            z = iz + 0.5 * (xg + 1.0)
            out[iz] = 0.5 * np.sum(wg * self.fluence(z))
        return out

    def reflectance(self) -> float:
        J0 = self.J(0.0)[0]
        up = self.mu < 0
        return float(np.sum(-self.mu[up] * self.w[up] * J0[up]))

    def transmittance(self) -> float:
        JL = self.J(self.tau_L)[0]
        down = self.mu > 0
        return float(np.sum(self.mu[down] * self.w[down] * JL[down]) + np.exp(-self.tau_L))

    def absorptance(self) -> float:
        return 1.0 - self.reflectance() - self.transmittance()
