"""Exact start-up solution of oscillatory flow in a plane channel (the
transient Poiseuille case of the paper's validation set, Sec. 4.1 /
Table 1 "tp1M", after Womersley 1955).

Fluid at rest in the channel 0 <= y <= H (no-slip walls) is driven from
t = 0 by a flow rate per unit depth Q(t) = u0 H sin(w t).  Far from the inlet
and the outlet the flow is parallel, u = u(y, t), with

    du/dt = G(t) + nu d2u/dy2,    u(0) = u(H) = 0,    int_0^H u dy = Q(t),

G = -dp/dx the unknown pressure gradient.  The solution is the periodic
(Womersley) part plus a decaying start-up part:

* periodic: u_p = Im[W(y) e^{iwt}], W = (G^/(iw)) (1 - cosh(k s)/cosh(k H/2)),
  s = y - H/2, k = sqrt(iw/nu), with G^ fixed by int W dy = u0 H;
* start-up: the modes of the flow-rate-constrained problem,
  v_j = cos(z_j s 2/H) - cos(z_j) with tan(z_j) = z_j (zero mean, zero at the
  walls, decay rate nu (2 z_j / H)^2); their coefficients make u(y, 0) = 0.
  The constrained operator is self-adjoint on zero-mean functions, so the
  v_j are L2-orthogonal and the coefficients are plain projections.

This is test infrastructure: it pins the oracle and checks GPU runs."""
from __future__ import annotations

import numpy as np


def _tan_roots(n: int) -> np.ndarray:
    """The first n positive roots of tan z = z (Newton from the asymptote
    z ~ (j + 1/2) pi - 1/((j + 1/2) pi))."""
    j = np.arange(1, n + 1, dtype=np.float64)
    z = (j + 0.5) * np.pi - 1.0 / ((j + 0.5) * np.pi)
    for _ in range(50):
        # f(z) = sin z - z cos z, f'(z) = z sin z
        f = np.sin(z) - z * np.cos(z)
        z = z - f / (z * np.sin(z))
    return z


class StartupChannel:
    """u(y, t) and G(t) of the start-up problem above."""

    def __init__(self, H: float, nu: float, u0: float, omega: float, modes: int = 400,
                 quad: int = 4000):
        self.H, self.nu, self.u0, self.omega = H, nu, u0, omega
        k = np.sqrt(1j * omega / nu)
        self._k = k
        a = k * H / 2
        # int_0^H [1 - cosh(k s)/cosh(a)] dy = H - (2/k) tanh(a)
        self._Ghat = u0 * H * 1j * omega / (H - (2.0 / k) * np.tanh(a))
        self.z = _tan_roots(modes)
        # projection of -u_p(y, 0) onto the start-up modes: composite
        # 20-point Gauss-Legendre on quad/20 equal panels
        x, w = np.polynomial.legendre.leggauss(20)
        panels = max(1, quad // 20)
        h = H / panels
        y = (np.arange(panels)[:, None] * h + 0.5 * h * (x[None, :] + 1.0)).ravel()
        wq = np.tile(0.5 * h * w, panels)
        f = -self._periodic(y, 0.0)
        V = self._modes(y)                       # [modes, quad]
        self.b = (V * (f * wq)).sum(1) / ((V * V) * wq).sum(1)
        self.lam = nu * (2.0 * self.z / H) ** 2

    def _W(self, y):
        s = np.asarray(y, dtype=np.float64) - self.H / 2
        a = self._k * self.H / 2
        return (self._Ghat / (1j * self.omega)) * (1.0 - np.cosh(self._k * s) / np.cosh(a))

    def _periodic(self, y, t):
        return np.imag(self._W(y) * np.exp(1j * self.omega * t))

    def _modes(self, y):
        s = np.asarray(y, dtype=np.float64) - self.H / 2
        zz = self.z[:, None]
        return np.cos(zz * s[None, :] * 2.0 / self.H) - np.cos(zz)

    def u(self, y, t: float) -> np.ndarray:
        y = np.atleast_1d(np.asarray(y, dtype=np.float64))
        tr = (self.b * np.exp(-self.lam * t)) @ self._modes(y)
        return self._periodic(y, t) + tr

    def G(self, t: float) -> float:
        """-dp/dx.  The start-up modes carry a pressure gradient too: for
        v_j, nu v_j'' = -nu (2 z_j/H)^2 cos(...) = -lam_j (v_j + cos z_j), so
        dv/dt - nu v'' = lam_j cos(z_j) b_j e^{-lam_j t}."""
        gp = np.imag(self._Ghat * np.exp(1j * self.omega * t))
        gt = float((self.b * self.lam * np.cos(self.z) * np.exp(-self.lam * t)).sum())
        return float(gp + gt)

    def Q(self, t: float) -> float:
        return self.u0 * self.H * np.sin(self.omega * t)
