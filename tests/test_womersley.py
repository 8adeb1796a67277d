"""Checks of the exact start-up solution of oscillatory channel flow
(tests/womersley.py) against what fixes it independently: the imposed flow
rate, the no-slip walls, the rest state at t = 0, the momentum equation with
a y-independent pressure gradient, and two textbook limits (quasi-steady
Poiseuille flow at small Womersley number, the periodic Womersley profile
once the start-up has decayed)."""
import numpy as np
import pytest

from womersley import StartupChannel, _tan_roots

H, NU, U0, W = 0.02, 3.3e-6, 0.01, np.pi          # the paper's tp1M parameters


def gauss(H, n=2000):
    x, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * H * (x + 1.0), 0.5 * H * w


def test_tan_roots():
    z = _tan_roots(50)
    assert np.abs(np.tan(z) - z).max() < 1e-9 * z.max()
    assert z[0] == pytest.approx(4.493409457909064, rel=1e-13)
    assert (np.diff(z) > 3.0).all()


@pytest.mark.parametrize("t", [1e-3, 0.02, 0.1, 0.5, 1.7])
def test_flow_rate_walls_and_rest(t):
    S = StartupChannel(H, NU, U0, W)
    y, w = gauss(H)
    assert (S.u(y, t) * w).sum() == pytest.approx(S.Q(t), rel=1e-9, abs=1e-18)
    assert np.abs(S.u([0.0, H], t)).max() < 1e-15
    assert np.abs(S.u(y, 0.0)).max() < 1e-4 * U0


@pytest.mark.parametrize("t", [0.01, 0.05, 0.3])
def test_momentum_equation(t):
    """du/dt - nu d2u/dy2 is the same at every y and equals G(t)."""
    S = StartupChannel(H, NU, U0, W)
    y = np.linspace(0.1 * H, 0.9 * H, 9)
    dt, dy = 1e-6, 2e-5
    ut = (S.u(y, t + dt) - S.u(y, t - dt)) / (2 * dt)
    uyy = (S.u(y + dy, t) - 2 * S.u(y, t) + S.u(y - dy, t)) / dy ** 2
    res = ut - NU * uyy
    assert np.abs(res - S.G(t)).max() < 1e-4 * abs(S.G(t))


def test_quasi_steady_poiseuille_limit():
    """At Womersley number 0.05 the profile is the parabola carrying Q(t)."""
    nu = 1.0
    w = 4 * (0.05 / (0.5 * H)) ** 2 * nu           # alpha = (H/2) sqrt(w/nu) = 0.05
    S = StartupChannel(H, nu, U0, w)
    t = 0.25 * 2 * np.pi / w
    y = np.linspace(0, H, 41)
    par = 6 * S.Q(t) / H * y * (H - y) / H ** 2
    assert np.abs(S.u(y, t) - par).max() < 1e-3 * par.max()
    assert S.G(t) == pytest.approx(12 * nu * S.Q(t) / H ** 3, rel=1e-3)


def test_start_up_decays_to_periodic_profile():
    """After many viscous times the solution repeats with the period."""
    nu = 3.3e-5                                     # slowest start-up mode decays at 6.7 1/s
    S = StartupChannel(H, nu, U0, W)
    y = np.linspace(0, H, 33)
    T = 2.0                                          # period of w = pi
    a, b = S.u(y, 40.3), S.u(y, 40.3 + T)
    assert np.abs(a - b).max() < 1e-12
    assert np.abs(S.u(y, 0.3) - S.u(y, 0.3 + T)).max() > 1e-4 * U0
