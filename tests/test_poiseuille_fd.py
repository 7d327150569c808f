"""Pins of the finite-difference Poiseuille reference (Appendix A) against
closed forms of the reduced equations of Sec. 3.1 and the discrete scheme's
own exact solutions."""
import math

import numpy as np
import pytest

from oracle import poiseuille_fd as fd
from paper_2302_04741_gb300 import workloads as W

C_D2Q37 = W.C_D2Q37


def test_small_gx_gives_parabola_and_quartic_heating():
    """g_y = 0, theta_b = theta_t: u = rho0 g_x y (H - y) / (2 mu) and, from
    mu u'^2 + lambda theta'' = 0, theta = theta_b + K [(H/2)^4 - (H/2 - y)^4]
    with K = rho0^2 g_x^2 / (12 mu lambda).  The central scheme differentiates a
    quadratic u exactly, and its second difference of the quartic exceeds
    dy^2 theta'' by dy^4 theta''''/12, so the discrete theta is the quartic
    minus (dy^2 theta''''/24) y (y - H) -- exact, up to the O(K) coupling of
    rho = p / theta that a small g_x makes negligible."""
    H, mu, lam, rho0 = 10.0, 0.3, 0.6, 1.0
    gx = 8 * mu * 1e-3 / (rho0 * H * H)  # U_c = 1e-3
    y, rho, u, th, _ = fd.solve(41, H, gx, 0.0, mu, lam, rho0=rho0)
    K = rho0 ** 2 * gx ** 2 / (12 * mu * lam)
    dy = y[1] - y[0]
    quartic = K * ((H / 2) ** 4 - (H / 2 - y) ** 4)
    d4 = -24 * K  # theta'''' of the quartic
    rise = quartic - dy * dy * d4 / 24 * y * (y - H)
    np.testing.assert_allclose(th - 1.0, rise, rtol=2e-5, atol=1e-16)
    np.testing.assert_allclose(u, rho0 * gx * y * (H - y) / (2 * mu), rtol=1e-6, atol=1e-18)
    assert abs(u.max() - 1e-3) < 1e-8  # U_c = rho0 g_x H^2 / (8 mu)


@pytest.mark.parametrize("theta_b,theta_t", [(1.0, 1.0), (0.7, 1.4)])
def test_hydrostatic_profile_converges_first_order(theta_b, theta_t):
    """g_x = 0: no flow and no heating, theta linear (exactly, in the scheme),
    and p = rho theta with p' = p g_y / theta, i.e. p ~ exp(g_y int dy/theta):
    (theta / theta_b)^(g_y H / (theta_t - theta_b)) for linear theta, or
    exp(g_y y / theta_b) when theta is uniform.  The forward difference makes
    rho first-order accurate: halving dy halves the error."""
    H, gy, rho0 = 150 * C_D2Q37, -2.8e-3, 1.0

    def exact(y):
        if theta_t == theta_b:
            th = np.full_like(y, theta_b)
            p = np.exp(gy * y / theta_b)
        else:
            th = theta_b + (theta_t - theta_b) * y / H
            p = (th / theta_b) ** (gy * H / (theta_t - theta_b))
        return p / th

    errs = []
    for N in (201, 401, 801):
        y, rho, u, th, _ = fd.solve(N, H, 0.0, gy, 0.3, 0.6, rho0=rho0, theta_b=theta_b,
                                    theta_t=theta_t)
        assert np.max(np.abs(u)) == 0.0
        np.testing.assert_allclose(th, np.linspace(theta_b, theta_t, N), rtol=0, atol=1e-12)
        # the exact profile normalised to mean density rho0 (its integral by
        # composite Simpson on 2^16 panels)
        r_e = exact(y)
        yy = np.linspace(0, H, 65537)
        rr = exact(yy)
        hh = yy[1] - yy[0]
        integral = hh / 3 * (rr[0] + rr[-1] + 4 * rr[1:-1:2].sum() + 2 * rr[2:-1:2].sum())
        r_e = r_e * rho0 * H / integral
        errs.append(np.max(np.abs(rho - r_e)))
        # density increases downward (g_y < 0)
        assert np.all(np.diff(rho * th) < 0)
    assert 1.8 < errs[0] / errs[1] < 2.2 and 1.8 < errs[1] / errs[2] < 2.2, errs
    assert errs[-1] < 1e-3


@pytest.mark.parametrize("theta_b,theta_t", [(1.0, 1.1), (0.7, 1.4)])
def test_paper_case_solves_the_discrete_system(theta_b, theta_t):
    """The validation case of Sec. 3.1 (U_c = 1.5, Re = 1800, g_y / g_x = -50,
    H = 150 c): every discrete equation of Appendix A holds to round-off, the
    velocity peak stays below U_c and moves off the centre (cross gravity and
    heating make rho and theta asymmetric), and the profiles converge with dy
    (first order, from the forward pressure difference)."""
    p = W.poiseuille_parameters(theta_b, theta_t)
    assert math.isclose(p["gx"] * p["H"] ** 2 / (8 * p["mu"]), 1.5, rel_tol=1e-14)
    out = {}
    for N in (451, 901, 1801):
        y, rho, u, th, it = fd.solve(N, p["H"], p["gx"], p["gy"], p["mu"], p["lam"],
                                     theta_b=theta_b, theta_t=theta_t)
        ru, rp, re, rm = fd.residuals(y, rho, u, th, p["gx"], p["gy"], p["mu"], p["lam"])
        assert max(ru, rp, re) < 1e-12 and rm < 1e-9 * N
        out[N] = (y, rho, u, th)
    y, rho, u, th = out[451]
    assert u.max() < 1.5
    assert abs(y[np.argmax(u)] / p["H"] - 0.5) > 1e-3
    assert rho[0] > rho[-1]
    # convergence at coinciding nodes: rho first order (the forward pressure
    # difference); theta mixes that with the central schemes' second order
    def diff(k, a, b):
        return np.max(np.abs(out[a][k] - out[b][k][::2]))
    r1, r2 = diff(1, 451, 901), diff(1, 901, 1801)
    assert 1.85 < r1 / r2 < 2.15, (r1, r2)
    t1, t2 = diff(3, 451, 901), diff(3, 901, 1801)
    assert 1.9 < t1 / t2 < 3.0, (t1, t2)
