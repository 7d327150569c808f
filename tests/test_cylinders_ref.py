"""Pins of the concentric-cylinder reference (Sec. 3.2) against closed forms
and independent quadrature."""
import math

import numpy as np
import pytest

from oracle import cylinders_ref as cr
from paper_2302_04741_gb300 import workloads as W


def test_parameters_follow_the_definitions():
    p = W.cylinders_parameters(1.0, 1.1)
    assert math.isclose(p["Ro"], 250 * W.C_D2Q37 / 2, rel_tol=1e-15)
    assert math.isclose(p["Ro"] / p["Ri"], 5.0, rel_tol=1e-15)
    assert math.isclose(p["alpha"] * (p["Ro"] + p["Ri"]) / 2, 0.3, rel_tol=1e-14)
    Re = p["rho0"] * p["alpha"] * (p["Ro"] ** 2 - p["Ri"] ** 2) / (2 * p["mu"])
    assert math.isclose(Re, 100.0, rel_tol=1e-14)


def test_theta_is_harmonic_with_wall_values():
    Ri, Ro = 3.0, 15.0
    R = np.linspace(Ri, Ro, 7)
    th = cr.theta(R, Ri, Ro, 1.4, 0.7)
    assert th[0] == pytest.approx(1.4, abs=1e-15) and th[-1] == pytest.approx(0.7, abs=1e-15)
    # (1/r) d/dr (r dtheta/dr) = 0: r dtheta/dr is constant
    h = 1e-4
    flux = [r * (cr.theta(r + h, Ri, Ro, 1.4, 0.7) - cr.theta(r - h, Ri, Ro, 1.4, 0.7)) / (2 * h)
            for r in R[1:-1]]
    np.testing.assert_allclose(flux, flux[0], rtol=1e-7)


def test_isothermal_density_is_gaussian_in_radius():
    """theta_i = theta_o = T: rho ~ exp(alpha^2 R^2 / (2 T))."""
    Ri, Ro, T, a = 20.0, 100.0, 1.2, 4e-3
    R = np.linspace(Ri, Ro, 11)
    shape = cr.density_shape(R, Ri, Ro, T, T, a)
    np.testing.assert_allclose(shape, np.exp(a * a * (R * R - Ri * Ri) / (2 * T)), rtol=1e-12)


@pytest.mark.parametrize("thetas", [(1.0, 1.1), (1.4, 0.7)])
def test_exponent_matches_adaptive_quadrature(thetas):
    p = W.cylinders_parameters(*thetas)
    R = np.linspace(p["Ri"], p["Ro"], 9)
    a = cr._exponent(R, p["Ri"], p["Ro"], *thetas, p["alpha"])
    b = cr.exponent_by_quad(R, p["Ri"], p["Ro"], *thetas, p["alpha"])
    np.testing.assert_allclose(a, b, rtol=1e-11, atol=1e-15)


@pytest.mark.parametrize("thetas", [(1.0, 1.1), (1.4, 0.7)])
def test_hydrostatic_balance_and_mean_density(thetas):
    """d(rho theta)/dR = rho alpha^2 R, and the area mean of rho is rho0."""
    p = W.cylinders_parameters(*thetas)
    Ri, Ro, a = p["Ri"], p["Ro"], p["alpha"]
    R = np.linspace(Ri + 1, Ro - 1, 9)
    h = 1e-3
    rho, th = cr.profiles(R, Ri, Ro, *thetas, a)
    rp, tp = cr.profiles(R + h, Ri, Ro, *thetas, a)
    rm, tm = cr.profiles(R - h, Ri, Ro, *thetas, a)
    dp = (rp * tp - rm * tm) / (2 * h)
    np.testing.assert_allclose(dp, rho * a * a * R, rtol=1e-6)
    r = np.linspace(Ri, Ro, 200001)
    rr, _ = cr.profiles(r, Ri, Ro, *thetas, a)
    trap = getattr(np, "trapezoid", None) or np.trapz
    mass = trap(2 * np.pi * r * rr, r)
    assert mass / (np.pi * (Ro ** 2 - Ri ** 2)) == pytest.approx(1.0, rel=1e-8)
