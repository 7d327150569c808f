"""Analytic reference of the concentric-cylinder test (Sec. 3.2).  Test
infrastructure, like the rest of ``oracle/``: only the test suite uses it.

In the frame rotating with both cylinders the fluid is static under the
centrifugal acceleration alpha^2 R.  Steady conduction with constant
conductivity between the walls at R_i (theta_i) and R_o (theta_o) gives
    theta(R) = theta_i + (theta_o - theta_i) ln(R / R_i) / ln(R_o / R_i),
and radial hydrostatic balance d(rho theta)/dR = rho alpha^2 R gives
    rho(R) = (rho_i theta_i / theta(R)) exp( int_{R_i}^{R} alpha^2 r / theta(r) dr ),
with rho_i fixed by the mean density.
"""
import math

import numpy as np
from scipy.integrate import quad


def theta(R, Ri, Ro, theta_i, theta_o):
    return theta_i + (theta_o - theta_i) * np.log(np.asarray(R) / Ri) / math.log(Ro / Ri)


def _exponent(R, Ri, Ro, theta_i, theta_o, alpha, panels=1 << 16):
    """int_{R_i}^{R} alpha^2 r / theta(r) dr: cumulative Simpson on a uniform
    grid of 2 * panels intervals over [R_i, R_o], then linear interpolation
    (both errors far below 1e-12 for this smooth integrand)."""
    r = np.linspace(Ri, Ro, 2 * panels + 1)
    f = alpha * alpha * r / theta(r, Ri, Ro, theta_i, theta_o)
    h = r[1] - r[0]
    # Simpson over each pair of intervals, accumulated at the even nodes
    pair = h / 3.0 * (f[0:-2:2] + 4.0 * f[1:-1:2] + f[2::2])
    even = np.concatenate(([0.0], np.cumsum(pair)))
    # odd nodes: even node before + Simpson-type quadrature over one interval
    # (quadratic through the three nodes of the pair)
    half = h / 12.0 * (5.0 * f[0:-2:2] + 8.0 * f[1:-1:2] - f[2::2])
    vals = np.empty_like(r)
    vals[0::2] = even
    vals[1::2] = even[:-1] + half
    return np.interp(np.asarray(R, dtype=np.float64), r, vals)


def exponent_by_quad(R, Ri, Ro, theta_i, theta_o, alpha):
    """The same integral by adaptive quadrature, point by point (for checks)."""
    f = lambda r: alpha * alpha * r / float(theta(r, Ri, Ro, theta_i, theta_o))
    R = np.atleast_1d(np.asarray(R, dtype=np.float64))
    return np.array([quad(f, Ri, x, epsabs=1e-15, epsrel=1e-13, limit=200)[0] for x in R])


def density_shape(R, Ri, Ro, theta_i, theta_o, alpha):
    """rho(R) / rho_i."""
    th = theta(R, Ri, Ro, theta_i, theta_o)
    return theta_i / th * np.exp(_exponent(R, Ri, Ro, theta_i, theta_o, alpha))


def profiles(R, Ri, Ro, theta_i, theta_o, alpha, rho0=1.0, mean_over=None):
    """(rho, theta) at radii R.  rho_i is set so that the mean density is rho0:
    over the continuous annulus (area weight 2 pi r dr) when mean_over is None,
    else over the radii ``mean_over`` (e.g. the fluid sites of a lattice, each
    of equal area)."""
    shape = density_shape(R, Ri, Ro, theta_i, theta_o, alpha)
    if mean_over is None:
        g = lambda r: 2.0 * math.pi * r * float(density_shape(r, Ri, Ro, theta_i, theta_o, alpha))
        mass = quad(g, Ri, Ro, epsabs=1e-12, epsrel=1e-12, limit=200)[0]
        rho_i = rho0 * math.pi * (Ro * Ro - Ri * Ri) / mass
    else:
        rho_i = rho0 / float(np.mean(density_shape(mean_over, Ri, Ro, theta_i, theta_o, alpha)))
    return rho_i * shape, theta(R, Ri, Ro, theta_i, theta_o)
