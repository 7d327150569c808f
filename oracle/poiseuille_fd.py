"""Finite-difference reference for compressible Poiseuille flow under cross
gravity (the paper's Appendix A).  Test infrastructure, like the rest of
``oracle/``: only the test suite uses it.

The steady, one-dimensional flow between plates at y = 0 and y = H (all
fields functions of y, u_y = 0) obeys the reduced Navier-Stokes-Fourier
equations of Sec. 3.1,

    -mu u''          = rho g_x          (horizontal momentum)
    (rho theta)'     = rho g_y          (vertical momentum)
    mu u'^2 + lambda theta'' = 0        (energy: viscous heating + conduction)

with constant mu and lambda, Dirichlet values u = U_b, U_t and theta =
theta_b, theta_t at the plates, and the mean density fixed to rho_0.

Discretisation (Appendix A): N nodes, dy = H / (N - 1); central second
differences for the horizontal momentum and energy equations, a forward first
difference for the vertical momentum equation, and the trapezoidal rule for
the mass constraint.  The viscous-heating term is lagged one iteration, which
leaves three linear problems solved in turn: theta (tridiagonal), rho (a
product recursion normalised by the mass constraint), u (tridiagonal).  The
iteration starts from the parabola of homogeneous rho and theta and stops when
no field changes by more than ``tol`` (relative to its scale).
"""
import numpy as np
from scipy.linalg import solve_banded


def _dirichlet_second_difference(rhs, left, right):
    """Solves v_{j+1} - 2 v_j + v_{j-1} = rhs_j (interior j) with v_0 = left,
    v_{N-1} = right.  rhs has N - 2 entries; returns the N values."""
    m = len(rhs)
    ab = np.zeros((3, m))
    ab[0, 1:] = 1.0
    ab[1, :] = -2.0
    ab[2, :-1] = 1.0
    b = np.array(rhs, dtype=np.float64)
    b[0] -= left
    b[-1] -= right
    v = np.empty(m + 2)
    v[0], v[-1] = left, right
    v[1:-1] = solve_banded((1, 1), ab, b)
    return v


def solve(N, H, gx, gy, mu, lam, rho0=1.0, U_b=0.0, U_t=0.0, theta_b=1.0, theta_t=1.0,
          tol=1e-14, max_iter=500):
    """Steady profiles on the N nodes y_k = k H / (N - 1).

    Returns (y, rho, u, theta, iterations)."""
    if N < 3:
        raise ValueError("need N >= 3 nodes")
    dy = H / (N - 1)
    y = np.linspace(0.0, H, N)
    # initial guess: the parabola of homogeneous rho = rho0
    u = -gx / (2.0 * mu) * y * (y - H) + (U_t - U_b) / H * y + U_b
    rho = np.full(N, rho0)
    theta = np.linspace(theta_b, theta_t, N)
    for it in range(1, max_iter + 1):
        # energy: 4 lam (theta_{j+1} - 2 theta_j + theta_{j-1}) = -mu (u_{j+1} - u_{j-1})^2
        heat = mu * (u[2:] - u[:-2]) ** 2
        theta_n = _dirichlet_second_difference(-heat / (4.0 * lam), theta_b, theta_t)
        # vertical momentum: rho_{j+1} theta_{j+1} = rho_j (theta_j + g_y dy), then
        # the trapezoidal mass constraint fixes the overall factor
        ratio = (theta_n[:-1] + gy * dy) / theta_n[1:]
        if np.any(ratio <= 0.0):
            raise ValueError("g_y dy too large for the forward pressure recursion")
        shape = np.concatenate(([1.0], np.cumprod(ratio)))
        mass = 0.5 * shape[0] + shape[1:-1].sum() + 0.5 * shape[-1]
        rho_n = shape * rho0 * (N - 1) / mass
        # horizontal momentum: u_{j+1} - 2 u_j + u_{j-1} = -(g_x dy^2 / mu) rho_j
        u_n = _dirichlet_second_difference(-(gx * dy * dy / mu) * rho_n[1:-1], U_b, U_t)
        du = np.max(np.abs(u_n - u)) / max(np.max(np.abs(u_n)), 1e-300)
        dt = np.max(np.abs(theta_n - theta)) / np.max(np.abs(theta_n))
        dr = np.max(np.abs(rho_n - rho)) / np.max(np.abs(rho_n))
        u, theta, rho = u_n, theta_n, rho_n
        if max(du, dt, dr) <= tol:
            return y, rho, u, theta, it
    raise RuntimeError(f"no convergence in {max_iter} iterations")


def residuals(y, rho, u, theta, gx, gy, mu, lam, rho0=1.0):
    """Max residual of each discrete equation of Appendix A (for checks)."""
    N = len(y)
    dy = y[1] - y[0]
    r_u = u[2:] - 2 * u[1:-1] + u[:-2] + gx * dy * dy / mu * rho[1:-1]
    r_p = rho[1:] * theta[1:] - rho[:-1] * (theta[:-1] + gy * dy)
    r_e = mu * (u[2:] - u[:-2]) ** 2 + 4 * lam * (theta[2:] - 2 * theta[1:-1] + theta[:-2])
    r_m = 0.5 * rho[0] + rho[1:-1].sum() + 0.5 * rho[-1] - rho0 * (N - 1)
    return (float(np.max(np.abs(r_u))), float(np.max(np.abs(r_p))), float(np.max(np.abs(r_e))),
            abs(float(r_m)))

