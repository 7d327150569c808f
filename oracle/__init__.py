"""FP64 CPU oracle of the thermal compressible LBM step (test infrastructure).

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline /
reference leg of ``bench.py`` may import this package.  The CUDA library and
its Python binding never import it, and it imports nothing from them.

``lbm_oracle.c`` holds the arithmetic (tensor-form Hermite algebra, Sec. 2 of
Li & Shan); this module only compiles it with gcc and marshals arguments
through ctypes.  Velocity ordering is the oracle's own (``lattice_info``);
compare with other implementations by matching velocity vectors.
"""
import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liblbm_oracle.so")
_lock = threading.Lock()
_lib = None

D2Q37, D3Q39 = 0, 1
PERIODIC, BOUNCE_BACK, THERMAL_WALL = 0, 1, 2

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)
_lp = ctypes.POINTER(ctypes.c_long)


def build(force=False):
    """Compile lbm_oracle.c into oracle/_build/liblbm_oracle.so (gcc, OpenMP)."""
    src = os.path.join(_HERE, "lbm_oracle.c")
    hdr = os.path.join(_HERE, "rules.h")
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= max(os.path.getmtime(src), os.path.getmtime(hdr))):
        return _LIB_PATH
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
           "-o", tmp, src, "-lm"]
    subprocess.check_call(cmd, cwd=_HERE)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.orc_create.restype = ctypes.c_void_p
            lib.orc_create.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                       ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                       _ip, _dp, _dp, _dp]
            lib.orc_destroy.argtypes = [ctypes.c_void_p]
            lib.orc_init.argtypes = [ctypes.c_void_p, _dp, _dp, _dp]
            lib.orc_step.argtypes = [ctypes.c_void_p, ctypes.c_int]
            lib.orc_moments.argtypes = [ctypes.c_void_p, _dp, _dp, _dp, _dp, _dp]
            lib.orc_get_state.argtypes = [ctypes.c_void_p, _dp]
            lib.orc_set_state.argtypes = [ctypes.c_void_p, _dp]
            lib.orc_pull_state.argtypes = [ctypes.c_void_p, _dp]
            lib.orc_step_sites.argtypes = [ctypes.c_void_p, _dp, _lp, ctypes.c_long, _dp]
            lib.orc_lattice_info.argtypes = [ctypes.c_int, _ip, _ip, _dp, _ip, _dp, _ip]
            lib.orc_hermite_tensor.argtypes = [ctypes.c_int, ctypes.c_int, _dp, _dp]
            lib.orc_maxwell_coeff.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, _dp,
                                              ctypes.c_double, _dp]
            lib.orc_equilibrium.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, _dp,
                                            ctypes.c_double, _dp]
            lib.orc_force.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, _dp,
                                      ctypes.c_double, _dp, _dp, _dp]
            lib.orc_set_solid.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_ubyte), _dp]
            lib.orc_set_threads.argtypes = [ctypes.c_int]
            lib.orc_get_threads.restype = ctypes.c_int
            _lib = lib
    return _lib


def _p(a, typ=_dp):
    return None if a is None else a.ctypes.data_as(typ)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def set_threads(n):
    _load().orc_set_threads(int(n))


def get_threads():
    return int(_load().orc_get_threads())


def lattice_info(lat):
    """(D, Q, c, e[Q,3] int, w[Q], neq) of the oracle's quadrature rule."""
    lib = _load()
    D, Q, neq = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    c = ctypes.c_double()
    e = np.zeros((39, 3), dtype=np.int32)
    w = np.zeros(39)
    if lib.orc_lattice_info(lat, ctypes.byref(D), ctypes.byref(Q), ctypes.byref(c), _p(e, _ip),
                            _p(w), ctypes.byref(neq)):
        raise ValueError(f"unknown lattice {lat}")
    q = Q.value
    return D.value, q, c.value, e[:q].copy(), w[:q].copy(), neq.value


def hermite_tensor(D, n, xi):
    out = np.zeros(D ** n)
    if _load().orc_hermite_tensor(D, n, _p(_f64(xi)), _p(out)):
        raise ValueError("bad arguments")
    return out.reshape((D,) * n) if n else out[0]


def maxwell_coeff(D, n, rho, u, theta):
    out = np.zeros(D ** n)
    if _load().orc_maxwell_coeff(D, n, float(rho), _p(_f64(u)), float(theta), _p(out)):
        raise ValueError("bad arguments")
    return out.reshape((D,) * n) if n else out[0]


def equilibrium(lat, rho, u, theta, neq=-1):
    D, Q = lattice_info(lat)[:2]
    out = np.zeros(Q)
    u3 = np.zeros(3)
    u3[:D] = u
    if _load().orc_equilibrium(lat, neq, float(rho), _p(u3), float(theta), _p(out)):
        raise ValueError("bad arguments")
    return out


def force(lat, order, rho, u, theta, g, sigma=None):
    D, Q = lattice_info(lat)[:2]
    out = np.zeros(Q)
    u3, g3 = np.zeros(3), np.zeros(3)
    u3[:D] = u
    g3[:D] = g
    sp = None if sigma is None else _f64(np.asarray(sigma).reshape(D * D))
    if _load().orc_force(lat, order, float(rho), _p(u3), float(theta), _p(g3), _p(sp), _p(out)):
        raise ValueError("bad arguments")
    return out


class OracleSim:
    """One simulation on the CPU oracle.

    Field layout: scalars (N,), vectors (D, N) with N = nx*ny*nz and x fastest.
    ``tau`` is the collision divisor tau-hat of Eq. lbm.  ``g`` is the (D, N)
    acceleration field.  ``bc`` per axis: PERIODIC, BOUNCE_BACK, THERMAL_WALL.
    ``mu`` > 0 selects constant dynamic viscosity: tau-hat = mu / (rho theta)
    + 1/2 per site (the paper's validation runs); ``tau`` is then unused.
    """

    def __init__(self, lat, nx, ny, nz, tau, g, force_order=2, include_sigma=False,
                 bc=(0, 0, 0), T_lo=(1.0, 1.0, 1.0), T_hi=(1.0, 1.0, 1.0), mu=0.0):
        self.lib = _load()
        self.D, self.Q, self.c, self.e, self.w, self.neq = lattice_info(lat)
        if self.D == 2:
            nz = 1
        self.shape = (nx, ny, nz)
        self.N = nx * ny * nz
        g = _f64(np.asarray(g).reshape(self.D, self.N))
        bca = np.asarray(list(bc) + [0] * (3 - len(bc)), dtype=np.int32)
        self.h = self.lib.orc_create(lat, nx, ny, nz, float(tau), float(mu), int(force_order),
                                     int(bool(include_sigma)), _p(bca, _ip),
                                     _p(_f64(T_lo)), _p(_f64(T_hi)), _p(g))
        if not self.h:
            raise ValueError("orc_create rejected the arguments")

    def __del__(self):
        if getattr(self, "h", None):
            self.lib.orc_destroy(self.h)
            self.h = None

    def set_solid(self, solid, T_wall):
        """Solid sites (N flags) with wall temperatures (N) -- curved walls as a
        staircase of diffuse thermal walls; fully periodic grids only, before
        init."""
        solid = np.ascontiguousarray(np.asarray(solid).reshape(self.N) != 0, dtype=np.uint8)
        T_wall = _f64(np.asarray(T_wall).reshape(self.N))
        if self.lib.orc_set_solid(self.h, solid.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte)),
                                  _p(T_wall)):
            raise ValueError("orc_set_solid rejected the arguments")

    def init(self, rho, u, T):
        rho = _f64(np.asarray(rho).reshape(self.N))
        u = _f64(np.asarray(u).reshape(self.D, self.N))
        T = _f64(np.asarray(T).reshape(self.N))
        self.lib.orc_init(self.h, _p(rho), _p(u), _p(T))

    def step(self, n=1):
        self.lib.orc_step(self.h, int(n))

    def moments(self, with_sigma=False):
        rho = np.zeros(self.N)
        u = np.zeros((self.D, self.N))
        T = np.zeros(self.N)
        q = np.zeros((self.D, self.N))
        sig = np.zeros((self.D * self.D, self.N)) if with_sigma else None
        self.lib.orc_moments(self.h, _p(rho), _p(u), _p(T), _p(q), _p(sig))
        if with_sigma:
            return rho, u, T, q, sig.reshape(self.D, self.D, self.N)
        return rho, u, T, q

    def get_state(self):
        f = np.zeros((self.Q, self.N))
        self.lib.orc_get_state(self.h, _p(f))
        return f

    def set_state(self, f):
        self.lib.orc_set_state(self.h, _p(_f64(np.asarray(f).reshape(self.Q, self.N))))

    def pulled(self):
        f = np.zeros((self.Q, self.N))
        self.lib.orc_pull_state(self.h, _p(f))
        return f

    def step_sites(self, state, sites):
        """One step from ``state`` (Q, N) evaluated at ``sites`` -> (len(sites), Q)."""
        sites = np.ascontiguousarray(sites, dtype=np.int64)
        out = np.zeros((len(sites), self.Q))
        self.lib.orc_step_sites(self.h, _p(_f64(np.asarray(state).reshape(self.Q, self.N))),
                                _p(sites, _lp), len(sites), _p(out))
        return out
