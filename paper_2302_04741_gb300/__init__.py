"""GB300-native thermal compressible lattice Boltzmann step with the
third-order Hermite body force of Li & Shan (arXiv 2302.04741).

This package is a thin ctypes binding of the C ABI in ``include/lbm.h``
(functions of the same names) plus ``Sim``, a convenience wrapper that only
allocates output arrays and marshals arguments.  Every step of the method
runs in the CUDA library ``_build/liblbm_gb300.so``; there is no CPU path:
if the library is missing or cannot be loaded, every call raises.

Arrays may be numpy arrays (host) or torch tensors (host or CUDA); they are
passed by pointer.  Device arrays must be contiguous float64 on the current
device.
"""
import ctypes
import os

import numpy as np

from . import workloads  # noqa: F401  (input generators, no method arithmetic)

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "liblbm_gb300.so")

LBM_D2Q37, LBM_D3Q39 = 0, 1
LBM_OK, LBM_EINVAL, LBM_ENOMEM, LBM_ECUDA, LBM_EUNSTABLE, LBM_ETIMEOUT, LBM_ESTATE, LBM_EIO = (
    0, -1, -2, -3, -4, -5, -6, -7)
LBM_G_UNIFORM, LBM_G_SINE, LBM_G_FIELD = 0, 1, 2
LBM_FP64, LBM_FP32_SHIFTED, LBM_FP16_SCALED = 0, 1, 2
LBM_PERIODIC, LBM_BOUNCE_BACK, LBM_THERMAL_WALL = 0, 1, 2
LBM_KERNEL_AUTO, LBM_KERNEL_PLAIN, LBM_KERNEL_TMA, LBM_KERNEL_PREFETCH, LBM_KERNEL_WAVE = 0, 1, 2, 3, 4
LBM_ARITH_DOUBLE, LBM_ARITH_FLOAT_PAIR = 0, 1
STATUS_NAMES = {0: "LBM_OK", -1: "LBM_EINVAL", -2: "LBM_ENOMEM", -3: "LBM_ECUDA",
                -4: "LBM_EUNSTABLE", -5: "LBM_ETIMEOUT", -6: "LBM_ESTATE", -7: "LBM_EIO"}


class lbm_gfield(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("g0", ctypes.c_double * 3), ("wave_axis", ctypes.c_int),
                ("field", ctypes.c_void_p)]


class lbm_options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("force_order", ctypes.c_int),
                ("include_sigma", ctypes.c_int), ("bc", ctypes.c_int * 3),
                ("T_lo", ctypes.c_double * 3), ("T_hi", ctypes.c_double * 3),
                ("stream", ctypes.c_void_p), ("block_x", ctypes.c_int),
                ("graph_steps", ctypes.c_int), ("kernel", ctypes.c_int),
                ("tma_stages", ctypes.c_int), ("mu", ctypes.c_double),
                ("overlap_steps", ctypes.c_int), ("storage_probe", ctypes.c_int),
                ("fp64_arith", ctypes.c_int)]


class LbmError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


_lib = None
_dp = ctypes.POINTER(ctypes.c_double)
_vp = ctypes.c_void_p


def lib():
    """The loaded CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"CUDA library not built: {LIB_PATH} is missing "
                               "(run paper_2302_04741_gb300.build.build())")
        L = ctypes.CDLL(LIB_PATH)
        L.lbm_options_size.restype = ctypes.c_size_t
        if L.lbm_options_size() != ctypes.sizeof(lbm_options):
            raise RuntimeError(f"lbm_options layout mismatch: library {L.lbm_options_size()} B, "
                               f"binding {ctypes.sizeof(lbm_options)} B")
        L.lbm_default_options.argtypes = [ctypes.POINTER(lbm_options)]
        L.lbm_default_options.restype = None
        L.lbm_lattice_info.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                       ctypes.POINTER(ctypes.c_int), _dp,
                                       ctypes.POINTER(ctypes.c_int), _dp]
        L.lbm_create.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                 ctypes.c_double, ctypes.POINTER(lbm_gfield),
                                 ctypes.POINTER(lbm_options), ctypes.POINTER(_vp)]
        for name in ("lbm_init",):
            getattr(L, name).argtypes = [_vp, _vp, _vp, _vp]
        L.lbm_step.argtypes = [_vp, ctypes.c_int]
        L.lbm_set_solid.argtypes = [_vp, ctypes.POINTER(ctypes.c_ubyte), _dp]
        L.lbm_moments.argtypes = [_vp, _vp, _vp, _vp, _vp]
        L.lbm_conserved.argtypes = [_vp, _dp, _dp, _dp]
        L.lbm_moments_async.argtypes = [_vp, _vp, _vp, _vp, _vp]
        L.lbm_set_params.argtypes = [_vp, ctypes.c_double, ctypes.POINTER(lbm_gfield)]
        for name in ("lbm_get_populations", "lbm_get_state", "lbm_set_state"):
            getattr(L, name).argtypes = [_vp, _vp]
        L.lbm_step_kernel.argtypes = [_vp]
        L.lbm_step_count.argtypes = [_vp]
        L.lbm_step_count.restype = ctypes.c_longlong
        L.lbm_fp16_scale.argtypes = [_vp]
        L.lbm_fp16_scale.restype = ctypes.c_double
        L.lbm_device_bytes.argtypes = [_vp]
        L.lbm_device_bytes.restype = ctypes.c_size_t
        L.lbm_save.argtypes = [_vp, ctypes.c_char_p]
        L.lbm_load.argtypes = [_vp, ctypes.c_char_p]
        L.lbm_last_error.argtypes = [_vp]
        L.lbm_last_error.restype = ctypes.c_char_p
        L.lbm_destroy.argtypes = [_vp]
        L.lbm_destroy.restype = None
        L.lbm_batch_create.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, _vp, ctypes.c_int,
                                       ctypes.POINTER(_vp)]
        for name in ("lbm_batch_add", "lbm_batch_remove"):
            getattr(L, name).argtypes = [_vp, _vp]
        L.lbm_batch_size.argtypes = [_vp]
        L.lbm_batch_set_config.argtypes = [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int]
        L.lbm_batch_get_config.argtypes = [_vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                           ctypes.POINTER(ctypes.c_int)]
        L.lbm_batch_step.argtypes = [_vp, ctypes.c_int]
        L.lbm_batch_set_staging.argtypes = [_vp, ctypes.c_int]
        L.lbm_batch_get_staging.argtypes = [_vp, ctypes.POINTER(ctypes.c_int)]
        L.lbm_batch_tune.argtypes = [_vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                     ctypes.POINTER(ctypes.c_int)]
        L.lbm_batch_last_error.argtypes = [_vp]
        L.lbm_batch_last_error.restype = ctypes.c_char_p
        L.lbm_batch_destroy.argtypes = [_vp]
        L.lbm_batch_destroy.restype = None
        L.lbm_create_slab.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                      ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                      ctypes.POINTER(lbm_gfield), ctypes.POINTER(lbm_options),
                                      ctypes.POINTER(_vp)]
        L.lbm_slab_exchange.argtypes = [_vp, _vp]
        L.lbm_slab_halo_bytes.argtypes = [_vp]
        L.lbm_slab_halo_bytes.restype = ctypes.c_size_t
        L.lbm_slab_halo_pack.argtypes = [_vp, ctypes.c_int, _vp]
        L.lbm_slab_halo_unpack.argtypes = [_vp, ctypes.c_int, _vp]
        L.lbm_slab_info.argtypes = [_vp] + [ctypes.POINTER(ctypes.c_int)] * 4
        L.lbm_set_fp16_scale.argtypes = [_vp, ctypes.c_double]
        L.lbm_conserved_static.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                           ctypes.POINTER(lbm_options), ctypes.POINTER(lbm_gfield),
                                           ctypes.c_double, _vp, _vp]
        _lib = L
    return _lib


def _check(rc, ctx=None):
    if rc != LBM_OK:
        raise LbmError(rc, lib().lbm_last_error(ctx).decode())
    return rc


def _ptr(a):
    """Raw address of a numpy array or torch tensor (must be contiguous float64)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        if a.dtype.__str__() != "torch.float64" or not a.is_contiguous():
            raise TypeError("torch tensors must be contiguous float64")
        return a.data_ptr()
    if not isinstance(a, np.ndarray) or a.dtype != np.float64 or not a.flags.c_contiguous:
        raise TypeError("numpy arrays must be C-contiguous float64")
    return a.ctypes.data


# ---------------------------------------------------------------- the C ABI
def lbm_default_options():
    o = lbm_options()
    lib().lbm_default_options(ctypes.byref(o))
    return o


def lbm_lattice_info(lat):
    """(D, Q, c, e[Q, 3] int, w[Q]) in the library's direction order."""
    D, Q = ctypes.c_int(), ctypes.c_int()
    c = ctypes.c_double()
    e = np.zeros((39, 3), dtype=np.int32)
    w = np.zeros(39)
    _check(lib().lbm_lattice_info(lat, ctypes.byref(D), ctypes.byref(Q), ctypes.byref(c),
                                  e.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                  w.ctypes.data_as(_dp)))
    q = Q.value
    return D.value, q, c.value, e[:q].copy(), w[:q].copy()


def make_gfield(g):
    """lbm_gfield from a workload descriptor dict (see workloads.g_field_array)."""
    gf = lbm_gfield()
    gf.kind = g["kind"]
    g0 = list(g.get("g0", (0.0, 0.0, 0.0))) + [0.0] * 3
    for a in range(3):
        gf.g0[a] = g0[a]
    gf.wave_axis = g.get("wave_axis", 0)
    gf.field = _ptr(g["field"]) if g["kind"] == LBM_G_FIELD else None
    return gf


def lbm_create(lat, nx, ny, nz, tau, g=None, opt=None):
    ctx = _vp()
    gf = make_gfield(g) if isinstance(g, dict) else g
    rc = lib().lbm_create(lat, nx, ny, nz, tau, ctypes.byref(gf) if gf is not None else None,
                          ctypes.byref(opt) if opt is not None else None, ctypes.byref(ctx))
    _check(rc)
    return ctx


def lbm_init(ctx, rho, u, T):
    _check(lib().lbm_init(ctx, _ptr(rho), _ptr(u), _ptr(T)), ctx)


def lbm_step(ctx, n):
    _check(lib().lbm_step(ctx, int(n)), ctx)


def lbm_set_solid(ctx, solid, T_wall):
    """solid: N flags (non-zero = solid); T_wall: N wall temperatures (host)."""
    s = np.ascontiguousarray(np.asarray(solid).ravel() != 0, dtype=np.uint8)
    t = np.ascontiguousarray(np.asarray(T_wall, dtype=np.float64).ravel())
    _check(lib().lbm_set_solid(ctx, s.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte)),
                               t.ctypes.data_as(_dp)), ctx)


def lbm_moments(ctx, rho=None, u=None, T=None, q=None):
    _check(lib().lbm_moments(ctx, _ptr(rho), _ptr(u), _ptr(T), _ptr(q)), ctx)


def lbm_moments_async(ctx, rho=None, u=None, T=None, q=None):
    """Enqueues the moments into device (or page-locked) float64 tensors."""
    _check(lib().lbm_moments_async(ctx, _ptr(rho), _ptr(u), _ptr(T), _ptr(q)), ctx)


def lbm_set_params(ctx, tau, g=None):
    """New tau-hat and uniform force (workload-style dict or None) for a context."""
    gf = make_gfield(g) if isinstance(g, dict) else g
    _check(lib().lbm_set_params(ctx, float(tau), ctypes.byref(gf) if gf is not None else None), ctx)


def lbm_conserved(ctx, D, raise_unstable=True):
    """(status, mass, momentum[D], energy)."""
    m, e = ctypes.c_double(), ctypes.c_double()
    mom = (ctypes.c_double * 3)()
    rc = lib().lbm_conserved(ctx, ctypes.byref(m), mom, ctypes.byref(e))
    if rc != LBM_EUNSTABLE or raise_unstable:
        _check(rc, ctx)
    return rc, m.value, np.array(mom[:D]), e.value


def lbm_get_populations(ctx, out):
    _check(lib().lbm_get_populations(ctx, _ptr(out)), ctx)


def lbm_get_state(ctx, out):
    _check(lib().lbm_get_state(ctx, _ptr(out)), ctx)


def lbm_set_state(ctx, inp):
    _check(lib().lbm_set_state(ctx, _ptr(inp)), ctx)


def lbm_step_kernel(ctx):
    return int(lib().lbm_step_kernel(ctx))


def lbm_step_count(ctx):
    return int(lib().lbm_step_count(ctx))


def lbm_fp16_scale(ctx):
    return float(lib().lbm_fp16_scale(ctx))


def lbm_device_bytes(ctx):
    return int(lib().lbm_device_bytes(ctx))


def lbm_save(ctx, path):
    _check(lib().lbm_save(ctx, os.fsencode(path)), ctx)


def lbm_load(ctx, path):
    _check(lib().lbm_load(ctx, os.fsencode(path)), ctx)


def lbm_last_error(ctx=None):
    return lib().lbm_last_error(ctx).decode()


def lbm_destroy(ctx):
    if ctx:
        lib().lbm_destroy(ctx)


def lbm_conserved_static(lat, nx, ny, nz, opt, g, fp16_scale, f, out):
    """Allocation-free conservation sums of a raw device population buffer
    ``f`` into the device array ``out`` (6 doubles); see include/lbm.h.
    ``f`` and ``out`` are device pointers (int) or CUDA tensors."""
    gf = make_gfield(g) if isinstance(g, dict) else g
    fp = f.data_ptr() if hasattr(f, "data_ptr") else f
    op = out.data_ptr() if hasattr(out, "data_ptr") else out
    _check(lib().lbm_conserved_static(lat, nx, ny, nz,
                                      ctypes.byref(opt) if opt is not None else None,
                                      ctypes.byref(gf) if gf is not None else None,
                                      float(fp16_scale), fp, op))


def lbm_create_slab(lat, nx, ny, nz, a_begin, a_end, tau, g=None, opt=None):
    """Slab [a_begin, a_end) of the last axis of an nx x ny x nz grid (see include/lbm.h)."""
    ctx = _vp()
    gf = make_gfield(g) if isinstance(g, dict) else g
    rc = lib().lbm_create_slab(lat, nx, ny, nz, a_begin, a_end, tau,
                               ctypes.byref(gf) if gf is not None else None,
                               ctypes.byref(opt) if opt is not None else None, ctypes.byref(ctx))
    _check(rc)
    return ctx


def lbm_slab_exchange(lo, hi):
    _check(lib().lbm_slab_exchange(lo, hi), lo)


def lbm_slab_halo_bytes(ctx):
    return int(lib().lbm_slab_halo_bytes(ctx))


def lbm_slab_halo_pack(ctx, side, dst):
    """dst: device pointer (int) or CUDA tensor of lbm_slab_halo_bytes(ctx) bytes."""
    _check(lib().lbm_slab_halo_pack(ctx, int(side), dst.data_ptr() if hasattr(dst, "data_ptr") else dst), ctx)


def lbm_slab_halo_unpack(ctx, side, src):
    _check(lib().lbm_slab_halo_unpack(ctx, int(side), src.data_ptr() if hasattr(src, "data_ptr") else src), ctx)


def lbm_slab_info(ctx):
    """(a_begin, a_end, ghosts_below, ghosts_above)."""
    v = [ctypes.c_int() for _ in range(4)]
    _check(lib().lbm_slab_info(ctx, *[ctypes.byref(x) for x in v]), ctx)
    return tuple(x.value for x in v)


def lbm_set_fp16_scale(ctx, scale):
    _check(lib().lbm_set_fp16_scale(ctx, float(scale)), ctx)


def _bcheck(rc, b):
    if rc != LBM_OK:
        raise LbmError(rc, lib().lbm_batch_last_error(b).decode())


def lbm_batch_create(lat, precision, force_order=2, stream=None, capacity=1024):
    b = _vp()
    rc = lib().lbm_batch_create(lat, precision, force_order, stream, capacity, ctypes.byref(b))
    _bcheck(rc, None)
    return b


def lbm_batch_add(b, ctx):
    _bcheck(lib().lbm_batch_add(b, ctx), b)


def lbm_batch_remove(b, ctx):
    _bcheck(lib().lbm_batch_remove(b, ctx), b)


def lbm_batch_size(b):
    return int(lib().lbm_batch_size(b))


def lbm_batch_set_config(b, block_x=128, sites_per_thread=1, graph_steps=0):
    _bcheck(lib().lbm_batch_set_config(b, block_x, sites_per_thread, graph_steps), b)


def lbm_batch_get_config(b):
    bx, spt, gs = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _bcheck(lib().lbm_batch_get_config(b, ctypes.byref(bx), ctypes.byref(spt), ctypes.byref(gs)), b)
    return bx.value, spt.value, gs.value


def lbm_batch_set_staging(b, staged):
    _bcheck(lib().lbm_batch_set_staging(b, int(staged)), b)


def lbm_batch_get_staging(b):
    v = ctypes.c_int()
    _bcheck(lib().lbm_batch_get_staging(b, ctypes.byref(v)), b)
    return v.value


def lbm_batch_step(b, n):
    _bcheck(lib().lbm_batch_step(b, int(n)), b)


def lbm_batch_tune(b, trial_steps=10):
    bx, spt = ctypes.c_int(), ctypes.c_int()
    _bcheck(lib().lbm_batch_tune(b, int(trial_steps), ctypes.byref(bx), ctypes.byref(spt)), b)
    return bx.value, spt.value


def lbm_batch_last_error(b):
    return lib().lbm_batch_last_error(b).decode()


def lbm_batch_destroy(b):
    if b:
        lib().lbm_batch_destroy(b)


# ------------------------------------------------------------ convenience
def options(precision=LBM_FP64, force_order=2, bc=(0, 0, 0), T_lo=(1.0, 1.0, 1.0),
            T_hi=(1.0, 1.0, 1.0), stream=None, block_x=0, graph_steps=0, kernel=LBM_KERNEL_AUTO,
            tma_stages=0, mu=0.0, include_sigma=False, overlap_steps=-1, storage_probe=0, fp64_arith=0):
    o = lbm_default_options()
    o.precision = precision
    o.force_order = force_order
    o.include_sigma = int(bool(include_sigma))
    for a in range(3):
        o.bc[a] = bc[a]
        o.T_lo[a] = T_lo[a]
        o.T_hi[a] = T_hi[a]
    o.stream = stream
    o.block_x = block_x
    o.graph_steps = graph_steps
    o.kernel = kernel
    o.tma_stages = tma_stages
    o.mu = mu
    o.overlap_steps = int(overlap_steps)
    o.storage_probe = int(storage_probe)
    o.fp64_arith = int(fp64_arith)
    return o


class Sim:
    """One simulation context: create / init / step / moments / destroy.

    ``w`` is a workload dict (see ``workloads``); ``stream`` an integer
    cudaStream_t (e.g. ``torch.cuda.current_stream().cuda_stream``) or None.
    """

    def __init__(self, w, stream=None, block_x=0, graph_steps=0, precision=None,
                 kernel=LBM_KERNEL_AUTO, tma_stages=0, overlap_steps=-1, storage_probe=0, fp64_arith=None):
        self.w = w
        self.lat = w["lattice"]
        self.D, self.Q, self.c, self.e, self.wts = lbm_lattice_info(self.lat)
        self.shape = w["shape"]
        self.N = self.shape[0] * self.shape[1] * self.shape[2]
        prec = w.get("precision", LBM_FP64) if precision is None else precision
        self.opt = options(prec, w.get("force_order", 2), w.get("bc", (0, 0, 0)),
                           w.get("T_lo", (1.0,) * 3), w.get("T_hi", (1.0,) * 3), stream,
                           block_x, graph_steps, kernel, tma_stages, w.get("mu", 0.0),
                           w.get("include_sigma", False), overlap_steps, storage_probe,
                           w.get("fp64_arith", 0) if fp64_arith is None else fp64_arith)
        g = w.get("g")
        self._gfield = g
        self.ctx = lbm_create(self.lat, *self.shape, w["tau"], g, self.opt)

    def __del__(self):
        self.close()

    def close(self):
        if getattr(self, "ctx", None):
            lbm_destroy(self.ctx)
            self.ctx = None

    def init(self, rho=None, u=None, T=None):
        if self.w.get("solid") is not None and not getattr(self, "_solid_set", False):
            lbm_set_solid(self.ctx, self.w["solid"], self.w["T_wall"])
            self._solid_set = True
        rho = self.w["rho"] if rho is None else rho
        u = self.w["u"] if u is None else u
        T = self.w["T"] if T is None else T
        lbm_init(self.ctx, np.ascontiguousarray(rho, dtype=np.float64) if isinstance(rho, np.ndarray) else rho,
                 np.ascontiguousarray(u, dtype=np.float64) if isinstance(u, np.ndarray) else u,
                 np.ascontiguousarray(T, dtype=np.float64) if isinstance(T, np.ndarray) else T)
        return self

    def step(self, n=1):
        lbm_step(self.ctx, n)

    def moments(self):
        rho = np.zeros(self.N)
        u = np.zeros((self.D, self.N))
        T = np.zeros(self.N)
        q = np.zeros((self.D, self.N))
        lbm_moments(self.ctx, rho, u, T, q)
        return rho, u, T, q

    def conserved(self, raise_unstable=True):
        return lbm_conserved(self.ctx, self.D, raise_unstable)

    def populations(self):
        out = np.zeros((self.Q, self.N))
        lbm_get_populations(self.ctx, out)
        return out

    def get_state(self):
        out = np.zeros((self.Q, self.N))
        lbm_get_state(self.ctx, out)
        return out

    def set_state(self, f):
        lbm_set_state(self.ctx, np.ascontiguousarray(f, dtype=np.float64))
