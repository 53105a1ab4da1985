"""Thin Python binding of the C ABI in include/dvm.h (argument marshalling only).

Every computation runs in the CUDA library ``_lib/libdvm_gb300.so``; there is no fallback: if the
library is missing or cannot be loaded, importing the functions raises.  PyTorch provides device
memory (through the allocator callback of ``dvm_options``) and the CUDA stream.
"""
import collections
import ctypes
import os
import threading

import numpy as np

from . import build as _build

DVM_OK, DVM_NOT_CONVERGED, DVM_EINVAL, DVM_ENOMEM, DVM_ECUDA, DVM_ETIMEOUT, DVM_ENUMERIC = 0, 1, -1, -2, -3, -4, -5
DVM_FP64, DVM_FP32, DVM_BF16_STORE = 0, 1, 2
DVM_LATERAL_SPECULAR, DVM_LATERAL_PERIODIC = 0, 1

_STATUS_NAMES = {0: "DVM_OK", 1: "DVM_NOT_CONVERGED", -1: "DVM_EINVAL", -2: "DVM_ENOMEM", -3: "DVM_ECUDA",
                 -4: "DVM_ETIMEOUT", -5: "DVM_ENUMERIC"}

ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)


class dvm_geometry(ctypes.Structure):
    _fields_ = [("dims", ctypes.c_int), ("n", ctypes.c_int64 * 3), ("solid", ctypes.c_void_p)]


class dvm_velocity_grid(ctypes.Structure):
    _fields_ = [("nv", ctypes.c_int), ("v", ctypes.c_void_p), ("w", ctypes.c_void_p)]


class dvm_options(ctypes.Structure):
    _fields_ = [
        ("precision", ctypes.c_int),
        ("stencil_order", ctypes.c_int),
        ("lateral_bc", ctypes.c_int),
        ("check_interval", ctypes.c_int),
        ("stream", ctypes.c_void_p),
        ("tile_x1", ctypes.c_int),
        ("band_rows", ctypes.c_int),
        ("alloc", ALLOC_FN),
        ("free", FREE_FN),
        ("alloc_user", ctypes.c_void_p),
        ("use_graph", ctypes.c_int),
        ("subdomains", ctypes.c_int * 3),
        ("group_warps", ctypes.c_int),
        ("temperature_term", ctypes.c_int),
        ("specular_fraction", ctypes.c_double),
        ("shakhov_prandtl", ctypes.c_double),
        ("es_prandtl", ctypes.c_double),
    ]


# (name, restype, argtypes) of every entry point declared in include/dvm.h
_P = ctypes.c_void_p
_SIGNATURES = [
    ("dvm_default_options", None, [ctypes.POINTER(dvm_options)]),
    ("dvm_gh_velocity_grid", ctypes.c_int, [ctypes.c_int, ctypes.c_int, _P, _P]),
    ("dvm_effective_pore_size", ctypes.c_int, [ctypes.c_int, ctypes.c_double, ctypes.c_double, _P]),
    ("dvm_create", ctypes.c_int, [ctypes.POINTER(dvm_geometry), ctypes.c_double, ctypes.POINTER(dvm_velocity_grid),
                                  ctypes.POINTER(dvm_options), ctypes.POINTER(_P)]),
    ("dvm_create_batch", ctypes.c_int, [ctypes.c_int, ctypes.POINTER(dvm_geometry), _P,
                                        ctypes.POINTER(dvm_velocity_grid), ctypes.POINTER(dvm_options),
                                        ctypes.POINTER(_P)]),
    ("dvm_iterate", ctypes.c_int, [_P, ctypes.c_int, ctypes.c_double, ctypes.POINTER(ctypes.c_int),
                                   ctypes.POINTER(ctypes.c_double)]),
    ("dvm_step", ctypes.c_int, [_P, ctypes.c_int]),
    ("dvm_sync", ctypes.c_int, [_P]),
    ("dvm_moments", ctypes.c_int, [_P, _P, _P, ctypes.c_int]),
    ("dvm_moments_at", ctypes.c_int, [_P, ctypes.c_int, _P, _P, ctypes.c_int]),
    ("dvm_temperature_at", ctypes.c_int, [_P, ctypes.c_int, _P, ctypes.c_int]),
    ("dvm_heat_flux_at", ctypes.c_int, [_P, ctypes.c_int, _P, ctypes.c_int]),
    ("dvm_stress_at", ctypes.c_int, [_P, ctypes.c_int, _P, ctypes.c_int]),
    ("dvm_permeability", ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]),
    ("dvm_permeability_at", ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                           ctypes.POINTER(ctypes.c_double)]),
    ("dvm_wall_density_at", ctypes.c_int, [_P, ctypes.c_int, _P]),
    ("dvm_info", ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int)]),
    ("dvm_last_error", ctypes.c_char_p, [_P]),
    ("dvm_destroy", None, [_P]),
    ("dvm_debug_set_wait", ctypes.c_int, [_P, ctypes.c_longlong, ctypes.c_int]),
    ("dvm_profile_enable", ctypes.c_int, [_P, ctypes.c_int]),
    ("dvm_profile_read", ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64),
                                        ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64)]),
    ("dvm_transfer_bytes", ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)]),
    ("dvm_autotune", ctypes.c_int, [ctypes.c_int, ctypes.POINTER(dvm_geometry), _P, ctypes.POINTER(dvm_velocity_grid),
                                    ctypes.POINTER(dvm_options), ctypes.c_int, ctypes.POINTER(ctypes.c_double)]),
    ("dvm_set_initial", ctypes.c_int, [_P, _P, _P]),
    ("dvm_set_initial_at", ctypes.c_int, [_P, ctypes.c_int, _P, _P]),
    ("dvm_get_state", ctypes.c_int, [_P, _P, ctypes.POINTER(ctypes.c_size_t)]),
    ("dvm_set_state", ctypes.c_int, [_P, _P, ctypes.c_size_t]),
    ("dvm_permeability_noalloc", ctypes.c_int, [_P, ctypes.c_int64, ctypes.c_double, _P, _P]),
    ("dvm_nn_conv3d", ctypes.c_int, [_P, _P, _P, _P] + [ctypes.c_int] * 6 + [_P, ctypes.c_int64, _P]),
    ("dvm_nn_conv3d_dgrad", ctypes.c_int, [_P, _P, _P] + [ctypes.c_int] * 6 + [_P, ctypes.c_int64, _P]),
    ("dvm_nn_conv3d_scratch_bytes", ctypes.c_int64, [ctypes.c_int] * 5),
    ("dvm_nn_status", ctypes.c_int, [_P]),
    ("dvm_nn_conv3d_wgrad", ctypes.c_int, [_P, _P, _P, _P, _P, ctypes.c_int64] + [ctypes.c_int] * 6 + [_P]),
    ("dvm_nn_wgrad_scratch_floats", ctypes.c_int64, [ctypes.c_int] * 5),
    ("dvm_nn_relu", ctypes.c_int, [_P, ctypes.c_int64, _P]),
    ("dvm_nn_relu_bwd", ctypes.c_int, [_P, _P, ctypes.c_int64, _P]),
    ("dvm_nn_pool2", ctypes.c_int, [_P, _P] + [ctypes.c_int] * 4 + [_P]),
    ("dvm_nn_pool2_bwd", ctypes.c_int, [_P, _P] + [ctypes.c_int] * 5 + [_P]),
    ("dvm_nn_up2", ctypes.c_int, [_P, _P] + [ctypes.c_int] * 4 + [_P]),
    ("dvm_nn_up2_bwd", ctypes.c_int, [_P, _P] + [ctypes.c_int] * 4 + [_P]),
    ("dvm_nn_mse", ctypes.c_int, [_P, _P, _P, _P, _P, ctypes.c_int, ctypes.c_int64, ctypes.c_float, _P]),
    ("dvm_nn_mse_partials", ctypes.c_int64, [ctypes.c_int, ctypes.c_int64]),
    ("dvm_nn_adam", ctypes.c_int, [_P, _P, _P, _P, _P, ctypes.c_int64, ctypes.c_float, ctypes.c_float,
                                   ctypes.c_float, ctypes.c_float, ctypes.c_int64, ctypes.c_float, _P]),
    ("dvm_nn_round_bf16", ctypes.c_int, [_P, _P, ctypes.c_int64, _P]),
    ("dvm_noalloc_last_error", ctypes.c_char_p, []),
    ("dvm_alu_peak", ctypes.c_int, [ctypes.c_int, _P, ctypes.c_int64, _P, ctypes.POINTER(ctypes.c_double)]),
]

_lib = None
_lock = threading.Lock()


def library_path():
    return _build.LIB


def load(build_if_missing=True):
    """Load (building first if needed) the CUDA library; raises if it is unavailable."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.LIB
            if not os.path.exists(path) or _build._stale():
                if not build_if_missing:
                    raise RuntimeError("CUDA library %s is missing; run the build first" % path)
                _build.build()
            lib = ctypes.CDLL(path)
            for name, res, args in _SIGNATURES:
                f = getattr(lib, name)
                f.restype = res
                f.argtypes = args
            _lib = lib
    return _lib


class DvmError(RuntimeError):
    def __init__(self, status, message):
        super().__init__("%s: %s" % (_STATUS_NAMES.get(status, status), message))
        self.status = status


def _check(status, ctx=None):
    if status < 0:
        msg = load().dvm_last_error(ctx)
        raise DvmError(status, msg.decode() if msg else "")
    return status


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


# --------------------------------------------------------------------------- same-name wrappers

def dvm_default_options():
    o = dvm_options()
    load().dvm_default_options(ctypes.byref(o))
    return o


def effective_pore_size(dims, k_inf, porosity):
    """L*/L of Eq. 14 from the continuum permeability k_inf and the porosity (library routine);
    the effective Knudsen number is Kn / (L*/L)."""
    r = ctypes.c_double()
    _check(load().dvm_effective_pore_size(int(dims), float(k_inf), float(porosity), ctypes.byref(r)))
    return r.value


def dvm_gh_velocity_grid(dims, n_per_axis):
    """Half-range Gauss-Hermite grid computed by the library: (v [nv, dims], w [nv])."""
    nv = n_per_axis ** dims
    v = np.zeros((nv, dims))
    w = np.zeros(nv)
    _check(load().dvm_gh_velocity_grid(int(dims), int(n_per_axis), _ptr(v), _ptr(w)))
    return v, w


def dvm_permeability_noalloc(u1_ptr, n, kn, out_ptr, stream=None):
    """Permeability of a device u1 field (n doubles at u1_ptr) into 2 device doubles at out_ptr,
    without any device allocation (scratch lives in a static device array; see include/dvm.h)."""
    lib = load()
    st = lib.dvm_permeability_noalloc(ctypes.c_void_p(int(u1_ptr)), int(n), float(kn), ctypes.c_void_p(int(out_ptr)),
                                      ctypes.c_void_p(int(stream)) if stream else None)
    if st < 0:
        raise DvmError(st, lib.dvm_noalloc_last_error().decode())
    return st


class _TorchAllocator:
    """Device memory from torch's caching allocator on the current device and stream."""

    def __init__(self):
        import torch
        self._torch = torch
        self.device = torch.cuda.current_device()
        self.live = {}

        def alloc(nbytes, user):
            try:
                ptr = torch.cuda.caching_allocator_alloc(int(nbytes), self.device)
            except Exception:
                return None
            self.live[ptr] = nbytes
            return ptr

        def free(ptr, nbytes, user):
            if ptr in self.live:
                del self.live[ptr]
                torch.cuda.caching_allocator_delete(ptr)

        self.alloc_fn = ALLOC_FN(alloc)
        self.free_fn = FREE_FN(free)


def alu_peak(precision="fp32"):
    """dvm_alu_peak: measured FMA throughput (TFLOP/s) of the current device, FP32 (packed) or FP64."""
    import torch
    lib = load()
    n = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count * 8 * 256 * 8
    buf = torch.empty(n, dtype=torch.uint8, device="cuda")
    out = ctypes.c_double(0.0)
    st = torch.cuda.current_stream().cuda_stream
    _check(lib.dvm_alu_peak({"fp64": DVM_FP64, "fp32": DVM_FP32}[precision], ctypes.c_void_p(buf.data_ptr()), n,
                            ctypes.c_void_p(st), ctypes.byref(out)), None)
    return out.value


def make_options(precision="fp64", stencil_order=2, lateral="specular", check_interval=100, stream=None,
                 tile_x1=0, band_rows=0, torch_memory=True, use_graph=False, subdomains=(1, 1, 1),
                 group_warps=0, temperature_term=False, specular_fraction=0.0,
                 shakhov_prandtl=0.0, es_prandtl=0.0):
    """dvm_options with torch's current stream (unless stream is given) and, by default, torch's
    caching allocator for device memory.  Returns (options, keepalive)."""
    o = dvm_default_options()
    o.precision = {"fp64": DVM_FP64, "fp32": DVM_FP32, "bf16_store": DVM_BF16_STORE}[precision]
    o.stencil_order = int(stencil_order)
    o.lateral_bc = {"specular": DVM_LATERAL_SPECULAR, "periodic": DVM_LATERAL_PERIODIC}[lateral]
    o.check_interval = int(check_interval)
    o.tile_x1 = int(tile_x1)
    o.band_rows = int(band_rows)
    o.use_graph = 1 if use_graph else 0
    o.group_warps = int(group_warps)
    o.temperature_term = 1 if temperature_term else 0
    o.specular_fraction = float(specular_fraction)
    o.shakhov_prandtl = float(shakhov_prandtl)
    o.es_prandtl = float(es_prandtl)
    for j in range(3):
        o.subdomains[j] = int(subdomains[j])
    keep = []
    if stream is None:
        import torch
        stream = torch.cuda.current_stream().cuda_stream
    o.stream = ctypes.c_void_p(int(stream)) if stream else None
    if torch_memory:
        al = _TorchAllocator()
        o.alloc = al.alloc_fn
        o.free = al.free_fn
        keep.append(al)
    return o, keep


def _geometries(masks, kn):
    """(uint8 masks, dvm_geometry array, Kn array) of one mask or a list of masks."""
    if isinstance(masks, np.ndarray):
        masks = [masks]
    kns = np.atleast_1d(np.asarray(kn, dtype=np.float64))
    if len(kns) == 1 and len(masks) > 1:
        kns = np.repeat(kns, len(masks))
    masks = [np.ascontiguousarray(np.asarray(m).astype(np.uint8)) for m in masks]
    geoms = (dvm_geometry * len(masks))()
    for g, m in zip(geoms, masks):
        g.dims = m.ndim
        shp = m.shape[::-1]
        for j in range(3):
            g.n[j] = shp[j] if j < m.ndim else 1
        g.solid = _ptr(m)
    return masks, geoms, np.ascontiguousarray(kns)


Tuning = collections.namedtuple("Tuning", "tile_x1 band_rows group_warps ms")


def autotune(masks, kn, v, w, iters=10, **options):
    """dvm_autotune: the fastest tile shape for these problems and options as a Tuning
    (tile_x1, band_rows, group_warps: pass them to Solver; ms: time per iteration)."""
    lib = load()
    masks, geoms, kns = _geometries(masks, kn)
    v = np.ascontiguousarray(np.asarray(v, dtype=np.float64))
    w = np.ascontiguousarray(np.asarray(w, dtype=np.float64))
    grid = dvm_velocity_grid(len(w), _ptr(v), _ptr(w))
    opt, keep = make_options(**options)
    best = ctypes.c_double(0.0)
    st = lib.dvm_autotune(len(masks), geoms, _ptr(kns), ctypes.byref(grid), ctypes.byref(opt), int(iters),
                          ctypes.byref(best))
    _check(st, None)
    return Tuning(opt.tile_x1, opt.band_rows, opt.group_warps, best.value)


class Solver:
    """A context (one problem or a batch) of the CUDA solver.

    masks: one mask or a list of masks (numpy, True = solid, shape (n2, n1), x1 fastest);
    kn: Knudsen number(s); v, w: velocity grid (e.g. from dvm_gh_velocity_grid)."""

    def __init__(self, masks, kn, v, w, **options):
        lib = load()
        self.masks, geoms, self._kn = _geometries(masks, kn)
        self.dims = self.masks[0].ndim
        self.v = np.ascontiguousarray(np.asarray(v, dtype=np.float64))
        self.w = np.ascontiguousarray(np.asarray(w, dtype=np.float64))
        grid = dvm_velocity_grid(len(self.w), _ptr(self.v), _ptr(self.w))
        self.options, self._keep = make_options(**options)
        ctx = ctypes.c_void_p()
        st = lib.dvm_create_batch(len(self.masks), geoms, _ptr(self._kn), ctypes.byref(grid),
                                  ctypes.byref(self.options), ctypes.byref(ctx))
        _check(st, None)
        self._ctx = ctx
        self._lib = lib

    def close(self):
        if getattr(self, "_ctx", None):
            self._lib.dvm_destroy(self._ctx)
            self._ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def nprob(self):
        return len(self.masks)

    def iterate(self, max_iter, tol=0.0):
        """dvm_iterate: returns (status, iterations done, Err)."""
        it = ctypes.c_int(0)
        err = ctypes.c_double(0.0)
        st = self._lib.dvm_iterate(self._ctx, int(max_iter), float(tol), ctypes.byref(it), ctypes.byref(err))
        _check(st, self._ctx)
        return st, it.value, err.value

    def step(self, n):
        _check(self._lib.dvm_step(self._ctx, int(n)), self._ctx)

    def sync(self):
        _check(self._lib.dvm_sync(self._ctx), self._ctx)

    @property
    def iterations(self):
        it = ctypes.c_int64(0)
        _check(self._lib.dvm_info(self._ctx, ctypes.byref(it), None), self._ctx)
        return it.value

    def moments(self, prob=0):
        m = self.masks[prob]
        rho = np.zeros(m.size)
        u = np.zeros(m.size * m.ndim)
        _check(self._lib.dvm_moments_at(self._ctx, int(prob), _ptr(rho), _ptr(u), 0), self._ctx)
        return rho.reshape(m.shape), u.reshape((m.ndim,) + m.shape)

    def temperature(self, prob=0):
        """Temperature perturbation tau (Eq. 4) of problem prob; needs temperature_term=True."""
        m = self.masks[prob]
        tau = np.zeros(m.size)
        _check(self._lib.dvm_temperature_at(self._ctx, int(prob), _ptr(tau), 0), self._ctx)
        return tau.reshape(m.shape)

    def heat_flux(self, prob=0):
        """Heat flux q = sum W v (|v|^2 - 5/2) h [3, *shape] of problem prob; needs shakhov_prandtl > 0."""
        m = self.masks[prob]
        q = np.zeros(3 * m.size)
        _check(self._lib.dvm_heat_flux_at(self._ctx, int(prob), _ptr(q), 0), self._ctx)
        return q.reshape((3,) + m.shape)

    def stress(self, prob=0):
        """Traceless stress [6, *shape] (11 22 33 12 13 23) of problem prob; needs es_prandtl > 0."""
        m = self.masks[prob]
        p = np.zeros(6 * m.size)
        _check(self._lib.dvm_stress_at(self._ctx, int(prob), _ptr(p), 0), self._ctx)
        return p.reshape((6,) + m.shape)

    def moments_device(self, prob, rho_ptr, u_ptr):
        _check(self._lib.dvm_moments_at(self._ctx, int(prob), ctypes.c_void_p(rho_ptr), ctypes.c_void_p(u_ptr), 1),
               self._ctx)

    def permeability(self, prob=0):
        k = ctypes.c_double(0.0)
        gp = ctypes.c_double(0.0)
        _check(self._lib.dvm_permeability_at(self._ctx, int(prob), ctypes.byref(k), ctypes.byref(gp)), self._ctx)
        return k.value, gp.value

    def wall(self, prob=0):
        m = self.masks[prob]
        out = np.zeros(m.size * m.ndim * 2)
        _check(self._lib.dvm_wall_density_at(self._ctx, int(prob), _ptr(out)), self._ctx)
        return out.reshape((m.ndim, 2) + m.shape)

    def set_initial(self, rho0, u0, prob=0):
        """dvm_set_initial_at: warm start of problem prob from rho0 (mask shape) and u0 ((dims,) +
        mask shape), both in the variables moments() returns."""
        m = self.masks[prob]
        r = np.ascontiguousarray(np.asarray(rho0, dtype=np.float64).reshape(m.size))
        u = np.ascontiguousarray(np.asarray(u0, dtype=np.float64).reshape(m.ndim * m.size))
        _check(self._lib.dvm_set_initial_at(self._ctx, int(prob), _ptr(r), _ptr(u)), self._ctx)

    def get_state(self):
        """dvm_get_state: the iteration state as bytes."""
        n = ctypes.c_size_t(0)
        _check(self._lib.dvm_get_state(self._ctx, None, ctypes.byref(n)), self._ctx)
        buf = ctypes.create_string_buffer(n.value)
        _check(self._lib.dvm_get_state(self._ctx, buf, ctypes.byref(n)), self._ctx)
        return buf.raw[:n.value]

    def set_state(self, blob):
        """dvm_set_state: resume from bytes written by get_state of a matching context."""
        buf = ctypes.create_string_buffer(bytes(blob), len(blob))
        _check(self._lib.dvm_set_state(self._ctx, buf, len(blob)), self._ctx)

    def profile_enable(self, on=True):
        _check(self._lib.dvm_profile_enable(self._ctx, 1 if on else 0), self._ctx)

    def profile_read(self):
        """(sweep_ms, sweep_launches, finalize_ms, finalize_launches) since the last read."""
        a, c = ctypes.c_double(0), ctypes.c_double(0)
        b, d = ctypes.c_int64(0), ctypes.c_int64(0)
        _check(self._lib.dvm_profile_read(self._ctx, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c),
                                          ctypes.byref(d)), self._ctx)
        return a.value, b.value, c.value, d.value

    def transfer_bytes(self):
        h, d = ctypes.c_int64(0), ctypes.c_int64(0)
        _check(self._lib.dvm_transfer_bytes(self._ctx, ctypes.byref(h), ctypes.byref(d)), self._ctx)
        return h.value, d.value

    def debug_set_wait(self, timeout_ns, withhold_item=-1):
        _check(self._lib.dvm_debug_set_wait(self._ctx, int(timeout_ns), int(withhold_item)), self._ctx)
