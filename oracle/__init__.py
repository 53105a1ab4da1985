"""FP64 CPU oracle of the discrete-velocity transport iteration (arXiv:1712.01132, Sec. 2-3).

TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the CPU-baseline leg of the
benchmark may import this package.  It shares no code with the CUDA library: the solver is the
plain C file ``dvm_oracle.c`` (built here with gcc), the velocity grid comes from
``quadrature.py``.

Parity status: every solver function here is pinned by the ``-m "not gpu"`` tests against
closed forms, invariants (symmetries, conservation, shift equivariance, formulation and traversal
equivalences), a textbook BGK flow rate, the paper's printed effective-Knudsen factors and an
independent dense linear solve (see ``tests/test_oracle_*.py``).  The paper's printed sphere-array
permeabilities (Table 3) are checked on the CUDA path, which agrees with this oracle.
"""
import ctypes
import math
import os
import subprocess
import threading

import numpy as np

from .quadrature import half_range_gauss_hermite, velocity_grid  # noqa: F401

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dvm_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


class _Cfg(ctypes.Structure):
    _fields_ = [
        ("dims", ctypes.c_int),
        ("n", ctypes.c_int * 3),
        ("solid", ctypes.c_void_p),
        ("kn", ctypes.c_double),
        ("jump", ctypes.c_double),
        ("nv", ctypes.c_int),
        ("v", ctypes.c_void_p),
        ("w", ctypes.c_void_p),
        ("order", ctypes.c_int),
        ("lateral", ctypes.c_int),
        ("form", ctypes.c_int),
        ("traversal", ctypes.c_int),
        ("dec", ctypes.c_int * 3),
        ("tau", ctypes.c_int),
        ("alpha", ctypes.c_double),
        ("shakhov_pr", ctypes.c_double),
        ("es_pr", ctypes.c_double),
    ]


def build(force=False):
    """Compile dvm_oracle.c into oracle/_build/liboracle.so (gcc, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11", "-D_GNU_SOURCE",
           "-o", tmp, _SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.ora_create.restype = ctypes.c_void_p
            lib.ora_create.argtypes = [ctypes.POINTER(_Cfg)]
            lib.ora_destroy.argtypes = [ctypes.c_void_p]
            lib.ora_iterate.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_int]
            lib.ora_iter.restype = ctypes.c_long
            lib.ora_iter.argtypes = [ctypes.c_void_p]
            for f in ("ora_get_moments",):
                getattr(lib, f).argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
            for f in ("ora_get_wall", "ora_get_flux", "ora_get_tau", "ora_get_q", "ora_get_pi"):
                getattr(lib, f).argtypes = [ctypes.c_void_p, ctypes.c_void_p]
            lib.ora_set_uniform.argtypes = [ctypes.c_void_p, ctypes.c_double]
            lib.ora_set_initial.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
            lib.ora_sweep_one.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]
            _lib = lib
    return _lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


class Oracle:
    """One problem: a solid mask (numpy bool/uint8, shape (n2, n1) or (n3, n2, n1), x1 fastest),
    Knudsen number kn and a velocity grid (v [nv, dims], W [nv], sum W = 1).

    form: "jump" (the paper's Eq. 7, default) or "source" (h' = h + J x1).
    lateral: "specular" (Eq. 8, default) or "periodic".
    order: 2 (Eq. 9 default) or 1.
    traversal: "raster" (the paper's raster scan) or "wavefront".
    decomposition: subdomain counts (c1, c2[, c3]) of the lagged-halo Omega_x decomposition.
    tau: keep the temperature term tau (|v|^2 - 3/2) of Eq. 2 with tau from Eq. 4 (3D only; the
    paper drops it for its isothermal flows).
    alpha: tangential momentum accommodation coefficient of the Maxwell wall condition (Eq. 5);
    1 (fully diffuse) is the paper's setting.
    shakhov_pr: 0 for the BGK model (the paper's); a Prandtl number > 0 selects the linearised
    Shakhov model, whose source adds (4/5)(1 - Pr) q.v (|v|^2 - 5/2) with the heat flux
    q = sum W v (|v|^2 - 5/2) h (needs tau).
    es_pr: 0 for the BGK model; a Prandtl number > 0 selects the linearised ES-BGK model: collision
    frequency Pr nu and the source adds (1 - 1/Pr) sum_ij P_ij v_i v_j with the traceless stress
    P_ij = 2 sum W (v_i v_j - delta_ij |v|^2 / 3) h (needs tau; not with shakhov_pr).
    """

    def __init__(self, solid, kn, v, w, *, jump=1.0, order=2, lateral="specular", form="jump",
                 traversal="raster", decomposition=(1, 1, 1), threads=0, tau=False, alpha=1.0, shakhov_pr=0.0,
                 es_pr=0.0):
        lib = _load()
        solid = np.ascontiguousarray(np.asarray(solid).astype(np.uint8))
        if solid.ndim not in (2, 3):
            raise ValueError("mask must be 2D or 3D")
        self.dims = solid.ndim
        self.shape = solid.shape
        self.solid = solid
        self.v = np.ascontiguousarray(np.asarray(v, dtype=np.float64).reshape(-1, self.dims))
        self.w = np.ascontiguousarray(np.asarray(w, dtype=np.float64).reshape(-1))
        self.kn = float(kn)
        self.threads = int(threads)
        cfg = _Cfg()
        cfg.dims = self.dims
        n = solid.shape[::-1]
        for j in range(3):
            cfg.n[j] = n[j] if j < self.dims else 1
        cfg.solid = _ptr(self.solid)
        cfg.kn = self.kn
        cfg.jump = float(jump)
        cfg.nv = self.v.shape[0]
        cfg.v = _ptr(self.v)
        cfg.w = _ptr(self.w)
        cfg.order = int(order)
        cfg.lateral = {"specular": 0, "periodic": 1}[lateral]
        cfg.form = {"jump": 0, "source": 1}[form]
        cfg.traversal = {"raster": 0, "wavefront": 1}[traversal]
        dec = tuple(decomposition) + (1,) * (3 - len(decomposition))
        for j in range(3):
            cfg.dec[j] = int(dec[j])
        cfg.tau = 1 if tau else 0
        cfg.alpha = float(alpha)
        cfg.shakhov_pr = float(shakhov_pr)
        cfg.es_pr = float(es_pr)
        self._cfg = cfg
        self._h = lib.ora_create(ctypes.byref(cfg))
        if not self._h:
            raise ValueError("oracle rejected the configuration")
        self._lib = lib
        self.k_history = []    # k after every iteration
        # Eq. 15 history: k at the last check (or of the start state, 0 for h = 0) and its iteration
        self.k_check = 0.0
        self.it_check = 0
        self.err = math.inf

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._lib.ora_destroy(h)
            self._h = None

    @property
    def iterations(self):
        return int(self._lib.ora_iter(self._h))

    def iterate(self, n):
        """Run n iterations; returns k after each of them."""
        out = np.zeros(max(n, 1))
        self._lib.ora_iterate(self._h, int(n), _ptr(out), self.threads)
        ks = out[:n].tolist()
        self.k_history.extend(ks)
        return np.array(ks)

    def run(self, tol, max_iter, check_interval=100):
        """Iterate until Err of Eq. 15 drops below tol at a check, or until the iteration count
        reaches max_iter.  Returns (iterations, k, Err of the last check).

        Sec. 3.1 steps iv-v: every check_interval iterations the permeability k(l) is evaluated and
        Err(l) = |k(l) - k(l - check_interval)| / (check_interval |k(l)|).  Checks fall on the
        iteration counts that are multiples of check_interval; k(l - check_interval) is the k of the
        previous check, at the first check the k of the start state (0 for h = 0).  After a warm
        start (set_initial) the previous check is the warm state, and the divisor becomes the
        iterations actually run since it.  k(l) = 0 gives Err = 0 when the previous k is 0 as well
        (no flow path), else infinity."""
        while self.iterations < max_iter:
            n = check_interval - self.iterations % check_interval
            n = min(n, max_iter - self.iterations)
            ks = self.iterate(n)
            if self.iterations % check_interval != 0:
                break
            k = float(ks[-1])
            gap = self.iterations - self.it_check
            if k != 0.0:
                self.err = abs((k - self.k_check) / k) / gap
            else:
                self.err = 0.0 if self.k_check == 0.0 else math.inf
            self.k_check, self.it_check = k, self.iterations
            if self.err < tol:
                break
        return self.iterations, self.permeability(), self.err

    def moments(self):
        """(rho [shape], u [dims, *shape]) in the paper's (jump-form) variables; solid = 0."""
        N = self.solid.size
        rho = np.zeros(N)
        u = np.zeros(N * self.dims)
        self._lib.ora_get_moments(self._h, _ptr(rho), _ptr(u))
        return rho.reshape(self.shape), u.reshape((self.dims,) + self.shape)

    def wall(self):
        """Wall densities [dims, 2, *shape] of faces (x, axis j, side -1/+1); 0 where no face."""
        out = np.zeros(self.solid.size * self.dims * 2)
        self._lib.ora_get_wall(self._h, _ptr(out))
        return out.reshape((self.dims, 2) + self.shape)

    def temperature(self):
        """Temperature tau of Eq. 4 [shape] (zero without the tau option; solid = 0)."""
        out = np.zeros(self.solid.size)
        self._lib.ora_get_tau(self._h, _ptr(out))
        return out.reshape(self.shape)

    def heat_flux(self):
        """Heat flux q [dims, *shape] of the Shakhov option (zero otherwise; solid = 0)."""
        out = np.zeros(self.solid.size * self.dims)
        self._lib.ora_get_q(self._h, _ptr(out))
        return out.reshape((self.dims,) + self.shape)

    def stress(self):
        """Traceless stress [6, *shape] (components 11 22 33 12 13 23) of the ES option."""
        out = np.zeros(self.solid.size * 6)
        self._lib.ora_get_pi(self._h, _ptr(out))
        return out.reshape((6,) + self.shape)

    def flux(self):
        """x1 face fluxes sum_{cross-section} sum_k W_k v1 h_upwind of the last iteration [n1]."""
        out = np.zeros(self.shape[-1])
        self._lib.ora_get_flux(self._h, _ptr(out))
        return out

    def permeability(self):
        """k = (2/sqrt(pi)) Kn G_p with G_p the mean of u1 over all points (Eq. 11-12)."""
        _, u = self.moments()
        return 2.0 / math.sqrt(math.pi) * self.kn * float(u[0].sum() / u[0].size)

    def set_uniform(self, c):
        self._lib.ora_set_uniform(self._h, float(c))
        self.k_check, self.it_check = self.permeability(), self.iterations

    def set_initial(self, rho0, u0):
        """Warm start: the state left by an iteration that produced h0 = rho0 + 2 u0 . v at every
        fluid point (rho0 [shape], u0 [dims, *shape], jump-form variables)."""
        r = np.ascontiguousarray(np.asarray(rho0, dtype=np.float64).reshape(-1))
        u = np.ascontiguousarray(np.asarray(u0, dtype=np.float64).reshape(-1))
        assert r.size == self.solid.size and u.size == self.solid.size * self.dims
        self._lib.ora_set_initial(self._h, _ptr(r), _ptr(u))
        self.k_check, self.it_check = self.permeability(), self.iterations

    def sweep_one(self, k):
        """Sweep velocity k from the current state without changing it; returns h [shape]."""
        h = np.zeros(self.solid.size)
        self._lib.ora_sweep_one(self._h, int(k), _ptr(h))
        return h.reshape(self.shape)


def effective_knudsen_factor(k_inf, porosity, dims):
    """Kn*/Kn = 1/(L*/L) with L*/L of Eq. 14: sqrt(12 k_inf/eps) in 2D, sqrt(8 k_inf/(pi eps)) in 3D."""
    if dims == 2:
        ratio = math.sqrt(12.0 * k_inf / porosity)
    else:
        ratio = math.sqrt(8.0 * k_inf / (math.pi * porosity))
    return 1.0 / ratio
