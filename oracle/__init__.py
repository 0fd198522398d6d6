"""FP64 CPU oracle of the hybrid LBM-FVM natural-convection step (arXiv 1908.08386, Section 5).

TEST INFRASTRUCTURE ONLY: the test-suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers.  The product path (the
CUDA library and its binding) never imports this package and shares no code
with it.

The arithmetic lives in ``lbmfvm_oracle.c`` (plain C, FP64, OpenMP over rows
for timing only; every reduction runs serially, so results do not depend on
the thread count).  This module compiles it with gcc and wraps it with ctypes.
"""

from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbmfvm_oracle.c")
_LIB = os.path.join(_HERE, "liblbmfvm_oracle.so")
_lock = threading.Lock()
_lib = None

# Side order and boundary kinds shared by convention with the C-ABI header
# (the values are part of the public interface, not of the method).
W, E, S, N = 0, 1, 2, 3
BC_DIRICHLET, BC_ADIABATIC, BC_PERIODIC, BC_MOVING = 0, 1, 2, 3


def build(force: bool = False) -> str:
    """Compile the oracle shared library in place (gcc, no FP contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = [
            "gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
            "-Wall", _SRC, "-o", _LIB + ".tmp", "-lm",
        ]
        subprocess.run(cmd, check=True)
        os.replace(_LIB + ".tmp", _LIB)
    return _LIB


def build_variant(source_text: str, out_path: str) -> str:
    """Compile a modified copy of the oracle source (used by the tests that
    plant mistakes in the oracle to show that its pins catch them)."""
    src = out_path + ".c"
    with open(src, "w") as fh:
        fh.write(source_text)
    subprocess.run(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
                    src, "-o", out_path, "-lm"], check=True)
    return out_path


def source_text() -> str:
    with open(_SRC) as fh:
        return fh.read()


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        build()
        _lib = load_library(_LIB)
        return _lib


def load_library(path: str):
    """Load an oracle shared library and declare its entry points."""
    lib = ctypes.CDLL(path)
    d, i, vp = ctypes.c_double, ctypes.c_int, ctypes.c_void_p
    dp = ctypes.POINTER(ctypes.c_double)
    lib.orc_create.restype = vp
    lib.orc_create.argtypes = [i, i, ctypes.POINTER(ctypes.c_int), dp, d, d, vp, d, d, d, d, d, d]
    lib.orc_destroy.argtypes = [vp]
    lib.orc_set_state.argtypes = [vp, vp, vp, vp, d]
    lib.orc_step.argtypes = [vp, ctypes.c_long]
    lib.orc_step_count.restype = ctypes.c_long
    lib.orc_step_count.argtypes = [vp]
    lib.orc_tau.restype = d
    lib.orc_tau.argtypes = [vp]
    lib.orc_fields.argtypes = [vp, vp, vp, vp, vp]
    lib.orc_get_f.argtypes = [vp, vp]
    lib.orc_set_f.argtypes = [vp, vp]
    lib.orc_set_T.argtypes = [vp, vp]
    lib.orc_classes.argtypes = [vp, vp, vp, vp]
    lib.orc_nusselt.argtypes = [vp, dp, vp, dp, vp]
    lib.orc_flux_nusselt.argtypes = [vp, vp]
    lib.orc_residual.restype = d
    lib.orc_residual.argtypes = [vp]
    lib.orc_cv_volumes.argtypes = [vp, vp]
    lib.orc_params_from_groups.argtypes = [d, d, d, d, d, dp, dp, dp, dp]
    lib.orc_num_threads.restype = i
    if hasattr(lib, "orc_set_fv"):
        lib.orc_set_fv.restype = i
        lib.orc_set_fv.argtypes = [vp, i, i]
    if hasattr(lib, "orc_set_energy"):
        lib.orc_set_energy.restype = i
        lib.orc_set_energy.argtypes = [vp, i]
    if hasattr(lib, "orc_set_wall_bc"):
        lib.orc_set_wall_bc.restype = i
        lib.orc_set_wall_bc.argtypes = [vp, i]
    if hasattr(lib, "orc_set_grid2"):
        lib.orc_set_grid2.restype = i
        lib.orc_set_grid2.argtypes = [vp, i]
    return lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def params_from_groups(Ra: float, Pr: float, Ma: float, H: float, dT: float = 1.0, lib=None):
    """(nu, alpha, gbeta, tau) in lattice units from Ra, Pr, Ma (Eqs. 83-89, 15)."""
    lib = lib if lib is not None else _load()
    out = [ctypes.c_double() for _ in range(4)]
    lib.orc_params_from_groups(Ra, Pr, Ma, H, dT, *[ctypes.byref(x) for x in out])
    return tuple(x.value for x in out)


def num_threads() -> int:
    return _load().orc_num_threads()


class Oracle:
    """One cavity (or periodic box) advanced by the FP64 reference step.

    Parameters are lattice units: ``nu`` kinematic viscosity (tau = 3 nu + 1/2),
    ``alpha`` thermal diffusivity, ``gbeta`` buoyancy coefficient so that the
    body force per unit mass is G = (fx, fy + gbeta (T - t_ref)).
    """

    def __init__(self, nx, ny, *, bc=(BC_DIRICHLET, BC_DIRICHLET, BC_ADIABATIC, BC_ADIABATIC),
                 t_wall=(1.0, 0.0, 0.0, 0.0), u_lid=0.0, t_init=0.5, mask=None,
                 nu, alpha, gbeta=0.0, t_ref=None, fx=0.0, fy=0.0, fv_scheme="central", fv_substeps=1,
                 energy="fv", wall_bc="nee", fv_grid=1, fv_every=1, lib=None):
        lib = lib if lib is not None else _load()
        self.nx, self.ny = int(nx), int(ny)
        self.t_wall = tuple(float(t) for t in t_wall)
        if t_ref is None:
            t_ref = self.t_wall[E]
        self._mask = None
        if mask is not None:
            self._mask = np.ascontiguousarray(mask, dtype=np.uint8).reshape(self.ny, self.nx)
        bc_arr = (ctypes.c_int * 4)(*[int(b) for b in bc])
        tw = (ctypes.c_double * 4)(*self.t_wall)
        h = lib.orc_create(self.nx, self.ny, bc_arr, tw, float(u_lid), float(t_init),
                           _ptr(self._mask), float(nu), float(alpha), float(gbeta), float(t_ref),
                           float(fx), float(fy))
        if not h:
            raise ValueError("oracle: invalid grid or boundary configuration")
        self._h = ctypes.c_void_p(h)
        self._lib = lib
        if fv_scheme not in ("central", "quick"):
            raise ValueError(f"oracle: fv_scheme must be 'central' or 'quick', not {fv_scheme!r}")
        if (fv_scheme, fv_substeps) != ("central", 1):
            if lib.orc_set_fv(self._h, int(fv_scheme == "quick"), int(fv_substeps)) != 0:
                raise ValueError(f"oracle: fv_substeps must be >= 1 (got {fv_substeps})")
        if energy not in ("fv", "lbm"):
            raise ValueError(f"oracle: energy must be 'fv' or 'lbm', not {energy!r}")
        if energy == "lbm" and lib.orc_set_energy(self._h, 1) != 0:
            raise ValueError("oracle: the D2Q5 energy populations could not be set up")
        self.energy = energy
        if wall_bc not in ("nee", "fd"):
            raise ValueError(f"oracle: wall_bc must be 'nee' or 'fd', not {wall_bc!r}")
        if wall_bc == "fd":
            lib.orc_set_wall_bc(self._h, 1)
        self.wall_bc = wall_bc
        if fv_grid not in (1, 2):
            raise ValueError(f"oracle: fv_grid must be 1 or 2, not {fv_grid!r}")
        if fv_grid == 2 and lib.orc_set_grid2(self._h, int(fv_every)) != 0:
            raise ValueError("oracle: grid setting 2 needs an even number of spacings (nodes along periodic axes), "
                             "no obstacle, the finite-volume energy update and fv_every >= 1")
        self.fv_grid = fv_grid
        self.nu, self.alpha, self.gbeta = float(nu), float(alpha), float(gbeta)
        self.t_init = float(t_init)

    @classmethod
    def from_groups(cls, nx, ny, Ra, Pr, Ma, **kw):
        """Cavity set up from Ra, Pr, Ma with H = ny - 1 and dT = T_W - T_E."""
        t_wall = kw.get("t_wall", (1.0, 0.0, 0.0, 0.0))
        nu, alpha, gbeta, _ = params_from_groups(Ra, Pr, Ma, ny - 1, t_wall[W] - t_wall[E], lib=kw.get("lib"))
        return cls(nx, ny, nu=nu, alpha=alpha, gbeta=gbeta, **kw)

    def close(self):
        if getattr(self, "_h", None):
            self._lib.orc_destroy(self._h)
            self._h = None

    __del__ = close

    @property
    def tau(self):
        return self._lib.orc_tau(self._h)

    @property
    def step_count(self):
        return self._lib.orc_step_count(self._h)

    def set_state(self, u=None, v=None, T=None):
        conv = lambda a: None if a is None else np.ascontiguousarray(a, dtype=np.float64).reshape(self.ny, self.nx)
        u, v, T = conv(u), conv(v), conv(T)
        self._lib.orc_set_state(self._h, _ptr(u), _ptr(v), _ptr(T), self.t_init)

    def step(self, n=1):
        self._lib.orc_step(self._h, int(n))

    def fields(self):
        shp = (self.ny, self.nx)
        rho, u, v, T = (np.empty(shp) for _ in range(4))
        self._lib.orc_fields(self._h, _ptr(rho), _ptr(u), _ptr(v), _ptr(T))
        return rho, u, v, T

    def f(self):
        out = np.empty((9, self.ny, self.nx))
        self._lib.orc_get_f(self._h, _ptr(out))
        return out

    def set_f(self, f):
        f = np.ascontiguousarray(f, dtype=np.float64).reshape(9, self.ny, self.nx)
        self._lib.orc_set_f(self._h, _ptr(f))

    def set_T(self, T):
        """Replace the temperature of the current state (f stays)."""
        T = np.ascontiguousarray(T, dtype=np.float64).reshape(self.ny, self.nx)
        self._lib.orc_set_T(self._h, _ptr(T))

    def classes(self):
        shp = (self.ny, self.nx)
        kind = np.empty(shp, np.uint8)
        therm = np.empty(shp, np.uint8)
        partner = np.empty(shp, np.int32)
        self._lib.orc_classes(self._h, _ptr(kind), _ptr(therm), _ptr(partner))
        return kind, therm, partner

    def nusselt(self):
        """(mean_hot, local_hot[ny], mean_cold, local_cold[ny])."""
        mh, mc = ctypes.c_double(), ctypes.c_double()
        lh, lc = np.empty(self.ny), np.empty(self.ny)
        self._lib.orc_nusselt(self._h, ctypes.byref(mh), _ptr(lh), ctypes.byref(mc), _ptr(lc))
        return mh.value, lh, mc.value, lc

    def flux_nusselt(self):
        out = np.empty(self.nx - 1)
        self._lib.orc_flux_nusselt(self._h, _ptr(out))
        return out

    def residual(self):
        return self._lib.orc_residual(self._h)

    def cv_volumes(self):
        out = np.empty((self.ny, self.nx))
        self._lib.orc_cv_volumes(self._h, _ptr(out))
        return out
