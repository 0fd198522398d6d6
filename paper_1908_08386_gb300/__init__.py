"""Python binding of ``liblbmfvm.so``, the GB300 coupled LBM-FVM solver.

The functions here carry the names of the C-ABI entry points declared in
``include/lbmfvm.h`` and only marshal arguments; every step of the method runs
in the CUDA kernels of the library.  PyTorch supplies device memory (the
handle's workspace) and the CUDA stream.  There is no CPU fallback: if the
library cannot be built or loaded, :func:`lib` raises.
"""

from __future__ import annotations

import ctypes
import math
import os
import threading

import numpy as np

from . import build as _build

# Status codes
LBMFVM_OK = 0
LBMFVM_ERR_ARG = -1
LBMFVM_ERR_UNSTABLE = -2
LBMFVM_ERR_CUDA = -3
LBMFVM_ERR_DIVERGED = -4
LBMFVM_ERR_TIMEOUT = -5
LBMFVM_ERR_NOMEM = -6
LBMFVM_ERR_IO = -7
# Sides
LBMFVM_SIDE_W, LBMFVM_SIDE_E, LBMFVM_SIDE_S, LBMFVM_SIDE_N = 0, 1, 2, 3
# Boundary kinds
LBMFVM_BC_DIRICHLET, LBMFVM_BC_ADIABATIC, LBMFVM_BC_PERIODIC, LBMFVM_BC_MOVING = 0, 1, 2, 3
# Step kernels
LBMFVM_KERNEL_AUTO, LBMFVM_KERNEL_GENERIC, LBMFVM_KERNEL_TMA = 0, 1, 2
KERNELS = {"auto": LBMFVM_KERNEL_AUTO, "generic": LBMFVM_KERNEL_GENERIC, "tma": LBMFVM_KERNEL_TMA}
LBMFVM_TMA_AUTOTUNE = -1
LBMFVM_TMA_DEFAULT = -2
# Storage precisions
LBMFVM_F64, LBMFVM_F32, LBMFVM_F16, LBMFVM_BF16, LBMFVM_F32X2 = 0, 1, 2, 3, 4
PRECISIONS = {"f64": LBMFVM_F64, "f32": LBMFVM_F32, "f16": LBMFVM_F16, "bf16": LBMFVM_BF16,
              "f32x2": LBMFVM_F32X2}
# Energy-update face temperatures and automatic sub-steps
LBMFVM_FV_CENTRAL, LBMFVM_FV_QUICK = 0, 1
FV_SCHEMES = {"central": LBMFVM_FV_CENTRAL, "quick": LBMFVM_FV_QUICK}
LBMFVM_FV_SUBSTEPS_AUTO = 0
# Energy solvers
LBMFVM_ENERGY_FV, LBMFVM_ENERGY_LBM_D2Q5 = 0, 1
ENERGY = {"fv": LBMFVM_ENERGY_FV, "lbm": LBMFVM_ENERGY_LBM_D2Q5}
# Box-wall treatments
LBMFVM_WALL_NEE, LBMFVM_WALL_FD = 0, 1
WALLS = {"nee": LBMFVM_WALL_NEE, "fd": LBMFVM_WALL_FD}

# Every entry point the header declares (checked by the test-suite).
EXPORTS = (
    "lbmfvm_opts_default", "lbmfvm_workspace_bytes", "lbmfvm_create", "lbmfvm_create_lattice",
    "lbmfvm_set_state", "lbmfvm_step", "lbmfvm_inject_stall", "lbmfvm_step_count", "lbmfvm_fields", "lbmfvm_fields_f32",
    "lbmfvm_nusselt", "lbmfvm_residual", "lbmfvm_run_to_steady", "lbmfvm_copy_state", "lbmfvm_launch_count", "lbmfvm_kernel_info", "lbmfvm_fv_info", "lbmfvm_params", "lbmfvm_residual_noalloc",
    "lbmfvm_save", "lbmfvm_load", "lbmfvm_checkpoint_info",
    "lbmfvm_destroy", "lbmfvm_last_error", "lbmfvm_batch_create", "lbmfvm_batch_set_state", "lbmfvm_batch_step",
    "lbmfvm_batch_residuals", "lbmfvm_batch_run", "lbmfvm_batch_fields", "lbmfvm_batch_nusselt", "lbmfvm_batch_info",
    "lbmfvm_batch_substeps", "lbmfvm_batch_set_polish", "lbmfvm_batch_kernel_info", "lbmfvm_batch_precision", "lbmfvm_batch_destroy", "lbmfvm_batch_last_error",
)


class lbmfvm_grid_t(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("bc", ctypes.c_int32 * 4),
                ("t_wall", ctypes.c_double * 4), ("u_lid", ctypes.c_double), ("t_init", ctypes.c_double)]


class lbmfvm_opts_t(ctypes.Structure):
    _fields_ = [("store", ctypes.c_int32), ("tile_y", ctypes.c_int32), ("kernel", ctypes.c_int32),
                ("tma_config", ctypes.c_int32), ("t_ref", ctypes.c_double),
                ("cuda_stream", ctypes.c_void_p), ("workspace", ctypes.c_void_p),
                ("workspace_bytes", ctypes.c_size_t), ("fv_scheme", ctypes.c_int32), ("fv_substeps", ctypes.c_int32),
                ("energy", ctypes.c_int32), ("wall_bc", ctypes.c_int32), ("fv_grid", ctypes.c_int32),
                ("fv_every", ctypes.c_int32)]


class lbmfvm_checkpoint_header_t(ctypes.Structure):
    _fields_ = [("magic", ctypes.c_char * 8), ("version", ctypes.c_uint32), ("header_bytes", ctypes.c_uint32),
                ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("store", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("steps", ctypes.c_int64), ("bc", ctypes.c_int32 * 4),
                ("t_wall", ctypes.c_double * 4), ("u_lid", ctypes.c_double), ("tau", ctypes.c_double),
                ("alpha", ctypes.c_double), ("gbeta", ctypes.c_double), ("t_ref", ctypes.c_double),
                ("force", ctypes.c_double * 2), ("payload_bytes", ctypes.c_uint64), ("code_crc", ctypes.c_uint32),
                ("payload_crc", ctypes.c_uint32), ("fv_scheme", ctypes.c_int32), ("fv_substeps", ctypes.c_int32),
                ("energy", ctypes.c_int32), ("wall_bc", ctypes.c_int32), ("pad", ctypes.c_uint8 * 76),
                ("header_crc", ctypes.c_uint32)]


class LbmfvmError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"lbmfvm error {code}: {msg}")
        self.code = code


_lock = threading.Lock()
_lib = None


def lib() -> ctypes.CDLL:
    """Load liblbmfvm.so (building it with nvcc if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build()
            if not os.path.exists(path):
                raise RuntimeError(f"liblbmfvm.so missing at {path}")
            L = ctypes.CDLL(path)
            vp, i32, i64, d = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
            G, O = ctypes.POINTER(lbmfvm_grid_t), ctypes.POINTER(lbmfvm_opts_t)
            pp = ctypes.POINTER(ctypes.c_void_p)
            dp, i64p = ctypes.POINTER(d), ctypes.POINTER(i64)
            sig = {
                "lbmfvm_opts_default": (None, [O]),
                "lbmfvm_workspace_bytes": (ctypes.c_int, [G, O, ctypes.POINTER(ctypes.c_size_t)]),
                "lbmfvm_create": (ctypes.c_int, [G, vp, d, d, d, O, pp]),
                "lbmfvm_create_lattice": (ctypes.c_int, [G, vp, d, d, d, vp, O, pp]),
                "lbmfvm_set_state": (ctypes.c_int, [vp, vp, vp, vp]),
                "lbmfvm_step": (ctypes.c_int, [vp, i64]),
                "lbmfvm_inject_stall": (ctypes.c_int, [vp]),
                "lbmfvm_step_count": (ctypes.c_int, [vp, i64p]),
                "lbmfvm_fields": (ctypes.c_int, [vp, vp, vp, vp, vp]),
                "lbmfvm_fields_f32": (ctypes.c_int, [vp, vp, vp, vp, vp]),
                "lbmfvm_nusselt": (ctypes.c_int, [vp, dp, vp, dp]),
                "lbmfvm_residual": (ctypes.c_int, [vp, dp]),
                "lbmfvm_run_to_steady": (ctypes.c_int, [vp, d, i64, i64, i64p, dp]),
                "lbmfvm_copy_state": (ctypes.c_int, [vp, vp]),
                "lbmfvm_kernel_info": (ctypes.c_int, [vp, ctypes.POINTER(i32), ctypes.POINTER(i32)]),
                "lbmfvm_fv_info": (ctypes.c_int, [vp, ctypes.POINTER(i32), ctypes.POINTER(i32)]),
                "lbmfvm_launch_count": (ctypes.c_int, [vp, i64p]),
                "lbmfvm_params": (ctypes.c_int, [vp, dp, dp, dp, dp]),
                "lbmfvm_residual_noalloc": (ctypes.c_int, [vp, vp, vp, vp, vp, i64, vp, dp]),
                "lbmfvm_save": (ctypes.c_int, [vp, ctypes.c_char_p]),
                "lbmfvm_load": (ctypes.c_int, [vp, ctypes.c_char_p]),
                "lbmfvm_checkpoint_info": (ctypes.c_int, [ctypes.c_char_p, ctypes.POINTER(lbmfvm_checkpoint_header_t)]),
                "lbmfvm_destroy": (None, [vp]),
                "lbmfvm_last_error": (ctypes.c_char_p, [vp]),
                "lbmfvm_batch_create": (ctypes.c_int, [i32, G, vp, dp, dp, dp, O, pp]),
                "lbmfvm_batch_set_state": (ctypes.c_int, [vp, i32, vp, vp, vp]),
                "lbmfvm_batch_step": (ctypes.c_int, [vp, i64]),
                "lbmfvm_batch_residuals": (ctypes.c_int, [vp, vp]),
                "lbmfvm_batch_run": (ctypes.c_int, [vp, d, i64, i64, vp, vp]),
                "lbmfvm_batch_fields": (ctypes.c_int, [vp, i32, vp, vp, vp, vp]),
                "lbmfvm_batch_nusselt": (ctypes.c_int, [vp, i32, dp, vp, dp]),
                "lbmfvm_batch_info": (ctypes.c_int, [vp, i32, i64p, ctypes.POINTER(i32), vp]),
                "lbmfvm_batch_substeps": (ctypes.c_int, [vp, i32, ctypes.POINTER(i32)]),
                "lbmfvm_batch_set_polish": (ctypes.c_int, [vp, i32, d, i32]),
                "lbmfvm_batch_precision": (ctypes.c_int, [vp, i32, ctypes.POINTER(i32)]),
                "lbmfvm_batch_kernel_info": (ctypes.c_int, [vp, i32, ctypes.POINTER(i32)]),
                "lbmfvm_batch_destroy": (None, [vp]),
                "lbmfvm_batch_last_error": (ctypes.c_char_p, [vp]),
            }
            for name, (res, args) in sig.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
        return _lib


def _check(code: int, handle=None):
    if code != LBMFVM_OK:
        msg = lib().lbmfvm_last_error(handle)
        raise LbmfvmError(code, msg.decode() if msg else "")


def _addr(a):
    """Address of a numpy array or torch tensor (None passes NULL)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return ctypes.c_void_p(a.data_ptr())
    return a.ctypes.data_as(ctypes.c_void_p)


def make_grid(nx, ny, bc=(LBMFVM_BC_DIRICHLET, LBMFVM_BC_DIRICHLET, LBMFVM_BC_ADIABATIC, LBMFVM_BC_ADIABATIC),
              t_wall=(1.0, 0.0, 0.0, 0.0), u_lid=0.0, t_init=0.5) -> lbmfvm_grid_t:
    g = lbmfvm_grid_t()
    g.nx, g.ny = int(nx), int(ny)
    for s in range(4):
        g.bc[s] = int(bc[s])
        g.t_wall[s] = float(t_wall[s])
    g.u_lid, g.t_init = float(u_lid), float(t_init)
    return g


def lbmfvm_opts_default() -> lbmfvm_opts_t:
    o = lbmfvm_opts_t()
    lib().lbmfvm_opts_default(ctypes.byref(o))
    return o


def lbmfvm_workspace_bytes(grid: lbmfvm_grid_t, opts: lbmfvm_opts_t | None = None) -> int:
    out = ctypes.c_size_t()
    _check(lib().lbmfvm_workspace_bytes(ctypes.byref(grid), ctypes.byref(opts) if opts else None, ctypes.byref(out)))
    return out.value


def lbmfvm_create(grid, mask, Ra, Pr, Ma, opts=None):
    h = ctypes.c_void_p()
    _check(lib().lbmfvm_create(ctypes.byref(grid), _addr(mask), float(Ra), float(Pr), float(Ma),
                               ctypes.byref(opts) if opts else None, ctypes.byref(h)))
    return h


def lbmfvm_create_lattice(grid, mask, nu, alpha, gbeta, force=None, opts=None):
    h = ctypes.c_void_p()
    fp = None
    if force is not None:
        fp = (ctypes.c_double * 2)(float(force[0]), float(force[1]))
    _check(lib().lbmfvm_create_lattice(ctypes.byref(grid), _addr(mask), float(nu), float(alpha), float(gbeta),
                                       fp, ctypes.byref(opts) if opts else None, ctypes.byref(h)))
    return h


def lbmfvm_set_state(h, u=None, v=None, T=None):
    _check(lib().lbmfvm_set_state(h, _addr(u), _addr(v), _addr(T)), h)


def lbmfvm_step(h, n):
    _check(lib().lbmfvm_step(h, int(n)), h)


def lbmfvm_inject_stall(h):
    _check(lib().lbmfvm_inject_stall(h), h)


def lbmfvm_step_count(h) -> int:
    out = ctypes.c_int64()
    _check(lib().lbmfvm_step_count(h, ctypes.byref(out)), h)
    return out.value


def lbmfvm_fields(h, rho=None, u=None, v=None, T=None):
    _check(lib().lbmfvm_fields(h, _addr(rho), _addr(u), _addr(v), _addr(T)), h)


def lbmfvm_fields_f32(h, rho=None, u=None, v=None, T=None):
    _check(lib().lbmfvm_fields_f32(h, _addr(rho), _addr(u), _addr(v), _addr(T)), h)


def lbmfvm_nusselt(h, local_hot=None):
    mh, mc = ctypes.c_double(), ctypes.c_double()
    _check(lib().lbmfvm_nusselt(h, ctypes.byref(mh), _addr(local_hot), ctypes.byref(mc)), h)
    return mh.value, mc.value


def lbmfvm_residual(h) -> float:
    r = ctypes.c_double()
    _check(lib().lbmfvm_residual(h, ctypes.byref(r)), h)
    return r.value


def lbmfvm_run_to_steady(h, tol=1e-8, check_every=1000, max_steps=10**8):
    done, r = ctypes.c_int64(), ctypes.c_double()
    _check(lib().lbmfvm_run_to_steady(h, float(tol), int(check_every), int(max_steps), ctypes.byref(done),
                                      ctypes.byref(r)), h)
    return done.value, r.value


def lbmfvm_launch_count(h) -> int:
    n = ctypes.c_int64()
    _check(lib().lbmfvm_launch_count(h, ctypes.byref(n)), h)
    return n.value


def lbmfvm_kernel_info(h):
    k, c = ctypes.c_int32(), ctypes.c_int32()
    _check(lib().lbmfvm_kernel_info(h, ctypes.byref(k), ctypes.byref(c)), h)
    return k.value, c.value


def lbmfvm_fv_info(h):
    """(scheme, sub-steps) of the handle's energy update."""
    sc, m = ctypes.c_int32(), ctypes.c_int32()
    _check(lib().lbmfvm_fv_info(h, ctypes.byref(sc), ctypes.byref(m)), h)
    return sc.value, m.value


def _tma_config(cfg):
    return {"auto": LBMFVM_TMA_AUTOTUNE, "default": LBMFVM_TMA_DEFAULT}.get(cfg, cfg) if isinstance(cfg, str) \
        else int(cfg)


def lbmfvm_copy_state(dst, src):
    _check(lib().lbmfvm_copy_state(dst, src), dst)


def lbmfvm_params(h):
    out = [ctypes.c_double() for _ in range(4)]
    _check(lib().lbmfvm_params(h, *[ctypes.byref(x) for x in out]), h)
    return tuple(x.value for x in out)


def lbmfvm_residual_noalloc(u, v, u_prev, v_prev, select=None, n=None, stream=None) -> float:
    """Residual of lbmfvm_residual on caller device arrays, without allocation."""
    r = ctypes.c_double()
    n = int(u.numel() if n is None else n)
    _check(lib().lbmfvm_residual_noalloc(_addr(u), _addr(v), _addr(u_prev), _addr(v_prev), _addr(select), n,
                                         None if stream is None else ctypes.c_void_p(stream), ctypes.byref(r)))
    return r.value


def lbmfvm_save(h, path):
    _check(lib().lbmfvm_save(h, os.fsencode(path)), h)


def lbmfvm_load(h, path):
    _check(lib().lbmfvm_load(h, os.fsencode(path)), h)


def lbmfvm_checkpoint_info(path) -> dict:
    """Header of the checkpoint at path, after its magic, sizes and CRCs are
    verified (no GPU needed)."""
    hd = lbmfvm_checkpoint_header_t()
    _check(lib().lbmfvm_checkpoint_info(os.fsencode(path), ctypes.byref(hd)))
    return dict(nx=hd.nx, ny=hd.ny, store=hd.store, steps=hd.steps, bc=tuple(hd.bc), t_wall=tuple(hd.t_wall),
                u_lid=hd.u_lid, tau=hd.tau, alpha=hd.alpha, gbeta=hd.gbeta, t_ref=hd.t_ref, force=tuple(hd.force),
                payload_bytes=hd.payload_bytes, code_crc=hd.code_crc, payload_crc=hd.payload_crc,
                fv_scheme=hd.fv_scheme, fv_substeps=max(1, hd.fv_substeps), energy=hd.energy, wall_bc=hd.wall_bc)


def lbmfvm_destroy(h):
    if h:
        lib().lbmfvm_destroy(h)


def lbmfvm_last_error(h=None) -> str:
    return lib().lbmfvm_last_error(h).decode()


class Cavity:
    """One cavity on the current CUDA device.

    Device memory for the state comes from a PyTorch uint8 tensor handed to
    the library as its workspace; work is ordered on PyTorch's current stream.
    Build it either from the nondimensional groups (``Ra``, ``Pr``, ``Ma``) or
    from lattice parameters (``nu``, ``alpha``, ``gbeta``, ``force``).
    """

    def __init__(self, nx, ny, *, Ra=None, Pr=None, Ma=None, nu=None, alpha=None, gbeta=0.0, force=None,
                 mask=None, store="f32", bc=(LBMFVM_BC_DIRICHLET, LBMFVM_BC_DIRICHLET, LBMFVM_BC_ADIABATIC,
                                             LBMFVM_BC_ADIABATIC),
                 t_wall=(1.0, 0.0, 0.0, 0.0), u_lid=0.0, t_init=0.5, t_ref=None, tile_y=0, kernel="auto",
                 tma_config="default", fv_scheme="central", fv_substeps=1, energy="fv", wall_bc="nee", fv_grid=1,
                 fv_every=1, device=None):
        import torch

        self.nx, self.ny = int(nx), int(ny)
        self.grid = make_grid(nx, ny, bc, t_wall, u_lid, t_init)
        self.opts = lbmfvm_opts_default()
        self.opts.store = PRECISIONS[store] if isinstance(store, str) else int(store)
        self.opts.tile_y = int(tile_y)
        self.opts.kernel = KERNELS[kernel] if isinstance(kernel, str) else int(kernel)
        self.opts.tma_config = _tma_config(tma_config)
        self.opts.t_ref = math.nan if t_ref is None else float(t_ref)
        self.opts.fv_scheme = FV_SCHEMES[fv_scheme] if isinstance(fv_scheme, str) else int(fv_scheme)
        self.opts.fv_substeps = int(fv_substeps)
        self.opts.energy = ENERGY[energy] if isinstance(energy, str) else int(energy)
        self.opts.wall_bc = WALLS[wall_bc] if isinstance(wall_bc, str) else int(wall_bc)
        self.opts.fv_grid = int(fv_grid)
        self.opts.fv_every = int(fv_every)
        dev = torch.device("cuda" if device is None else device)
        self.device = dev
        nbytes = lbmfvm_workspace_bytes(self.grid, self.opts)
        self._ws = torch.empty(nbytes + 256, dtype=torch.uint8, device=dev)
        base = self._ws.data_ptr()
        aligned = (base + 255) // 256 * 256
        self.opts.workspace = aligned
        self.opts.workspace_bytes = nbytes
        self.opts.cuda_stream = torch.cuda.current_stream(dev).cuda_stream
        self._mask = None if mask is None else np.ascontiguousarray(mask, dtype=np.uint8).reshape(self.ny, self.nx)
        with torch.cuda.device(dev):
            if Ra is not None:
                self.h = lbmfvm_create(self.grid, self._mask, Ra, Pr, Ma, self.opts)
            else:
                self.h = lbmfvm_create_lattice(self.grid, self._mask, nu, alpha, gbeta, force, self.opts)
        self.nu, self.alpha, self.gbeta, self.tau = lbmfvm_params(self.h)

    def close(self):
        if getattr(self, "h", None):
            lbmfvm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_state(self, u=None, v=None, T=None):
        conv = lambda a: None if a is None else (a if hasattr(a, "data_ptr") else
                                                np.ascontiguousarray(a, dtype=np.float32).reshape(self.ny, self.nx))
        u, v, T = conv(u), conv(v), conv(T)
        lbmfvm_set_state(self.h, u, v, T)

    def step(self, n=1):
        lbmfvm_step(self.h, n)

    @property
    def steps(self):
        return lbmfvm_step_count(self.h)

    def fields(self):
        shp = (self.ny, self.nx)
        rho, u, v, T = (np.empty(shp) for _ in range(4))
        lbmfvm_fields(self.h, rho, u, v, T)
        return rho, u, v, T

    def nusselt(self):
        loc = np.empty(self.ny)
        mh, mc = lbmfvm_nusselt(self.h, loc)
        return mh, loc, mc

    def residual(self):
        return lbmfvm_residual(self.h)

    def run_to_steady(self, tol=1e-8, check_every=1000, max_steps=10**8):
        return lbmfvm_run_to_steady(self.h, tol, check_every, max_steps)

    @property
    def tma_config(self):
        """TMA tile shape in use (-1 on the generic kernel)."""
        return lbmfvm_kernel_info(self.h)[1]

    @property
    def substeps(self):
        """Energy-update sub-steps per lattice step."""
        return lbmfvm_fv_info(self.h)[1]

    def copy_state_from(self, other: "Cavity"):
        """Take ``other``'s state (populations, temperature, step count,
        residual snapshot), converted to this cavity's storage precision."""
        lbmfvm_copy_state(self.h, other.h)

    def save(self, path):
        """Write this cavity's state to a checkpoint file."""
        lbmfvm_save(self.h, path)

    def load(self, path):
        """Resume from a checkpoint saved by a cavity of the same geometry,
        storage and parameters."""
        lbmfvm_load(self.h, path)


def _bcheck(code: int, b):
    if code != LBMFVM_OK:
        msg = lib().lbmfvm_batch_last_error(b)
        raise LbmfvmError(code, msg.decode() if msg else "")


class Batch:
    """Many cavities advanced together by one persistent launch per step.

    ``cases``: sequence of objects with ``nx, ny, Ra, Pr, Ma`` and optional
    ``mask`` (ny x nx, 1 = solid) and ``t_init`` attributes (for example
    ``workloads.CavityCase``).  The library allocates the memory; work runs on
    PyTorch's current stream.
    """

    def __init__(self, cases, store="f32", tma_config="auto", fv_scheme="central", fv_substeps=1, device=None):
        import torch

        self.n = len(cases)
        self.shapes = [(int(c.ny), int(c.nx)) for c in cases]
        grids = (lbmfvm_grid_t * self.n)()
        for k, c in enumerate(cases):
            grids[k] = make_grid(c.nx, c.ny, t_init=getattr(c, "t_init", 0.5))
        self._masks = [None if getattr(c, "mask", None) is None else
                       np.ascontiguousarray(c.mask, dtype=np.uint8).reshape(c.ny, c.nx) for c in cases]
        mptrs = (ctypes.c_void_p * self.n)(*[None if m is None else m.ctypes.data for m in self._masks])
        arr = lambda xs: (ctypes.c_double * self.n)(*[float(x) for x in xs])
        ra, pr, ma = arr([c.Ra for c in cases]), arr([c.Pr for c in cases]), arr([c.Ma for c in cases])
        self.opts = lbmfvm_opts_default()
        self.opts.store = PRECISIONS[store] if isinstance(store, str) else int(store)
        self.opts.tma_config = _tma_config(tma_config)
        self.opts.fv_scheme = FV_SCHEMES[fv_scheme] if isinstance(fv_scheme, str) else int(fv_scheme)
        self.opts.fv_substeps = int(fv_substeps)
        dev = torch.device("cuda" if device is None else device)
        self.opts.cuda_stream = torch.cuda.current_stream(dev).cuda_stream
        self.b = ctypes.c_void_p()
        with torch.cuda.device(dev):
            _bcheck(lib().lbmfvm_batch_create(self.n, grids, ctypes.cast(mptrs, ctypes.c_void_p), ra, pr, ma,
                                              ctypes.byref(self.opts), ctypes.byref(self.b)), None)

    def close(self):
        if getattr(self, "b", None):
            lib().lbmfvm_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_state(self, i, u=None, v=None, T=None):
        """Initial (u, v, T) of cavity i: host arrays or float32 device tensors
        of ny x nx values (None: rest, t_init)."""
        ny, nx = self.shapes[i]
        conv = lambda a: None if a is None else (a if hasattr(a, "data_ptr") else
                                                np.ascontiguousarray(a, dtype=np.float32).reshape(ny, nx))
        u, v, T = conv(u), conv(v), conv(T)
        _bcheck(lib().lbmfvm_batch_set_state(self.b, int(i), _addr(u), _addr(v), _addr(T)), self.b)

    def step(self, n=1):
        _bcheck(lib().lbmfvm_batch_step(self.b, int(n)), self.b)

    def residuals(self):
        r = np.empty(self.n)
        _bcheck(lib().lbmfvm_batch_residuals(self.b, _addr(r)), self.b)
        return r

    def run(self, tol=1e-8, check_every=1000, max_steps=10**8):
        steps = np.empty(self.n, dtype=np.int64)
        r = np.empty(self.n)
        _bcheck(lib().lbmfvm_batch_run(self.b, float(tol), int(check_every), int(max_steps), _addr(steps), _addr(r)),
                self.b)
        return steps, r

    def fields(self, i):
        shp = self.shapes[i]
        rho, u, v, T = (np.empty(shp) for _ in range(4))
        _bcheck(lib().lbmfvm_batch_fields(self.b, int(i), _addr(rho), _addr(u), _addr(v), _addr(T)), self.b)
        return rho, u, v, T

    def nusselt(self, i):
        loc = np.empty(self.shapes[i][0])
        mh, mc = ctypes.c_double(), ctypes.c_double()
        _bcheck(lib().lbmfvm_batch_nusselt(self.b, int(i), ctypes.byref(mh), _addr(loc), ctypes.byref(mc)), self.b)
        return mh.value, loc, mc.value

    def info(self, i):
        steps, active = ctypes.c_int64(), ctypes.c_int32()
        params = np.empty(4)
        _bcheck(lib().lbmfvm_batch_info(self.b, int(i), ctypes.byref(steps), ctypes.byref(active), _addr(params)),
                self.b)
        return steps.value, bool(active.value), tuple(params)

    def substeps(self, i):
        """Energy-update sub-steps per lattice step of cavity i."""
        m = ctypes.c_int32()
        _bcheck(lib().lbmfvm_batch_substeps(self.b, int(i), ctypes.byref(m)), self.b)
        return m.value

    def set_polish(self, prec, r_switch, stall_checks=0):
        """Ladder switch of the cavities stepped in ``prec``: the residual
        below which ``run`` moves them one precision up (<= 0: never), and the
        checks without halving that also do (<= 0: off)."""
        p = PRECISIONS[prec] if isinstance(prec, str) else int(prec)
        _bcheck(lib().lbmfvm_batch_set_polish(self.b, p, float(r_switch), int(stall_checks)), self.b)

    def tma_config(self, prec):
        """TMA tile shape of the packed grid in ``prec`` (-1 before it exists)."""
        p = PRECISIONS[prec] if isinstance(prec, str) else int(prec)
        c = ctypes.c_int32()
        _bcheck(lib().lbmfvm_batch_kernel_info(self.b, p, ctypes.byref(c)), self.b)
        return c.value

    def precision(self, i):
        """Storage precision cavity i is stepped in ("f32", "f16" or "bf16")."""
        p = ctypes.c_int32()
        _bcheck(lib().lbmfvm_batch_precision(self.b, int(i), ctypes.byref(p)), self.b)
        return {v: k for k, v in PRECISIONS.items()}[p.value]
