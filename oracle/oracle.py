"""Python face of the FP64 CPU oracle (olbm_oracle.c), loaded through ctypes.

TEST INFRASTRUCTURE ONLY: tests/, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` use it. The product package never imports it,
and it imports nothing from the product package.

Paper: arXiv 2602.21242 (generalized Onsager-regularised LBM on D2Q9). Each
wrapped C function names the equation it follows in olbm_core.inc.

Readings of the paper taken here (see the C file for the rest):
  * viscosity and relaxation time: nu = theta * (tau - 1/2), i.e. the printed
    "tau = nu / theta" (Sec. 1) plus the 1/2 that the (1 - dt/2tau) factors of
    the Chapman-Enskog result (Eq. 5) imply for dt = 1.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = [os.path.join(_HERE, "olbm_oracle.c"), os.path.join(_HERE, "olbm_core.inc")]
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

LBGK, OREG, OREG_PARTIAL, OREG_COMPLETE, OREG_COMPLETE_NEQ, LBGK_POLY = 0, 1, 2, 3, 4, 5
NO_COLLISION = -1  # test hook: streaming only

# D2Q9 velocities, Fig. 1a numbering (the oracle's own copy).
CX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1], dtype=np.int64)
CY = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1], dtype=np.int64)


def build(force: bool = False) -> str:
    """Compile olbm_oracle.c into oracle/_build/liboracle.so (gcc, OpenMP, no FMA contraction).

    Test hook: when OLBM_ORACLE_LIB names a library, that library is loaded instead
    (tests/test_oracle_mutants_cpu.py runs the pins against copies of the oracle with a
    planted mistake this way)."""
    override = os.environ.get("OLBM_ORACLE_LIB")
    if override:
        return override
    os.makedirs(_BUILD_DIR, exist_ok=True)
    newest = max(os.path.getmtime(p) for p in _SRC)
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= newest:
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-std=c11", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-o", tmp, _SRC[0], "-lm"]
    subprocess.run(cmd, check=True, cwd=_HERE)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        d, i, p = ctypes.c_double, ctypes.c_int, ctypes.c_void_p
        sig = {
            "oracle_version": ([], i),
            "oracle_set_threads": ([i], i),
            "oracle_geq": ([d, d, d, d, p], None),
            "oracle_collide_node": ([p, d, d, i, p], None),
            "oracle_node_terms": ([p, d, p, p, p, p, p, p, p, p], None),
            "oracle_oreg_node": ([p, p, d, d, d, d, p], None),
            "oracle_init": ([i, i, d, p, p, p, p], None),
            "oracle_run": ([i, i, d, d, i, i, p, p], None),
            "oracle_run_cplx": ([i, i, d, d, i, i, p, p], None),
            "oracle_run_walls": ([i, i, d, d, i, i, p, p, p], None),
            "oracle_run_walls_cplx": ([i, i, d, d, i, i, p, p, p], None),
            "oracle_init_cplx": ([i, i, d, p, p, p, p], None),
            "oracle_collide_node_cplx": ([p, d, d, i, p], None),
            "oracle_moments_field": ([i, i, p, p, p, p], None),
            "oracle_moments_field_cplx": ([i, i, p, p, p, p], None),
            "oracle_diagnostics": ([i, i, p, p], None),
        }
        for name, (args, res) in sig.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        _lib = lib
        return lib


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


def _f64(a, shape=None) -> np.ndarray:
    out = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None and out.shape != shape:
        raise ValueError(f"expected shape {shape}, got {out.shape}")
    return out


def _c128(a, shape=None) -> np.ndarray:
    out = np.ascontiguousarray(a, dtype=np.complex128)
    if shape is not None and out.shape != shape:
        raise ValueError(f"expected shape {shape}, got {out.shape}")
    return out


def tau_from_nu(nu: float, theta: float) -> float:
    """Relaxation time for lattice viscosity nu at reduced temperature theta: tau = nu/theta + 1/2."""
    return nu / theta + 0.5


def set_threads(n: int = 0) -> int:
    """Set the OpenMP thread count used by run() (0 = leave as is); returns the count in use."""
    return int(_load().oracle_set_threads(int(n)))


def geq(rho: float, ux: float, uy: float, theta: float) -> np.ndarray:
    """Guided equilibrium at one node (Eq. 10)."""
    out = np.empty(9)
    _load().oracle_geq(float(rho), float(ux), float(uy), float(theta), _ptr(out))
    return out


def collide_node(f9, theta: float, tau: float, model: int) -> np.ndarray:
    """Post-collision populations at one node (Eq. 1a with the model's g)."""
    f9 = _f64(f9, (9,))
    out = np.empty(9)
    _load().oracle_collide_node(_ptr(f9), float(theta), float(tau), int(model), _ptr(out))
    return out


def collide_node_cplx(f9, theta: float, tau: float, model: int) -> np.ndarray:
    f9 = _c128(f9, (9,))
    out = np.empty(9, dtype=np.complex128)
    _load().oracle_collide_node_cplx(_ptr(f9), float(theta), float(tau), int(model), _ptr(out))
    return out


def node_terms(f9, theta: float) -> dict:
    """Every intermediate of one collision: moments, f^eq, f^OReg, psi, pref, Pi~, Psi^P, Psi^C."""
    f9 = _f64(f9, (9,))
    mom, feq, foreg = np.empty(3), np.empty(9), np.empty(9)
    psi, pref, pit = np.empty(2), np.empty(1), np.empty(3)
    psiP, psiC = np.empty(9), np.empty(9)
    _load().oracle_node_terms(_ptr(f9), float(theta), _ptr(mom), _ptr(feq), _ptr(foreg),
                              _ptr(psi), _ptr(pref), _ptr(pit), _ptr(psiP), _ptr(psiC))
    return {"rho": mom[0], "ux": mom[1], "uy": mom[2], "feq": feq, "foreg": foreg,
            "psi": psi, "pref": float(pref[0]), "pitilde": pit, "PsiP": psiP, "PsiC": psiC}


def oreg_node(f9, feq9, rho: float, ux: float, uy: float, theta: float) -> np.ndarray:
    """Eq. 2 for given (f, f^eq, rho, u)."""
    f9, feq9 = _f64(f9, (9,)), _f64(feq9, (9,))
    out = np.empty(9)
    _load().oracle_oreg_node(_ptr(f9), _ptr(feq9), float(rho), float(ux), float(uy),
                             float(theta), _ptr(out))
    return out


def init(rho, ux, uy, theta: float) -> np.ndarray:
    """Pre-collision populations f(x, 0) = f^eq(rho0, u0), shape (9, ny, nx)."""
    rho = _f64(rho)
    ny, nx = rho.shape
    ux, uy = _f64(ux, (ny, nx)), _f64(uy, (ny, nx))
    f = np.empty((9, ny, nx))
    _load().oracle_init(nx, ny, float(theta), _ptr(rho), _ptr(ux), _ptr(uy), _ptr(f))
    return f


def _walls(walls, ny, nx):
    if walls is None:
        return None, None
    w = np.ascontiguousarray(np.asarray(walls) != 0, dtype=np.uint8)
    if w.shape != (ny, nx):
        raise ValueError(f"walls must have shape {(ny, nx)}, got {w.shape}")
    return w, _ptr(w)


def run(f, theta: float, tau: float, model: int, nsteps: int, walls=None) -> np.ndarray:
    """Advance pre-collision populations (9, ny, nx) by nsteps LBE steps (Eq. 1); returns a new array.

    walls: optional (ny, nx) flags; a nonzero node is a fullway bounce-back wall (Sec. 5.2)."""
    f = np.array(f, dtype=np.float64, order="C", copy=True)
    if f.ndim != 3 or f.shape[0] != 9:
        raise ValueError("populations must have shape (9, ny, nx)")
    _, ny, nx = f.shape
    work = np.empty_like(f)
    w, wp = _walls(walls, ny, nx)
    _load().oracle_run_walls(nx, ny, float(theta), float(tau), int(model), int(nsteps), wp, _ptr(f), _ptr(work))
    return f


def run_cplx(f, theta: float, tau: float, model: int, nsteps: int, walls=None) -> np.ndarray:
    """Complex-step twin of run() (complex128 populations)."""
    f = np.array(f, dtype=np.complex128, order="C", copy=True)
    _, ny, nx = f.shape
    work = np.empty_like(f)
    w, wp = _walls(walls, ny, nx)
    _load().oracle_run_walls_cplx(nx, ny, float(theta), float(tau), int(model), int(nsteps), wp, _ptr(f),
                                  _ptr(work))
    return f


def init_cplx(rho, ux, uy, theta: float) -> np.ndarray:
    rho = _c128(rho)
    ny, nx = rho.shape
    ux, uy = _c128(ux, (ny, nx)), _c128(uy, (ny, nx))
    f = np.empty((9, ny, nx), dtype=np.complex128)
    _load().oracle_init_cplx(nx, ny, float(theta), _ptr(rho), _ptr(ux), _ptr(uy), _ptr(f))
    return f


def moments(f):
    """(rho, u_x, u_y) of pre-collision populations (9, ny, nx)."""
    f = _f64(f)
    _, ny, nx = f.shape
    rho, ux, uy = np.empty((ny, nx)), np.empty((ny, nx)), np.empty((ny, nx))
    _load().oracle_moments_field(nx, ny, _ptr(f), _ptr(rho), _ptr(ux), _ptr(uy))
    return rho, ux, uy


def moments_cplx(f):
    f = _c128(f)
    _, ny, nx = f.shape
    rho = np.empty((ny, nx), dtype=np.complex128)
    ux, uy = np.empty_like(rho), np.empty_like(rho)
    _load().oracle_moments_field_cplx(nx, ny, _ptr(f), _ptr(rho), _ptr(ux), _ptr(uy))
    return rho, ux, uy


def diagnostics(f) -> np.ndarray:
    """[sum rho, sum rho u_x, sum rho u_y, sum rho |u|^2 / 2, non-finite node count]."""
    f = _f64(f)
    _, ny, nx = f.shape
    out = np.empty(5)
    _load().oracle_diagnostics(nx, ny, _ptr(f), _ptr(out))
    return out
