"""FP64 CPU oracle for leading-order Stokesian dynamics (arXiv:1205.6333).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` are the only
callers.  The CUDA library never imports this package and this package never
imports the CUDA library; the two share no code.  The arithmetic lives in
``sd_oracle.c`` (plain C, IEEE double, no fast-math); this module compiles it
with gcc and marshals numpy arrays through ctypes.

Every function is the paper's definition written out:

* ``mu0``                 -- Stokes mobility 1/(6 pi eta a)            (Sec. 2.2)
* ``pair_tensor``         -- T(r): Rotne-Prager / Oseen / RPY          (Sec. 2.2, Eqs. rotneMobility, oseenTensor)
* ``mobility_apply``      -- v_i = mu0 F_i + sum_{j!=i} T(r_i-r_j) F_j  (Sec. 2.2, Eq. rotneMobility; Algorithm 1)
* ``mobility_rows``       -- the same sum for selected rows i
* ``assemble``            -- the 3N x 3N matrix mu (second formulation, tests only)
* ``forces``              -- F_ext + gravity + truncated (2a/r)^12 repulsion (Sec. 3.1, step 2)
* ``lubrication``         -- -sum_j zeta^sing_ij (v_i - v_j), cut at r = 3a (Sec. 2.3 Eq. lubrication)
* ``euler``               -- x <- x + dt M(x) F(x)                     (Sec. 3.1, steps 1-3)
* ``vjp``                 -- (dv/dx)^T w and M w, closed-form derivative of T
* ``adjoint``             -- reverse sweep through Euler steps

Parity notes: no function here is "parity unpinned"; the pins live in
``tests/test_oracle_pins.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sd_oracle.c")
_LIB = os.path.join(_HERE, "libsd_oracle.so")

RPY, RP, OSEEN = 0, 1, 2
TENSORS = {"rpy": RPY, "rp": RP, "oseen": OSEEN}

_lib = None


def build(force: bool = False) -> str:
    """Compile sd_oracle.c into libsd_oracle.so (gcc -O2, no fast-math, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        cmd = ["gcc", "-O2", "-fno-fast-math", "-ffp-contract=off", "-fPIC", "-shared",
               "-fopenmp", "-std=c99", _SRC, "-o", tmp, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        # SD_ORACLE_LIB: load another build of sd_oracle.c (the mutation tests plant
        # mistakes in a copy and check that the pins catch them)
        path = os.environ.get("SD_ORACLE_LIB")
        if not path:
            build()
            path = _LIB
        lib = ctypes.CDLL(path)
        D, I, P, L = ctypes.c_double, ctypes.c_int, ctypes.c_void_p, ctypes.c_int64
        lib.sdo_mu0.restype = D
        lib.sdo_mu0.argtypes = [D, D]
        lib.sdo_pair_tensor.argtypes = [I, D, D, P, P]
        lib.sdo_mobility_apply.argtypes = [I, D, D, P, I, P, P, P, I]
        lib.sdo_mobility_rows.argtypes = [I, D, D, P, I, P, P, I, P, P, I]
        lib.sdo_assemble.argtypes = [I, D, D, P, I, P, P]
        lib.sdo_forces.argtypes = [D, P, I, P, P, P, D, D, P]
        lib.sdo_euler.argtypes = [I, D, D, P, I, P, P, P, D, D, I, D, L, L, P, I]
        lib.sdo_lubrication.argtypes = [D, D, P, I, P, P, P]
        lib.sdo_vjp.argtypes = [I, D, D, P, I, P, P, P, P, P, I]
        lib.sdo_adjoint.argtypes = [I, D, D, P, I, P, P, P, D, L, P, P, P, I]
        lib.sdo_has_openmp.restype = I
        _lib = lib
    return _lib


class OracleError(RuntimeError):
    pass


def _check(st: int):
    if st == 4:
        raise OracleError("coincident distinct particles (r = 0) in RP/Oseen mode")
    if st != 0:
        raise OracleError("oracle status %d" % st)


def _d(a) -> np.ndarray:
    """Exact widening to a C-contiguous float64 array (float32 inputs widen exactly)."""
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _box(box):
    if box is None:
        return None
    b = _d(box).reshape(3)
    return b if np.any(b > 0) else None


def _t(tensor) -> int:
    return TENSORS[tensor] if isinstance(tensor, str) else int(tensor)


def _threads(nthreads):
    return int(nthreads) if nthreads else 1


def mu0(a: float = 1.0, eta: float = 1.0) -> float:
    return _load().sdo_mu0(float(a), float(eta))


def pair_tensor(r, tensor="rpy", a=1.0, eta=1.0) -> np.ndarray:
    r = _d(r).reshape(3)
    T = np.zeros(9)
    _check(_load().sdo_pair_tensor(_t(tensor), float(a), float(eta), _p(r), _p(T)))
    return T.reshape(3, 3)


def mobility_apply(x, F, tensor="rpy", a=1.0, eta=1.0, box=None, nthreads=None) -> np.ndarray:
    x, F = _d(x).reshape(-1, 3), _d(F).reshape(-1, 3)
    n = x.shape[0]
    assert F.shape[0] == n
    v = np.zeros((n, 3))
    b = _box(box)
    _check(_load().sdo_mobility_apply(_t(tensor), float(a), float(eta), _p(b), n, _p(x), _p(F), _p(v),
                                      _threads(nthreads)))
    return v


def mobility_rows(x, F, rows, tensor="rpy", a=1.0, eta=1.0, box=None, nthreads=None) -> np.ndarray:
    x, F = _d(x).reshape(-1, 3), _d(F).reshape(-1, 3)
    rows = np.ascontiguousarray(np.asarray(rows, dtype=np.int32))
    v = np.zeros((rows.size, 3))
    b = _box(box)
    _check(_load().sdo_mobility_rows(_t(tensor), float(a), float(eta), _p(b), x.shape[0], _p(x), _p(F),
                                     rows.size, _p(rows), _p(v), _threads(nthreads)))
    return v


def assemble(x, tensor="rpy", a=1.0, eta=1.0, box=None) -> np.ndarray:
    x = _d(x).reshape(-1, 3)
    n = x.shape[0]
    M = np.zeros((3 * n, 3 * n))
    b = _box(box)
    _check(_load().sdo_assemble(_t(tensor), float(a), float(eta), _p(b), n, _p(x), _p(M)))
    return M


def forces(x, fext=None, gravity=(0.0, 0.0, 0.0), rep_eps=0.0, rep_rc=2.5, a=1.0, box=None) -> np.ndarray:
    x = _d(x).reshape(-1, 3)
    n = x.shape[0]
    fe = None if fext is None else _d(fext).reshape(n, 3)
    g = _d(gravity).reshape(3)
    F = np.zeros((n, 3))
    b = _box(box)
    _check(_load().sdo_forces(float(a), _p(b), n, _p(x), _p(fe), _p(g), float(rep_eps), float(rep_rc), _p(F)))
    return F


def lubrication(x, v, a=1.0, eta=1.0, box=None) -> np.ndarray:
    """The lubrication friction forces -sum_j zeta_ij (v_i - v_j) of Sec. 2.3 / 3.1 step 2."""
    x, v = _d(x).reshape(-1, 3), _d(v).reshape(-1, 3)
    F = np.zeros_like(x)
    b = _box(box)
    _check(_load().sdo_lubrication(float(a), float(eta), _p(b), x.shape[0], _p(x), _p(v), _p(F)))
    return F


def euler(x0, nsteps, dt, fext=None, gravity=(0.0, 0.0, 0.0), rep_eps=0.0, rep_rc=2.5, tensor="rpy",
          a=1.0, eta=1.0, box=None, every=0, nthreads=None, lubrication=False):
    """Returns x after nsteps, and the positions after every `every`-th step if every > 0.
    With lubrication=True each step's forces include the lubrication friction of
    close pairs computed from the previous step's velocities (zero at the start)."""
    x = _d(x0).reshape(-1, 3).copy()
    n = x.shape[0]
    fe = None if fext is None else _d(fext).reshape(n, 3)
    g = _d(gravity).reshape(3)
    traj = None
    if every and every > 0:
        traj = np.zeros((int(nsteps) // int(every), n, 3))
    b = _box(box)
    _check(_load().sdo_euler(_t(tensor), float(a), float(eta), _p(b), n, _p(x), _p(fe), _p(g), float(rep_eps),
                             float(rep_rc), int(bool(lubrication)), float(dt), int(nsteps), int(every or 0),
                             _p(traj), _threads(nthreads)))
    return (x, traj) if traj is not None else x


def vjp(x, F, w, tensor="rpy", a=1.0, eta=1.0, box=None, nthreads=None):
    """(gx, gF) = ((d(M(x)F)/dx)^T w, M(x)^T w)."""
    x, F, w = _d(x).reshape(-1, 3), _d(F).reshape(-1, 3), _d(w).reshape(-1, 3)
    n = x.shape[0]
    gx = np.zeros((n, 3))
    gF = np.zeros((n, 3))
    b = _box(box)
    _check(_load().sdo_vjp(_t(tensor), float(a), float(eta), _p(b), n, _p(x), _p(F), _p(w), _p(gx), _p(gF),
                           _threads(nthreads)))
    return gx, gF


def adjoint(x0, fext, gxT, nsteps, dt, gravity=(0.0, 0.0, 0.0), tensor="rpy", a=1.0, eta=1.0, box=None,
            nthreads=None):
    """(dL/dx0, dL/dF_ext) for x_{n+1} = x_n + dt M(x_n)(F_ext + g), given gxT = dL/dx_T."""
    x0 = _d(x0).reshape(-1, 3)
    n = x0.shape[0]
    fe = _d(fext).reshape(n, 3)
    g = _d(gravity).reshape(3)
    gxT = _d(gxT).reshape(n, 3)
    gx0 = np.zeros((n, 3))
    gF = np.zeros((n, 3))
    b = _box(box)
    _check(_load().sdo_adjoint(_t(tensor), float(a), float(eta), _p(b), n, _p(x0), _p(fe), _p(g), float(dt),
                               int(nsteps), _p(gxT), _p(gx0), _p(gF), _threads(nthreads)))
    return gx0, gF


def has_openmp() -> bool:
    return bool(_load().sdo_has_openmp())
