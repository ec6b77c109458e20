"""FP64 CPU oracle for two-link staggered quark smearing (arXiv:2301.05518, Sec. 2).

TEST INFRASTRUCTURE ONLY.  The tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` are the only callers.  The oracle shares no code
with the CUDA library ``paper_2301_05518_gb300``, and neither imports the
other.  The arithmetic lives in ``oracle.c`` (plain C, FP64, periodic 4-D
coordinates); this module only compiles it with gcc and marshals numpy arrays.

Functions (all FP64, complex numbers as numpy complex128):

- ``twolink(U)``               W_i(x) = U_i(x) U_i(x+i)           (Sec. 2)
- ``apply_lap(W, psi, t0)``    4 Lap_two psi                       (Eq. tlLapl1)
- ``apply_lap_unfused(U, psi, t0)``  same from single links        (Eq. tlLapl2)
- ``smear(W, psi, n, sigma, t0)``    (1 + (sigma/n) Lap_two)^n psi (Eq. tlSmear)
- ``smear_unfused(U, psi, n, sigma, t0)``
- ``apply_hop(U, psi, t0)``         one-link hopping H psi          (Eq. 2)
- ``smear_onelink(U, psi, n, alpha, t0)``  (1 + alpha H)^n psi     (Eq. 3, C = 1)
- ``su3_project(M)``                projection of 3x3 matrices onto SU(3)
- ``ape_smear(U, alpha, n)``        APE-smeared spatial links (Sec. 2, the remark
                                    on gauge-smeared links after Eq. tlSmear)

Array shapes: ``U`` is ``[Lt, Lz, Ly, Lx, nd, 3, 3]`` (nd = 3 or 4, mu order
x, y, z[, t]); ``W`` is ``[Lt, Lz, Ly, Lx, 3, 3, 3]``; ``psi`` is
``[nvec, Lt, Lz, Ly, Lx, 3]`` or ``[Lt, Lz, Ly, Lx, 3]``.  ``t0 = -1`` acts on
every time slice, ``t0 >= 0`` on that slice only.

Parity status: every function is pinned by tests/test_oracle_pins.py (fused =
unfused, free-field closed forms, gauge covariance, Hermiticity, decoupling,
SU(3) closure, staggered-phase invariance, dense brute force).  The paper
prints no worked numerical example, so no value of the paper itself pins it.
"""

from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so with gcc (OpenMP, no FP contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
               _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        I = ctypes.c_int
        D = ctypes.c_double
        lib.oracle_twolink.argtypes = [P, I, P, P]
        lib.oracle_twolink.restype = None
        lib.oracle_apply_lap.argtypes = [P, P, P, P, I]
        lib.oracle_apply_lap.restype = None
        lib.oracle_apply_lap_unfused.argtypes = [P, I, P, P, P, I]
        lib.oracle_apply_lap_unfused.restype = None
        lib.oracle_smear.argtypes = [P, P, P, I, I, D, I]
        lib.oracle_smear.restype = I
        lib.oracle_smear_unfused.argtypes = [P, I, P, P, I, I, D, I]
        lib.oracle_smear_unfused.restype = I
        lib.oracle_apply_hop.argtypes = [P, I, P, P, P, I]
        lib.oracle_apply_hop.restype = None
        lib.oracle_smear_onelink.argtypes = [P, I, P, P, I, I, D, I]
        lib.oracle_smear_onelink.restype = I
        lib.oracle_su3_project.argtypes = [P, P]
        lib.oracle_su3_project.restype = I
        lib.oracle_ape.argtypes = [P, I, P, D, I, P]
        lib.oracle_ape.restype = I
        lib.oracle_threads.argtypes = []
        lib.oracle_threads.restype = I
        _lib = lib
    return _lib


def _dims(shape5) -> np.ndarray:
    Lt, Lz, Ly, Lx = shape5[:4]
    return np.array([Lx, Ly, Lz, Lt], dtype=np.int32)


def _c128(a) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.complex128)
    return a


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def threads() -> int:
    """OpenMP threads the oracle's parallel loops use."""
    return int(_load().oracle_threads())


def twolink(U) -> np.ndarray:
    """W_i(x) = U_i(x) U_i(x + i) for i = x, y, z (Sec. 2)."""
    U = _c128(U)
    assert U.ndim == 7 and U.shape[5:] == (3, 3) and U.shape[4] in (3, 4)
    dims = _dims(U.shape)
    W = np.zeros(U.shape[:4] + (3, 3, 3), dtype=np.complex128)
    _load().oracle_twolink(_ptr(U), U.shape[4], _ptr(dims), _ptr(W))
    return W


def _as_vecs(psi):
    psi = _c128(psi)
    single = psi.ndim == 5
    if single:
        psi = psi[None]
    assert psi.ndim == 6 and psi.shape[-1] == 3
    return np.ascontiguousarray(psi), single


def apply_lap(W, psi, t0: int = -1) -> np.ndarray:
    """Delta psi = 4 Lap_two psi (Eq. tlLapl1); unselected slices are 0."""
    W = _c128(W)
    psi5 = _c128(psi)
    assert psi5.ndim == 5
    dims = _dims(psi5.shape)
    out = np.zeros_like(psi5)
    _load().oracle_apply_lap(_ptr(W), _ptr(dims), _ptr(psi5), _ptr(out), int(t0))
    return out


def apply_lap_unfused(U, psi, t0: int = -1) -> np.ndarray:
    """Delta psi from single links applied twice (Eq. tlLapl2)."""
    U = _c128(U)
    psi5 = _c128(psi)
    assert psi5.ndim == 5
    dims = _dims(psi5.shape)
    out = np.zeros_like(psi5)
    _load().oracle_apply_lap_unfused(_ptr(U), U.shape[4], _ptr(dims), _ptr(psi5),
                                     _ptr(out), int(t0))
    return out


def smear(W, psi, n: int, sigma: float, t0: int = -1) -> np.ndarray:
    """(1 + (sigma/n) Lap_two)^n psi (Eq. tlSmear); returns a new array."""
    W = _c128(W)
    vecs, single = _as_vecs(psi)
    out = vecs.copy()
    dims = _dims(out.shape[1:])
    rc = _load().oracle_smear(_ptr(W), _ptr(dims), _ptr(out), out.shape[0], int(n),
                              float(sigma), int(t0))
    if rc != 0:
        raise ValueError("oracle_smear failed (%d)" % rc)
    return out[0] if single else out


def smear_unfused(U, psi, n: int, sigma: float, t0: int = -1) -> np.ndarray:
    """Eq. tlSmear with the operator of Eq. tlLapl2 (never forms W)."""
    U = _c128(U)
    vecs, single = _as_vecs(psi)
    out = vecs.copy()
    dims = _dims(out.shape[1:])
    rc = _load().oracle_smear_unfused(_ptr(U), U.shape[4], _ptr(dims), _ptr(out),
                                      out.shape[0], int(n), float(sigma), int(t0))
    if rc != 0:
        raise ValueError("oracle_smear_unfused failed (%d)" % rc)
    return out[0] if single else out


def apply_hop(U, psi, t0: int = -1) -> np.ndarray:
    """One-link hopping H psi (Eq. 2); unselected slices are 0."""
    U = _c128(U)
    psi5 = _c128(psi)
    assert psi5.ndim == 5
    dims = _dims(psi5.shape)
    out = np.zeros_like(psi5)
    _load().oracle_apply_hop(_ptr(U), U.shape[4], _ptr(dims), _ptr(psi5), _ptr(out), int(t0))
    return out


def smear_onelink(U, psi, n: int, alpha: float, t0: int = -1) -> np.ndarray:
    """Gaussian smearing (1 + alpha H)^n psi (Eq. 3 with C = 1); returns a new array."""
    U = _c128(U)
    vecs, single = _as_vecs(psi)
    out = vecs.copy()
    dims = _dims(out.shape[1:])
    rc = _load().oracle_smear_onelink(_ptr(U), U.shape[4], _ptr(dims), _ptr(out), out.shape[0], int(n),
                                      float(alpha), int(t0))
    if rc != 0:
        raise ValueError("oracle_smear_onelink failed (%d)" % rc)
    return out[0] if single else out


def su3_project(M) -> np.ndarray:
    """Nearest SU(3) matrix of each 3x3 complex matrix in M (shape [..., 3, 3]):
    the unitary polar factor by Newton's iteration, then the determinant phase
    removed by its principal cube root."""
    M = _c128(M)
    assert M.shape[-2:] == (3, 3)
    flat = np.ascontiguousarray(M.reshape(-1, 3, 3))
    out = np.empty_like(flat)
    lib = _load()
    for k in range(flat.shape[0]):
        src = np.ascontiguousarray(flat[k])
        dst = np.empty_like(src)
        if lib.oracle_su3_project(_ptr(src), _ptr(dst)) != 0:
            raise ValueError("oracle_su3_project: singular or not converged")
        out[k] = dst
    return out.reshape(M.shape)


def ape_smear(U, alpha: float, n: int) -> np.ndarray:
    """n APE steps on the spatial links (staples in the three spatial
    directions, weight alpha, projection onto SU(3)); returns [Lt, Lz, Ly, Lx, 3, 3, 3]."""
    U = _c128(U)
    assert U.ndim == 7 and U.shape[5:] == (3, 3) and U.shape[4] in (3, 4)
    dims = _dims(U.shape)
    out = np.zeros(U.shape[:4] + (3, 3, 3), dtype=np.complex128)
    rc = _load().oracle_ape(_ptr(U), U.shape[4], _ptr(dims), float(alpha), int(n), _ptr(out))
    if rc != 0:
        raise ValueError("oracle_ape: a projection failed")
    return out
