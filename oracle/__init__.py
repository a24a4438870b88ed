"""CPU oracle for the 3D 7-point Jacobi library -- TEST INFRASTRUCTURE ONLY.

Only the tests, the package smoke check and the benchmark's CPU-baseline leg
may import this package.  The library's own code path never does, and this
package imports nothing from the library.

The arithmetic lives in ``jacobi_oracle.c`` (plain C, FP64 unless stated,
built with -O2 -ffp-contract=off -fno-fast-math -fopenmp); this module only
compiles it and marshals numpy/torch CPU arrays.  ``poisson_dst`` solves the
discrete Poisson problem exactly with SciPy's DST-I (a library routine used
as an independent check of the residual and of refinement).

Every function and the passage it follows:
  jacobi(A, B, T)            Eq. (1) sweeps, grids A and B in turn (Sect. 1.1)
  jacobi_pipelined(...)      pipelined temporal blocking order (Sect. 2.1,
                             Fig. 1; distances of Eq. 3, Sect. 2.2)
  jacobi_multihalo(...)      multi-layer halo decomposition (Sect. 3.1)
  jacobi_compressed(A0, T)   compressed grid: one array, results shifted by
                             (-1,-1,-1) / (+1,+1,+1) on alternate sweeps with
                             the loops reversed (Sect. 2.1), sequential
  poisson_residual(u, f, h)  r = f - A_h u, 7-point Laplacian
  norm2(x)                   interior Euclidean norm
  poisson_jacobi(u, f, h, n) plain FP64 Jacobi for -Lap_h u = f
  refine(u, f, h, ...)       mixed-precision iterative refinement
  poisson_dst(f, h)          exact discrete solution (DST-I diagonalisation)
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "jacobi_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

CFLAGS = ["-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC", "-shared"]


def build(force: bool = False) -> str:
    """Compiles the oracle with gcc (idempotent)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.run(["gcc", *CFLAGS, "-o", tmp, _SRC, "-lm"], check=True)
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB)
            P, l, d = ctypes.c_void_p, ctypes.c_long, ctypes.c_double
            L.oracle_set_threads.argtypes = [ctypes.c_int]
            L.oracle_set_threads.restype = ctypes.c_int
            L.oracle_jacobi_f64.argtypes = [P, P, l, l, l, l]
            L.oracle_jacobi_f32.argtypes = [P, P, l, l, l, l]
            L.oracle_halo_copy_f64.argtypes = [P, P, l, l, l]
            L.oracle_jacobi_pipelined_f64.argtypes = [P, P, l, l, l, l, l, l, l, l, l, l, l, l]
            L.oracle_jacobi_multihalo_f64.argtypes = [P, P, l, l, l, P, l, l, l]
            L.oracle_jacobi_compressed_f64.argtypes = [P, l, l, l, l]
            L.oracle_jacobi_compressed_f32.argtypes = [P, l, l, l, l]
            L.oracle_poisson_residual.argtypes = [P, P, P, l, l, l, d]
            L.oracle_poisson_residual.restype = None
            L.oracle_norm2_interior.argtypes = [P, l, l, l]
            L.oracle_norm2_interior.restype = d
            L.oracle_poisson_jacobi_f64.argtypes = [P, P, P, l, l, l, d, l]
            L.oracle_poisson_jacobi_f64.restype = None
            L.oracle_refine.argtypes = [P, P, l, l, l, d, d, l, l,
                                        ctypes.POINTER(l), ctypes.POINTER(d)]
            _lib = L
    return _lib


def _np(a, dtype=np.float64) -> np.ndarray:
    """numpy view of a contiguous host array (numpy or torch CPU tensor)."""
    if hasattr(a, "numpy"):
        a = a.numpy()
    assert isinstance(a, np.ndarray) and a.dtype == dtype and a.flags.c_contiguous
    return a


def _dims(a):
    nz, ny, nx = (s - 2 for s in a.shape)
    return nx, ny, nz


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def jacobi(A, B, T: int) -> int:
    """In place on host arrays shaped (nz+2, ny+2, nx+2); float64 or float32.
    Returns 0 if the result is in A, 1 if in B."""
    a = A.numpy() if hasattr(A, "numpy") else A
    dt = a.dtype
    a, b = _np(A, dt), _np(B, dt)
    nx, ny, nz = _dims(a)
    f = lib().oracle_jacobi_f64 if dt == np.float64 else lib().oracle_jacobi_f32
    r = f(_ptr(a), _ptr(b), nx, ny, nz, int(T))
    if r < 0:
        raise ValueError("oracle_jacobi: bad arguments")
    return r


def jacobi_result(A0, T: int):
    """Convenience: returns a new array holding T sweeps applied to A0."""
    a = np.array(_np(A0, (A0.numpy() if hasattr(A0, "numpy") else A0).dtype), copy=True)
    b = np.empty_like(a)
    return a if jacobi(a, b, T) == 0 else b


def jacobi_pipelined(A, B, T, n_teams, t_team, T_upd, d_l, d_t, bx, by, bz) -> int:
    a, b = _np(A), _np(B)
    nx, ny, nz = _dims(a)
    r = lib().oracle_jacobi_pipelined_f64(_ptr(a), _ptr(b), nx, ny, nz, int(T), n_teams,
                                          t_team, T_upd, d_l, d_t, bx, by, bz)
    if r < 0:
        raise ValueError("oracle_jacobi_pipelined: bad arguments")
    return r


def jacobi_multihalo(A, B, depths, bx, by) -> int:
    a, b = _np(A), _np(B)
    nx, ny, nz = _dims(a)
    d = (ctypes.c_long * max(1, len(depths)))(*depths)
    r = lib().oracle_jacobi_multihalo_f64(_ptr(a), _ptr(b), nx, ny, nz, d, len(depths), bx, by)
    if r < 0:
        raise ValueError("oracle_jacobi_multihalo: bad arguments")
    return r


def jacobi_compressed(A0, T: int):
    """T sweeps of grid A0 (FP64 or FP32, halo included) in ONE array of
    (nx+3)(ny+3)(nz+3) cells by the sequential compressed grid (Sect. 2.1);
    returns the result grid (a copy taken out of that array)."""
    a = np.asarray(A0.numpy() if hasattr(A0, "numpy") else A0)
    dt = np.float32 if a.dtype == np.float32 else np.float64
    a = np.ascontiguousarray(a, dtype=dt)
    nz, ny, nx = (s - 2 for s in a.shape)
    E = np.zeros((nz + 3, ny + 3, nx + 3), dtype=dt)
    E[1:, 1:, 1:] = a
    f = lib().oracle_jacobi_compressed_f32 if dt == np.float32 else lib().oracle_jacobi_compressed_f64
    pos = f(E.ctypes.data, nx, ny, nz, int(T))
    if pos < 0:
        raise ValueError("bad arguments")
    return E[pos:pos + nz + 2, pos:pos + ny + 2, pos:pos + nx + 2].copy()


def poisson_residual(u, f, h: float) -> np.ndarray:
    u, f = _np(u), _np(f)
    r = np.empty_like(u)
    nx, ny, nz = _dims(u)
    lib().oracle_poisson_residual(_ptr(u), _ptr(f), _ptr(r), nx, ny, nz, float(h))
    return r


def norm2(x) -> float:
    x = _np(x)
    nx, ny, nz = _dims(x)
    return lib().oracle_norm2_interior(_ptr(x), nx, ny, nz)


def poisson_jacobi(u, f, h: float, sweeps: int):
    u, f = _np(u), _np(f)
    tmp = np.empty_like(u)
    nx, ny, nz = _dims(u)
    lib().oracle_poisson_jacobi_f64(_ptr(u), _ptr(tmp), _ptr(f), nx, ny, nz, float(h), int(sweeps))
    return u


def refine(u, f, h: float, tol: float, inner: int, max_outer: int):
    """In place on u.  Returns (status, outer_done, final_rel)."""
    u, f = _np(u), _np(f)
    nx, ny, nz = _dims(u)
    od, fr = ctypes.c_long(0), ctypes.c_double(0.0)
    st = lib().oracle_refine(_ptr(u), _ptr(f), nx, ny, nz, float(h), float(tol), int(inner),
                             int(max_outer), ctypes.byref(od), ctypes.byref(fr))
    if st < 0:
        raise MemoryError("oracle_refine")
    return st, od.value, fr.value


def poisson_dst(f, h: float) -> np.ndarray:
    """Exact solution of -Lap_h u = f with zero halo: the 7-point Laplacian is
    diagonal in the DST-I basis sin(pi p i/(n+1)); eigenvalue
    sum over axes of (2 - 2 cos(pi p/(n+1)))/h^2."""
    from scipy.fft import dstn, idstn

    f = _np(f)
    nz, ny, nx = (s - 2 for s in f.shape)
    fi = f[1:-1, 1:-1, 1:-1]
    fh = dstn(fi, type=1)
    lam = []
    for n in (nz, ny, nx):
        p = np.arange(1, n + 1, dtype=np.float64)
        lam.append((2.0 - 2.0 * np.cos(np.pi * p / (n + 1))) / (h * h))
    den = lam[0][:, None, None] + lam[1][None, :, None] + lam[2][None, None, :]
    u = np.zeros_like(f)
    u[1:-1, 1:-1, 1:-1] = idstn(fh / den, type=1)
    return u


def set_threads(n: int) -> int:
    """Sets the OpenMP threads of later oracle calls (results do not depend
    on it); returns the number in effect."""
    return int(lib().oracle_set_threads(int(n)))


def threads() -> int:
    """OpenMP threads the oracle will use (OMP_NUM_THREADS, else the cores
    this process may run on)."""
    v = os.environ.get("OMP_NUM_THREADS")
    if v and v.isdigit():
        return int(v)
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1
