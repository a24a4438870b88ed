"""Python binding of libjacobi.so: the C ABI's entry points under the same
names, taking torch tensors (device memory) and torch streams.

Argument marshalling only -- every step of a sweep runs in the library's
CUDA kernels.  There is no fallback: if libjacobi.so is missing or cannot be
loaded, every call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

import torch

from . import build as _build

F64 = 0
F32 = 1
KERNEL_AUTO, KERNEL_PLAIN, KERNEL_TB, KERNEL_PLAIN_X2, KERNEL_TB_CTA, KERNEL_TB_REG, KERNEL_TB_CHAIN = 0, 1, 2, 3, 4, 5, 6
BATCH_PERSISTENT, BATCH_SWEEPS = 0, 1

STATUS = {
    0: "JACOBI_OK", -1: "JACOBI_ERR_ARG", -2: "JACOBI_ERR_DTYPE", -3: "JACOBI_ERR_ALLOC",
    -4: "JACOBI_ERR_CUDA", -5: "JACOBI_ERR_TIMEOUT", -6: "JACOBI_ERR_BOUNDS",
    -7: "JACOBI_ERR_NOT_CONVERGED", -8: "JACOBI_ERR_ALIGN", -9: "JACOBI_ERR_UNSUPPORTED",
}

_lock = threading.Lock()
_lib = None


class JacobiError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        msg = "%s failed: %s (%d)" % (what, STATUS.get(code, "?"), code)
        if code == -4 and _lib is not None:
            msg += ": " + _lib.jacobi_last_cuda_error().decode()
        super().__init__(msg)


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Loads libjacobi.so (building it first if allowed and needed)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if build_if_missing and not _build.up_to_date():
            _build.build()
        if not os.path.exists(_build.LIB):
            raise RuntimeError("libjacobi.so not built (%s); run __graft_entry__.build()" % _build.LIB)
        L = ctypes.CDLL(_build.LIB)
        P, i, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
        pi = ctypes.POINTER(ctypes.c_int)
        sig = {
            "jacobi_status_string": ([i], ctypes.c_char_p),
            "jacobi_version": ([], i),
            "jacobi_last_cuda_error": ([], ctypes.c_char_p),
            "jacobi_create": ([ctypes.POINTER(P), i, i, i, i], i),
            "jacobi_destroy": ([P], i),
            "jacobi_sweep": ([P, P, P, i, P], i),
            "jacobi_sweep_host": ([P, P, P, i, P], i),
            "jacobi_set_plan": ([P, i, i, i, i, i, i, i], i),
            "jacobi_get_plan": ([P, pi, pi, pi, pi, pi, pi, pi], i),
            "jacobi_tune": ([P, P, P, P, ctypes.POINTER(d)], i),
            "jacobi_tune_candidates": ([P, pi, i], i),
            "jacobi_get_status": ([P, pi], i),
            "jacobi_debug_set_fault": ([P, i, i], i),
            "jacobi_build_checked": ([], i),
            "jacobi_plan_passes": ([i, i, pi, i], i),
            "jacobi_profile_enable": ([P, i], i),
            "jacobi_poisson_residual": ([P, P, P, d, P, ctypes.POINTER(d)], i),
            "jacobi_poisson_jacobi": ([P, P, P, P, d, i, P], i),
            "jacobi_poisson_residual_noalloc": ([P, P, i, i, i, d, P, ctypes.POINTER(d)], i),
            "jacobi_refine": ([P, P, P, d, d, i, i, P, pi, ctypes.POINTER(d)], i),
            "jacobi_batch_create": ([ctypes.POINTER(P), i, pi, pi, pi, pi, pi], i),
            "jacobi_batch_run": ([P, ctypes.POINTER(P), ctypes.POINTER(P), P], i),
            "jacobi_batch_destroy": ([P], i),
            "jacobi_batch_set_tile": ([P, i, i, i], i),
            "jacobi_batch_set_engine": ([P, i, i], i),
            "jacobi_batch_get_engine": ([P, pi, pi], i),
            "jacobi_compressed_set_plan": ([P, i, i, i], i),
            "jacobi_compressed_get_plan": ([P, pi, pi, pi, ctypes.POINTER(ctypes.c_longlong)], i),
            "jacobi_sweep_compressed": ([P, P, i, i, pi, P], i),
            "jacobi_batch_set_fp32_depth": ([P, i], i),
            "jacobi_batch_get_fp32_depth": ([P, pi], i),
            "jacobi_batch_run_rhs": ([P, ctypes.POINTER(P), ctypes.POINTER(P), ctypes.POINTER(P), P], i),
            "jacobi_batch_tune": ([P, ctypes.POINTER(P), ctypes.POINTER(P), P, ctypes.POINTER(d)], i),
            "jacobi_batch_get_info": ([P, pi, pi, pi, ctypes.POINTER(ctypes.c_longlong), pi], i),
            "jacobi_batch_get_status": ([P, pi], i),
            "jacobi_batch_debug_set_fault": ([P, i, i], i),
            "jacobi_check_addition": ([ctypes.c_ulonglong, ctypes.c_ulonglong, ctypes.POINTER(ctypes.c_ulonglong),
                                       ctypes.POINTER(ctypes.c_ulonglong)], i),
            "jacobi_check_division": ([ctypes.c_ulonglong, ctypes.c_ulonglong, ctypes.POINTER(ctypes.c_ulonglong),
                                       ctypes.POINTER(ctypes.c_ulonglong)], i),
            "jacobi_profile_read": ([P, ctypes.POINTER(d), pi, pi], i),
        }
        for name, (args, res) in sig.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = res
        _lib = L
        return L


def _check(code: int, what: str):
    if code != 0:
        raise JacobiError(code, what)


def _stream(stream) -> ctypes.c_void_p:
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def _dtype_code(dtype) -> int:
    if dtype in (torch.float64, F64, "f64", "float64"):
        return F64
    if dtype in (torch.float32, F32, "f32", "float32"):
        return F32
    raise ValueError("dtype must be float64 or float32")


def _grid_ptr(t: torch.Tensor, shape, dtype) -> ctypes.c_void_p:
    if not t.is_cuda or not t.is_contiguous() or t.dtype != dtype or tuple(t.shape) != tuple(shape):
        raise ValueError("grid must be a contiguous CUDA %s tensor of shape %s" % (dtype, shape))
    return ctypes.c_void_p(t.data_ptr())


class Handle:
    """Owns a jacobi_h.  Grids are tensors shaped (nz+2, ny+2, nx+2)."""

    def __init__(self, nx: int, ny: int, nz: int, dtype=torch.float64):
        L = load()
        self.nx, self.ny, self.nz = int(nx), int(ny), int(nz)
        self.dtype = torch.float64 if _dtype_code(dtype) == F64 else torch.float32
        self.shape = (self.nz + 2, self.ny + 2, self.nx + 2)
        h = ctypes.c_void_p()
        _check(L.jacobi_create(ctypes.byref(h), self.nx, self.ny, self.nz, _dtype_code(dtype)), "jacobi_create")
        self._h = h

    @property
    def ptr(self):
        return self._h

    def close(self):
        if self._h:
            load().jacobi_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def jacobi_create(nx, ny, nz, dtype=torch.float64) -> Handle:
    return Handle(nx, ny, nz, dtype)


def jacobi_destroy(h: Handle):
    h.close()


def jacobi_sweep(h: Handle, A: torch.Tensor, B: torch.Tensor, T: int, stream=None) -> torch.Tensor:
    """T sweeps of Eq. (1), A and B in turn; returns the grid holding the
    result (B if T is odd, A if even)."""
    pa = _grid_ptr(A, h.shape, h.dtype)
    pb = _grid_ptr(B, h.shape, h.dtype)
    _check(load().jacobi_sweep(h.ptr, pa, pb, int(T), _stream(stream)), "jacobi_sweep")
    return B if T % 2 == 1 else A


def jacobi_sweep_host(h: Handle, A_host: torch.Tensor, out_host: torch.Tensor, T: int, stream=None):
    for t in (A_host, out_host):
        if t.is_cuda or not t.is_contiguous() or t.dtype != h.dtype or tuple(t.shape) != h.shape:
            raise ValueError("host grids must be contiguous CPU tensors of shape %s" % (h.shape,))
    _check(load().jacobi_sweep_host(h.ptr, ctypes.c_void_p(A_host.data_ptr()),
                                    ctypes.c_void_p(out_host.data_ptr()), int(T), _stream(stream)),
           "jacobi_sweep_host")
    return out_host


def jacobi_set_plan(h: Handle, kernel: int, depth: int = 1, bx: int = 0, by: int = 0, bz: int = 0,
                    ring: int = 0, threads: int = 0):
    _check(load().jacobi_set_plan(h.ptr, int(kernel), int(depth), int(bx), int(by), int(bz), int(ring),
                                  int(threads)), "jacobi_set_plan")


def jacobi_get_plan(h: Handle) -> dict:
    v = [ctypes.c_int() for _ in range(7)]
    _check(load().jacobi_get_plan(h.ptr, *[ctypes.byref(x) for x in v]), "jacobi_get_plan")
    return dict(zip(("kernel", "depth", "bx", "by", "bz", "ring", "threads"), (x.value for x in v)))


def jacobi_tune(h: Handle, scratchA: torch.Tensor, scratchB: torch.Tensor, stream=None) -> float:
    g = ctypes.c_double()
    _check(load().jacobi_tune(h.ptr, _grid_ptr(scratchA, h.shape, h.dtype), _grid_ptr(scratchB, h.shape, h.dtype),
                              _stream(stream), ctypes.byref(g)), "jacobi_tune")
    return g.value


def jacobi_tune_candidates(h: Handle) -> list:
    """The tuner's first-stage candidate plans that this device can launch,
    as tuples (kernel, depth, bx, by, bz, ring, threads)."""
    L = load()
    n = L.jacobi_tune_candidates(h.ptr, None, 0)
    if n < 0:
        raise JacobiError(n, "jacobi_tune_candidates")
    buf = (ctypes.c_int * (7 * max(n, 1)))()
    m = L.jacobi_tune_candidates(h.ptr, buf, n)
    if m < 0:
        raise JacobiError(m, "jacobi_tune_candidates")
    return [tuple(buf[7 * k:7 * k + 7]) for k in range(min(n, m))]


def jacobi_get_status(h: Handle) -> int:
    v = ctypes.c_int()
    _check(load().jacobi_get_status(h.ptr, ctypes.byref(v)), "jacobi_get_status")
    return v.value


def jacobi_debug_set_fault(h: Handle, mode: int, limit_ms: int = 2000):
    _check(load().jacobi_debug_set_fault(h.ptr, int(mode), int(limit_ms)), "jacobi_debug_set_fault")


def jacobi_status_string(code: int) -> str:
    return load().jacobi_status_string(int(code)).decode()


def jacobi_plan_passes(T: int, depth: int) -> list:
    buf = (ctypes.c_int * (max(T, 1) + 1))()
    n = load().jacobi_plan_passes(int(T), int(depth), buf, max(T, 1) + 1)
    if n < 0:
        raise JacobiError(-1, "jacobi_plan_passes")
    return list(buf[:n])


def jacobi_profile_enable(h: Handle, enable: bool = True):
    _check(load().jacobi_profile_enable(h.ptr, 1 if enable else 0), "jacobi_profile_enable")


def jacobi_profile_read(h: Handle) -> dict:
    ms, npass, nother = ctypes.c_double(), ctypes.c_int(), ctypes.c_int()
    _check(load().jacobi_profile_read(h.ptr, ctypes.byref(ms), ctypes.byref(npass), ctypes.byref(nother)),
           "jacobi_profile_read")
    return {"pass_ms": ms.value, "pass_launches": npass.value, "other_launches": nother.value}


def jacobi_check_division(count: int, seed: int = 1) -> tuple:
    """(mismatches, first failing input bits) of the exact FP64 division."""
    m, f = ctypes.c_ulonglong(), ctypes.c_ulonglong()
    _check(load().jacobi_check_division(int(count), int(seed), ctypes.byref(m), ctypes.byref(f)),
           "jacobi_check_division")
    return m.value, f.value


class Batch:
    """Owns a jacobi_batch_h for grids of the given sizes, dtypes and sweeps."""

    def __init__(self, dims, dtypes, Ts):
        L = load()
        n = len(dims)
        arr = lambda xs: (ctypes.c_int * n)(*xs)
        self.n = n
        self.dims = [tuple(int(v) for v in d) for d in dims]
        self.dtypes = [torch.float64 if _dtype_code(t) == F64 else torch.float32 for t in dtypes]
        self.Ts = [int(t) for t in Ts]
        h = ctypes.c_void_p()
        _check(L.jacobi_batch_create(ctypes.byref(h), n, arr([d[0] for d in self.dims]),
                                     arr([d[1] for d in self.dims]), arr([d[2] for d in self.dims]),
                                     arr([_dtype_code(t) for t in self.dtypes]), arr(self.Ts)),
               "jacobi_batch_create")
        self._h = h

    @property
    def ptr(self):
        return self._h

    def shape(self, g):
        nx, ny, nz = self.dims[g]
        return (nz + 2, ny + 2, nx + 2)

    def _ptrs(self, grids):
        if len(grids) != self.n:
            raise ValueError("need %d grids" % self.n)
        return (ctypes.c_void_p * self.n)(*[_grid_ptr(t, self.shape(g), self.dtypes[g]).value
                                            for g, t in enumerate(grids)])

    def close(self):
        if self._h:
            load().jacobi_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def jacobi_batch_create(dims, dtypes, Ts) -> Batch:
    return Batch(dims, dtypes, Ts)


def jacobi_batch_run(b: Batch, A, B, stream=None):
    """Runs all sweeps; returns the list of result grids (B_g if T_g odd)."""
    pa, pb = b._ptrs(A), b._ptrs(B)
    _check(load().jacobi_batch_run(b.ptr, pa, pb, _stream(stream)), "jacobi_batch_run")
    return [B[g] if b.Ts[g] % 2 == 1 else A[g] for g in range(b.n)]


def jacobi_batch_destroy(b: Batch):
    b.close()


def jacobi_batch_set_tile(b: Batch, bx: int, by: int, bz: int = 0):
    _check(load().jacobi_batch_set_tile(b.ptr, int(bx), int(by), int(bz)), "jacobi_batch_set_tile")


def jacobi_batch_set_engine(b: Batch, engine: int, kz: int = 0):
    _check(load().jacobi_batch_set_engine(b.ptr, int(engine), int(kz)), "jacobi_batch_set_engine")


def jacobi_batch_get_engine(b: Batch) -> dict:
    e, kz = ctypes.c_int(), ctypes.c_int()
    _check(load().jacobi_batch_get_engine(b.ptr, ctypes.byref(e), ctypes.byref(kz)), "jacobi_batch_get_engine")
    return {"engine": e.value, "kz": kz.value}


def jacobi_compressed_set_plan(h: Handle, depth: int = 0, bz: int = 0, waves: int = 0):
    """Compressed-grid plan; a zero field takes the dtype's default."""
    _check(load().jacobi_compressed_set_plan(h.ptr, int(depth), int(bz), int(waves)), "jacobi_compressed_set_plan")


def jacobi_compressed_get_plan(h: Handle) -> dict:
    d, bz, w, S = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_longlong()
    _check(load().jacobi_compressed_get_plan(h.ptr, ctypes.byref(d), ctypes.byref(bz), ctypes.byref(w),
                                             ctypes.byref(S)), "jacobi_compressed_get_plan")
    return {"depth": d.value, "bz": bz.value, "waves": w.value, "shift_planes": S.value}


def compressed_buffer(h: Handle, device="cuda") -> torch.Tensor:
    """An uninitialised buffer for jacobi_sweep_compressed: nz + 2 + S planes."""
    S = jacobi_compressed_get_plan(h)["shift_planes"]
    return torch.empty((h.nz + 2 + S, h.ny + 2, h.nx + 2), dtype=h.dtype, device=device)


def compressed_view(h: Handle, U: torch.Tensor, upper: int) -> torch.Tensor:
    """The grid inside U in position `upper` (1: planes S .. S+nz+1, 0: 0 .. nz+1)."""
    S = jacobi_compressed_get_plan(h)["shift_planes"]
    o = S if upper else 0
    return U[o:o + h.nz + 2]


def jacobi_sweep_compressed(h: Handle, U: torch.Tensor, T: int, upper: int = 1, stream=None) -> int:
    """T sweeps in the single buffer U (see compressed_buffer); returns the
    position of the result (1: upper, 0: lower)."""
    S = jacobi_compressed_get_plan(h)["shift_planes"]
    need = (h.nz + 2 + S) * (h.ny + 2) * (h.nx + 2)
    if not U.is_cuda or not U.is_contiguous() or U.numel() < need or U.dtype != h.dtype:
        raise ValueError("U: contiguous CUDA tensor of %d elements of the handle's dtype" % need)
    out = ctypes.c_int()
    _check(load().jacobi_sweep_compressed(h.ptr, ctypes.c_void_p(U.data_ptr()), int(T), int(upper),
                                          ctypes.byref(out), _stream(stream)), "jacobi_sweep_compressed")
    return out.value


def jacobi_batch_set_fp32_depth(b: Batch, depth: int):
    """FP32 grids in temporally blocked passes of depth <= depth (1: the engine)."""
    _check(load().jacobi_batch_set_fp32_depth(b.ptr, int(depth)), "jacobi_batch_set_fp32_depth")


def jacobi_batch_get_fp32_depth(b: Batch) -> int:
    d = ctypes.c_int()
    _check(load().jacobi_batch_get_fp32_depth(b.ptr, ctypes.byref(d)), "jacobi_batch_get_fp32_depth")
    return d.value


def jacobi_batch_run_rhs(b: Batch, A, B, RHS, stream=None):
    """Poisson form: grid g uses the source term RHS[g] (= h^2 f, or None)."""
    pa, pb = b._ptrs(A), b._ptrs(B)
    pr = (ctypes.c_void_p * b.n)(*[None if r is None else _grid_ptr(r, b.shape(g), b.dtypes[g]).value
                                   for g, r in enumerate(RHS)])
    _check(load().jacobi_batch_run_rhs(b.ptr, pa, pb, pr, _stream(stream)), "jacobi_batch_run_rhs")
    return [B[g] if b.Ts[g] % 2 == 1 else A[g] for g in range(b.n)]


def jacobi_batch_tune(b: Batch, scratchA, scratchB, stream=None) -> float:
    g = ctypes.c_double()
    _check(load().jacobi_batch_tune(b.ptr, b._ptrs(scratchA), b._ptrs(scratchB), _stream(stream),
                                    ctypes.byref(g)), "jacobi_batch_tune")
    return g.value


def jacobi_batch_get_info(b: Batch) -> dict:
    bx, by, bz, blocks, items = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_longlong()
    _check(load().jacobi_batch_get_info(b.ptr, ctypes.byref(bx), ctypes.byref(by), ctypes.byref(bz),
                                        ctypes.byref(items), ctypes.byref(blocks)), "jacobi_batch_get_info")
    return {"bx": bx.value, "by": by.value, "bz": bz.value, "items": items.value, "blocks": blocks.value}


def jacobi_batch_get_status(b: Batch) -> int:
    v = ctypes.c_int()
    _check(load().jacobi_batch_get_status(b.ptr, ctypes.byref(v)), "jacobi_batch_get_status")
    return v.value


def jacobi_batch_debug_set_fault(b: Batch, mode: int, limit_ms: int = 2000):
    _check(load().jacobi_batch_debug_set_fault(b.ptr, int(mode), int(limit_ms)), "jacobi_batch_debug_set_fault")


def jacobi_poisson_residual(h: Handle, u: torch.Tensor, f: torch.Tensor, hgrid: float, stream=None) -> float:
    rel = ctypes.c_double()
    _check(load().jacobi_poisson_residual(h.ptr, _grid_ptr(u, h.shape, h.dtype), _grid_ptr(f, h.shape, h.dtype),
                                          float(hgrid), _stream(stream), ctypes.byref(rel)), "jacobi_poisson_residual")
    return rel.value


def jacobi_poisson_jacobi(h: Handle, u: torch.Tensor, tmp: torch.Tensor, f: torch.Tensor, hgrid: float,
                          sweeps: int, stream=None) -> torch.Tensor:
    _check(load().jacobi_poisson_jacobi(h.ptr, _grid_ptr(u, h.shape, h.dtype), _grid_ptr(tmp, h.shape, h.dtype),
                                        _grid_ptr(f, h.shape, h.dtype), float(hgrid), int(sweeps), _stream(stream)),
           "jacobi_poisson_jacobi")
    return tmp if sweeps % 2 == 1 else u


def jacobi_refine(h: Handle, u: torch.Tensor, f: torch.Tensor, hgrid: float, rel_tol: float, inner_sweeps: int,
                  max_outer: int, stream=None):
    """Returns (status, outer_done, final_rel); status 0 or -7 (not converged)."""
    od, fr = ctypes.c_int(), ctypes.c_double()
    st = load().jacobi_refine(h.ptr, _grid_ptr(u, h.shape, h.dtype), _grid_ptr(f, h.shape, h.dtype), float(hgrid),
                              float(rel_tol), int(inner_sweeps), int(max_outer), _stream(stream), ctypes.byref(od),
                              ctypes.byref(fr))
    if st not in (0, -7):
        raise JacobiError(st, "jacobi_refine")
    return st, od.value, fr.value


def jacobi_poisson_residual_noalloc(u: torch.Tensor, f: torch.Tensor, hgrid: float, stream=None) -> float:
    """Relative residual without any device allocation (library-internal
    fixed scratch; nz <= JACOBI_NOALLOC_MAX_NZ; calls must not overlap)."""
    nz, ny, nx = (s - 2 for s in u.shape)
    shape = tuple(u.shape)
    rel = ctypes.c_double()
    _check(load().jacobi_poisson_residual_noalloc(_grid_ptr(u, shape, torch.float64),
                                                  _grid_ptr(f, shape, torch.float64), nx, ny, nz, float(hgrid),
                                                  _stream(stream), ctypes.byref(rel)),
           "jacobi_poisson_residual_noalloc")
    return rel.value


def jacobi_check_addition(count: int, seed: int = 1) -> tuple:
    """(mismatches, failing pair) of the integer-pipe FP64 addition."""
    m = ctypes.c_ulonglong()
    f = (ctypes.c_ulonglong * 2)()
    _check(load().jacobi_check_addition(int(count), int(seed), ctypes.byref(m), f), "jacobi_check_addition")
    return m.value, (f[0], f[1])
