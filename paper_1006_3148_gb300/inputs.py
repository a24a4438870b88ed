"""Seeded synthetic inputs for the Jacobi workloads.

This module is shared by the CUDA path's tests and benchmark and by the CPU
oracle's tests.  It holds no arithmetic of the method itself (no stencil,
no sweep, no residual): only random fields and the fixed initial/boundary
values of the workloads.  Every value is produced from integer arithmetic
(bit-identical on any device) except where a transcendental function is
named (Box-Muller normals, the sine mode), which are always evaluated on the
host in float64.

Random stream (counter-based SplitMix64, Steele/Lea/Flood 2014, the
finaliser published as ``splitmix64`` by S. Vigna): draw ``n`` (0-based) of
stream ``seed`` is ``mix(seed + (n + 1) * 0x9E3779B97F4A7C15 mod 2**64)``
with ``mix(z) = z3`` where ``z1 = (z ^ z>>30) * 0xBF58476D1CE4E5B9``,
``z2 = (z1 ^ z1>>27) * 0x94D049BB133111EB``, ``z3 = z2 ^ z2>>31``.  A uniform
double in [0, 1) is ``(draw >> 11) * 2**-53``.  Arrays are filled in memory
order of the dense layout ``idx = (k*(ny+2) + j)*(nx+2) + i`` (x fastest),
over the whole array including the halo.

Workload recipes (sizes and value distributions follow the five workloads of
the library; the paper itself runs a 600^3 grid of unstated values, Sect. 2.4):

* ``uniform_grid``: interior and halo i.i.d. U[0,1) (64^3 parity case, the
  batched grids).
* ``dirichlet_z0_grid``: interior U[0,1), halo 0 except the whole k=0 plane,
  which is 1 (the 512^3 FP64 workload).
* ``mode_grid``: interior U[0,1) plus one discrete sine mode of amplitude 1,
  halo 0 (the 1024^3 FP32 workload).
* ``batch_dims``: per-grid interior sizes drawn uniformly from 32..192 per
  axis, and a seeded shuffle that marks half of the grids FP32.
* ``normal_rhs``: i.i.d. N(0,1) right-hand side (Box-Muller on consecutive
  pairs of uniforms), zero halo (the 96^3 Poisson workload).
"""
from __future__ import annotations

import math

import numpy as np
import torch

GAMMA = 0x9E3779B97F4A7C15
_M1 = 0xBF58476D1CE4E5B9
_M2 = 0x94D049BB133111EB
_CHUNK = 1 << 24


def _s64(v: int) -> int:
    """Reinterpret an unsigned 64-bit constant as a signed int64."""
    v &= (1 << 64) - 1
    return v - (1 << 64) if v >= (1 << 63) else v


def _srl(x: torch.Tensor, k: int) -> torch.Tensor:
    """Logical right shift of int64 bit patterns."""
    return (x >> k) & ((1 << (64 - k)) - 1)


def splitmix64(seed: int, start: int, count: int, device="cpu") -> torch.Tensor:
    """Draws ``start .. start+count-1`` of stream ``seed`` as int64 bit patterns."""
    n = torch.arange(start + 1, start + count + 1, dtype=torch.int64, device=device)
    z = n * _s64(GAMMA) + _s64(seed)
    z = (z ^ _srl(z, 30)) * _s64(_M1)
    z = (z ^ _srl(z, 27)) * _s64(_M2)
    return z ^ _srl(z, 31)


def uniform(seed: int, start: int, count: int, device="cpu") -> torch.Tensor:
    """U[0,1) doubles: top 53 bits of each draw times 2**-53 (exact)."""
    return _srl(splitmix64(seed, start, count, device), 11).to(torch.float64) * (2.0 ** -53)


def uniform_fill(out: torch.Tensor, seed: int) -> torch.Tensor:
    """Fills a float64/float32 tensor (any shape, contiguous) in memory order."""
    flat = out.view(-1)
    for s in range(0, flat.numel(), _CHUNK):
        c = min(_CHUNK, flat.numel() - s)
        flat[s:s + c] = uniform(seed, s, c, out.device).to(out.dtype)
    return out


def normal(seed: int, count: int) -> np.ndarray:
    """N(0,1) doubles by Box-Muller on draws (2m, 2m+1), host float64."""
    m = (count + 1) // 2
    u = uniform(seed, 0, 2 * m).numpy()
    u1, u2 = u[0::2], u[1::2]
    rad = np.sqrt(-2.0 * np.log1p(-u1))
    out = np.empty(2 * m)
    out[0::2] = rad * np.cos(2.0 * math.pi * u2)
    out[1::2] = rad * np.sin(2.0 * math.pi * u2)
    return out[:count]


def grid_shape(nx: int, ny: int, nz: int) -> tuple:
    """Array shape (z, y, x) of an nx*ny*nz interior with a one-cell halo."""
    return (nz + 2, ny + 2, nx + 2)


def uniform_grid(nx, ny, nz, seed, dtype=torch.float64, device="cpu") -> torch.Tensor:
    """Interior and halo i.i.d. U[0,1)."""
    a = torch.empty(grid_shape(nx, ny, nz), dtype=dtype, device=device)
    return uniform_fill(a, seed)


def zero_halo(a: torch.Tensor) -> torch.Tensor:
    a[0].zero_()
    a[-1].zero_()
    a[:, 0].zero_()
    a[:, -1].zero_()
    a[:, :, 0].zero_()
    a[:, :, -1].zero_()
    return a


def dirichlet_z0_grid(nx, ny, nz, seed, dtype=torch.float64, device="cpu") -> torch.Tensor:
    """Interior U[0,1); halo 0 on five faces and 1 on the whole k=0 plane."""
    a = uniform_grid(nx, ny, nz, seed, dtype, device)
    zero_halo(a)
    a[0].fill_(1.0)
    return a


def sine_mode_1d(n: int, p: int) -> torch.Tensor:
    """sin(pi*p*i/(n+1)) for i = 0..n+1 (host float64), exact 0 at both ends."""
    i = np.arange(n + 2, dtype=np.float64)
    v = np.sin(math.pi * p * i / (n + 1))
    v[0] = 0.0
    v[-1] = 0.0
    return torch.from_numpy(v)


def mode_grid(nx, ny, nz, seed, pqr=(16, 16, 16), amp=1.0, dtype=torch.float32,
              device="cpu") -> torch.Tensor:
    """Interior U[0,1) plus amp*phi, phi = sx[i]*sy[j]*sz[k] (float64, left to
    right), halo 0; the sum is formed in float64 and rounded once to ``dtype``."""
    sx = sine_mode_1d(nx, pqr[0]).to(device)
    sy = sine_mode_1d(ny, pqr[1]).to(device)
    sz = sine_mode_1d(nz, pqr[2]).to(device)
    out = torch.empty(grid_shape(nx, ny, nz), dtype=dtype, device=device)
    plane = (ny + 2) * (nx + 2)
    sxy = sy[:, None] * sx[None, :]
    for k in range(nz + 2):
        u = uniform(seed, k * plane, plane, device).view(ny + 2, nx + 2)
        out[k] = (u + (sxy * sz[k]) * amp).to(dtype)
    return zero_halo(out)


def mode_only_grid(nx, ny, nz, pqr, dtype=torch.float64) -> torch.Tensor:
    """The pure sine mode phi on the full array (zero halo)."""
    sx = sine_mode_1d(nx, pqr[0])
    sy = sine_mode_1d(ny, pqr[1])
    sz = sine_mode_1d(nz, pqr[2])
    return ((sy[:, None] * sx[None, :])[None, :, :] * sz[:, None, None]).to(dtype).contiguous()


def batch_dims(n_grids: int, seed: int, lo: int = 32, hi: int = 192):
    """Per-grid interior sizes (nx, ny, nz) uniform over lo..hi, and dtype flags.

    Size draw g*3+a of stream ``seed`` gives axis a of grid g:
    ``lo + floor(u * (hi - lo + 1))``.  Dtypes: the first half of a seeded
    Fisher-Yates permutation (stream ``seed + 1``) is FP64, the rest FP32.
    Returns (dims list, is_f32 list)."""
    u = uniform(seed, 0, 3 * n_grids).numpy()
    span = hi - lo + 1
    d = [lo + int(math.floor(x * span)) for x in u]
    dims = [(d[3 * g], d[3 * g + 1], d[3 * g + 2]) for g in range(n_grids)]
    perm = list(range(n_grids))
    v = uniform(seed + 1, 0, n_grids).numpy()
    for i in range(n_grids - 1, 0, -1):
        j = int(math.floor(v[i] * (i + 1)))
        perm[i], perm[j] = perm[j], perm[i]
    is_f32 = [False] * n_grids
    for g in perm[n_grids // 2:]:
        is_f32[g] = True
    return dims, is_f32


def normal_rhs(nx, ny, nz, seed) -> torch.Tensor:
    """Interior i.i.d. N(0,1) in memory order of the interior, zero halo (float64)."""
    f = torch.zeros(grid_shape(nx, ny, nz), dtype=torch.float64)
    f[1:-1, 1:-1, 1:-1] = torch.from_numpy(normal(seed, nx * ny * nz)).view(nz, ny, nx)
    return f
