// Bounds-checked build.  Compiled with -DJACOBI_CHECKED (build tag
// "checked": libjacobi_checked.so), every global, shared and distributed
// shared memory access of the sweep kernels is first checked against the
// extent of the buffer it belongs to; an access outside records
// JACOBI_ERR_BOUNDS in the launch's status word (first error wins) and is
// skipped.  Nothing traps.  In the normal build the checks are compile-time
// true and cost nothing.  A test hook (jacobi_debug_set_fault mode 2)
// declares every grid `shrink` elements shorter than it is, so that the
// checker's own reporting can be tested on accesses that are in fact valid.
#pragma once

#include "jacobi.h"

namespace jac {

#ifdef JACOBI_CHECKED
constexpr bool kChecked = true;
#else
constexpr bool kChecked = false;
#endif

// [off, off + n) inside [0, size)?  Records JACOBI_ERR_BOUNDS if not.
__device__ __forceinline__ bool in_bounds(long long off, long long n, long long size, int *status)
{
    if (!kChecked) return true;
    if (off >= 0 && n >= 0 && off + n <= size) return true;
    if (status) atomicCAS(status, 0, JACOBI_ERR_BOUNDS);
    return false;
}

// Number of elements of a grid of interior nx*ny*nz, as the checks see it.
__host__ __device__ __forceinline__ long long checked_grid_elems(int nx, int ny, int nz, long long shrink)
{
    return (long long)(nx + 2) * (ny + 2) * (long long)(nz + 2) - shrink;
}

}  // namespace jac
