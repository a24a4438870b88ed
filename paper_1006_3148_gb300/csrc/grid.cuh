// Index helpers for a grid of interior nx*ny*nz cells stored densely with
// its one-cell halo, x fastest: cell (i, j, k), 0 <= i <= nx+1 etc., sits
// at (k*(ny+2) + j)*(nx+2) + i.
#pragma once

namespace jac {

// Number of halo cells read by the 7-point stencil or kept by the boundary
// copy: the k = 0 and k = nz+1 planes, the j = 0 and j = ny+1 rows of the
// interior planes, and the i = 0 and i = nx+1 cells of the interior rows.
__host__ __device__ __forceinline__ long long halo_count(int nx, int ny, int nz)
{
    const long long NXP = nx + 2, NYP = ny + 2;
    return 2 * NXP * NYP + 2 * NXP * (long long)nz + 2 * (long long)ny * nz;
}

// Linear index of halo cell t (0 <= t < halo_count) in the order above.
__device__ __forceinline__ long long halo_cell(long long t, int nx, int ny, int nz)
{
    const long long NXP = nx + 2, NYP = ny + 2;
    const long long nzf = 2 * NXP * NYP, nyf = 2 * NXP * (long long)nz;
    long long i, j, k;
    if (t < nzf) {
        const long long p = t % (NXP * NYP);
        k = (t < NXP * NYP) ? 0 : nz + 1;
        j = p / NXP;
        i = p % NXP;
    } else if (t < nzf + nyf) {
        const long long u = t - nzf, half = NXP * nz;
        j = (u < half) ? 0 : ny + 1;
        const long long p = u % half;
        k = 1 + p / NXP;
        i = p % NXP;
    } else {
        const long long u = t - nzf - nyf, half = (long long)ny * nz;
        i = (u < half) ? 0 : nx + 1;
        const long long p = u % half;
        k = 1 + p / ny;
        j = 1 + p % ny;
    }
    return (k * NYP + j) * NXP + i;
}

}  // namespace jac
