/*
 * CPU oracle for the 3D 7-point Jacobi library.  TEST INFRASTRUCTURE ONLY:
 * it is called by the tests, by the package's smoke check and by the
 * benchmark's CPU-baseline leg, never by the library itself.  It shares no
 * code, header or constant with the CUDA path.
 *
 * Plain, slow, obviously correct loops.  Build flags: -O2 -ffp-contract=off
 * -fno-fast-math (no FMA contraction, no reassociation), OpenMP over z-planes
 * only (every cell is computed by exactly one thread with the same operation
 * order, so results do not depend on the thread count).
 *
 * Grid layout (all functions): interior nx*ny*nz with a one-cell halo, dense,
 * x fastest: idx(i,j,k) = (k*(ny+2) + j)*(nx+2) + i, 0 <= i <= nx+1.
 * Halo cells are Dirichlet values: read, never written (Sect. 1.1: Jacobi
 * solves boundary value problems; the halo is the boundary).
 *
 * Functions and the passages they follow:
 *   oracle_jacobi_f64        Eq. (1) + alternating grids A/B (Sect. 1.1)
 *   oracle_jacobi_f32        same, single precision, multiply by RN(1/6)
 *                            (the "one multiplication and five additions"
 *                            count of Sect. 2.3)
 *   oracle_jacobi_pipelined  pipelined temporal blocking, Sect. 2.1 / Fig. 1:
 *                            threads in a team, T updates per thread per
 *                            block, blocks shifted by one cell per update,
 *                            minimum thread distance d_l >= 1 block, team
 *                            delay d_t (Sect. 2.2)
 *   oracle_jacobi_multihalo  multi-layer halo decomposition, Sect. 3.1: each
 *                            x/y subdomain performs h updates on a private
 *                            copy; update s covers a region h-s layers larger
 *   oracle_poisson_*         -Lap_h u = f with the 7-point Laplacian (the
 *                            Poisson operator whose Jacobi smoother is Eq. 1)
 *   oracle_refine            mixed-precision iterative refinement around the
 *                            FP32 Jacobi smoother (workload definition, not
 *                            in the paper)
 * Parity pins for every function live in tests/test_oracle_*.py.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define IDX(i, j, k) ((((size_t)(k)) * (size_t)(ny + 2) + (size_t)(j)) * (size_t)(nx + 2) + (size_t)(i))

/* Number of OpenMP threads of the following calls (n >= 1); results do
 * not depend on it.  Returns the number in effect. */
int oracle_set_threads(int n)
{
#ifdef _OPENMP
    if (n >= 1) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

/* ---------------------------------------------------------------- Eq. (1) */

/* One sweep dst <- J(src) on the interior.  Term order exactly as printed in
 * Eq. (1): i-1, i+1, j-1, j+1, k-1, k+1, summed left to right, then divided
 * by 6 (true IEEE division). */
static void sweep_f64(const double *src, double *dst, long nx, long ny, long nz)
{
    long k;
#pragma omp parallel for schedule(static)
    for (k = 1; k <= nz; ++k)
        for (long j = 1; j <= ny; ++j)
            for (long i = 1; i <= nx; ++i) {
                double s = src[IDX(i - 1, j, k)];
                s = s + src[IDX(i + 1, j, k)];
                s = s + src[IDX(i, j - 1, k)];
                s = s + src[IDX(i, j + 1, k)];
                s = s + src[IDX(i, j, k - 1)];
                s = s + src[IDX(i, j, k + 1)];
                dst[IDX(i, j, k)] = s / 6.0;
            }
}

static void sweep_f32(const float *src, float *dst, long nx, long ny, long nz)
{
    const float sixth = 1.0f / 6.0f; /* RN_f32(1/6) */
    long k;
#pragma omp parallel for schedule(static)
    for (k = 1; k <= nz; ++k)
        for (long j = 1; j <= ny; ++j)
            for (long i = 1; i <= nx; ++i) {
                float s = src[IDX(i - 1, j, k)];
                s = s + src[IDX(i + 1, j, k)];
                s = s + src[IDX(i, j - 1, k)];
                s = s + src[IDX(i, j + 1, k)];
                s = s + src[IDX(i, j, k - 1)];
                s = s + src[IDX(i, j, k + 1)];
                dst[IDX(i, j, k)] = s * sixth;
            }
}

static int is_halo(long i, long j, long k, long nx, long ny, long nz)
{
    return i == 0 || j == 0 || k == 0 || i == nx + 1 || j == ny + 1 || k == nz + 1;
}

/* Copies every halo cell of A into B, so both grids carry the same boundary. */
void oracle_halo_copy_f64(const double *A, double *B, long nx, long ny, long nz)
{
    for (long k = 0; k <= nz + 1; ++k)
        for (long j = 0; j <= ny + 1; ++j)
            for (long i = 0; i <= nx + 1; ++i)
                if (is_halo(i, j, k, nx, ny, nz)) B[IDX(i, j, k)] = A[IDX(i, j, k)];
}

void oracle_halo_copy_f32(const float *A, float *B, long nx, long ny, long nz)
{
    for (long k = 0; k <= nz + 1; ++k)
        for (long j = 0; j <= ny + 1; ++j)
            for (long i = 0; i <= nx + 1; ++i)
                if (is_halo(i, j, k, nx, ny, nz)) B[IDX(i, j, k)] = A[IDX(i, j, k)];
}

/* T sweeps writing to grids A and B in turn (Sect. 1.1).  Sweep s (0-based)
 * reads A if s is even, B if odd.  Returns 0 if the result is in A (T even),
 * 1 if in B (T odd); returns -1 on bad arguments. */
int oracle_jacobi_f64(double *A, double *B, long nx, long ny, long nz, long T)
{
    if (nx < 1 || ny < 1 || nz < 1 || T < 0) return -1;
    oracle_halo_copy_f64(A, B, nx, ny, nz);
    for (long s = 0; s < T; ++s) {
        if (s % 2 == 0) sweep_f64(A, B, nx, ny, nz);
        else sweep_f64(B, A, nx, ny, nz);
    }
    return (int)(T % 2);
}

int oracle_jacobi_f32(float *A, float *B, long nx, long ny, long nz, long T)
{
    if (nx < 1 || ny < 1 || nz < 1 || T < 0) return -1;
    oracle_halo_copy_f32(A, B, nx, ny, nz);
    for (long s = 0; s < T; ++s) {
        if (s % 2 == 0) sweep_f32(A, B, nx, ny, nz);
        else sweep_f32(B, A, nx, ny, nz);
    }
    return (int)(T % 2);
}

/* ------------------------------------- pipelined blocking, Sect. 2.1 / 2.2 */

/* Bounds of block m (0 <= m < nb) of a 1D partition of [1, n] into blocks of
 * length bs, shifted by -shift cells and clipped to [1, n]; the last block
 * always ends at n (so every shifted partition still covers the interior). */
static void block_range(long m, long nb, long bs, long n, long shift, long *lo, long *hi)
{
    long a = 1 + m * bs - shift;
    long b = (m == nb - 1) ? n + 1 : 1 + (m + 1) * bs - shift;
    if (a < 1) a = 1;
    if (b > n + 1) b = n + 1;
    *lo = a;
    *hi = b; /* exclusive; empty if hi <= lo */
}

/* update_block(): one Jacobi update (Eq. 1) of the cells of one block. */
static void update_block_f64(const double *src, double *dst, long nx, long ny, long nz,
                             long x0, long x1, long y0, long y1, long z0, long z1)
{
    for (long k = z0; k < z1; ++k)
        for (long j = y0; j < y1; ++j)
            for (long i = x0; i < x1; ++i) {
                double s = src[IDX(i - 1, j, k)];
                s = s + src[IDX(i + 1, j, k)];
                s = s + src[IDX(i, j - 1, k)];
                s = s + src[IDX(i, j + 1, k)];
                s = s + src[IDX(i, j, k - 1)];
                s = s + src[IDX(i, j, k + 1)];
                dst[IDX(i, j, k)] = s / 6.0;
            }
}

/* Pipelined temporal blocking, emulated sequentially.  n_teams teams of
 * t_team threads; each thread applies T_upd updates to a block before
 * handing it on, so one team sweep applies L = n_teams*t_team*T_upd updates.
 * Blocks (bx*by*bz, lexicographic order, x fastest) are visited by thread i
 * at pipeline step tau as block m = tau - off_i, where off_i = i*d_l plus
 * d_t for every team boundary before thread i (Eq. 3 with a rigid lockstep
 * at the minimum distance d_l; the schedule is one legal interleaving of the
 * relaxed one).  Update number lam of the team sweep works on the block
 * shifted by -lam cells in every direction (Fig. 1).  The last team sweep
 * applies only the remaining updates.  Returns 0/1 (result in A/B) like
 * oracle_jacobi_f64, or -1 on bad arguments. */
int oracle_jacobi_pipelined_f64(double *A, double *B, long nx, long ny, long nz, long T,
                                long n_teams, long t_team, long T_upd, long d_l, long d_t,
                                long bx, long by, long bz)
{
    if (nx < 1 || ny < 1 || nz < 1 || T < 0 || n_teams < 1 || t_team < 1 || T_upd < 1 ||
        d_l < 1 || d_t < 0 || bx < 1 || by < 1 || bz < 1)
        return -1;
    oracle_halo_copy_f64(A, B, nx, ny, nz);
    const long nth = n_teams * t_team;
    const long L = nth * T_upd;
    const long nbx = (nx + bx - 1) / bx, nby = (ny + by - 1) / by, nbz = (nz + bz - 1) / bz;
    const long nblocks = nbx * nby * nbz;
    long *off = (long *)malloc(sizeof(long) * (size_t)nth);
    if (!off) return -1;
    for (long i = 0; i < nth; ++i) off[i] = i * d_l + (i / t_team) * d_t;

    long done = 0; /* updates applied so far */
    while (done < T) {
        const long L_now = (T - done < L) ? (T - done) : L;
        /* grid holding the data at the start of this team sweep */
        double *X = (done % 2 == 0) ? A : B;
        double *Y = (done % 2 == 0) ? B : A;
        const long last_step = nblocks - 1 + off[nth - 1];
        for (long tau = 0; tau <= last_step; ++tau)
            for (long i = 0; i < nth; ++i) {
                const long m = tau - off[i];
                if (m < 0 || m >= nblocks) continue;
                const long mx = m % nbx, my = (m / nbx) % nby, mz = m / (nbx * nby);
                for (long u = 0; u < T_upd; ++u) {
                    const long lam = i * T_upd + u;
                    if (lam >= L_now) break;
                    long x0, x1, y0, y1, z0, z1;
                    block_range(mx, nbx, bx, nx, lam, &x0, &x1);
                    block_range(my, nby, by, ny, lam, &y0, &y1);
                    block_range(mz, nbz, bz, nz, lam, &z0, &z1);
                    if (x1 <= x0 || y1 <= y0 || z1 <= z0) continue;
                    const double *src = (lam % 2 == 0) ? X : Y;
                    double *dst = (lam % 2 == 0) ? Y : X;
                    update_block_f64(src, dst, nx, ny, nz, x0, x1, y0, y1, z0, z1);
                }
            }
        done += L_now;
    }
    free(off);
    return (int)(T % 2);
}

/* ------------------------------------------------ multi-layer halo, Sect. 3.1 */

/* Passes of depth depths[0..n_pass-1] (sum = total update count).  In each
 * pass of depth h, every x/y subdomain [x0, x0+bx) x [y0, y0+by) (all z)
 * copies its region widened by h layers (clipped to the array) from the
 * source grid into two private buffers, performs update s = 1..h on the
 * region widened by h-s layers (clipped to the interior), and writes its own
 * cells of update h into the destination grid.  Grids alternate per pass.
 * Returns 0/1 = grid holding the result (n_pass even/odd), -1 on error. */
int oracle_jacobi_multihalo_f64(double *A, double *B, long nx, long ny, long nz,
                                const long *depths, long n_pass, long bx, long by)
{
    if (nx < 1 || ny < 1 || nz < 1 || n_pass < 0 || bx < 1 || by < 1) return -1;
    for (long p = 0; p < n_pass; ++p)
        if (depths[p] < 1) return -1;
    oracle_halo_copy_f64(A, B, nx, ny, nz);
    for (long p = 0; p < n_pass; ++p) {
        const double *src = (p % 2 == 0) ? A : B;
        double *dst = (p % 2 == 0) ? B : A;
        const long h = depths[p];
        for (long ty = 1; ty <= ny; ty += by)
            for (long tx = 1; tx <= nx; tx += bx) {
                const long tx1 = (tx + bx <= nx + 1) ? tx + bx : nx + 1;
                const long ty1 = (ty + by <= ny + 1) ? ty + by : ny + 1;
                /* private region: widened by h, clipped to the array */
                const long rx0 = (tx - h < 0) ? 0 : tx - h;
                const long rx1 = (tx1 + h > nx + 2) ? nx + 2 : tx1 + h;
                const long ry0 = (ty - h < 0) ? 0 : ty - h;
                const long ry1 = (ty1 + h > ny + 2) ? ny + 2 : ty1 + h;
                const long lx = rx1 - rx0, ly = ry1 - ry0, lz = nz + 2;
                const size_t cells = (size_t)lx * (size_t)ly * (size_t)lz;
                double *L0 = (double *)malloc(cells * sizeof(double));
                double *L1 = (double *)malloc(cells * sizeof(double));
                if (!L0 || !L1) {
                    free(L0);
                    free(L1);
                    return -1;
                }
#define LIDX(i, j, k) ((((size_t)(k)) * (size_t)ly + (size_t)((j) - ry0)) * (size_t)lx + (size_t)((i) - rx0))
                for (long k = 0; k < lz; ++k)
                    for (long j = ry0; j < ry1; ++j)
                        for (long i = rx0; i < rx1; ++i) {
                            L0[LIDX(i, j, k)] = src[IDX(i, j, k)];
                            L1[LIDX(i, j, k)] = src[IDX(i, j, k)];
                        }
                for (long s = 1; s <= h; ++s) {
                    const double *ls = (s % 2 == 1) ? L0 : L1;
                    double *ld = (s % 2 == 1) ? L1 : L0;
                    const long w = h - s;
                    const long cx0 = (tx - w < 1) ? 1 : tx - w;
                    const long cx1 = (tx1 + w > nx + 1) ? nx + 1 : tx1 + w;
                    const long cy0 = (ty - w < 1) ? 1 : ty - w;
                    const long cy1 = (ty1 + w > ny + 1) ? ny + 1 : ty1 + w;
                    for (long k = 1; k <= nz; ++k)
                        for (long j = cy0; j < cy1; ++j)
                            for (long i = cx0; i < cx1; ++i) {
                                double v = ls[LIDX(i - 1, j, k)];
                                v = v + ls[LIDX(i + 1, j, k)];
                                v = v + ls[LIDX(i, j - 1, k)];
                                v = v + ls[LIDX(i, j + 1, k)];
                                v = v + ls[LIDX(i, j, k - 1)];
                                v = v + ls[LIDX(i, j, k + 1)];
                                ld[LIDX(i, j, k)] = v / 6.0;
                            }
                }
                const double *res = (h % 2 == 1) ? L1 : L0;
                for (long k = 1; k <= nz; ++k)
                    for (long j = ty; j < ty1; ++j)
                        for (long i = tx; i < tx1; ++i) dst[IDX(i, j, k)] = res[LIDX(i, j, k)];
#undef LIDX
                free(L0);
                free(L1);
            }
    }
    return (int)(n_pass % 2);
}

/* ------------------------------------------------------------ Poisson part */

/* r = f - A_h u on the interior, A_h u = (6u - sum of the six neighbours)/h^2,
 * neighbour sum in the order of Eq. (1).  Halo of r set to 0. */
void oracle_poisson_residual(const double *u, const double *f, double *r, long nx, long ny,
                             long nz, double h)
{
    const double h2 = h * h;
    memset(r, 0, sizeof(double) * (size_t)(nx + 2) * (size_t)(ny + 2) * (size_t)(nz + 2));
    long k;
#pragma omp parallel for schedule(static)
    for (k = 1; k <= nz; ++k)
        for (long j = 1; j <= ny; ++j)
            for (long i = 1; i <= nx; ++i) {
                double s = u[IDX(i - 1, j, k)];
                s = s + u[IDX(i + 1, j, k)];
                s = s + u[IDX(i, j - 1, k)];
                s = s + u[IDX(i, j + 1, k)];
                s = s + u[IDX(i, j, k - 1)];
                s = s + u[IDX(i, j, k + 1)];
                const double au = (6.0 * u[IDX(i, j, k)] - s) / h2;
                r[IDX(i, j, k)] = f[IDX(i, j, k)] - au;
            }
}

/* Euclidean norm over the interior (plain sequential sum of squares). */
double oracle_norm2_interior(const double *x, long nx, long ny, long nz)
{
    double acc = 0.0;
    for (long k = 1; k <= nz; ++k)
        for (long j = 1; j <= ny; ++j)
            for (long i = 1; i <= nx; ++i) acc += x[IDX(i, j, k)] * x[IDX(i, j, k)];
    return sqrt(acc);
}

/* Jacobi smoother for -Lap_h e = g/h^2 in single precision, with zero halo:
 * e_new = (neighbour sum in the order of Eq. (1) + g) * RN_f32(1/6), where
 * g = RN_f32(h^2 * r) is formed once per outer step in double. */
static void sweep_rhs_f32(const float *src, float *dst, const float *g, long nx, long ny, long nz)
{
    const float sixth = 1.0f / 6.0f;
    long k;
#pragma omp parallel for schedule(static)
    for (k = 1; k <= nz; ++k)
        for (long j = 1; j <= ny; ++j)
            for (long i = 1; i <= nx; ++i) {
                float s = src[IDX(i - 1, j, k)];
                s = s + src[IDX(i + 1, j, k)];
                s = s + src[IDX(i, j - 1, k)];
                s = s + src[IDX(i, j + 1, k)];
                s = s + src[IDX(i, j, k - 1)];
                s = s + src[IDX(i, j, k + 1)];
                s = s + g[IDX(i, j, k)];
                dst[IDX(i, j, k)] = s * sixth;
            }
}

/* Plain FP64 Jacobi for -Lap_h u = f: u_new = (neighbour sum + h^2 f)/6. */
void oracle_poisson_jacobi_f64(double *u, double *tmp, const double *f, long nx, long ny,
                               long nz, double h, long sweeps)
{
    const double h2 = h * h;
    oracle_halo_copy_f64(u, tmp, nx, ny, nz);
    for (long s = 0; s < sweeps; ++s) {
        const double *src = (s % 2 == 0) ? u : tmp;
        double *dst = (s % 2 == 0) ? tmp : u;
        long k;
#pragma omp parallel for schedule(static)
        for (k = 1; k <= nz; ++k)
            for (long j = 1; j <= ny; ++j)
                for (long i = 1; i <= nx; ++i) {
                    double v = src[IDX(i - 1, j, k)];
                    v = v + src[IDX(i + 1, j, k)];
                    v = v + src[IDX(i, j - 1, k)];
                    v = v + src[IDX(i, j + 1, k)];
                    v = v + src[IDX(i, j, k - 1)];
                    v = v + src[IDX(i, j, k + 1)];
                    v = v + h2 * f[IDX(i, j, k)];
                    dst[IDX(i, j, k)] = v / 6.0;
                }
    }
    if (sweeps % 2 == 1)
        memcpy(u, tmp, sizeof(double) * (size_t)(nx + 2) * (size_t)(ny + 2) * (size_t)(nz + 2));
}

/* Mixed-precision iterative refinement for -Lap_h u = f, zero Dirichlet halo.
 * Outer step: r = f - A_h u (FP64); stop if ||r||/||f|| <= tol or max_outer
 * corrections were applied; else g = RN_f32(h^2 r), e = 0, `inner` FP32
 * Jacobi sweeps on A_h e = r (ping-pong), then u += (double)e (FP64).
 * Returns 0 if converged, 1 if not, -1 on error. */
int oracle_refine(double *u, const double *f, long nx, long ny, long nz, double h, double tol,
                  long inner, long max_outer, long *outer_done, double *final_rel)
{
    const size_t n = (size_t)(nx + 2) * (size_t)(ny + 2) * (size_t)(nz + 2);
    double *r = (double *)calloc(n, sizeof(double));
    float *g = (float *)calloc(n, sizeof(float));
    float *e0 = (float *)calloc(n, sizeof(float));
    float *e1 = (float *)calloc(n, sizeof(float));
    if (!r || !g || !e0 || !e1) {
        free(r); free(g); free(e0); free(e1);
        return -1;
    }
    const double fn = oracle_norm2_interior(f, nx, ny, nz);
    const double h2 = h * h;
    long outer = 0;
    double rel = 0.0;
    int status = 1;
    for (;;) {
        oracle_poisson_residual(u, f, r, nx, ny, nz, h);
        rel = (fn > 0.0) ? oracle_norm2_interior(r, nx, ny, nz) / fn : 0.0;
        if (rel <= tol) { status = 0; break; }
        if (outer >= max_outer) break;
        for (size_t q = 0; q < n; ++q) {
            g[q] = (float)(h2 * r[q]);
            e0[q] = 0.0f;
            e1[q] = 0.0f;
        }
        for (long s = 0; s < inner; ++s) {
            if (s % 2 == 0) sweep_rhs_f32(e0, e1, g, nx, ny, nz);
            else sweep_rhs_f32(e1, e0, g, nx, ny, nz);
        }
        const float *e = (inner % 2 == 0) ? e0 : e1;
        for (long k = 1; k <= nz; ++k)
            for (long j = 1; j <= ny; ++j)
                for (long i = 1; i <= nx; ++i) u[IDX(i, j, k)] = u[IDX(i, j, k)] + (double)e[IDX(i, j, k)];
        ++outer;
    }
    *outer_done = outer;
    *final_rel = rel;
    free(r); free(g); free(e0); free(e1);
    return status;
}

/* ------------------------------------------------------- compressed grid */

/* The compressed grid of Sect. 2.1, run sequentially: ONE array E of
 * (nx+3)(ny+3)(nz+3) cells holds the grid (halo included, indices 0..n+1
 * per axis), shifted by one cell along every axis on alternate sweeps.
 * Position 1: cell (i,j,k) at E(i+1, j+1, k+1); position 0: at E(i, j, k).
 * A sweep from position 1 writes every cell to position 0, i.e. shifted by
 * (-1,-1,-1), with the loops over k, j, i running upward; a sweep from
 * position 0 writes shifted by (+1,+1,+1) with the loops running downward.
 * Halo cells are carried along unchanged; interior cells get Eq. (1) with
 * the term order and division of sweep_f64 / sweep_f32.  A write destroys
 * the old value of the cell one step back along every axis (in loop
 * direction), and every cell that reads that value (its six neighbours and,
 * for a halo cell, itself) comes earlier in the loop order.  Returns the
 * position of the result: 1 if T is even, else 0. */
#define EIDX(i, j, k) ((((k) * (ny + 3)) + (j)) * (nx + 3) + (i))

static void cg_sweep_f64(double *E, long nx, long ny, long nz, long from)
{
    const long o = from, w = 1 - from;
    for (long kk = 0; kk <= nz + 1; ++kk) {
        const long k = from ? kk : nz + 1 - kk;
        for (long jj = 0; jj <= ny + 1; ++jj) {
            const long j = from ? jj : ny + 1 - jj;
            for (long ii = 0; ii <= nx + 1; ++ii) {
                const long i = from ? ii : nx + 1 - ii;
                double v;
                if (is_halo(i, j, k, nx, ny, nz)) {
                    v = E[EIDX(i + o, j + o, k + o)];
                } else {
                    double s = E[EIDX(i - 1 + o, j + o, k + o)];
                    s = s + E[EIDX(i + 1 + o, j + o, k + o)];
                    s = s + E[EIDX(i + o, j - 1 + o, k + o)];
                    s = s + E[EIDX(i + o, j + 1 + o, k + o)];
                    s = s + E[EIDX(i + o, j + o, k - 1 + o)];
                    s = s + E[EIDX(i + o, j + o, k + 1 + o)];
                    v = s / 6.0;
                }
                E[EIDX(i + w, j + w, k + w)] = v;
            }
        }
    }
}

static void cg_sweep_f32(float *E, long nx, long ny, long nz, long from)
{
    const float sixth = 1.0f / 6.0f; /* RN_f32(1/6) */
    const long o = from, w = 1 - from;
    for (long kk = 0; kk <= nz + 1; ++kk) {
        const long k = from ? kk : nz + 1 - kk;
        for (long jj = 0; jj <= ny + 1; ++jj) {
            const long j = from ? jj : ny + 1 - jj;
            for (long ii = 0; ii <= nx + 1; ++ii) {
                const long i = from ? ii : nx + 1 - ii;
                float v;
                if (is_halo(i, j, k, nx, ny, nz)) {
                    v = E[EIDX(i + o, j + o, k + o)];
                } else {
                    float s = E[EIDX(i - 1 + o, j + o, k + o)];
                    s = s + E[EIDX(i + 1 + o, j + o, k + o)];
                    s = s + E[EIDX(i + o, j - 1 + o, k + o)];
                    s = s + E[EIDX(i + o, j + 1 + o, k + o)];
                    s = s + E[EIDX(i + o, j + o, k - 1 + o)];
                    s = s + E[EIDX(i + o, j + o, k + 1 + o)];
                    v = s * sixth;
                }
                E[EIDX(i + w, j + w, k + w)] = v;
            }
        }
    }
}

int oracle_jacobi_compressed_f64(double *E, long nx, long ny, long nz, long T)
{
    if (nx < 1 || ny < 1 || nz < 1 || T < 0) return -1;
    long pos = 1;
    for (long s = 0; s < T; ++s) {
        cg_sweep_f64(E, nx, ny, nz, pos);
        pos = 1 - pos;
    }
    return (int)pos;
}

int oracle_jacobi_compressed_f32(float *E, long nx, long ny, long nz, long T)
{
    if (nx < 1 || ny < 1 || nz < 1 || T < 0) return -1;
    long pos = 1;
    for (long s = 0; s < T; ++s) {
        cg_sweep_f32(E, nx, ny, nz, pos);
        pos = 1 - pos;
    }
    return (int)pos;
}
