/*
 * jacobi.h -- C ABI of the GB300 (sm_103a) temporally blocked 3D Jacobi
 * library (libjacobi.so).
 *
 * The operation (Sect. 1.1, Eq. 1): for every interior cell
 *     B[i,j,k] = (A[i-1,j,k] + A[i+1,j,k] + A[i,j-1,k] + A[i,j+1,k]
 *                 + A[i,j,k-1] + A[i,j,k+1]) / 6
 * and successive sweeps write to grids A and B in turn.  Temporal blocking
 * (Sect. 2.1: several updates per cell while it is on chip; Sect. 3.1: a
 * subdomain with an h-layer halo takes h updates, update s on a region h-s
 * layers wider) applies d sweeps per pass over HBM.
 *
 * Grid layout (every entry point): interior nx*ny*nz plus a one-cell
 * Dirichlet halo, dense, x fastest:
 *     idx(i,j,k) = (k*(ny+2) + j)*(nx+2) + i,   0 <= i <= nx+1, ...
 * element type double (JACOBI_F64) or float (JACOBI_F32).  Halo cells are
 * boundary values: read, never changed.
 *
 * Arithmetic: FP64 adds the six neighbours left to right in the order of
 * Eq. (1) and divides the sum by 6.0 with IEEE round-to-nearest; results are
 * bit-identical to a plain CPU loop doing the same.  FP32 adds in the same
 * order and multiplies by RN_f32(1/6) (the paper's count of one
 * multiplication and five additions per update, Sect. 2.3).
 *
 * Ownership and errors: the caller owns every grid buffer (device memory of
 * the current device, 16-byte aligned); the library owns handles and its
 * own scratch.  Every call returns an int status, JACOBI_OK (0) or a
 * negative JACOBI_ERR_* code; no call aborts or prints.  Device work is
 * enqueued on the caller's stream (cudaStream_t passed as jacobi_stream_t;
 * NULL = legacy default stream) with no implicit device synchronisation
 * unless stated.  Calls on one handle must not overlap on different streams.
 */
#ifndef JACOBI_H
#define JACOBI_H

#ifdef __cplusplus
extern "C" {
#endif

/* Same type as cudaStream_t; declared here so that this header needs no
 * CUDA header. */
typedef struct CUstream_st *jacobi_stream_t;

typedef enum { JACOBI_F64 = 0, JACOBI_F32 = 1 } jacobi_dtype;

enum {
    JACOBI_OK = 0,
    JACOBI_ERR_ARG = -1,           /* bad size, count, pointer or option      */
    JACOBI_ERR_DTYPE = -2,         /* dtype not JACOBI_F64 / JACOBI_F32       */
    JACOBI_ERR_ALLOC = -3,         /* device or host allocation failed        */
    JACOBI_ERR_CUDA = -4,          /* a CUDA call failed (see last_cuda_error) */
    JACOBI_ERR_TIMEOUT = -5,       /* a device-side wait ran out its limit    */
    JACOBI_ERR_BOUNDS = -6,        /* a device-side index check failed        */
    JACOBI_ERR_NOT_CONVERGED = -7, /* refinement stopped at max_outer         */
    JACOBI_ERR_ALIGN = -8,         /* grid pointer not 16-byte aligned        */
    JACOBI_ERR_UNSUPPORTED = -9    /* plan not launchable on this device      */
};

/* Kernel families selectable by jacobi_set_plan. */
enum {
    JACOBI_KERNEL_AUTO = 0,  /* tuned (or default) plan                      */
    JACOBI_KERNEL_PLAIN = 1, /* one sweep per launch, every operand from
                                global memory: the single-pass baseline       */
    JACOBI_KERNEL_TB = 2,    /* z-streaming pass; depth d > 1 runs the
                                time-skewed cluster pipeline                  */
    JACOBI_KERNEL_PLAIN_X2 = 3, /* single-pass kernel with two x cells per
                                thread (vector loads, shuffled x-neighbours,
                                packed FP32 additions); even nx only          */
    JACOBI_KERNEL_TB_CTA = 4, /* temporal blocking inside one CTA: depth 1..4
                                levels applied to a tile's planes in shared
                                memory (T updates per thread, Sect. 2.1)     */
    JACOBI_KERNEL_TB_REG = 5, /* temporal blocking inside one CTA with
                                register-blocked cells (FP32 only): every
                                thread keeps a 4 x 4 cell block of each level
                                in registers and exchanges only its block
                                boundary through shared memory; depth 1..4  */
    JACOBI_KERNEL_TB_CHAIN = 6 /* temporal blocking by a chain of 2..4 CTAs
                                of a thread-block cluster (FP32 only), each
                                applying up to 4 levels of the register-
                                blocked step and handing its last level to
                                the next CTA through distributed shared
                                memory: depth up to 16 per pass (the team
                                of threads x T updates of Sect. 2.1)      */
};

typedef struct jacobi_plan_s *jacobi_h;
typedef struct jacobi_batch_s *jacobi_batch_h;

/* Text of a status code (static storage, never NULL). */
const char *jacobi_status_string(int status);
/* Library version as major*10000 + minor*100 + patch. */
int jacobi_version(void);
/* Text of the last CUDA error seen by this thread's calls ("" if none). */
const char *jacobi_last_cuda_error(void);

/* Creates a handle for grids of interior nx*ny*nz (each >= 1, and
 * (nx+2)(ny+2)(nz+2) < 2^40 elements) of element type dtype, on the current
 * device.  Allocates a 4-byte device status word.  *out is set to NULL on
 * error. */
int jacobi_create(jacobi_h *out, int nx, int ny, int nz, int dtype);

/* Frees the handle.  The caller must have synchronised every stream that
 * has work of this handle in flight.  NULL is accepted. */
int jacobi_destroy(jacobi_h h);

/* Applies T >= 0 sweeps of Eq. (1), grids A and B in turn (Sect. 1.1).
 * First copies the halo of A into B (so both carry the same Dirichlet
 * values), then runs ceil-ish(T/d) passes of depth <= d, pass p reading the
 * grid written by pass p-1.  The number of passes always has the parity of
 * T, so the result is in B if T is odd and in A if T is even, exactly as
 * with single sweeps; the other grid's interior is left unspecified.  T = 0
 * does nothing.  A and B: device pointers, 16-byte aligned, not
 * overlapping, each (nx+2)(ny+2)(nz+2) elements.  Asynchronous on stream.
 * Device-side wait timeouts are reported by jacobi_get_status.  Once a call
 * with the same plan has run uncaptured (it sets the kernels' shared-memory
 * limits), the call enqueues kernel launches only and can be captured into
 * a CUDA graph. */
int jacobi_sweep(jacobi_h h, void *A, void *B, int T, jacobi_stream_t stream);

/* Same operation with host buffers (end-to-end entry point): copies
 * A_host (pageable or pinned, (nx+2)(ny+2)(nz+2) elements) to library-owned
 * device grids (allocated on first use, freed by jacobi_destroy), runs
 * jacobi_sweep, and copies the result grid back to out_host.  Synchronises
 * stream before returning. */
int jacobi_sweep_host(jacobi_h h, const void *A_host, void *out_host, int T,
                      jacobi_stream_t stream);

/* Forces a plan: kernel (JACOBI_KERNEL_*) and temporal depth (1..16;
 * taken as 1 for PLAIN).  For TB: tile interior bx*by (bx, by >= 1), z chunk
 * bz >= 1 interior planes per cluster, ring = plane slots between two
 * pipeline levels (4, 8 or 16; 0 = the deepest that fits 100 KB of shared
 * memory), and threads = CTA width (128, 256 or 512; 0 = automatic).  The
 * ring depth is the pipeline looseness of Sect. 2.2 (a producer may run up
 * to ring planes ahead of its consumer; at least one plane, Eq. 3).
 * Depths > 8 need the non-portable cluster size.  For TB_CTA: depth 1..4
 * (1: one sweep per pass with the input planes staged in shared memory),
 * tile bx*by, z chunk bz, threads 256 or 512 (0 = 512), at most 8 cells
 * (FP64) or 4 quads of 4 cells (FP32) of the widened tile (bx+2d)(by+2d)
 * per thread; ring ignored.  For TB_REG (FP32 grids only): bx*by is the
 * region the CTA streams -- the output tile widened by depth cells on each
 * side -- one of 64x32, 64x64 or 128x32 (threads = bx*by/16, each owning
 * 4 x 4 cells), depth 1..4, z chunk bz; the output tile is (bx - 2 depth,
 * rounded down to even when nx is even) x (by - 2 depth); ring and threads
 * ignored.  For TB_CHAIN (FP32 grids only): depth d = total levels per pass,
 * ring = c, the CTAs of the chain (2..4, c <= d <= 4c; levels are split as
 * evenly as possible, d/c rounded up per CTA at most), bx*by = region, 64x32
 * (d <= 15) or 64x64, as for TB_REG at depth d, z chunk bz; threads ignored.
 * Passes of depth below c run on the one-CTA TB_REG kernel.  For PLAIN and
 * PLAIN_X2:
 * bx*by = CTA shape in threads (bx a multiple of 32, bx*by <= 1024; a
 * PLAIN_X2 thread covers two x cells) and bz = planes each thread walks in
 * z; ring and threads are ignored.  A zero bx, by or bz takes the family's
 * default (PLAIN 32 x 8 x 8; PLAIN_X2 32 x 8 x 16; TB 64 x 16 x 64; TB_CTA
 * 64 x 32 x 64; TB_REG region 64 x 32, 64 planes; TB_CHAIN region
 * 64 x 64, 64 planes, 2 CTAs; tiles clamped to the grid).  JACOBI_KERNEL_AUTO returns to
 * the tuned/default plan.  Returns JACOBI_ERR_ARG for out-of-range fields and JACOBI_ERR_UNSUPPORTED
 * if the plan cannot launch on this device (shared memory, registers,
 * cluster occupancy). */
int jacobi_set_plan(jacobi_h h, int kernel, int depth, int bx, int by, int bz, int ring,
                    int threads);

/* Reads back the plan jacobi_sweep will use, defaults resolved
 * (ring/threads 0 = automatic). */
int jacobi_get_plan(jacobi_h h, int *kernel, int *depth, int *bx, int *by, int *bz, int *ring,
                    int *threads);

/* Autotuner (experiment-driven parameter choice, Sect. 2.4): fills the
 * caller's scratch grids (same size as the handle's grids; contents
 * overwritten, never the user's data) with a constant and times candidate
 * plans on them -- the single-pass kernel over CTA shapes and planes per
 * thread, and pass kernels of depth 1..8 over tile shapes, then z chunks,
 * ring depths and CTA widths around the best -- and
 * keeps the fastest as the handle's AUTO plan.  Results are
 * cached per process by (dtype, nx, ny, nz, SM count).  Synchronises
 * stream.  *glups (may be NULL) receives the best measured GLUP/s. */
int jacobi_tune(jacobi_h h, void *scratchA, void *scratchB, jacobi_stream_t stream,
                double *glups);

/* The autotuner's first-stage candidate plans for this handle (the plans
 * jacobi_tune times before refining the winner), restricted to those this
 * device can launch: writes up to max_plans plans as 7 ints each (kernel,
 * depth, bx, by, bz, ring, threads, the fields of jacobi_set_plan) to
 * plans[0 .. 7*max_plans-1] and returns the total number of candidates
 * (which may exceed max_plans), or a negative JACOBI_ERR_* code.  No device
 * work beyond occupancy queries.  Serves tests that force every plan the
 * tuner can choose (Sect. 2.4's parameter sweeps). */
int jacobi_tune_candidates(jacobi_h h, int *plans, int max_plans);

/* Pass planning (host only, no device work): splits T >= 0 sweeps into
 * passes of depth <= depth (>= 1) whose count has the parity of T, as even
 * as possible (a team sweep of Sect. 2.1 applies t*T updates; here a pass
 * applies d).  Writes the depths to depths[0..n-1] and returns n, or -1 if
 * more than max_passes passes would be needed or an argument is bad. */
int jacobi_plan_passes(int T, int depth, int *depths, int max_passes);

/* Self-test of the exact FP64 division used by the FP64 kernels (the sum of
 * Eq. 1 divided by 6 is computed on the integer pipe): compares it bit for bit with the device's IEEE division for
 * `count` pseudo-random bit patterns (SplitMix64 stream `seed`, NaNs
 * skipped) and for mantissas near 2^52, 3*2^51 and 2^53-1 at every exponent
 * and sign.  Synchronises the device.  *mismatches = number of differing
 * results; *first_bad (may be NULL) = one failing input's bits. */
int jacobi_check_division(unsigned long long count, unsigned long long seed,
                          unsigned long long *mismatches, unsigned long long *first_bad);

/* Self-test of the exact FP64 addition that part of the FP64 sums use (the
 * additions of Eq. 1 moved to the integer pipe): compares it bit for bit
 * with the device's FP64 addition for 4*count pairs -- random bit patterns,
 * and same-sign pairs whose exponents differ by 0..63 (carries, sticky
 * bits, ties) -- from SplitMix64 stream `seed`.  Synchronises the device.
 * *mismatches = differing results; first_bad[0..1] (may be NULL) = one
 * failing pair. */
int jacobi_check_addition(unsigned long long count, unsigned long long seed,
                          unsigned long long *mismatches, unsigned long long *first_bad);

/* Reads and clears the handle's device status word (synchronises the
 * device).  *device_status: 0 = fine, else the first JACOBI_ERR_* code a
 * kernel recorded (JACOBI_ERR_TIMEOUT, JACOBI_ERR_BOUNDS). */
int jacobi_get_status(jacobi_h h, int *device_status);

/* Kernel timing for benchmarks.  While enabled, every pass-kernel launch of
 * this handle's sweeps is bracketed by two CUDA events recorded on the
 * launch stream, and every other kernel launch of the handle (halo copies,
 * and the Poisson and refinement kernels) is counted.  enable = 0 stops
 * recording (already recorded launches stay until read). */
int jacobi_profile_enable(jacobi_h h, int enable);

/* Synchronises the recorded events and returns, since the previous read:
 * *pass_ms = summed device time of the pass launches (ms), *pass_launches,
 * *other_launches (halo copies and other helper kernels).  Resets the
 * record.  Any output pointer may be NULL. */
int jacobi_profile_read(jacobi_h h, double *pass_ms, int *pass_launches, int *other_launches);

/* Test hook for failure detection: mode 1 makes the next pass kernel omit
 * one mbarrier arrival (TB: a cp.async arrival; TB_CHAIN: the first CTA's
 * hand-off of one plane; the compressed grid: the first item's completion
 * flag) so that its bounded waits run out (after limit_ms milliseconds);
 * the kernel records JACOBI_ERR_TIMEOUT and returns without faulting.  Mode 2 (bounds-checked build only, else
 * JACOBI_ERR_UNSUPPORTED): the kernels check their accesses against grids
 * declared one element shorter than they are, so the accesses to each
 * grid's last element are reported as JACOBI_ERR_BOUNDS and skipped (every
 * skipped access is in fact valid: nothing faults).  mode 0 disables both.
 * limit_ms also sets the wait limit of later launches (default 2000). */
int jacobi_debug_set_fault(jacobi_h h, int mode, int limit_ms);

/* 1 if this library is the bounds-checked build (compiled with
 * -DJACOBI_CHECKED: every global, shared and distributed shared memory
 * access of the sweep, batch, compressed-grid and refinement kernels is checked against its
 * buffer, and an access outside records JACOBI_ERR_BOUNDS in the status word
 * and is skipped instead of performed), else 0. */
int jacobi_build_checked(void);

/* -------------------------------------------------------------- Poisson
 * -Lap_h u = f with the 7-point Laplacian, (A_h u) = (6u - sum of the six
 * neighbours)/h^2, on a handle created with JACOBI_F64; the halo of u holds
 * the Dirichlet values (0 for the homogeneous problem); f's halo is not
 * read.  Scratch grids are allocated on the handle at first use. */

/* *rel = ||f - A_h u||_2 / ||f||_2 over the interior, FP64, sums of squares
 * reduced in a fixed order.  Synchronises stream. */
int jacobi_poisson_residual(jacobi_h h, const void *u, const void *f, double hgrid,
                            jacobi_stream_t stream, double *rel);

/* Plain FP64 Jacobi for the Poisson problem: `sweeps` sweeps of
 * u <- (neighbour sum + h^2 f)/6 (order of Eq. 1, h^2 f added last, IEEE
 * division), u and tmp in turn: one single-pass sweep kernel per sweep,
 * replayed from a CUDA graph cached on the handle; result in tmp if sweeps
 * is odd, else in u (tmp's halo is set from u's).  Asynchronous. */
int jacobi_poisson_jacobi(jacobi_h h, void *u, void *tmp, const void *f, double hgrid, int sweeps,
                          jacobi_stream_t stream);

/* Mixed-precision iterative refinement (u updated in place):
 *   loop: r = f - A_h u in FP64, rel = ||r||/||f||; stop if rel <= rel_tol
 *         or max_outer corrections were applied; g = RN_f32(h^2 r);
 *         e = 0 and inner_sweeps FP32 Jacobi sweeps e <- (sum(e) + g)/6 on
 *         A_h e = r (zero halo; single-pass sweep kernels replayed from
 *         a CUDA graph cached on the handle); u += (double)e.
 * Only the residual and the update run in FP64.  *outer_done = corrections
 * applied, *final_rel_residual = last rel (both may be NULL).  Returns
 * JACOBI_ERR_NOT_CONVERGED if rel_tol was not reached.  Synchronises stream
 * once per outer step (to read the residual norm). */
int jacobi_refine(jacobi_h h, double *u, const double *f, double hgrid, double rel_tol,
                  int inner_sweeps, int max_outer, jacobi_stream_t stream, int *outer_done,
                  double *final_rel_residual);

/* Largest nz accepted by jacobi_poisson_residual_noalloc (its scratch holds
 * two partial sums per z-plane plus two totals: 2*16384+2 doubles, 256 KB,
 * held on every GPU that loads this library until the process exits). */
#define JACOBI_NOALLOC_MAX_NZ 16384

/* The relative residual ||f - A_h u||_2 / ||f||_2 of jacobi_poisson_residual
 * (same operator and arithmetic, sums reduced per z-plane, so the last bits
 * may differ), computed without allocating anything: no cudaMalloc, no
 * cudaFree, no allocating library call, and no handle.  The paper has no
 * counterpart; this exists for callers that cannot allocate device memory --
 * code whose device memory is owned entirely by another allocator (a
 * framework's caching pool, a fixed memory budget) and code on a
 * latency-critical path where an allocation's implicit device
 * synchronisation, or its failure under memory pressure, is not acceptable.
 * Its scratch is a fixed device array inside the library (size: see
 * JACOBI_NOALLOC_MAX_NZ); nz > JACOBI_NOALLOC_MAX_NZ returns JACOBI_ERR_ARG.
 * u, f: device grids of interior nx*ny*nz as in jacobi_create; the result
 * is read back, so the call synchronises stream.  Every call looks up the
 * array's device address in the current device's context (a lookup, not an
 * allocation), so the address is never stale after a context reset.  All
 * calls share the one array: calls that overlap on the GPU (several streams
 * or threads at once) race and must be serialised by the caller. */
int jacobi_poisson_residual_noalloc(const void *u, const void *f, int nx, int ny, int nz,
                                    double hgrid, jacobi_stream_t stream, double *rel);

/* ------------------------------------------------------- compressed grid
 * Sweeps in ONE buffer, without the second grid (the compressed grid of
 * Sect. 2.1).  The buffer U holds nz + 2 + S planes of (nx+2)(ny+2)
 * elements of the handle's dtype; the grid (the usual layout, halo
 * included) sits either in the UPPER position (its plane k at buffer plane
 * k + S, i.e. starting S*(nx+2)*(ny+2) elements into U) or in the LOWER
 * position (starting at U).  Each pass of `depth` sweeps reads the grid in
 * one position and leaves the result, halo included, in the other: the
 * write shift of S planes alternates in direction, as the paper's shift by
 * (-1,-1,-1) and (+1,+1,+1) does, and the order of the z chunks is reversed
 * on alternate passes.  S = waves*bz + depth + 1 (jacobi_compressed_get_plan):
 * the grid is swept in items (x-y tile, z chunk of bz planes), and an item
 * starts only after the items of its tile and the neighbouring tiles, in
 * the two chunks whose input it overwrites (`waves` and waves+1 chunks
 * back in sweep order), have finished (bounded waits: JACOBI_ERR_TIMEOUT in
 * the status word if one runs out).  Results are bit-identical to
 * jacobi_sweep with T sweeps. */

/* Plan of the compressed sweeps: depth 1..4 sweeps per pass (FP32: the
 * register-blocked one-CTA body of JACOBI_KERNEL_TB_REG, 64 x 32 regions;
 * FP64: depth 1 only, else JACOBI_ERR_UNSUPPORTED), z chunk bz >= 2*depth+2,
 * waves 1..8 (JACOBI_ERR_ARG otherwise; the plan is then unchanged).  A zero
 * field takes the default: FP32 depth 3, bz 128, waves 1 (S = 132); FP64
 * depth 1, bz 64, waves 1 (S = 66). */
int jacobi_compressed_set_plan(jacobi_h h, int depth, int bz, int waves);

/* The current compressed plan and its shift S in planes (any may be NULL). */
int jacobi_compressed_get_plan(jacobi_h h, int *depth, int *bz, int *waves, long long *shift_planes);

/* T sweeps of the grid held in U (device pointer, 16-byte aligned, at least
 * (nx+2)(ny+2)(nz+2+S) elements) starting in position `upper` (1: upper,
 * 0: lower).  Runs ceil(T/depth) passes (the last one shallower if depth
 * does not divide T); *upper_out (may be NULL) receives the position of the
 * result: upper XOR (number of passes odd).  Cells of U outside the grid's
 * position are scratch.  Asynchronous on stream; allocates its small
 * counter array on first use, and a larger one when a plan needs more
 * (kept on the handle, the replaced ones too, until jacobi_destroy); after
 * one uncaptured call with the plan, a call enqueues memsets and kernel
 * launches only and can be captured into a CUDA graph, which stays valid
 * until the handle is destroyed.  Calls on one handle must not overlap. */
int jacobi_sweep_compressed(jacobi_h h, void *U, int T, int upper, int *upper_out, jacobi_stream_t stream);

/* ---------------------------------------------------------------- batch
 * Many independent grids (each its own size, element type and sweep count
 * T_g), swept by a CUDA graph that one of two engines builds:
 *   JACOBI_BATCH_SWEEPS (default): one kernel launch per sweep covers every
 *     grid, one CTA per (grid, row block, z chunk) unit; FP64 and FP32
 *     units are dealt out alternately so both kinds share the SMs.
 *   JACOBI_BATCH_PERSISTENT: ONE persistent launch.  Work items are (grid,
 *     x-y tile column, sweep), taken in pass-major order from a device-side
 *     queue; an item waits (bounded) until its tile and the face-neighbour
 *     tiles finished the previous sweep -- per-tile progress counters, the
 *     counters c_i of the relaxed synchronisation of Sect. 2.2.
 * Each grid ends exactly as after jacobi_sweep with T_g sweeps: result in
 * B_g if T_g is odd, else in A_g. */
enum { JACOBI_BATCH_PERSISTENT = 0, JACOBI_BATCH_SWEEPS = 1 };

/* Creates a batch of n (1..65535) grids; nx/ny/nz/dtype/T are host arrays
 * of n entries (sizes >= 1, dtype JACOBI_F64/F32, T >= 0, each grid below
 * 2^31 elements).  Allocates the device descriptor table and counters and
 * captures the graph (item-counter reset, halo copy of every grid,
 * persistent launch).  Synchronous. */
int jacobi_batch_create(jacobi_batch_h *out, int n, const int *nx, const int *ny, const int *nz,
                        const int *dtype, const int *T);

/* Binds the grids and launches the graph on stream.  A, B: host arrays of
 * n device pointers (grid g: (nx+2)(ny+2)(nz+2) elements of its dtype,
 * A[g] != B[g]); the pointer table is copied to the device on stream before
 * the graph launch.  Asynchronous.  Runs of one batch must not overlap.
 * Not for stream capture: the call launches the batch's own graph after a
 * copy from host memory. */
int jacobi_batch_run(jacobi_batch_h b, void *const *A, void *const *B, jacobi_stream_t stream);

/* Same, for the Poisson problem -Lap_h u = f: grid g is swept with the
 * source term RHS[g] (device pointer, same shape and dtype, holding
 * g = h^2 f; halo ignored), i.e. update = (neighbour sum + g)/6 in the
 * order of Eq. (1) with g added last.  RHS = NULL or RHS[g] = NULL: plain
 * Jacobi for that grid. */
int jacobi_batch_run_rhs(jacobi_batch_h b, void *const *A, void *const *B, const void *const *RHS,
                         jacobi_stream_t stream);

/* Frees the batch (after the caller synchronised its streams). */
int jacobi_batch_destroy(jacobi_batch_h b);

/* Selects the persistent engine with a work-item tile of bx*by cells
 * (bx*by <= 4096) and bz planes (bz = 0: the whole z column; bz > 0 also
 * splits z, and an item then also waits on the tiles above and below).
 * Re-captures the graph. */
int jacobi_batch_set_tile(jacobi_batch_h b, int bx, int by, int bz);

/* Selects the engine (JACOBI_BATCH_*); kz > 0 sets the sweep engine's
 * planes per thread (0 keeps the current value, initially 16).  Re-captures
 * the graph.  JACOBI_ERR_ARG for an unknown engine or kz < 0. */
int jacobi_batch_set_engine(jacobi_batch_h b, int engine, int kz);

/* Current engine and sweep-engine planes per thread (either may be NULL). */
int jacobi_batch_get_engine(jacobi_batch_h b, int *engine, int *kz);

/* Temporal depth of the batch's FP32 grids (Sect. 2.1 and 3.1): depth 1
 * (initially) sweeps them with the selected engine like the FP64 grids;
 * depth 2..4 takes them out of that engine and sweeps each FP32 grid g in
 * passes of depth <= depth (the pass count has the parity of T_g, so the
 * result buffer is unchanged) by the register-blocked one-CTA kernel of
 * JACOBI_KERNEL_TB_REG with 64 x 32 regions and z chunks of 128 planes, all
 * FP32 grids of one pass in one launch, on a branch of the graph that runs
 * beside the FP64 grids' launches.  Results stay bit-identical to depth 1.
 * Such grids take no source term: jacobi_batch_run_rhs returns
 * JACOBI_ERR_UNSUPPORTED if RHS[g] is non-NULL for one of them.
 * Re-captures the graph; JACOBI_ERR_ARG for a depth outside 1..4. */
int jacobi_batch_set_fp32_depth(jacobi_batch_h b, int depth);
int jacobi_batch_get_fp32_depth(jacobi_batch_h b, int *depth);

/* Autotuner for the batch: fills the caller's scratch grids (arrays of n
 * device pointers, same shapes as the batch) with a constant, times the
 * sweep engine at several planes per thread, the persistent engine at
 * several tiles and, where the batch has FP32 grids, FP32 depths 2 and 3,
 * and keeps the fastest.  Synchronises stream. */
int jacobi_batch_tune(jacobi_batch_h b, void *const *scratchA, void *const *scratchB,
                      jacobi_stream_t stream, double *glups);

/* Current tile, number of work items and persistent CTAs (any may be NULL). */
int jacobi_batch_get_info(jacobi_batch_h b, int *bx, int *by, int *bz, long long *items, int *blocks);

/* Reads and clears the batch's device status word (synchronises). */
int jacobi_batch_get_status(jacobi_batch_h b, int *device_status);

/* Test hook: mode 1 makes the persistent kernel never publish sweep 2 of
 * the first tile, so that dependent waits run out after limit_ms and the
 * kernel records JACOBI_ERR_TIMEOUT (no fault); re-captures the graph.
 * Mode 1 needs the persistent engine (else JACOBI_ERR_UNSUPPORTED).  Mode 2
 * (bounds-checked build only): grids are checked as one element shorter than
 * they are, as in jacobi_debug_set_fault. */
int jacobi_batch_debug_set_fault(jacobi_batch_h b, int mode, int limit_ms);

#ifdef __cplusplus
}
#endif
#endif /* JACOBI_H */
