// Internal declarations shared by the library's translation units.
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include <vector>

#include "jacobi.h"

namespace jac {

// Arguments of one temporally blocked pass (one launch).
struct TbArgs {
    const void *src;
    void *dst;
    int nx, ny, nz;     // interior size
    int depth;          // D: levels per pass = CTAs per cluster
    int bx, by, bz;     // tile interior (x, y) and z chunk (interior planes)
    int ntx;            // number of x tiles (grid.x = D * ntx)
    int W, H, Wp;       // ring plane: width bx+2D, height by+2D, padded pitch
    int R;              // ring slots per CTA (power of two, <= 16)
    int rshift;         // log2(R)
    int *status;        // device status word (first error code wins)
    unsigned long long limit_ns;  // bound of every device-side wait
    int fault_mode;     // test hook: 1 = drop one arrival (see jacobi.h)
    long long shrink = 0;  // checked build: grids declared this many elements short
};

// Arguments of one pass of the one-CTA temporally blocked kernel.
struct TbcArgs {
    const void *src;
    void *dst;
    int nx, ny, nz;
    int bx, by, bz;  // tile interior (x, y) and z chunk
    int W, H, WH;    // region: tile widened by the depth on each side
    int *status = nullptr;  // checked build: bounds errors
    long long shrink = 0;
};

// Arguments of one pass of the register-blocked one-CTA kernel (FP32).
// Tile t in x covers output columns [1 + t*bx, 1 + (t+1)*bx); its region
// starts at x_first + t*bx (a multiple of the copy piece A), off cells left
// of the tile's D-cell margin.
struct TbrArgs {
    const void *src;
    void *dst;
    int nx, ny, nz;
    int bx, by, bz;  // output tile (x, y) and z chunk
    int x_first;     // region origin of tile 0: 1 - D - off
    int off;         // alignment slack left of the region's margin
    int *status = nullptr;  // checked build: bounds errors
    long long shrink = 0;
};

// Arguments of one pass of the chained-cluster kernel (FP32): a cluster of
// `cluster` CTAs per tile, CTA r applying levels[r] of the pass's `depth`
// time levels (lev_before[r] = levels of CTAs 0..r-1); tile geometry as for
// the one-CTA register-blocked kernel at that depth.
struct TbxArgs {
    const void *src;
    void *dst;
    int nx, ny, nz;
    int bx, by, bz;
    int x_first, off;
    int depth, cluster;
    int levels[4], lev_before[4];
    int *status = nullptr;
    unsigned long long limit_ns = 2000000000ull;
    int fault_mode = 0;  // test hook: 1 = CTA 0 never hands over its third plane
    long long shrink = 0;
};

struct PlainArgs {
    const void *src;
    void *dst;
    int nx, ny, nz;
    const void *rhs = nullptr;  // source term g: (sum + g) / 6, or nullptr
    int kz;      // planes per thread
    int tx, ty;  // CTA shape in cells
    int gy, gz;  // row blocks, z chunks (set by plain_launch)
    int *status = nullptr;  // checked build: bounds errors
    long long shrink = 0;
};

// Plan of one handle.
// PLAIN, PLAIN_X2: bx x by = CTA shape in threads, bz = planes per thread.
// TB: bx x by = tile interior, bz = interior planes per cluster.
struct Plan {
    int kernel = JACOBI_KERNEL_TB;
    int depth = 1;
    int bx = 64, by = 16, bz = 64;
    int ring = 0;     // ring slots per CTA (4, 8, 16); 0 = largest that fits the budget
    int threads = 0;  // threads per CTA (128, 256, 512); 0 = automatic
};

// Launch resources of a TB plan (host side), filled by tb_configure.
struct TbLaunch {
    int nc = 0, maxc = 0;   // compute threads, cells per thread (template)
    size_t smem = 0;        // dynamic shared memory bytes
    int R = 4;
    int W = 0, H = 0, Wp = 0;
};


// Kernels (sweep_kernels.cu).  All return cudaError_t of the launch.
cudaError_t tb_configure(int dtype, int depth, int bx, int by, int ring, int threads, TbLaunch *out);
cudaError_t tb_launch(int dtype, const TbArgs &a, const TbLaunch &L, cudaStream_t s);
cudaError_t tb_max_clusters(int dtype, const TbLaunch &L, int depth, int *clusters);
// Kernel entry of a cluster pass variant (threads, groups per thread), or
// nullptr: parts 0/1 hold the FP64 variants, 2/3 the FP32 ones.
const void *tb_kernel_part0(int nc, int maxg);
const void *tb_kernel_part1(int nc, int maxg);
const void *tb_kernel_part2(int nc, int maxg);
const void *tb_kernel_part3(int nc, int maxg);
cudaError_t plain_launch(int dtype, PlainArgs a, cudaStream_t s);
// One-CTA temporal blocking: checks a plan (depth 1..4, CTA of 256 or 512
// threads, at most 8 cells per thread, shared memory) and fills the region
// fields of a; launches one pass.
int tbc_configure(int dtype, int depth, int bx, int by, int threads, TbcArgs *a, size_t *smem);
cudaError_t tbc_launch(int dtype, int depth, int threads, const TbcArgs &a, cudaStream_t s);
cudaError_t plain_x2_launch(int dtype, PlainArgs a, cudaStream_t s);  // nx even
// Chained-cluster temporal blocking (FP32): `cluster` (2..4) CTAs of a
// thread-block cluster, `depth` (>= cluster, <= 4 * cluster) levels split as
// evenly as possible; region W x H in {64x32, 64x64}.  Fills a; launches one pass.
int tbx_configure(int depth, int cluster, int W, int H, TbxArgs *a, size_t *smem);
cudaError_t tbx_launch(int depth, int cluster, int W, int H, const TbxArgs &a, cudaStream_t s);
cudaError_t tbx_max_clusters(int depth, int cluster, int W, int H, int nx, int *clusters);
// Register-blocked one-CTA temporal blocking (FP32): region W x H (W in
// {64, 128}, H in {32, 64}; 16 cells per thread), depth 1..4.  Checks the
// plan and fills the tile fields of a; launches one pass.
int tbr_configure(int depth, int W, int H, TbrArgs *a, size_t *smem, int *threads);
cudaError_t tbr_launch(int depth, int W, int H, const TbrArgs &a, cudaStream_t s);
cudaError_t tbr_launch_a1(int depth, int W, int H, const TbrArgs &a, size_t smem, cudaStream_t s);
cudaError_t tbr_launch_a2(int depth, int W, int H, const TbrArgs &a, size_t smem, cudaStream_t s);
cudaError_t fill_launch(int dtype, void *p, long long n, double v, cudaStream_t s);
cudaError_t halo_copy_launch(int dtype, const void *A, void *B, int nx, int ny, int nz, cudaStream_t s,
                             int *status = nullptr, long long shrink = 0);

// Pass planning: split T sweeps into passes of depth <= d whose count has
// the parity of T (so the result ends in the grid single sweeps would use).
int plan_passes(int T, int d, int *depths, int max_passes);

}  // namespace jac

// Library-owned state behind a jacobi_h.
struct jacobi_plan_s {
    int nx = 0, ny = 0, nz = 0, dtype = 0, device = 0, sms = 0;
    jac::Plan plan;
    bool forced = false;
    int *d_status = nullptr;
    int fault_mode = 0;
    unsigned long long limit_ns = 2000000000ull;
    void *hostA = nullptr, *hostB = nullptr;  // device grids of jacobi_sweep_host
    bool prof = false;                          // profiling of pass launches
    std::vector<cudaEvent_t> ev_pool;           // events, reused after a read
    size_t ev_used = 0;
    int prof_pass = 0, prof_other = 0;
    long long check_shrink = 0;  // checked build test hook (jacobi_debug_set_fault mode 2)
    // compressed grid: depth, z chunk, chunk waves (0: the dtype's default,
    // FP32 3 / 128 / 1, FP64 1 / 64 / 1); item ticket and per-item flags
    int cg_depth = 0, cg_bz = 0, cg_waves = 0;
    int *cg_ctl = nullptr;
    size_t cg_ctl_n = 0;
    std::vector<int *> cg_old;  // replaced counter arrays, kept for captured graphs until destroy
    // Poisson / refinement scratch (allocated on first use, freed by destroy)
    void *g = nullptr;          // source term h^2 r (FP32) or h^2 f (FP64)
    void *e0 = nullptr, *e1 = nullptr;  // FP32 correction grids
    double *partials = nullptr;  // per-block partial sums of squares
    double *h_sum = nullptr;     // pinned host mirror of one reduced sum
    cudaGraphExec_t inner_exec = nullptr;  // K single-pass sweeps with a source term
    int inner_dtype = -1, inner_K = -1;
    const void *inner_A = nullptr, *inner_B = nullptr, *inner_G = nullptr;
};

namespace jac {
// Raises fn's dynamic shared memory limit on the current device to at least
// smem bytes.  The attribute call is made only when the limit grows (once
// per kernel and device in practice), so the launches that follow are plain
// stream work and can be captured into a CUDA graph.
cudaError_t ensure_smem_limit(const void *fn, size_t smem);
// The cluster kernels' attributes (largest dynamic shared memory, full
// shared-memory carveout, clusters above 8 CTAs), set once per kernel and
// device.
cudaError_t ensure_cluster_attrs(const void *fn, int smem_max);
void free_poisson_scratch(jacobi_plan_s *h);
// compressed grid (compressed.cu)
long long cg_shift_planes(int depth, int bz, int waves);
int cg_check(const jacobi_plan_s *h, int depth, int bz, int waves);
int cg_sweep(jacobi_plan_s *h, void *U, int T, int upper, int *upper_out, cudaStream_t s);
}

