// Internal declarations shared by the batch engine (batch.cu) and the
// batched register-blocked FP32 passes (batch_tbr.cu).
#pragma once
#include <cuda_runtime.h>

#include <vector>

namespace jac {

struct BatchGrid {
    void *A;
    void *B;
    const void *rhs;  // optional source term g (same dtype): update (sum + g)/6
    int nx, ny, nz, dtype, T;
    int Te;  // sweeps done by the sweep or persistent engine: T, or 0 for an
             // FP32 grid that the batched blocked passes take
    int ntx, nty, ntz;
    int tile_base;  // global index of this grid's tile 0
    int nbxy, nbz;  // sweep engine: runs of kSweepThreads x-y cells, z chunks
};

// One FP32 grid in one launch of batched temporally blocked passes: its
// tiles are the launch's blocks unit_base .. unit_base + ntx*nty*ntz - 1;
// tile geometry as for the one-CTA register-blocked kernel (64 x 32 regions).
struct TbrBatchEntry {
    long long unit_base;
    int grid;
    int ntx, nty, ntz;
    int bx, by, off, x_first;
};

// One launch: pass `pass` of every listed grid at `depth`, copy pieces of A
// elements; its entries are tab[tab_off .. tab_off + count - 1].
struct TbrBatchLaunch {
    int pass, depth, A;
    long long tab_off;
    int count;
    long long units;
};

constexpr int kBatchTbrZ = 128;  // z chunk of the batched passes

// Splits every FP32 grid's T sweeps into passes of depth <= depth (count
// with the parity of T) and groups the grids of each pass by (depth, A).
void batch_tbr_plan(const std::vector<BatchGrid> &grids, int depth, std::vector<TbrBatchEntry> &tab,
                    std::vector<TbrBatchLaunch> &launches);
// Sets the launch's kernel attributes (before stream capture).
cudaError_t batch_tbr_configure(const TbrBatchLaunch &L);
cudaError_t batch_tbr_launch(const TbrBatchLaunch &L, const BatchGrid *d_grids, const TbrBatchEntry *d_tab,
                             int *status, long long shrink, cudaStream_t s);

}  // namespace jac
