// Device tables of the batched step (internal to the library).
#pragma once

#include "kernels.h"

namespace lbm {

constexpr int BATCH_RESCALE_EVERY = 64;  // FP16 storage: steps between scale checks

// One box of a batch, in device memory. The host writes it once at admission;
// afterwards only the step kernel's closing block changes cur, step, scale
// and amax.
struct BatchDomain {
    StepArgs a;          // sizes, periodicity, g (pre, post, dscale, seed unused)
    void* buf[2];        // ping-pong state records
    int ntx, ntiles;     // tiles in x, tiles per plane
    uint32_t cur;        // buf[cur] holds the current state
    int64_t step;        // steps taken
    float scale[2][8];   // 16-bit: {S, 1/S} of the contents of buf[0], buf[1]
    unsigned amax[4];    // 16-bit: max |value| stored this step (float bits)
    float gfloor;        // 64 |g|_max, the floor of the headroom rule
    int tma;             // 1: full tiles, stepped by the staged (TMA) tile column
};

// Header of a batch in device memory; the step kernel's only argument.
struct BatchTable {
    int nitems;              // work items (tile columns) of all live boxes
    int ndom;                // live boxes
    unsigned done;           // blocks finished in the current step
    unsigned next;           // items handed out beyond the first one of each block
    int chunk;               // planes per work item (the same for every box)
    const int* live;         // [ndom] slot of each live box
    const int* item_begin;   // [ndom] first item of each live box
    BatchDomain* dom;        // [capacity] by slot
    const CUtensorMap* maps; // [capacity][2] tensor maps of buf[0], buf[1] (boxes with tma)
};

// Persistent grid size and tile height (2H) of a kernel variant, in its
// staged (tma) or register instance.
cudaError_t batch_prepare(int q, int storage, int variant, bool tma, int* grid, int* tile_h);
cudaError_t launch_tau1_batch(int q, int storage, int variant, bool tma, BatchTable* T, int grid, cudaStream_t s);

}  // namespace lbm
