// Host interface of the gridding kernels (grid.cu).
#pragma once

#include <cstring>

#include "cf_internal.cuh"

namespace cf {

// Temporaries of one grid build (device memory, carved from the workspace).
struct GridTemps {
    uint32_t *cell_of;   // n
    uint32_t *slot;      // n
    int *tmp_idx;        // n + 3 * ncols (padded index space)
    unsigned long long *tmp_key;  // n + 3 * ncols: order-preserving keys of z
    uint32_t *counts;    // ncells + 1 (the last: the in-cell sort's claim counter)
    uint32_t *pad;       // ncols
    uint32_t *bsum;      // ceil(ncells / 4096)
};

// Grid one catalogue into `out` (whose arrays are preallocated).
cudaError_t build_grid(cf_dtype dt, const void *x, const void *y, const void *z, const double *w,
                       long long n, const Geom &g, const GridTemps &t, Gridded &out, int sms,
                       unsigned *err, cudaStream_t st);

// Bounding box of a catalogue: out6 = order-preserving keys of (min x,y,z, max x,y,z);
// initialise out6[0..2] to ~0 and out6[3..5] to 0 first.
cudaError_t launch_bbox(cf_dtype dt, const void *x, const void *y, const void *z, long long n,
                        unsigned long long *out6, int sms, unsigned *err, cudaStream_t st);

double decode_dkey(unsigned long long k);

// ---- batched gridding: every catalogue of every job of a batch, one launch per stage
// One catalogue of a batch (a segment; device record).
struct GridSeg {
    const void *x, *y, *z;  // coordinates (device)
    int f32;                // 1: float32 coordinates, 0: binary64
    int job;                // index of the job's geometry
    long long n;            // points
    long long c0;           // first entry of the segment in the concatenated per-cell arrays
                            // (ncells + 1 entries per segment)
    Gridded out;            // output arrays (preallocated; no weights, no residuals)
    uint32_t *cell_of, *slot;      // n each
    int *tmp_idx;                  // n + 3 ncols
    unsigned long long *tmp_key;   // n + 3 ncols
    uint32_t *pad;                 // ncols
    unsigned *err;                 // the job's error word
};

// Block shapes of the batched stages; a stage's blocks are split among the
// segments by a prefix array pre[0..nseg] (segment s owns [pre[s], pre[s + 1])).
enum GridBatchShape {
    GB_POINTS,    // 256 points per block
    GB_COLWARPS,  // 8 columns per block (one warp each)
    GB_COLS,      // 256 columns per block (one thread each)
    GB_COLBLK,    // one column per block
    GB_CELLS,     // 256 entries of cell_start per block
    GB_SHAPES
};

struct GridBatch {
    const GridSeg *seg;         // device, nseg
    const Geom *geom;           // device, one per job
    int nseg;
    long long ctot;             // entries of the concatenated per-cell arrays
    uint32_t *counts;           // device, ctot + 1: raw cell counts, then the sort's claim counter
    uint32_t *scan;             // device, ctot: padded counts, scanned in place
    uint32_t *bsum;             // device, scan_block_sums(ctot)
    const unsigned *pre[GB_SHAPES];  // device prefix arrays (nseg + 1 each)
    unsigned blocks[GB_SHAPES];      // host copies of pre[k][nseg]
};

// Block-sum entries the scan of n elements needs.
long long scan_block_sums(long long n);

// Blocks of segment-shape k for a catalogue of n points on geometry g.
unsigned grid_batch_blocks(int k, long long n, const Geom &g);

// Grid every segment (the same outputs build_grid writes for each catalogue).
cudaError_t build_grid_batch(const GridBatch &B, int sms, cudaStream_t st);

// Kernel launches (and memsets) of one build_grid_batch.
inline int grid_batch_kernels() { return 11; }

// Kernels launched by build_grid / launch_bbox for a catalogue of n points.
inline int grid_kernels(long long n, bool residuals = false)
{
    return (n > 0 ? 9 : 6) + (residuals ? 1 : 0);
}
inline int bbox_kernels(long long n) { return n > 0 ? 1 : 0; }

}  // namespace cf
