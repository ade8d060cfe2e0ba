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

// Kernels launched by build_grid / launch_bbox for a catalogue of n points.
inline int grid_kernels(long long n, bool residuals = false)
{
    return (n > 0 ? 9 : 6) + (residuals ? 1 : 0);
}
inline int bbox_kernels(long long n) { return n > 0 ? 1 : 0; }

}  // namespace cf
