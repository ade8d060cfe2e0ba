// Host interface of the pair kernels (pairs.cu).
#pragma once

#include "cf_internal.cuh"

namespace cf {

__host__ __device__ inline int align_up(int v, int a) { return (v + a - 1) / a * a; }

// Shared-memory layout of the binary64 kernels (identical on host and device):
// [0, 128) barrier + work item; tile of tile_max + 32 points (x, y, z, w);
// squared edges; pi edges (rp-pi); histograms.
struct Smem64 {
    int tile, e2, p, hist, total;
};

__host__ __device__ inline Smem64 smem64_layout(int tile_max, int nbins, int npibins, int hist_words)
{
    Smem64 L;
    int off = 128;
    L.tile = off;
    off += (tile_max + 32) * 32;
    L.e2 = off = align_up(off, 16);
    off += (nbins + 1) * 8;
    L.p = off = align_up(off, 16);
    off += (npibins > 0 ? npibins + 1 : 0) * 8;
    L.hist = off = align_up(off, 128);
    off += hist_words * 4;
    L.total = align_up(off, 128);
    return L;
}

struct PairLaunch {
    int f64;         // 1: binary64 path
    int chunk;       // primary lanes per warp chunk (8, 16 or 32)
    int pp;          // primaries per lane (1 or 2; float32 DD(r))
    int evals;       // count evaluations
    int verify;      // verify float32 decisions against binary64
    int blocks;      // persistent CTAs
    int smem;        // dynamic shared memory bytes
    int hist_words;  // shared histogram words
};

// Fill the shared-memory plan of a launch: L.smem, L.hist_words and, for
// rp-pi, P.hcopies and P.hist_off.  Needs P.kind, P.nbins, P.npibins,
// P.tile_max and L.f64.
void plan_pairs(PairParams &P, PairLaunch &L);

// Configure (max dynamic smem), pick the occupancy-based grid and launch.
cudaError_t launch_pairs(const PairParams &P, PairLaunch &L, int sms, cudaStream_t st);

}  // namespace cf
