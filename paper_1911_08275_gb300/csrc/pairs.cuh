// Host interface of the pair kernels (pairs.cu).
#pragma once

#include "cf_internal.cuh"

namespace cf {

// Shared-memory layout of a pair-kernel CTA (identical on host and device).
struct SmemLayout {
    int tile, lut, thr, e2, pilut, pithr, p, hist, total;
};

__host__ __device__ inline int align_up(int v, int a) { return (v + a - 1) / a * a; }

__host__ __device__ inline SmemLayout smem_layout(int tile_max, int pt_bytes, int lut_n, int nthr,
                                                  int nbins, int pilut_n, int pi_nthr, int npibins,
                                                  int hist_words)
{
    SmemLayout L;
    int off = 128;  // [0, 128): mbarrier, work item, flags
    L.tile = off;
    off += (tile_max + 32) * pt_bytes;
    L.lut = off = align_up(off, 16);
    off += lut_n * 2;
    L.thr = off = align_up(off, 16);
    off += nthr * 4;
    L.e2 = off = align_up(off, 16);
    off += (nbins + 1) * 8;
    L.pilut = off = align_up(off, 16);
    off += pilut_n * 2;
    L.pithr = off = align_up(off, 16);
    off += pi_nthr * 4;
    L.p = off = align_up(off, 16);
    off += (npibins > 0 ? npibins + 1 : 0) * 8;
    L.hist = off = align_up(off, 16);
    off += hist_words * 4;
    L.total = align_up(off, 128);
    return L;
}

struct PairLaunch {
    int f64;         // 1: binary64 path
    int chunk;       // primary points per warp chunk (8, 16 or 32)
    int evals;       // count evaluations
    int verify;      // verify float32 decisions against binary64
    int blocks;      // persistent CTAs
    int smem;        // dynamic shared memory bytes
    int hist_words;  // shared histogram words
};

// Dynamic shared memory of the float32 DD(r) kernel for nbins bins.
int xi32_smem_bytes(int nbins);

// Hist words of one CTA for a given kind / bin count (xi: per-lane rows per warp;
// rp-pi: one row per warp).
int pair_hist_words(int kind, int nbins, int npibins);

// Configure (max dynamic smem), pick the occupancy-based grid and launch.
cudaError_t launch_pairs(const PairParams &P, PairLaunch &L, int sms, cudaStream_t st);

}  // namespace cf
