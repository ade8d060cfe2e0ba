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

constexpr int SMEM_MAX = 232448;  // dynamic shared memory a CTA may opt in to (227 KB)

struct PairLaunch {
    int f64;         // 1: binary64 path
    int chunk;       // primary lanes per warp chunk (8, 16 or 32)
    int pp;          // primaries per lane (1 or 2; float32 DD(r))
    int evals;       // count evaluations
    int verify;      // verify float32 decisions against binary64
    int blocks;      // persistent CTAs
    int smem;        // dynamic shared memory bytes
    int hist_words;  // shared histogram words
    int max_blocks;  // upper bound on the persistent grid (0 = none)
    int pipe;        // float32 DD(r) without sums: two tile buffers (no CTA barrier per item)
    int kernels;     // kernels the launch issued (work list, window pre-pass, pair kernel)
};

// Primaries per chunk of the float32 DD(r) kernel for a requested shape (chunk
// lanes x primaries per lane; the weighted sweep runs 16 x 1, the verifying
// one 8 x 1); the window pre-pass writes one record per chunk of this size.
inline int xi32_chunk(int chunk, int pp, bool weighted, bool verify)
{
    if (verify)
        return 8;
    if (weighted)
        return 16;
    if (pp == 4)
        return 32;
    if (pp == 2)
        return chunk == 8 ? 16 : 32;
    return chunk == 16 || chunk == 32 ? chunk : 8;
}

// Upper bound on the window records of one launch: every kept column pair
// (at most nstencil per column of d1) has one record per chunk of its column a,
// and the columns of d1 hold n1 points plus at most 3 padding points each.
inline long long win_bound(long long n1, int ncols, int nstencil, int chunk)
{
    return (long long)nstencil * ((n1 + 3ll * ncols) / chunk + ncols + 1);
}

// Fill the shared-memory plan of a launch: L.smem, L.hist_words and, for
// rp-pi, P.hcopies and P.hist_off.  Needs P.kind, P.nbins, P.npibins,
// P.tile_max and L.f64.
void plan_pairs(PairParams &P, PairLaunch &L);

// Configure (max dynamic smem), pick the occupancy-based grid and launch
// (the work-list kernel, then the pair kernel).
cudaError_t launch_pairs(const PairParams &P, PairLaunch &L, int sms, cudaStream_t st);

// ---- batched launch: jobs of these paths share one persistent kernel
enum : int {
    BATCH_XI32 = 0,       // float32 DD(r), chunks of 16 lanes x 2 primaries
    BATCH_XI64 = 1,
    BATCH_RPPI32 = 2,
    BATCH_RPPI64 = 3,
    BATCH_XI32_8x2 = 4,   // float32 DD(r) with the other tuned shapes
    BATCH_XI32_16x1 = 5,
    BATCH_XI32_32x1 = 6,
};
constexpr int BATCH_MAX = 1024;  // jobs per batched launch

struct BatchParams {
    const PairParams *jobs;  // device array, one per job (work lists already built)
    const int *path;         // device array: BATCH_* per job
    int njobs;
    unsigned *offsets;       // device, njobs + 1 (written by the launch)
    unsigned *item_counter;  // device, zeroed before the launch
};

// Path of a job: float32 (float32 DD(r) in the kernel shape chunk x pp: 16 x 2,
// 8 x 2, 16 x 1 or 32 x 1, else 16 x 2) or binary64, DD(r) or DD(rp, pi);
// unweighted only.
int batch_path(const PairParams &P, int f64, int chunk = 16, int pp = 2);

// The work-list kernel of one job (kept column pairs into P.work, count into
// *P.work_count, which must be zero).
cudaError_t launch_worklist(const PairParams &P, cudaStream_t st);

// The work lists of njobs jobs (device parameter array) in one launch; job j
// owns blocks [pre[j], pre[j + 1]) of 256 candidates, blocks = pre[njobs].
cudaError_t launch_worklist_batch(const PairParams *jobs, const unsigned *pre, int njobs,
                                  unsigned blocks, cudaStream_t st);

// Offsets over the jobs' kept pairs, then the batched persistent kernel with
// smem bytes of dynamic shared memory (the largest job's plan); blocks returns
// the grid size.
cudaError_t launch_batch(const BatchParams &B, int smem, int sms, int &blocks, cudaStream_t st);

}  // namespace cf
