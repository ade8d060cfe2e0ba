// Internal definitions shared by the cfgpu translation units (not installed).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "cf.h"

namespace cf {

// ----------------------------------------------------------------- limits
constexpr int NB_MAX = 64;          // radial (xi) or rp bins
constexpr int NBINS2D_MAX = 4096;   // rp bins * pi bins
constexpr int NPI_MAX = 4096;
constexpr int LUT_MAX = 16384;      // entries (bytes) of the float32 bin lookup table
constexpr int TILE32 = 2048;        // secondary points per staged float32 tile
constexpr int MAX_REACH = 4;        // column stencil half-width per axis
constexpr int MAX_STENCIL = (2 * MAX_REACH + 1) * (2 * MAX_REACH + 1);
constexpr int WARPS = 8;            // warps per pair-kernel CTA
constexpr int THREADS = WARPS * 32;
constexpr unsigned FULL = 0xffffffffu;

// Error-word bits written by kernels (read back once per call).
enum : unsigned {
    ERR_COORD = 1u,     // non-finite coordinate or outside [0, L) in periodic mode
    ERR_TIMEOUT = 2u,   // a bounded mbarrier wait gave up
    ERR_INTERNAL = 4u,  // an index or table inconsistency that must never happen
};

// Lookup-table entry (one byte): 0..nbins-1 -> the bin (the cell lies wholly
// between hi_k and lo_{k+1}); nbins -> surely not counted; TAB_FLAGGED (0xff)
// -> the cell touches a threshold or a band (settled by the thresholds, maybe
// a binary64 re-check).  Loaded sign-extended the flagged entry is -1, so its
// sign bit marks the pair: the float32 kernels keep a histogram row for each
// of the values -1 .. nbins (the row of -1 just before bin 0, never read) and
// an entry is a row index without a clamp.
constexpr unsigned char TAB_FLAGGED = 0xff;

// Shared layout of the float32 DD(r) kernel (compile-time offsets):
// [0,128) barrier + work item; LUT; x, y, z tiles of TILE32 + 64 floats each;
// thresholds; squared edges; histogram copies ((nbins + 2) rows of 32 lanes each:
// the flagged row, the bins, the not-counted row).
constexpr int XI32_LUT_OFF = 128;
constexpr int XI32_TX_OFF = XI32_LUT_OFF + LUT_MAX;
constexpr int XI32_TSTRIDE = (TILE32 + 64) * 4;
constexpr int XI32_THR_OFF = XI32_TX_OFF + 3 * XI32_TSTRIDE;
constexpr int XI32_E2_OFF = XI32_THR_OFF + 2 * (NB_MAX + 1) * 4;
constexpr int XI32_HIST_OFF = XI32_E2_OFF + (NB_MAX + 1) * 8;

// The pipelined float32 DD(r) kernel keeps one histogram copy shared by all
// warps and places its second tile buffer after it.
__host__ __device__ constexpr int pipe_slot1_off(int nbins)
{
    return (XI32_HIST_OFF + (nbins + 2) * 128 + 127) & ~127;
}

// The weighted float32 DD(rp, pi) kernel stages a weight tile after the squared
// edges.
constexpr int XIW_W_OFF = XI32_HIST_OFF;
static_assert(XIW_W_OFF % 16 == 0, "bulk-copy destinations need 16 B");

// The float32 DD(rp, pi) kernel uses the DD(r) layout up to the thresholds and
// squared rp edges, then a weight tile (as above), the pi edges (binary64) and,
// from a run-time offset, its histograms: hcopies copies of (nbins + 1) rows
// of (npibins + 1) words (row nbins and column npibins collect pairs that are
// not counted), then for weighted sums binary64 [copy][slot][w, r w].
constexpr int RPPI_P_OFF = XIW_W_OFF + XI32_TSTRIDE;

// Grid geometry: columns in (x, y), z-cells inside each column (sort keys).
struct Geom {
    int periodic;
    int ncx, ncy, nz;
    int ncols;
    long long ncells;
    int reach_x, reach_y;
    int reach_z;            // z refinement (z-cells of the in-column sort per Rmax)
    double origin[3];   // grid frame origin (0 in periodic mode)
    double extent[3];   // grid extent (= box in periodic mode)
    double inv_w[3];    // cells per unit length along each axis
    double box[3];      // periodic box (0 when open)
    float inv_wf[3];    // fl32(inv_w): cell indices are computed in float32
    long long box_bits[3];  // bit pattern of box (binary64 inputs: 0 <= x < box)
    int box_bits32[3];      // bits of the smallest float >= box (float32 inputs)
};

// A gridded catalogue, in (column, z, original index) order; every column is
// padded with NaN entries to a multiple of 4 (see grid.cu).
struct Gridded {
    long long n;
    float *xs, *ys, *zs;  // float32 coordinates in the grid frame (padded columns)
    float *ws;            // float32 weights (padded columns, 64 floats of slack; NULL without weights)
    unsigned *wmax;       // bit pattern of max |w| as float (written by gridding; NULL without weights)
    float *xl, *yl, *zl;  // rounding residuals fl32((X - O) - xs) of the float32 coordinates
                          // (float32 mean separations from float64 inputs; else NULL)
    double4_32a *pos64;       // (x, y, z, w) binary64, exact inputs
    int *perm;            // original index of each sorted point
    uint32_t *cell_start; // ncells + 1
    double4_32a *colbox;      // per column (xmin, xmax, ymin, ymax)
};

// One kept column pair (Sec. 2.2 pruning done), written by the work-list kernel.
struct __align__(16) WorkItem {
    int a0, a1, b0, b1;  // point ranges of columns a and b
    double dzmax;        // z reach of the pair (binary64, already widened)
    int code;            // bits 0-1: qx + 1, bits 2-3: qy + 1 (periodic image), bit 4: self pair,
                         // bits 5-31: column b
    int wbase;           // first window record of the pair's chunks (window pre-pass), else 0
};

// Window record of one chunk of column a against column b (window pre-pass):
// for each periodic z image k = -1, 0, +1 the range [lo, hi) of column b (point
// indices) whose float32 z can lie within the pair's z reach of the chunk; an
// empty range (lo == hi) when the image does not apply.
struct __align__(8) Win {
    int lo[3], hi[3];
};

// Cell index along one axis from a float32 frame coordinate (monotone in it):
// the gridding's rule, also used to locate a z value among a column's z-cells.
__device__ __forceinline__ int cell_index_f(float t, float inv_w, int n)
{
    const float c = floorf(__fmul_rn(t, inv_w));
    return (int)fminf(fmaxf(c, 0.0f), (float)(n - 1));
}

// Everything a pair kernel needs (passed by value, lives in the constant bank).
struct PairParams {
    Gridded A, B;
    Geom g;
    int autocorr;
    int kind;           // 0 = xi, 1 = rp-pi
    int nstencil;
    int2 stencil[MAX_STENCIL];
    int n_items;        // (column, stencil offset) candidates
    int shard_k, shard_n;  // keep columns whose first point lies in slice k of n (n > 1)
    WorkItem *work;     // kept column pairs (work-list kernel output)
    unsigned *work_count;  // number of kept column pairs
    Win *win;           // window records (window pre-pass), NULL = windows found in the sweep
    unsigned *win_count;   // window records handed out by the work-list kernel
    long long win_cap;  // capacity of win (records)
    int win_chunk;      // primaries per chunk the windows are computed for (0 = no pre-pass)
    int tile_max;       // points per staged tile
    uint32_t flags;
    uint64_t wait_ns;   // limit of every tile-barrier wait (then the error word gets ERR_TIMEOUT)
    // radii (binary64 decisions on bounding boxes)
    double prune_r2;    // prune a column pair if its xy gap^2 >= prune_r2
    double rz;          // z reach: Rmax (xi) or pimax (rp-pi)
    double rxy2;        // squared xy reach for the z window: Rmax^2
    float zslack;       // float32 slack added to z windows
    float boxf[3];      // fl32(L)
    // binning
    int nbins;          // xi or rp bins
    int npibins;        // rp-pi only
    int nthr;           // 2 * nbins + 2 float32 thresholds
    int lut_n, lut_shift; // table entries (last one = out of range), cell width 2^shift
    uint32_t u0;          // (float bit pattern of the table's first cell) >> lut_shift
    int lut_lin;          // 1: cells linear in d2 (cell = round(d2 * lut_scale)), else logarithmic
    float lut_scale;
    float pscale;       // rp-pi: fl32(npibins / pimax), pi edges at integer t = |dz| * pscale
    float pband;        // rp-pi: |t - 1/2 - round(t - 1/2)| > pband means t is near an edge
    int hcopies;        // rp-pi: shared histogram copies per CTA (warp w uses w % hcopies)
    int hist_off;       // byte offset of the shared histograms (rp-pi kernels)
    // weighted sums (Code 1's weight per bin) and mean separation
    int weighted;       // pair weight w_i * w_j (else 1)
    int want_r;         // accumulate r (xi) or rp (rp-pi) times the pair weight
    int wacc;           // weighted || want_r
    int rlo;            // float32 mean separation corrected with the coordinates' residuals
    int acc_off;        // byte offset of the binary64 accumulators in shared memory
    long long *wscratch;  // float32 weighted DD(r): per-thread [bin][count, w, r w] int64 sums
    const float *thr;        // nthr
    const uint8_t *lut;      // lut_n
    const double *E2;        // nbins + 1
    const double *P;         // npibins + 1 pi edges (rp-pi)
    // outputs
    unsigned long long *hist;  // nbins (xi) or nbins * npibins
    double *wsum, *rsum;       // same shape (accumulated only when wacc)
    unsigned long long *diag;  // [0] kept items, [1] evaluations, [2] rechecks, [3] band violations
    unsigned *err;
    unsigned *item_counter;
};

// ----------------------------------------------------------------- device helpers
__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

// Plain arrive (no transaction bytes): completes a phase that carries no copy.
__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Nanoseconds of the GPU's global timer.
__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// One bounded wait on phase `parity`: true once the phase completed, false
// after limit_ns nanoseconds (or 2^26 tries, whichever comes first).
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, unsigned parity, uint64_t limit_ns)
{
    const uint32_t a = smem_u32(bar);
    uint64_t t0 = 0;
    for (unsigned it = 0; it < (1u << 26); ++it) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            " selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done)
            return true;
        if ((it & 31u) == 0u) {
            const uint64_t t = global_ns();
            if (it == 0u)
                t0 = t;
            else if (t - t0 > limit_ns)
                return false;
        }
    }
    return false;
}

// 1-D bulk copy global -> shared (TMA, no tensor map), completion on `bar`.
// dst, src 16-byte aligned; bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
            "r"(smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Canonical binary64 squared separation of point j (image shifted by S) from i:
// d = fl(x_j - x_i), then fl(d + S) when S != 0; rp2 = dx*dx + dy*dy; r2 = rp2 + dz*dz.
// With S equal to the periodic image of j, this is bit-identical to the
// minimum-image wrap for every pair closer than L/2.
__device__ __forceinline__ double canon_comp(double xi, double xj, double S)
{
    double d = __dsub_rn(xj, xi);
    if (S != 0.0)
        d = __dadd_rn(d, S);
    return d;
}

}  // namespace cf
